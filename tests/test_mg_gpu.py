"""Parity of the CUDA block multigrid (through the C-ABI) with the oracle V-cycle:
eigenvalue estimates per level and the V-cycle output of both blocks, for the
FP64 and the FP32 V-cycle (tolerances 1e-10 and 1e-5 relative)."""
import numpy as np
import pytest

from harness import LAMBDA_RTOL, Pair, random_active, random_linearisation, rel_err
from oracle import mg as omg
from oracle import operators as ops

pytestmark = pytest.mark.gpu

_cache = {}


def setup_pair(name, frac, seed=0):
    key = (name, frac, seed)
    if key in _cache:
        return _cache[key]
    P = Pair(name, 1)
    mat = P.material(kappa=1e-3, p=0.05)
    u, phi, phit = random_linearisation(P, seed=seed, u_std=1e-2)
    active = random_active(P, seed=5, frac=frac) if frac > 0 else np.zeros(P.om.nn, bool)
    M = omg.MG(P.om, ops.Material(**mat), u, phi, phit, active)
    _cache[key] = (P, mat, u, phi, phit, active, M)
    return _cache[key]


def lib_mg(P, mat, u, phi, phit, active, prec):
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64, Problem
    dev = torch.device("cuda:0")
    pb = Problem(P.lm, **mat)
    pb.set_state(torch.tensor(P.to_slots(u).T.copy(), device=dev), torch.tensor(P.to_slots(phi), device=dev),
                 torch.tensor(P.to_slots(phit), device=dev))
    pb.set_active(torch.tensor(P.to_slots(active.astype(np.uint8)), device=dev))
    mg = MG(pb, PFF_F64 if prec == "f64" else PFF_F32)
    mg.setup()
    return pb, mg


@pytest.mark.parametrize("name,frac", [("tiny", 0.0), ("small", 0.0), ("small", 0.05), ("band4_2_4", 0.0)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lambda_estimates(name, frac, prec):
    """lambda_max per level against the oracle's FP64 CG: 1e-9 for the FP64 V-cycle,
    LAMBDA_RTOL for the FP32 one (its CG applies the level operators in FP32; the
    small active-set mesh has a 3-DoF level whose Krylov space the run exhausts)."""
    P, mat, u, phi, phit, active, M = setup_pair(name, frac)
    pb, mg = lib_mg(P, mat, u, phi, phit, active, prec)
    for b, blk in ((0, "uu"), (1, "pp")):
        lam = mg.lam(b)
        ref = np.array([0.0] + [M.B[blk][l].lam for l in range(1, len(M.B[blk]))])
        assert np.allclose(lam[1:], ref[1:], rtol=LAMBDA_RTOL[prec], atol=1e-300), (blk, lam, ref)


@pytest.mark.parametrize("name,frac", [("tiny", 0.0), ("small", 0.0), ("small", 0.05), ("band4_2_4", 0.0)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
@pytest.mark.parametrize("fused", [True, False])
def test_vcycle_parity(name, frac, prec, tol, fused):
    """Both smoother paths: Chebyshev steps fused into the level sweeps' stores, and
    apply and update as separate kernels."""
    import torch
    P, mat, u, phi, phit, active, M = setup_pair(name, frac)
    pb, mg = lib_mg(P, mat, u, phi, phit, active, prec)
    mg.set_fused_smoother(fused)
    om = P.om
    nn = om.nn
    rng = np.random.default_rng(3)
    for b, blk, nc in ((0, "uu", 2), (1, "pp", 1)):
        r = rng.normal(size=(nn, nc))
        zref = M.vcycle(blk, np.concatenate([r[:, c] for c in range(nc)]))
        zref = np.stack([zref[c * nn:(c + 1) * nn] for c in range(nc)], 1)
        rs = P.to_slots(r)
        rs[~P.valid] = 1e30   # holes must be ignored
        rt = torch.tensor(rs.T.copy() if nc == 2 else rs[:, 0].copy(), device="cuda")
        zt = torch.full_like(rt, float("nan"))
        mg.vcycle(b, rt, zt)
        torch.cuda.synchronize()
        zs = zt.cpu().numpy()
        zs = zs.T if nc == 2 else zs[:, None]
        assert np.all(zs[~P.valid] == 0.0)
        z = P.from_slots(zs)
        assert np.all(z[om.is_hanging] == 0.0)
        inf, two = rel_err(z, zref)
        assert inf < tol and two < tol, (blk, prec, inf, two)


@pytest.mark.parametrize("name,frac", [("small", 0.0), ("small", 0.05), ("band4_2_4", 0.0)])
def test_inverse_diagonal(name, frac):
    """pff_inverse_diagonal against the oracle's 1/diag(A_l) on interior rows, 0 elsewhere (1e-12)."""
    P, mat, u, phi, phit, active, M = setup_pair(name, frac)
    pb, mg = lib_mg(P, mat, u, phi, phit, active, "f64")
    for b, blk, nc in ((0, "uu", 2), (1, "pp", 1)):
        for l, lm in enumerate(M.levels):
            d, X, Y = mg.inverse_diagonal(l, b)
            d = d.cpu().numpy().reshape(nc, -1)
            valid = X >= 0
            assert np.all(d[:, ~valid] == 0.0)
            key = Y[valid].astype(np.int64) * (lm.Xmax + 1) + X[valid]
            node = np.searchsorted(lm.key, key)
            assert np.array_equal(lm.key[node], key)
            ref = M.B[blk][l].dinv.reshape(nc, -1)[:, node]
            got = d[:, valid]
            assert np.array_equal(got == 0.0, ref == 0.0), (blk, l)
            scale = np.abs(ref).max() if np.abs(ref).max() > 0 else 1.0
            assert np.abs(got - ref).max() <= 1e-12 * scale, (blk, l)


@pytest.mark.parametrize("name,frac", [("small", 0.0), ("small", 0.05), ("band4_2_4", 0.0)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_vcycle_chebyshev_coarse(name, frac, prec, tol):
    """V-cycle with the Chebyshev coarse solver of Sec. 3.2 against the oracle's (same
    reading of interval and degree), and the level-0 lambda_max (1e-9)."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64, Problem
    P, mat, u, phi, phit, active, _ = setup_pair(name, frac)
    om = P.om
    nn = om.nn
    M = omg.MG(om, ops.Material(**mat), u, phi, phit, active, coarse="chebyshev")
    pb = Problem(P.lm, **mat)
    pb.set_state(torch.tensor(P.to_slots(u).T.copy(), device="cuda"), torch.tensor(P.to_slots(phi), device="cuda"),
                 torch.tensor(P.to_slots(phit), device="cuda"))
    pb.set_active(torch.tensor(P.to_slots(active.astype(np.uint8)), device="cuda"))
    mg = MG(pb, PFF_F64 if prec == "f64" else PFF_F32, coarse="chebyshev")
    mg.setup()
    rng = np.random.default_rng(3)
    for b, blk, nc in ((0, "uu", 2), (1, "pp", 1)):
        lam = mg.lam(b)
        ref = M.B[blk][0].cheb[1] / 1.2
        assert abs(lam[0] - ref) <= 1e-9 * max(abs(ref), 1e-300), (blk, lam[0], ref)
        r = rng.normal(size=(nn, nc))
        zref = M.vcycle(blk, np.concatenate([r[:, c] for c in range(nc)]))
        zref = np.stack([zref[c * nn:(c + 1) * nn] for c in range(nc)], 1)
        rs = P.to_slots(r)
        rt = torch.tensor(rs.T.copy() if nc == 2 else rs[:, 0].copy(), device="cuda")
        zt = torch.full_like(rt, float("nan"))
        mg.vcycle(b, rt, zt)
        torch.cuda.synchronize()
        zs = zt.cpu().numpy()
        z = P.from_slots(zs.T if nc == 2 else zs[:, None])
        inf, two = rel_err(z, zref)
        assert inf < tol and two < tol, (blk, prec, inf, two)


def lib_mg_schedule(P, mat, u, phi, phit, active, prec, sched):
    """lib_mg with the Q1 cell loop forced to one strip schedule (before the set-up,
    which captures the V-cycle)."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64, Problem
    dev = torch.device("cuda:0")
    pb = Problem(P.lm, **mat)
    pb.set_cell_loop(sched)
    pb.set_state(torch.tensor(P.to_slots(u).T.copy(), device=dev), torch.tensor(P.to_slots(phi), device=dev),
                 torch.tensor(P.to_slots(phit), device=dev))
    pb.set_active(torch.tensor(P.to_slots(active.astype(np.uint8)), device=dev))
    mg = MG(pb, PFF_F64 if prec == "f64" else PFF_F32)
    mg.setup()
    return pb, mg


@pytest.mark.parametrize("name,frac", [("small", 0.05), ("band4_2_4", 0.0)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_vcycle_parity_every_strip_schedule(name, frac, prec, tol):
    """The level block operators (Sec. 3.2) under each strip schedule of the cell
    loop (one, three or fifteen strips per brick): V-cycle output against the
    oracle, and bitwise equal across the schedules (same arithmetic per cell and
    the same summation order of every nodal sum)."""
    import torch
    P, mat, u, phi, phit, active, M = setup_pair(name, frac)
    om = P.om
    nn = om.nn
    outs = {}
    for sched in (15, 5, 1):
        pb, mg = lib_mg_schedule(P, mat, u, phi, phit, active, prec, sched)
        rng = np.random.default_rng(3)
        for b, blk, nc in ((0, "uu", 2), (1, "pp", 1)):
            r = rng.normal(size=(nn, nc))
            rs = P.to_slots(r)
            rt = torch.tensor(rs.T.copy() if nc == 2 else rs[:, 0].copy(), device="cuda")
            zt = torch.full_like(rt, float("nan"))
            mg.vcycle(b, rt, zt)
            torch.cuda.synchronize()
            zs = zt.cpu().numpy()
            outs.setdefault(b, []).append(zs)
            zref = M.vcycle(blk, np.concatenate([r[:, c] for c in range(nc)]))
            zref = np.stack([zref[c * nn:(c + 1) * nn] for c in range(nc)], 1)
            z = P.from_slots(zs.T if nc == 2 else zs[:, None])
            inf, two = rel_err(z, zref)
            assert inf < tol and two < tol, (sched, blk, prec, inf, two)
    for b, zs in outs.items():
        assert np.array_equal(zs[0], zs[1]) and np.array_equal(zs[0], zs[2]), b


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_setup_graph_replay(prec):
    """From its second set-up on, an MG replays its set-up chains as a captured graph,
    re-captured when the pressure (a constant baked into the launches) changes.  After
    a pressure change the replaying MG gives bitwise the lambda estimates and V-cycle
    outputs of a fresh MG set up directly at the new pressure, and a further replay
    gives them again."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64
    P, mat, u, phi, phit, active, M = setup_pair("small", 0.05)
    pb, mg = lib_mg(P, mat, u, phi, phit, active, prec)   # first set-up: direct launches
    p2 = 0.5 * mat["p"]
    pb.set_pressure(p2)
    mg.setup()                                              # key changed: capture, then replay

    def state(m):
        nn = P.om.nn
        rng = np.random.default_rng(7)
        out = [m.lam(0), m.lam(1)]
        for b, nc in ((0, 2), (1, 1)):
            rs = P.to_slots(rng.normal(size=(nn, nc)))
            rt = torch.tensor(rs.T.copy() if nc == 2 else rs[:, 0].copy(), device="cuda")
            zt = torch.full_like(rt, float("nan"))
            m.vcycle(b, rt, zt)
            torch.cuda.synchronize()
            out.append(zt.cpu().numpy())
        return out

    a = state(mg)
    mg.setup()                                              # same key: replay
    b = state(mg)
    mat2 = dict(mat, p=p2)
    pb2, mg2 = lib_mg(P, mat2, u, phi, phit, active, prec)
    c = state(mg2)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)
