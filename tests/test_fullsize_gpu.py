"""Full-size checks, in the launch configuration bench.py times.

* Leaf Jacobian apply on the 4,096,509-DoF Q1 apply workload (16x16 coarse, 6
  global + 2 box refinements; the bench's own seeded inputs): sampled rows
  against the oracle, which assembles only the cells that touch the sampled
  nodes and their hanging children, so that each sampled row of
  G~ = M_f C^T G C M_f + I_fixed is exact (1e-12 FP64, 1e-5 FP32, relative to
  the largest sampled |y|).  Sampled: random nodes, hanging nodes (rows must be
  0), their parents, Dirichlet nodes (identity rows), and nodes on brick edges.
  Whole-vector properties at any size: holes 0, hanging rows 0, FP32 = FP64 to
  1e-5.
* Load step on the 1,043,811-DoF band-refined crack mesh (p = 1e-3): properties
  that hold at any size (convergence, phi <= phi_old, phi = phi_old on the
  active set, TCV within the error of the comparable rows of Table 2, FP32-MG and
  FP64-MG solutions equal to 1e-7).
* Symmetry of the FP64 V-cycle of both diagonal blocks on that mesh.
"""
import numpy as np
import pytest

import synthetic as synth
from harness import Pair, rel_err
from oracle import operators as ops

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_cache = {}


def apply_pair():
    if "apply" not in _cache:
        _cache["apply"] = Pair("apply", 1)
    return _cache["apply"]


def sampled_rows(P, rng):
    om = P.om
    nn = om.nn
    hang = np.nonzero(om.is_hanging)[0]
    Cc = om.C.tocsc()
    h_s = rng.choice(hang, size=min(100, len(hang)), replace=False)
    parents = np.unique(np.concatenate([om.C[h].indices for h in h_s]))
    dirich = rng.choice(np.nonzero(om.dirichlet)[0], size=100, replace=False)
    rand = rng.choice(nn, size=1000, replace=False)
    # nodes on brick edges of their level (30 x 30 node slots per brick)
    X, Y, F = P.slot_X, P.slot_Y, P.slot_F
    edge_slots = np.nonzero(((F & 1) == 1) & (((np.arange(len(X)) % 900) % 30 == 0)
                                              | ((np.arange(len(X)) % 900) // 30 == 29)))[0]
    edge_nodes = P.onode[np.searchsorted(P.slots, rng.choice(edge_slots, size=300, replace=False))]
    S = np.unique(np.concatenate([h_s, parents, dirich, rand, edge_nodes]))
    # cells touching S or a hanging child of S
    touch = set(S.tolist())
    for i in S:
        touch.update(Cc.indices[Cc.indptr[i]:Cc.indptr[i + 1]].tolist())
    touch = np.array(sorted(touch))
    cn = om.cell_nodes
    mask = np.isin(cn, touch).any(axis=1)
    return S, np.nonzero(mask)[0], h_s


def test_apply_fullsize_sampled():
    import torch
    from paper_2404_03265_gb300 import PFF_OP_JACOBIAN, Problem
    P = apply_pair()
    om = P.om
    nn = om.nn
    h = om.h_min_diag()
    mat = dict(E=1.0, nu=0.2, Gc=1.0, eps=2.0 * h, kappa=1e-10, p=1e-3)
    # the bench's inputs: linearisation seed 0 (u ~ N(0, 1e-3^2)), x seed 1, no active set
    u, phi, phit = synth.linearisation(om.X, om.Y, om.Xmax, om.Ymax, seed=0, u_std=1e-3)
    x = synth.vector(om.X, om.Y, seed=1)
    pb = Problem(P.lm, **mat)
    dv = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dt)
    pb.set_state(dv(P.to_slots(u).T), dv(P.to_slots(phi)), dv(P.to_slots(phit)))
    xs = P.to_slots(x)
    out = {}
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        xu, xp = dv(xs[:, :2].T, dt), dv(xs[:, 2], dt)
        yu, yp = torch.full_like(xu, float("nan")), torch.full_like(xp, float("nan"))
        pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN)
        torch.cuda.synchronize()
        ys = np.concatenate([yu.cpu().double().numpy().T, yp.cpu().double().numpy()[:, None]], 1)
        assert np.all(ys[~P.valid] == 0.0), "holes must be written as zero"
        out[name] = P.from_slots(ys)
    for name in out:
        assert np.all(np.isfinite(out[name]))
        assert np.all(out[name][om.is_hanging] == 0.0)
    assert max(rel_err(out["f32"], out["f64"])) < 1e-5
    # sampled rows against the oracle
    rng = np.random.Generator(np.random.PCG64(11))
    S, cells, h_s = sampled_rows(P, rng)
    st = ops.State(om, u, phi, phit)
    G = ops.assemble_jacobian(om, ops.Material(**mat), st, cell_idx=cells)
    active = np.zeros(nn, bool)
    v = np.concatenate([x[:, 0], x[:, 1], x[:, 2]])
    y = ops.constrained_operator(om, G, active) @ v
    ref = np.stack([y[:nn], y[nn:2 * nn], y[2 * nn:]], 1)[S]
    assert np.all(ref[np.isin(S, h_s)] == 0.0)
    for name, tol in (("f64", 1e-12), ("f32", 1e-5)):
        err = np.abs(out[name][S] - ref).max() / np.abs(ref).max()
        assert err < tol, (name, err)
    # identity rows on Dirichlet u
    d = np.nonzero(om.dirichlet)[0]
    assert np.array_equal(out["f64"][d, :2], x[d, :2])
    # every strip schedule of the cell loop gives the same bits (the schedule by
    # mesh size, taken above, runs regular bricks as one strip and irregular ones
    # as three)
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        xu, xp = dv(xs[:, :2].T, dt), dv(xs[:, 2], dt)
        ref_bits = None
        for sched in (0, 15, 5, 1):
            pb.set_cell_loop(sched)
            yu, yp = torch.full_like(xu, float("nan")), torch.full_like(xp, float("nan"))
            pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN)
            torch.cuda.synchronize()
            bits = torch.cat([yu.reshape(-1), yp]).cpu().numpy()
            if ref_bits is None:
                ref_bits = bits
            assert np.array_equal(bits, ref_bits), (name, sched)
    pb.set_cell_loop(0)


def solve_setup():
    import torch
    from paper_2404_03265_gb300 import Mesh, Problem
    if "solve" in _cache:
        return _cache["solve"]
    mesh = Mesh.from_recipe(synth.recipe("solve")).finalize(1)
    info = mesh.info
    X, Y, F = mesh.slots()
    valid = (F & 1) == 1
    x, y = synth.node_xy(X[valid], Y[valid], info["x_max"], info["y_max"])
    h = info["h_min"]
    po = np.ones(info["n_slots"])
    po[valid] = synth.crack_phi_old(x, y, h)
    m = synth.material(h_min=h)
    mat = dict(E=m["E"], nu=m["nu"], Gc=m["Gc"], eps=m["eps"], kappa=m["kappa"], p=1e-3, c=m["c"])
    _cache["solve"] = (mesh, valid, torch.tensor(po, device="cuda"), mat)
    return _cache["solve"]


def test_load_step_fullsize_properties():
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64, Problem, newton_step
    mesh, valid, po, mat = solve_setup()
    ns = mesh.info["n_slots"]
    res = {}
    for prec in (PFF_F32, PFF_F64):
        pb = Problem(mesh, **mat)
        mg = MG(pb, prec)
        u = torch.zeros((2, ns), dtype=torch.float64, device="cuda")
        phi = po.clone()
        act = torch.zeros(ns, dtype=torch.uint8, device="cuda")
        info = newton_step(pb, mg, u, phi, po, act)
        assert info["converged"] and info["newton"] <= 12 and info["linesearch_failures"] == 0, info
        res[prec] = (u.cpu().numpy()[:, valid], phi.cpu().numpy()[valid], act.cpu().numpy()[valid].astype(bool),
                     pb.tcv(u, phi))
    u32, p32, a32, t32 = res[PFF_F32]
    u64, p64, a64, t64 = res[PFF_F64]
    pov = po.cpu().numpy()[valid]
    # irreversibility and the active constraint
    assert np.all(p32 <= pov + 1e-12)
    assert np.all(p32[a32] == pov[a32])
    assert np.array_equal(a32, a64)
    assert np.linalg.norm(u32 - u64) / np.linalg.norm(u64) < 1e-7
    assert np.linalg.norm(p32 - p64) / np.linalg.norm(p64) < 1e-7
    # TCV against 2 pi p l0^2 / E' (Sec. 4): Table 2 lists errors of 0.5-2.9 % at comparable h
    eprime = mat["E"] / (1.0 - mat["nu"] ** 2)
    tref = 2.0 * np.pi * mat["p"] / eprime
    assert abs(t32 - tref) / tref < 0.03, (t32, tref)


@pytest.mark.parametrize("frac", [0.0, 0.05])
def test_vcycle_fullsize_symmetry(frac):
    """<a, MG b> = <MG a, b> for the FP64 V-cycle of both blocks (symmetric level
    operators, same polynomial before and after the coarse correction)."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F64, Problem
    mesh, valid, po, mat = solve_setup()
    ns = mesh.info["n_slots"]
    X, Y, F = mesh.slots()
    Xv, Yv = X[valid], Y[valid]
    info = mesh.info
    u, phi, phit = synth.linearisation(Xv, Yv, info["x_max"], info["y_max"], seed=4, u_std=1e-3)

    def slots(a):
        o = np.zeros((ns,) + a.shape[1:])
        o[valid] = a
        return o

    pb = Problem(mesh, **mat)
    dv = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    pb.set_state(dv(slots(u).T), dv(slots(phi)), dv(slots(phit)))
    rng = np.random.Generator(np.random.PCG64(9))
    act = slots((rng.uniform(size=len(Xv)) < frac).astype(np.float64)).astype(np.uint8)
    pb.set_active(dv(act))
    mg = MG(pb, PFF_F64)
    mg.setup()
    for b, nc in ((0, 2), (1, 1)):
        shape = (2, ns) if nc == 2 else (ns,)
        a = dv(rng.normal(size=shape))
        c = dv(rng.normal(size=shape))
        za, zc = torch.empty_like(a), torch.empty_like(c)
        mg.vcycle(b, a, za)
        mg.vcycle(b, c, zc)
        torch.cuda.synchronize()
        # holes and hanging entries are 0 in both outputs; compare on all slots
        l = float((c * za).sum())
        r = float((a * zc).sum())
        assert abs(l - r) <= 1e-10 * max(abs(l), abs(r)), (b, l, r)


def test_vcycle_fullsize_schedules_bitwise():
    """On the 1,043,811-DoF crack mesh (13 levels, from a few bricks to over a
    thousand per level) the FP32 V-cycle of both blocks is bitwise the same under
    every strip schedule of the level block operators, with a 5% active set."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem
    mesh, valid, po, mat = solve_setup()
    ns = mesh.info["n_slots"]
    X, Y, F = mesh.slots()
    Xv, Yv = X[valid], Y[valid]
    info = mesh.info
    u, phi, phit = synth.linearisation(Xv, Yv, info["x_max"], info["y_max"], seed=4, u_std=1e-3)

    def slots(a):
        o = np.zeros((ns,) + a.shape[1:])
        o[valid] = a
        return o

    dv = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    rng = np.random.Generator(np.random.PCG64(9))
    act = slots((rng.uniform(size=len(Xv)) < 0.05).astype(np.float64)).astype(np.uint8)
    r = {0: dv(rng.normal(size=(2, ns))), 1: dv(rng.normal(size=ns))}
    ref = {}
    for sched in (0, 15, 5, 1):
        pb = Problem(mesh, **mat)
        pb.set_cell_loop(sched)
        pb.set_state(dv(slots(u).T), dv(slots(phi)), dv(slots(phit)))
        pb.set_active(dv(act))
        mg = MG(pb, PFF_F32)
        mg.setup()
        for b in (0, 1):
            z = torch.full_like(r[b], float("nan"))
            mg.vcycle(b, r[b], z)
            torch.cuda.synchronize()
            zb = z.cpu().numpy()
            assert np.all(np.isfinite(zb))
            if b not in ref:
                ref[b] = zb
            assert np.array_equal(zb, ref[b]), (sched, b)
