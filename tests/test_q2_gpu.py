"""Parity of the Q2 (k = 2) operators through the C-ABI with the oracle: leaf
Jacobian, transpose and condensed apply (1e-12 FP64, 1e-5 FP32), residual,
lumped mass and TCV (1e-12), cell modulus, TCV gradient and parameter VJP
(1e-12), the block V-cycle (lambda_max 1e-9 FP64 and LAMBDA_RTOL FP32, V-cycle 1e-10 FP64, 1e-5 FP32) and
a Sneddon load step of Algorithm 2 (same active set, u and phi within 1e-7)."""
import numpy as np
import pytest

import synthetic as synth
from harness import LAMBDA_RTOL, Pair, oracle_apply, random_active, random_linearisation, rel_err
from oracle import adjoint as adj
from oracle import mg as omg
from oracle import operators as ops
from oracle import solvers

pytestmark = pytest.mark.gpu

_pairs = {}


def pair(name):
    if name not in _pairs:
        _pairs[name] = Pair(name, 2)
    return _pairs[name]


def dev(a, dtype=None):
    import torch
    t = torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t if dtype is None else t.to(dtype)


def lib_problem(P, mat, u, phi, phit, active, E=None):
    from paper_2404_03265_gb300 import Problem
    pb = Problem(P.lm, **mat)
    pb.set_state(dev(P.to_slots(u).T), dev(P.to_slots(phi)), dev(P.to_slots(phit)))
    pb.set_active(dev(P.to_slots(active.astype(np.uint8))))
    if E is not None:
        pb.set_cell_modulus(dev(E))
    return pb


def cell_E(P):
    c = P.om.cells
    assert np.array_equal(P.lm.leaf_cells(), c)
    return synth.cell_modulus(c[:, 0], c[:, 1], c[:, 2], seed=1)


@pytest.mark.parametrize("name", ["tiny", "small", "band4_2_4"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("op", ["jacobian", "transpose", "condensed"])
@pytest.mark.parametrize("modulus", [False, True])
def test_q2_apply(name, prec, tol, op, modulus):
    import torch
    from paper_2404_03265_gb300 import PFF_OP_CONDENSED, PFF_OP_JACOBIAN, PFF_OP_TRANSPOSE
    P = pair(name)
    mat = P.material(kappa=1e-2, p=0.4, Gc=2.0)
    u, phi, phit = random_linearisation(P, seed=0, u_std=0.3)
    active = random_active(P, seed=5, frac=0.05)
    E = cell_E(P) if modulus else None
    x = synth.vector(P.om.X, P.om.Y, seed=1)
    ref = oracle_apply(P, mat, u, phi, phit, active, x, op=op, E_cells=E)
    pb = lib_problem(P, mat, u, phi, phit, active, E)
    dt = torch.float64 if prec == "f64" else torch.float32
    xs = P.to_slots(x)
    xs[~P.valid] = 1e30                                   # holes ignored
    hang = P.slots[(P.slot_F[P.slots] & 4) != 0]
    xs[hang] = 7.0                                        # hanging entries ignored
    xu, xp = dev(xs[:, :2].T, dt), dev(xs[:, 2], dt)
    yu, yp = torch.full_like(xu, float("nan")), torch.full_like(xp, float("nan"))
    opc = {"jacobian": PFF_OP_JACOBIAN, "transpose": PFF_OP_TRANSPOSE, "condensed": PFF_OP_CONDENSED}[op]
    pb.apply(xu, xp, yu, yp, op=opc)
    torch.cuda.synchronize()
    ys = np.concatenate([yu.cpu().double().numpy().T, yp.cpu().double().numpy()[:, None]], 1)
    assert np.all(ys[~P.valid] == 0.0)
    y = P.from_slots(ys)
    assert np.all(y[P.om.is_hanging] == 0.0)
    inf, two = rel_err(y, ref)
    assert inf < tol and two < tol, (inf, two)


@pytest.mark.parametrize("name", ["tiny", "small", "band4_2_4"])
def test_q2_residual_mass_tcv_gradient_vjp(name):
    import torch
    P = pair(name)
    om = P.om
    nn = om.nn
    mat = P.material(kappa=1e-3, p=0.2, Gc=1.3)
    u, phi, phit = random_linearisation(P, seed=2, u_std=0.05)
    active = random_active(P, seed=5, frac=0.05)
    E = cell_E(P)
    pb = lib_problem(P, mat, u, phi, phit, active, E)
    st = ops.State(om, u, phi, phit, E)
    us, ps, pts = dev(P.to_slots(u).T), dev(P.to_slots(phi)), dev(P.to_slots(phit))
    R = torch.full((3, P.n_slots), float("nan"), dtype=torch.float64, device="cuda")
    pb.residual(us, ps, pts, R)
    B = torch.full((P.n_slots,), float("nan"), dtype=torch.float64, device="cuda")
    pb.lumped_mass(B)
    g = torch.full((3, P.n_slots), float("nan"), dtype=torch.float64, device="cuda")
    pb.tcv_gradient(us, ps, g)
    torch.cuda.synchronize()
    Rref = ops.condense(om, -ops.residual_form(om, ops.Material(**mat), st))
    Rref = np.stack([Rref[:nn], Rref[nn:2 * nn], Rref[2 * nn:]], 1)
    Rref[om.dirichlet, :2] = 0.0
    inf, two = rel_err(P.from_slots(R.cpu().numpy().T), Rref)
    assert inf < 1e-12 and two < 1e-12, ("residual", inf, two)
    Bref = ops.lumped_mass(om)
    assert np.abs(P.from_slots(B.cpu().numpy()) - Bref).max() < 1e-13 * Bref.max()
    tcv = pb.tcv(us, ps)
    tref = ops.tcv(om, ops.State(om, u, phi, phit))
    assert abs(tcv - tref) <= 1e-12 * abs(tref)
    gref = ops.condense(om, adj.tcv_gradient(om, ops.State(om, u, phi, phi)))
    gref[ops.fixed_dofs(om, active)] = 0.0
    gref = np.stack([gref[:nn], gref[nn:2 * nn], gref[2 * nn:]], 1)
    inf, two = rel_err(P.from_slots(g.cpu().numpy().T), gref)
    assert inf < 1e-12 and two < 1e-12, ("tcv gradient", inf, two)
    w = synth.vector(om.X, om.Y, seed=7)
    wv = np.concatenate([w[:, 0], w[:, 1], w[:, 2]])
    wv[ops.fixed_dofs(om, active)] = 0.0
    rp, rg, re = adj.param_vjp(om, ops.Material(**mat), st, wv)
    gE = torch.full((len(E),), float("nan"), dtype=torch.float64, device="cuda")
    gp, ggc = pb.param_vjp(dev(P.to_slots(w).T), gE)
    assert abs(gp - rp) <= 1e-12 * abs(rp) and abs(ggc - rg) <= 1e-12 * abs(rg), (gp, rp, ggc, rg)
    inf, two = rel_err(gE.cpu().numpy(), re)
    assert inf < 1e-12 and two < 1e-12, ("vjp", inf, two)


@pytest.mark.parametrize("name,frac", [("tiny", 0.0), ("small", 0.0), ("band4_2_4", 0.0)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
@pytest.mark.parametrize("fused", [True, False])
def test_q2_vcycle(name, frac, prec, tol, fused):
    """Q2 V-cycle against the oracle's, with the Chebyshev steps fused into the level
    applies' stores and as separate kernels."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64
    P = pair(name)
    om = P.om
    nn = om.nn
    mat = P.material(kappa=1e-3, p=0.05)
    u, phi, phit = random_linearisation(P, seed=0, u_std=1e-2)
    active = np.zeros(nn, bool)
    M = omg.MG(om, ops.Material(**mat), u, phi, phit, active)
    pb = lib_problem(P, mat, u, phi, phit, active)
    mg = MG(pb, PFF_F64 if prec == "f64" else PFF_F32)
    mg.setup()
    mg.set_fused_smoother(fused)
    rng = np.random.default_rng(3)
    for b, blk, nc in ((0, "uu", 2), (1, "pp", 1)):
        lam = mg.lam(b)
        ref = np.array([0.0] + [M.B[blk][l].lam for l in range(1, len(M.B[blk]))])
        assert np.allclose(lam[1:], ref[1:], rtol=LAMBDA_RTOL[prec], atol=1e-300), (blk, lam, ref)
        r = rng.normal(size=(nn, nc))
        zref = M.vcycle(blk, np.concatenate([r[:, c] for c in range(nc)]))
        zref = np.stack([zref[c * nn:(c + 1) * nn] for c in range(nc)], 1)
        rs = P.to_slots(r)
        rt = dev(rs.T if nc == 2 else rs[:, 0])
        zt = torch.full_like(rt, float("nan"))
        mg.vcycle(b, rt, zt)
        torch.cuda.synchronize()
        zs = zt.cpu().numpy()
        z = P.from_slots(zs.T if nc == 2 else zs[:, None])
        inf, two = rel_err(z, zref)
        assert inf < tol and two < tol, (blk, prec, inf, two)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_q2_load_step(prec):
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64, Problem, newton_step
    P = pair("small")
    om = P.om
    mat = P.material()
    u0, po = solvers.sneddon_initial(om, om.h_min_diag())
    uo, pho, ao, io = solvers.load_step(om, ops.Material(**mat), 1e4, u0, po.copy(), po)
    assert io.converged
    pb = Problem(P.lm, **mat)
    mg = MG(pb, PFF_F64 if prec == "f64" else PFF_F32)
    us = torch.zeros((2, P.n_slots), dtype=torch.float64, device="cuda")
    ps = dev(P.to_slots(po))
    pos = ps.clone()
    act = torch.zeros(P.n_slots, dtype=torch.uint8, device="cuda")
    info = newton_step(pb, mg, us, ps, pos, act)
    assert info["converged"], info
    assert np.array_equal(P.from_slots(act.cpu().numpy()).astype(bool), ao)
    ug = P.from_slots(us.cpu().numpy().T)
    pg = P.from_slots(ps.cpu().numpy())
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) < 1e-7
    assert np.linalg.norm(pg - pho) / np.linalg.norm(pho) < 1e-7
