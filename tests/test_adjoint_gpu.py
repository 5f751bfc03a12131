"""Parity of the differentiation path (through the C-ABI) with the oracle.

* per-cell modulus E_K in the leaf Jacobian apply (1e-12 FP64, 1e-5 FP32), the
  residual (1e-12) and the level operators of the V-cycle (lambda_max 1e-9,
  V-cycle 1e-10 FP64, 1e-5 FP32);
* TCV gradient M_f C^T dJ/dU and the parameter VJP (1e-12);
* adjoint gradient of a converged load step (Sneddon, lognormal E_K) against the
  oracle's adjoint at the oracle's own converged state (1e-6: both load steps are
  solved to a relative residual of 1e-12, and the two converged states agree to
  about 1e-7, the parity bar of a converged solution), and against central
  differences of GPU load steps at relative step 1e-6 (1e-5), on the 4,293-DoF
  mesh and the 65,001-DoF mesh of the same box-refined recipe;
* the torch autograd wrapper returns the same gradients.

At p = 1e-3, |G_c dJ/dG_c| is about 1e-7 J, below what a difference of J at
relative step 1e-6 resolves; G_c is checked against differences at p = 0.2 and
against the oracle adjoint at both pressures.
"""
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
        _pairs[name] = Pair(name, 1)
    return _pairs[name]


def dev(a, dtype=None):
    import torch
    t = torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t if dtype is None else t.to(dtype)


def cell_E(P, seed=1):
    c = P.om.cells
    assert np.array_equal(P.lm.leaf_cells(), c), "leaf-cell orders differ"
    return synth.cell_modulus(c[:, 0], c[:, 1], c[:, 2], seed=seed)


def lib_problem(P, mat, u, phi, phit, active, E):
    from paper_2404_03265_gb300 import Problem
    pb = Problem(P.lm, **mat)
    pb.set_state(dev(P.to_slots(u).T), dev(P.to_slots(phi)), dev(P.to_slots(phit)))
    pb.set_active(dev(P.to_slots(active.astype(np.uint8))))
    pb.set_cell_modulus(dev(E))
    return pb


@pytest.mark.parametrize("name", ["tiny", "small", "band4_2_4"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("op", ["jacobian", "transpose"])
def test_apply_with_cell_modulus(name, prec, tol, op):
    import torch
    from paper_2404_03265_gb300 import PFF_OP_JACOBIAN, PFF_OP_TRANSPOSE
    P = pair(name)
    mat = P.material(kappa=1e-2, p=0.4, Gc=2.0)
    u, phi, phit = random_linearisation(P, seed=0, u_std=0.3)
    active = random_active(P, seed=5, frac=0.05)
    E = cell_E(P)
    x = synth.vector(P.om.X, P.om.Y, seed=1)
    ref = oracle_apply(P, mat, u, phi, phit, active, x, op=op, E_cells=E)
    # the field matters: the uniform-modulus operator differs by far more than tol
    ref1 = oracle_apply(P, mat, u, phi, phit, active, x, op=op)
    assert rel_err(ref1, ref)[1] > 1e-3
    pb = lib_problem(P, mat, u, phi, phit, active, E)
    dt = torch.float64 if prec == "f64" else torch.float32
    xs = P.to_slots(x)
    xu, xp = dev(xs[:, :2].T, dt), dev(xs[:, 2], dt)
    yu, yp = torch.full_like(xu, float("nan")), torch.full_like(xp, float("nan"))
    pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN if op == "jacobian" else PFF_OP_TRANSPOSE)
    torch.cuda.synchronize()
    y = P.from_slots(np.concatenate([yu.cpu().double().numpy().T, yp.cpu().double().numpy()[:, None]], 1))
    inf, two = rel_err(y, ref)
    assert inf < tol and two < tol, (inf, two)
    # back to the uniform modulus
    pb.set_cell_modulus(None)
    pb.apply(xu, xp, yu, yp, op=PFF_OP_JACOBIAN if op == "jacobian" else PFF_OP_TRANSPOSE)
    torch.cuda.synchronize()
    y1 = P.from_slots(np.concatenate([yu.cpu().double().numpy().T, yp.cpu().double().numpy()[:, None]], 1))
    inf, two = rel_err(y1, ref1)
    assert inf < tol and two < tol, (inf, two)


@pytest.mark.parametrize("name", ["small", "band4_2_4"])
def test_residual_with_cell_modulus(name):
    import torch
    P = pair(name)
    om = P.om
    mat = P.material(kappa=1e-3, p=0.2)
    u, phi, phit = random_linearisation(P, seed=2, u_std=0.05)
    E = cell_E(P)
    pb = lib_problem(P, mat, u, phi, phit, np.zeros(om.nn, bool), E)
    R = torch.full((3, P.n_slots), float("nan"), dtype=torch.float64, device="cuda")
    pb.residual(dev(P.to_slots(u).T), dev(P.to_slots(phi)), dev(P.to_slots(phit)), R)
    torch.cuda.synchronize()
    Rref = ops.condense(om, -ops.residual_form(om, ops.Material(**mat), ops.State(om, u, phi, phit, E)))
    nn = om.nn
    Rref = np.stack([Rref[:nn], Rref[nn:2 * nn], Rref[2 * nn:]], 1)
    Rref[om.dirichlet, :2] = 0.0
    inf, two = rel_err(P.from_slots(R.cpu().numpy().T), Rref)
    assert inf < 1e-12 and two < 1e-12, (inf, two)


@pytest.mark.parametrize("name", ["small", "band4_2_4"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_vcycle_with_cell_modulus(name, prec, tol):
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, PFF_F64
    P = pair(name)
    om = P.om
    nn = om.nn
    mat = P.material(kappa=1e-3, p=0.05)
    u, phi, phit = random_linearisation(P, seed=0, u_std=1e-2)
    active = np.zeros(nn, bool)
    E = cell_E(P)
    M = omg.MG(om, ops.Material(**mat), u, phi, phit, active, E_cells=E)
    pb = lib_problem(P, mat, u, phi, phit, active, E)
    mg = MG(pb, PFF_F64 if prec == "f64" else PFF_F32)
    mg.setup()
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


@pytest.mark.parametrize("name", ["tiny", "small", "band4_2_4"])
def test_tcv_gradient_and_param_vjp(name):
    import torch
    P = pair(name)
    om = P.om
    nn = om.nn
    mat = P.material(kappa=1e-3, p=0.2, Gc=1.3)
    u, phi, phit = random_linearisation(P, seed=2, u_std=0.3)
    active = random_active(P, seed=5, frac=0.05)
    E = cell_E(P)
    pb = lib_problem(P, mat, u, phi, phit, active, E)
    st = ops.State(om, u, phi, phit, E)
    # TCV gradient: M_f C^T dJ/dU
    g = torch.full((3, P.n_slots), float("nan"), dtype=torch.float64, device="cuda")
    pb.tcv_gradient(dev(P.to_slots(u).T), dev(P.to_slots(phi)), g)
    torch.cuda.synchronize()
    gref = ops.condense(om, adj.tcv_gradient(om, ops.State(om, u, phi, phi)))
    gref[ops.fixed_dofs(om, active)] = 0.0
    gref = np.stack([gref[:nn], gref[nn:2 * nn], gref[2 * nn:]], 1)
    gs = g.cpu().numpy().T
    assert np.all(gs[~P.valid] == 0.0)
    inf, two = rel_err(P.from_slots(gs), gref)
    assert inf < 1e-12 and two < 1e-12, (inf, two)
    # VJP: (C M_f w) . dR/dtheta
    w = synth.vector(om.X, om.Y, seed=7)
    wv = np.concatenate([w[:, 0], w[:, 1], w[:, 2]])
    wv[ops.fixed_dofs(om, active)] = 0.0
    rp, rg, re = adj.param_vjp(om, ops.Material(**mat), st, wv)
    ws = P.to_slots(w)
    hang = P.slots[(P.slot_F[P.slots] & 4) != 0]
    ws[hang] = 5.0            # hanging entries of w are ignored
    gE = torch.full((len(E),), float("nan"), dtype=torch.float64, device="cuda")
    gp, ggc = pb.param_vjp(dev(ws.T), gE)
    assert abs(gp - rp) <= 1e-12 * abs(rp), (gp, rp)
    assert abs(ggc - rg) <= 1e-12 * abs(rg), (ggc, rg)
    inf, two = rel_err(gE.cpu().numpy(), re)
    assert inf < 1e-12 and two < 1e-12, (inf, two)


def gpu_load_step(P, pb, mg, phi_old, tol=1e-12):
    """One Sneddon load step from U = (0, phi_old) on the GPU; returns device tensors."""
    import torch
    from paper_2404_03265_gb300 import newton_step
    us = torch.zeros((2, P.n_slots), dtype=torch.float64, device="cuda")
    ps = dev(P.to_slots(phi_old))
    pos = ps.clone()
    act = torch.zeros(P.n_slots, dtype=torch.uint8, device="cuda")
    info = newton_step(pb, mg, us, ps, pos, act, tol=tol, atol=1e-15)
    assert info["converged"], info
    return us, ps, pos, act


def oracle_adjoint(P, mat, E):
    om = P.om
    u0, po = solvers.sneddon_initial(om, om.h_min_diag())
    uo, pho, ao, io = solvers.load_step(om, ops.Material(**mat), 1e4, u0, po.copy(), po, E_cells=E, tol=1e-12,
                                        atol=1e-15)
    assert io.converged
    st = ops.State(om, uo, pho, po, E)
    go = adj.tcv_adjoint(om, ops.Material(**mat), st, ao)
    go["u"], go["phi"] = st.u, st.phi
    return go, ao, ops.tcv(om, st), po


def close(a, b, rel, floor):
    return abs(a - b) <= rel * abs(b) + floor


@pytest.mark.parametrize("name,p", [("small", 1e-3), ("small", 0.2), ("band4_3_3", 1e-3)])
def test_tcv_adjoint_vs_oracle(name, p):
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem, tcv_adjoint
    P = pair(name)
    mat = P.material(p=p)
    E = cell_E(P)
    go, ao, J, po = oracle_adjoint(P, mat, E)
    pb = Problem(P.lm, **mat)
    pb.set_cell_modulus(dev(E))
    mg = MG(pb, PFF_F32)
    us, ps, pos, act = gpu_load_step(P, pb, mg, po)
    assert np.array_equal(P.from_slots(act.cpu().numpy()).astype(bool), ao)
    eu = np.linalg.norm(P.from_slots(us.cpu().numpy().T) - go["u"]) / np.linalg.norm(go["u"])
    ep = np.linalg.norm(P.from_slots(ps.cpu().numpy()) - go["phi"]) / np.linalg.norm(go["phi"])
    assert eu < 1e-7 and ep < 1e-7, (eu, ep)
    gE = torch.full((len(E),), float("nan"), dtype=torch.float64, device="cuda")
    r = tcv_adjoint(pb, mg, us, ps, pos, act, gE=gE, rtol=1e-12)
    assert r["converged"]
    assert close(r["p"], go["p"], 1e-6, 0.0), (r["p"], go["p"])
    # G_c: relative 1e-6, with a floor of 1e-10 J / G_c for the tiny derivative at small p
    assert close(r["Gc"], go["Gc"], 1e-6, 1e-10 * J / mat["Gc"]), (r["Gc"], go["Gc"])
    inf, two = rel_err(gE.cpu().numpy(), go["E"])
    assert inf < 1e-6 and two < 1e-6, (inf, two)


def test_tcv_adjoint_vs_central_difference_gpu():
    """GPU adjoint against central differences of GPU load steps, p = 0.2 (relative
    step 1e-6, bound 1e-5), for p, G_c and the two cells of largest |dJ/dE_K|."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem, tcv_adjoint
    P = pair("small")
    mat = P.material(p=0.2)
    E = cell_E(P)
    om = P.om
    _, po = solvers.sneddon_initial(om, om.h_min_diag())
    pb = Problem(P.lm, **mat)
    pb.set_cell_modulus(dev(E))
    mg = MG(pb, PFF_F32)
    us, ps, pos, act = gpu_load_step(P, pb, mg, po)
    act0 = act.clone()
    gE = torch.empty(len(E), dtype=torch.float64, device="cuda")
    r = tcv_adjoint(pb, mg, us, ps, pos, act, gE=gE, rtol=1e-12)
    gE = gE.cpu().numpy()

    def J(kw, Ec):
        pb.set_params(**kw)
        pb.set_cell_modulus(dev(Ec))
        u2, p2, _, a2 = gpu_load_step(P, pb, mg, po)
        assert torch.equal(a2, act0), "active set changed under the perturbation"
        return pb.tcv(u2, p2)

    rel = 1e-6
    for key in ("p", "Gc"):
        hh = rel * mat[key]
        fd = (J({key: mat[key] + hh}, E) - J({key: mat[key] - hh}, E)) / (2 * hh)
        pb.set_params(**{key: mat[key]})
        assert abs(fd - r[key]) <= 1e-5 * abs(fd), (key, fd, r[key])
    for c in np.argsort(-np.abs(gE))[:2]:
        hh = rel * E[c]
        Ep, Em = E.copy(), E.copy()
        Ep[c] += hh
        Em[c] -= hh
        fd = (J({}, Ep) - J({}, Em)) / (2 * hh)
        assert abs(fd - gE[c]) <= 1e-5 * abs(fd), (c, fd, gE[c])


def test_autograd_load_step_65k():
    """The 65,001-DoF box-refined crack mesh with lognormal E_K (sigma_log 0.1, seed 1),
    p = 1e-3: J.backward() through the torch wrapper against the oracle adjoint and
    central differences (relative step 1e-6) of GPU load steps for p and two E_K."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem
    from paper_2404_03265_gb300.autograd import tcv_load_step
    P = pair("adjoint")
    mat = P.material(p=1e-3)
    E = cell_E(P)
    go, ao, Jo, po = oracle_adjoint(P, mat, E)
    pb = Problem(P.lm, **mat)
    mg = MG(pb, PFF_F32)
    pt = torch.tensor(mat["p"], dtype=torch.float64, requires_grad=True)
    gct = torch.tensor(mat["Gc"], dtype=torch.float64, requires_grad=True)
    Et = dev(E).requires_grad_(True)
    us = torch.zeros((2, P.n_slots), dtype=torch.float64, device="cuda")
    ps = dev(P.to_slots(po))
    pos = ps.clone()
    act = torch.zeros(P.n_slots, dtype=torch.uint8, device="cuda")
    J = tcv_load_step(pb, mg, pt, gct, Et, us, ps, pos, act, newton_kw=dict(tol=1e-12, atol=1e-15),
                      adjoint_kw=dict(rtol=1e-12))
    assert abs(J.item() - Jo) <= 1e-9 * abs(Jo), (J.item(), Jo)
    J.backward()
    assert close(pt.grad.item(), go["p"], 1e-6, 0.0), (pt.grad.item(), go["p"])
    assert close(gct.grad.item(), go["Gc"], 1e-6, 1e-10 * Jo / mat["Gc"]), (gct.grad.item(), go["Gc"])
    gE = Et.grad.cpu().numpy()
    inf, two = rel_err(gE, go["E"])
    assert inf < 1e-6 and two < 1e-6, (inf, two)
    act0 = act.clone()

    def Jfd(kw, Ec):
        pb.set_params(**kw)
        pb.set_cell_modulus(dev(Ec))
        u2, p2, _, a2 = gpu_load_step(P, pb, mg, po)
        assert torch.equal(a2, act0), "active set changed under the perturbation"
        return pb.tcv(u2, p2)

    hh = 1e-6 * mat["p"]
    fd = (Jfd({"p": mat["p"] + hh}, E) - Jfd({"p": mat["p"] - hh}, E)) / (2 * hh)
    pb.set_params(p=mat["p"])
    assert abs(fd - pt.grad.item()) <= 1e-5 * abs(fd), (fd, pt.grad.item())
    for c in np.argsort(-np.abs(gE))[:2]:
        hh = 1e-6 * E[c]
        Ep, Em = E.copy(), E.copy()
        Ep[c] += hh
        Em[c] -= hh
        fd = (Jfd({}, Ep) - Jfd({}, Em)) / (2 * hh)
        assert abs(fd - gE[c]) <= 1e-5 * abs(fd), (c, fd, gE[c])


def gpu_steps(P, pb, mg, po, ps, tol=1e-12):
    """Load steps at pressures ps from the initial crack on the GPU; checkpoints per step."""
    import torch
    from paper_2404_03265_gb300 import newton_step
    us = [torch.zeros((2, P.n_slots), dtype=torch.float64, device="cuda")]
    phis = [dev(P.to_slots(po))]
    acts = []
    act = torch.zeros(P.n_slots, dtype=torch.uint8, device="cuda")
    for p in ps:
        pb.set_pressure(p)
        u = us[-1].clone()
        phi = phis[-1].clone()
        info = newton_step(pb, mg, u, phi, phis[-1], act, tol=tol, atol=1e-15)
        assert info["converged"], info
        us.append(u)
        phis.append(phi)
        acts.append(act.clone())
    return us, phis, acts


def test_multi_step_adjoint_vs_oracle_and_differences():
    """Three load steps (p = 0.1, 0.15, 0.2) on the 4,293-DoF mesh with lognormal E_K:
    the checkpointed GPU adjoint against the oracle's (1e-6; states agree to about
    1e-7) and against central differences of three-step GPU solves (1e-5)."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem, tcv_adjoint_steps
    P = pair("small")
    om = P.om
    E = cell_E(P)
    ps = [0.1, 0.15, 0.2]
    base = P.material()
    # oracle
    _, po = solvers.sneddon_initial(om, om.h_min_diag())
    mats, ous, ophis, oacts = [], [np.zeros((om.nn, 2))], [po], []
    u, phi, act = ous[0], po.copy(), None
    for p in ps:
        mat = ops.Material(**dict(base, p=p))
        u, phi_n, act, info = solvers.load_step(om, mat, 1e4, u, phi.copy(), phi, active_prev=act, E_cells=E,
                                                tol=1e-12, atol=1e-15)
        assert info.converged
        phi = phi_n
        mats.append(mat)
        ous.append(u)
        ophis.append(phi)
        oacts.append(act)
    go = adj.tcv_adjoint_steps(om, mats, ous, ophis, oacts, E)
    # GPU
    pb = Problem(P.lm, **base)
    pb.set_cell_modulus(dev(E))
    mg = MG(pb, PFF_F32)
    us, phis, acts = gpu_steps(P, pb, mg, po, ps)
    for a_g, a_o in zip(acts, oacts):
        assert np.array_equal(P.from_slots(a_g.cpu().numpy()).astype(bool), a_o)
    gE = torch.full((len(E),), float("nan"), dtype=torch.float64, device="cuda")
    r = tcv_adjoint_steps(pb, mg, us, phis, acts, ps, gE=gE, rtol=1e-12)
    assert r["converged"]
    J = ops.tcv(om, ops.State(om, ous[-1], ophis[-1], ophis[-1]))
    for n in range(len(ps)):
        assert close(r["p"][n], go["p"][n], 1e-6, 0.0), (n, r["p"][n], go["p"][n])
    assert close(r["Gc"], go["Gc"], 1e-6, 1e-10 * J / base["Gc"]), (r["Gc"], go["Gc"])
    inf, two = rel_err(gE.cpu().numpy(), go["E"])
    assert inf < 1e-6 and two < 1e-6, (inf, two)

    # central differences of three-step GPU solves
    def Jfd(kw, pss, Ec):
        pb.set_params(**kw)
        pb.set_cell_modulus(dev(Ec))
        u2, p2, a2 = gpu_steps(P, pb, mg, po, pss)
        for x0, x1 in zip(a2, acts):
            assert torch.equal(x0, x1), "active set changed under the perturbation"
        return pb.tcv(u2[-1], p2[-1])

    rel = 1e-6
    hh = rel * ps[0]
    fd = (Jfd({}, [ps[0] + hh] + ps[1:], E) - Jfd({}, [ps[0] - hh] + ps[1:], E)) / (2 * hh)
    assert abs(fd - r["p"][0]) <= 1e-5 * abs(fd), (fd, r["p"][0])
    hh = rel * base["Gc"]
    fd = (Jfd({"Gc": base["Gc"] + hh}, ps, E) - Jfd({"Gc": base["Gc"] - hh}, ps, E)) / (2 * hh)
    pb.set_params(Gc=base["Gc"])
    assert abs(fd - r["Gc"]) <= 1e-5 * abs(fd), (fd, r["Gc"])
    gEn = gE.cpu().numpy()
    c = int(np.argmax(np.abs(gEn)))
    hh = rel * E[c]
    Ep, Em = E.copy(), E.copy()
    Ep[c] += hh
    Em[c] -= hh
    fd = (Jfd({}, ps, Ep) - Jfd({}, ps, Em)) / (2 * hh)
    assert abs(fd - gEn[c]) <= 1e-5 * abs(fd), (c, fd, gEn[c])


def test_autograd_load_steps_three():
    """J = TCV after three load steps (p = 0.1, 0.15, 0.2, lognormal E_K) through the
    several-step torch wrapper: J.backward() against the oracle's checkpointed
    adjoint (1e-6) and central differences of three-step GPU solves (1e-5) for the
    first pressure, G_c and the largest E_K gradient."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem
    from paper_2404_03265_gb300.autograd import tcv_load_steps
    P = pair("small")
    om = P.om
    E = cell_E(P)
    ps = [0.1, 0.15, 0.2]
    base = P.material()
    _, po = solvers.sneddon_initial(om, om.h_min_diag())
    mats, ous, ophis, oacts = [], [np.zeros((om.nn, 2))], [po], []
    u, phi, act = ous[0], po.copy(), None
    for p in ps:
        mat = ops.Material(**dict(base, p=p))
        u, phi_n, act, info = solvers.load_step(om, mat, 1e4, u, phi.copy(), phi, active_prev=act, E_cells=E,
                                                tol=1e-12, atol=1e-15)
        assert info.converged
        phi = phi_n
        mats.append(mat)
        ous.append(u)
        ophis.append(phi)
        oacts.append(act)
    go = adj.tcv_adjoint_steps(om, mats, ous, ophis, oacts, E)
    Jo = ops.tcv(om, ops.State(om, ous[-1], ophis[-1], ophis[-1]))

    pb = Problem(P.lm, **base)
    mg = MG(pb, PFF_F32)
    pt = torch.tensor(ps, dtype=torch.float64, requires_grad=True)
    gct = torch.tensor(base["Gc"], dtype=torch.float64, requires_grad=True)
    Et = dev(E).requires_grad_(True)
    u0 = torch.zeros((2, P.n_slots), dtype=torch.float64, device="cuda")
    phi0 = dev(P.to_slots(po))
    out = {}
    J = tcv_load_steps(pb, mg, pt, gct, Et, u0, phi0, newton_kw=dict(tol=1e-12, atol=1e-15),
                       adjoint_kw=dict(rtol=1e-12), out=out)
    assert abs(J.item() - Jo) <= 1e-7 * abs(Jo), (J.item(), Jo)
    for a_g, a_o in zip(out["active"], oacts):
        assert np.array_equal(P.from_slots(a_g.cpu().numpy()).astype(bool), a_o)
    J.backward()
    gp = pt.grad.numpy()
    for n in range(len(ps)):
        assert close(gp[n], go["p"][n], 1e-6, 0.0), (n, gp[n], go["p"][n])
    assert close(gct.grad.item(), go["Gc"], 1e-6, 1e-10 * Jo / base["Gc"]), (gct.grad.item(), go["Gc"])
    gE = Et.grad.cpu().numpy()
    inf, two = rel_err(gE, go["E"])
    assert inf < 1e-6 and two < 1e-6, (inf, two)

    # central differences of three-step GPU solves, through the same wrapper's forward
    def Jfd(pss, gc, Ec):
        with torch.no_grad():
            return tcv_load_steps(pb, mg, torch.tensor(pss, dtype=torch.float64),
                                  torch.tensor(gc, dtype=torch.float64), dev(Ec), u0,
                                  phi0, newton_kw=dict(tol=1e-12, atol=1e-15)).item()

    rel = 1e-6
    hh = rel * ps[0]
    fd = (Jfd([ps[0] + hh] + ps[1:], base["Gc"], E) - Jfd([ps[0] - hh] + ps[1:], base["Gc"], E)) / (2 * hh)
    assert abs(fd - gp[0]) <= 1e-5 * abs(fd), (fd, gp[0])
    hh = rel * base["Gc"]
    fd = (Jfd(ps, base["Gc"] + hh, E) - Jfd(ps, base["Gc"] - hh, E)) / (2 * hh)
    assert abs(fd - gct.grad.item()) <= 1e-5 * abs(fd), (fd, gct.grad.item())
    c = int(np.argmax(np.abs(gE)))
    hh = rel * E[c]
    Ep, Em = E.copy(), E.copy()
    Ep[c] += hh
    Em[c] -= hh
    fd = (Jfd(ps, base["Gc"], Ep) - Jfd(ps, base["Gc"], Em)) / (2 * hh)
    assert abs(fd - gE[c]) <= 1e-5 * abs(fd), (c, fd, gE[c])


def oracle_steps_extrapolated(om, base, E, po, ps):
    """Oracle load steps from (u = 0, phi^0 = po), phi_tilde of step n >= 2 extrapolated
    (clip(2 phi^(n-1) - phi^(n-2), 0, 1), Sec. 2); the clip masks of steps 2..N."""
    mats, us, phis, acts, chis = [], [np.zeros((om.nn, 2))], [po], [], []
    u, phi, act = us[0], po.copy(), None
    for n, p in enumerate(ps, start=1):
        mat = ops.Material(**dict(base, p=p))
        phit = None
        if n >= 2:
            phit = solvers.extrapolate_phi(phis[-1], phis[-2])
            raw = 2.0 * phis[-1] - phis[-2]
            chis.append((raw > 0.0) & (raw < 1.0))
        u, phi_n, act, info = solvers.load_step(om, mat, 1e4, u, phi.copy(), phi, active_prev=act, E_cells=E,
                                                tol=1e-12, atol=1e-15, phi_tilde=phit)
        assert info.converged
        phi = phi_n
        mats.append(mat)
        us.append(u)
        phis.append(phi)
        acts.append(act)
    return mats, us, phis, acts, chis


def test_load_steps_extrapolated_phi_tilde_gradient():
    """Three load steps (p = 0.1, 0.15, 0.2, lognormal E_K, 4,293 DoFs) whose phi_tilde
    of steps 2 and 3 is extrapolated from the two previous steps (Sec. 2), through the
    several-step torch wrapper: J and the GPU states' active sets and clip masks equal
    the oracle's; J.backward() (pff_tcv_adjoint_steps, PFF_PHIT_EXTRAPOLATED) against
    the oracle's extrapolated adjoint (1e-6) and central differences of three-step GPU
    solves (1e-5) for p_1, p_2, G_c and the largest E_K gradient; another
    phi_tilde_mode is refused."""
    import ctypes
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem, _lib, tcv_adjoint_steps
    from paper_2404_03265_gb300.autograd import tcv_load_steps
    P = pair("small")
    om = P.om
    E = cell_E(P)
    ps = [0.1, 0.15, 0.2]
    base = P.material()
    _, po = solvers.sneddon_initial(om, om.h_min_diag())
    mats, ous, ophis, oacts, ochis = oracle_steps_extrapolated(om, base, E, po, ps)
    go = adj.tcv_adjoint_steps(om, mats, ous, ophis, oacts, E, extrapolate=True)
    Jo = ops.tcv(om, ops.State(om, ous[-1], ophis[-1], ophis[-1]))

    pb = Problem(P.lm, **base)
    mg = MG(pb, PFF_F32)
    pt = torch.tensor(ps, dtype=torch.float64, requires_grad=True)
    gct = torch.tensor(base["Gc"], dtype=torch.float64, requires_grad=True)
    Et = dev(E).requires_grad_(True)
    u0 = torch.zeros((2, P.n_slots), dtype=torch.float64, device="cuda")
    phi0 = dev(P.to_slots(po))
    out = {}
    kw = dict(newton_kw=dict(tol=1e-12, atol=1e-15), extrapolated=True)
    J = tcv_load_steps(pb, mg, pt, gct, Et, u0, phi0, adjoint_kw=dict(rtol=1e-12), out=out, **kw)
    assert abs(J.item() - Jo) <= 1e-7 * abs(Jo), (J.item(), Jo)
    for a_g, a_o in zip(out["active"], oacts):
        assert np.array_equal(P.from_slots(a_g.cpu().numpy()).astype(bool), a_o)
    gphis = [P.from_slots(t.cpu().numpy()) for t in out["phi"]]
    for n, c_o in enumerate(ochis, start=2):
        raw = 2.0 * gphis[n - 1] - gphis[n - 2]
        assert np.array_equal((raw > 0.0) & (raw < 1.0), c_o), n
    J.backward()
    gp = pt.grad.numpy()
    for n in range(len(ps)):
        assert close(gp[n], go["p"][n], 1e-6, 0.0), (n, gp[n], go["p"][n])
    assert close(gct.grad.item(), go["Gc"], 1e-6, 1e-10 * Jo / base["Gc"]), (gct.grad.item(), go["Gc"])
    gE = Et.grad.cpu().numpy()
    inf, two = rel_err(gE, go["E"])
    assert inf < 1e-6 and two < 1e-6, (inf, two)

    # the same checkpoints with phi_tilde = phi^(k-1) give another gradient
    pb.set_cell_modulus(dev(E))
    r_prev = tcv_adjoint_steps(pb, mg, out["u"], out["phi"], out["active"], ps, rtol=1e-12)
    assert np.max(np.abs(r_prev["p"] - gp)) > 1e-2 * np.max(np.abs(gp))

    # phi_tilde_mode other than PFF_PHIT_PREVIOUS / PFF_PHIT_EXTRAPOLATED
    VP = ctypes.c_void_p
    N = len(ps)
    ua = (VP * (N + 1))(*[_lib.ptr(t) for t in out["u"]])
    pa = (VP * (N + 1))(*[_lib.ptr(t) for t in out["phi"]])
    aa = (VP * N)(*[_lib.ptr(t) for t in out["active"]])
    p_host = np.asarray(ps, dtype=np.float64)
    gpo, ggc = np.zeros(N), np.zeros(1)
    st = _lib.lib().pff_tcv_adjoint_steps(pb._h, mg._h, N, ua, pa, aa, _lib.ptr(p_host), 2, 1e-12, 50, 2000, None,
                                          _lib.ptr(gpo), _lib.ptr(ggc), None, _lib.stream_ptr())
    assert st == 1 and b"phi_tilde_mode" in _lib.lib().pff_last_error()

    # central differences of three-step GPU solves, through the same wrapper's forward
    def Jfd(pss, gc, Ec):
        with torch.no_grad():
            o = {}
            v = tcv_load_steps(pb, mg, torch.tensor(pss, dtype=torch.float64), torch.tensor(gc, dtype=torch.float64),
                               dev(Ec), u0, phi0, out=o, **kw).item()
        for x0, x1 in zip(o["active"], out["active"]):
            assert torch.equal(x0, x1), "active set changed under the perturbation"
        for n in range(2, len(pss) + 1):
            c0 = (lambda r: (r > 0) & (r < 1))(2.0 * o["phi"][n - 1] - o["phi"][n - 2])
            c1 = (lambda r: (r > 0) & (r < 1))(2.0 * out["phi"][n - 1] - out["phi"][n - 2])
            assert torch.equal(c0, c1), "clip pattern changed under the perturbation"
        return v

    rel = 1e-6
    for n in (0, 1):
        hh = rel * ps[n]
        pp_, pm_ = list(ps), list(ps)
        pp_[n] += hh
        pm_[n] -= hh
        fd = (Jfd(pp_, base["Gc"], E) - Jfd(pm_, base["Gc"], E)) / (2 * hh)
        assert abs(fd - gp[n]) <= 1e-5 * abs(fd), (n, fd, gp[n])
    hh = rel * base["Gc"]
    fd = (Jfd(ps, base["Gc"] + hh, E) - Jfd(ps, base["Gc"] - hh, E)) / (2 * hh)
    assert abs(fd - gct.grad.item()) <= 1e-5 * abs(fd), (fd, gct.grad.item())
    c = int(np.argmax(np.abs(gE)))
    hh = rel * E[c]
    Ep, Em = E.copy(), E.copy()
    Ep[c] += hh
    Em[c] -= hh
    fd = (Jfd(ps, base["Gc"], Ep) - Jfd(ps, base["Gc"], Em)) / (2 * hh)
    assert abs(fd - gE[c]) <= 1e-5 * abs(fd), (c, fd, gE[c])
