"""Pins of the oracle's adjoint TCV gradient (oracle/adjoint.py).

* dJ/dU against central differences of the TCV functional: J = integral of
  u . grad phi is bilinear in (u, phi), so a central difference is exact up to
  rounding (the quadratic term cancels).
* dA/dp, dA/dG_c, dA/dE_K against central differences of the residual form:
  A is linear in each of them (Problem 2), so again exact up to rounding.
* The adjoint gradient against central differences of converged load steps
  (Algorithm 2) with relative step 1e-6, the active set checked unchanged.
"""
import numpy as np
import pytest

import synthetic as synth
from oracle import adjoint as adj
from oracle import operators as ops
from oracle import solvers
from oracle.mesh import LeafMesh, build_recipe

_meshes = {}


def mesh(name, k=1):
    if (name, k) not in _meshes:
        _meshes[(name, k)] = LeafMesh(build_recipe(synth.recipe(name)), k)
    return _meshes[(name, k)]


def cell_E(om, seed=1):
    return synth.cell_modulus(om.cells[:, 0], om.cells[:, 1], om.cells[:, 2], seed=seed)


def random_state(om, seed=0, E=None):
    u, phi, phit = synth.linearisation(om.X, om.Y, om.Xmax, om.Ymax, seed=seed, u_std=0.3)
    return u, phi, phit


@pytest.mark.parametrize("name,k", [("tiny", 1), ("small", 1), ("tiny", 2)])
def test_tcv_gradient_central_difference(name, k):
    om = mesh(name, k)
    u, phi, phit = random_state(om)
    st = ops.State(om, u, phi, phit)
    g = ops.condense(om, adj.tcv_gradient(om, st))
    rng = np.random.Generator(np.random.PCG64(4))
    v = rng.normal(size=3 * om.nn)
    nn = om.nn
    eps = 1e-3

    def J(s):
        U = np.concatenate([u[:, 0], u[:, 1], phi]) + s * v
        return ops.tcv(om, ops.State(om, np.stack([U[:nn], U[nn:2 * nn]], 1), U[2 * nn:], phit))

    fd = (J(eps) - J(-eps)) / (2 * eps)
    assert abs(fd - g @ v) <= 1e-10 * max(abs(fd), np.abs(g).sum() * 1e-3)
    # hanging rows of the condensed gradient are zero
    assert np.all(g[np.tile(om.is_hanging, 3)] == 0.0)


@pytest.mark.parametrize("name,k", [("tiny", 1), ("small", 1), ("tiny", 2)])
def test_param_derivatives_central_difference(name, k):
    om = mesh(name, k)
    u, phi, phit = random_state(om, seed=2)
    E = cell_E(om)
    h = om.h_min_diag()
    base = dict(E=1.0, nu=0.2, Gc=1.3, eps=2.0 * h, kappa=1e-3, p=0.2)
    mat = ops.Material(**base)
    st = ops.State(om, u, phi, phit, E)
    d_p, d_gc, d_e = adj.residual_param_derivatives(om, mat, st)
    scale = np.abs(ops.residual_form(om, mat, st)).max()

    def A(**kw):
        m = dict(base)
        m.update(kw)
        return ops.residual_form(om, ops.Material(**m), st)

    for name_, dv, val in (("p", d_p, base["p"]), ("Gc", d_gc, base["Gc"])):
        hh = 1e-3 * val
        fd = (A(**{name_: val + hh}) - A(**{name_: val - hh})) / (2 * hh)
        assert np.abs(fd - dv).max() <= 1e-9 * scale / val, name_
    for c in (0, len(om.cells) // 2, len(om.cells) - 1):
        hh = 1e-3 * E[c]
        Ep, Em = E.copy(), E.copy()
        Ep[c] += hh
        Em[c] -= hh
        fd = (ops.residual_form(om, mat, ops.State(om, u, phi, phit, Ep))
              - ops.residual_form(om, mat, ops.State(om, u, phi, phit, Em))) / (2 * hh)
        assert np.abs(fd - d_e[:, c].toarray().ravel()).max() <= 1e-9 * scale / E[c]
    # A depends on E_K only through the nodes of cell K
    col = d_e[:, 0].toarray().ravel()
    nz = np.nonzero(col)[0] % om.nn
    assert set(nz) <= set(om.cell_nodes[0])


def sneddon_solve(om, mat_kw, E, tol=1e-13):
    h = om.h_min_diag()
    u0, po = solvers.sneddon_initial(om, h)
    mat = ops.Material(**mat_kw)
    u, phi, act, info = solvers.load_step(om, mat, 1e4, u0, po.copy(), po, E_cells=E, tol=tol, atol=1e-15,
                                          gmres_rtol=1e-12)
    assert info.converged
    return u, phi, po, act, mat


@pytest.mark.parametrize("name,p", [("tiny", 1e-3), ("tiny", 0.2), ("band4_2_2", 1e-3), ("band4_2_2", 0.2)])
def test_adjoint_gradient_central_difference(name, p):
    """dJ/dtheta from one adjoint solve against central differences of J over
    two converged load steps each (relative step 1e-6, bound 1e-5 relative).

    At p = 1e-3 the phase field hardly responds to G_c (|G_c dJ/dG_c| ~ 1e-7 J),
    below what a difference of J at relative step 1e-6 resolves, so G_c is
    checked at p = 0.2, where it is 1e-3 J."""
    om = mesh(name)
    h = om.h_min_diag()
    E = cell_E(om)
    base = dict(E=1.0, nu=0.2, Gc=1.0, eps=2.0 * h, kappa=1e-10, p=p)
    u, phi, po, act, mat = sneddon_solve(om, base, E)
    st = ops.State(om, u, phi, po, E)
    g = adj.tcv_adjoint(om, mat, st, act)
    # the VJP of the residual with the adjoint gives the same gradient
    vp, vg, ve = adj.param_vjp(om, mat, st, g["lam"])
    assert abs(vp - g["p"]) <= 1e-12 * abs(g["p"])
    assert abs(vg - g["Gc"]) <= 1e-10 * abs(g["Gc"])
    assert np.allclose(ve, g["E"], rtol=0, atol=1e-12 * np.abs(g["E"]).max())

    def J(mat_kw, Ec):
        uu, pp, po_, aa, _ = sneddon_solve(om, mat_kw, Ec)
        assert np.array_equal(aa, act), "active set changed under the perturbation"
        return ops.tcv(om, ops.State(om, uu, pp, po_))

    rel = 1e-6
    for key in ("p", "Gc") if p > 0.1 else ("p",):
        hh = rel * base[key]
        kp, km = dict(base), dict(base)
        kp[key] += hh
        km[key] -= hh
        fd = (J(kp, E) - J(km, E)) / (2 * hh)
        assert abs(fd - g[key]) <= 1e-5 * abs(fd), (key, fd, g[key])
    for c in np.argsort(-np.abs(g["E"]))[:2]:
        hh = rel * E[c]
        Ep, Em = E.copy(), E.copy()
        Ep[c] += hh
        Em[c] -= hh
        fd = (J(base, Ep) - J(base, Em)) / (2 * hh)
        assert abs(fd - g["E"][c]) <= 1e-5 * abs(fd), (c, fd, g["E"][c])


@pytest.mark.parametrize("name,k", [("tiny", 1), ("small", 1), ("tiny", 2)])
def test_phit_vjp_central_difference(name, k):
    """A is quadratic in phi_tilde, so a central difference of w . A in direction v is exact."""
    om = mesh(name, k)
    u, phi, phit = random_state(om, seed=3)
    E = cell_E(om)
    mat = ops.Material(E=1.0, nu=0.2, Gc=1.3, eps=2.0 * om.h_min_diag(), kappa=1e-3, p=0.2)
    rng = np.random.Generator(np.random.PCG64(8))
    w = rng.normal(size=3 * om.nn)
    v = rng.normal(size=om.nn)
    got = v @ adj.phit_vjp(om, mat, ops.State(om, u, phi, phit, E), w)
    wf = ops.C3(om) @ w
    eps = 1e-3
    Ap = ops.residual_form(om, mat, ops.State(om, u, phi, phit + eps * v, E))
    Am = ops.residual_form(om, mat, ops.State(om, u, phi, phit - eps * v, E))
    fd = wf @ (Ap - Am) / (2 * eps)
    assert abs(got - fd) <= 1e-10 * max(abs(fd), 1e-12), (got, fd)


def sneddon_steps(om, base, E, ps, tol=1e-13):
    """Load steps at pressures ps from the initial crack; returns mats, us, phis, actives."""
    h = om.h_min_diag()
    u0, po = solvers.sneddon_initial(om, h)
    mats, us, phis, acts = [], [u0], [po], []
    u, phi, act = u0, po.copy(), None
    for p in ps:
        kw = dict(base, p=p)
        mat = ops.Material(**kw)
        u, phi_new, act, info = solvers.load_step(om, mat, 1e4, u, phi.copy(), phi, active_prev=act, E_cells=E,
                                                  tol=tol, atol=1e-15, gmres_rtol=1e-12)
        assert info.converged
        phi = phi_new
        mats.append(mat)
        us.append(u)
        phis.append(phi)
        acts.append(act)
    return mats, us, phis, acts


def test_multi_step_adjoint_central_difference():
    """Three load steps: dJ/dp_n, dJ/dG_c and dJ/dE_K of the final TCV from one
    backward sweep against central differences of three-step solves (relative
    step 1e-6, bound 1e-5)."""
    om = mesh("tiny")
    E = cell_E(om)
    base = dict(E=1.0, nu=0.2, Gc=1.0, eps=2.0 * om.h_min_diag(), kappa=1e-10)
    ps = [0.1, 0.15, 0.2]
    mats, us, phis, acts = sneddon_steps(om, base, E, ps)
    g = adj.tcv_adjoint_steps(om, mats, us, phis, acts, E)
    # the single-step formula agrees for one step
    g1 = adj.tcv_adjoint_steps(om, mats[:1], us[:2], phis[:2], acts[:1], E)
    r1 = adj.tcv_adjoint(om, mats[0], ops.State(om, us[1], phis[1], phis[0], E), acts[0])
    assert abs(g1["p"][0] - r1["p"]) <= 1e-12 * abs(r1["p"]) and abs(g1["Gc"] - r1["Gc"]) <= 1e-10 * abs(r1["Gc"])

    def J(bkw, pss, Ec):
        _, uu, pp, aa = sneddon_steps(om, bkw, Ec, pss)
        for a0, a1 in zip(aa, acts):
            assert np.array_equal(a0, a1), "active set changed under the perturbation"
        return ops.tcv(om, ops.State(om, uu[-1], pp[-1], pp[-1]))

    rel = 1e-6
    for n in range(len(ps)):
        hh = rel * ps[n]
        pp_, pm_ = list(ps), list(ps)
        pp_[n] += hh
        pm_[n] -= hh
        fd = (J(base, pp_, E) - J(base, pm_, E)) / (2 * hh)
        assert abs(fd - g["p"][n]) <= 1e-5 * abs(fd), (n, fd, g["p"][n])
    hh = rel * base["Gc"]
    fd = (J(dict(base, Gc=base["Gc"] + hh), ps, E) - J(dict(base, Gc=base["Gc"] - hh), ps, E)) / (2 * hh)
    assert abs(fd - g["Gc"]) <= 1e-5 * abs(fd), (fd, g["Gc"])
    for c in np.argsort(-np.abs(g["E"]))[:2]:
        hh = rel * E[c]
        Ep, Em = E.copy(), E.copy()
        Ep[c] += hh
        Em[c] -= hh
        fd = (J(base, ps, Ep) - J(base, ps, Em)) / (2 * hh)
        assert abs(fd - g["E"][c]) <= 1e-5 * abs(fd), (c, fd, g["E"][c])


def sneddon_steps_extrapolated(om, base, E, ps, tol=1e-13):
    """sneddon_steps with phi_tilde of step n >= 2 extrapolated from the two previous
    steps (clip(2 phi^(n-1) - phi^(n-2), 0, 1), oracle/solvers.extrapolate_phi);
    returns mats, us, phis, actives and the clip masks of steps 2..N."""
    h = om.h_min_diag()
    u0, po = solvers.sneddon_initial(om, h)
    mats, us, phis, acts, chis = [], [u0], [po], [], []
    u, phi, act = u0, po.copy(), None
    for n, p in enumerate(ps, start=1):
        mat = ops.Material(**dict(base, p=p))
        phit = None
        if n >= 2:
            phit = solvers.extrapolate_phi(phis[-1], phis[-2])
            raw = 2.0 * phis[-1] - phis[-2]
            chis.append((raw > 0.0) & (raw < 1.0))
        u, phi_new, act, info = solvers.load_step(om, mat, 1e4, u, phi.copy(), phi, active_prev=act, E_cells=E,
                                                  tol=tol, atol=1e-15, gmres_rtol=1e-12, phi_tilde=phit)
        assert info.converged
        phi = phi_new
        mats.append(mat)
        us.append(u)
        phis.append(phi)
        acts.append(act)
    return mats, us, phis, acts, chis


def test_multi_step_adjoint_extrapolated_phi_tilde():
    """Three load steps whose phi_tilde (Sec. 2) is extrapolated from the two previous
    steps: dJ/dp_n and dJ/dG_c of the final TCV from one backward sweep against central
    differences of three-step solves (relative step 1e-6, bound 1e-5), active sets and
    clip pattern unchanged under the perturbations.  The gradient differs from the one
    with phi_tilde = phi_old of the same states (the extrapolation's two-step coupling
    matters)."""
    om = mesh("tiny")
    E = cell_E(om)
    base = dict(E=1.0, nu=0.2, Gc=1.0, eps=2.0 * om.h_min_diag(), kappa=1e-10)
    ps = [0.1, 0.15, 0.2]
    mats, us, phis, acts, chis = sneddon_steps_extrapolated(om, base, E, ps)
    assert all(c.any() for c in chis)
    g = adj.tcv_adjoint_steps(om, mats, us, phis, acts, E, extrapolate=True)
    g_old = adj.tcv_adjoint_steps(om, mats, us, phis, acts, E)
    assert np.max(np.abs(g["p"] - g_old["p"])) > 1e-2 * np.max(np.abs(g["p"]))

    def J(bkw, pss):
        _, uu, pp, aa, cc = sneddon_steps_extrapolated(om, bkw, E, pss)
        for a0, a1 in zip(aa, acts):
            assert np.array_equal(a0, a1), "active set changed under the perturbation"
        for c0, c1 in zip(cc, chis):
            assert np.array_equal(c0, c1), "clip pattern changed under the perturbation"
        return ops.tcv(om, ops.State(om, uu[-1], pp[-1], pp[-1]))

    rel = 1e-6
    for n in range(len(ps)):
        hh = rel * ps[n]
        pp_, pm_ = list(ps), list(ps)
        pp_[n] += hh
        pm_[n] -= hh
        fd = (J(base, pp_) - J(base, pm_)) / (2 * hh)
        assert abs(fd - g["p"][n]) <= 1e-5 * abs(fd), (n, fd, g["p"][n])
    hh = rel * base["Gc"]
    fd = (J(dict(base, Gc=base["Gc"] + hh), ps) - J(dict(base, Gc=base["Gc"] - hh), ps)) / (2 * hh)
    assert abs(fd - g["Gc"]) <= 1e-5 * abs(fd), (fd, g["Gc"])
