"""Failure reporting through the C-ABI, made on the host (no GPU fault): a NaN in
a host-generated input and iteration caps that cannot be met.  Each call returns
its status code with pff_solve_info filled, and the context stays usable: a
normal call afterwards succeeds (status codes of include/pff.h:
PFF_ERR_INVALID_ARG = 1, PFF_ERR_NOT_CONVERGED = 4, PFF_ERR_NONFINITE = 6)."""
import numpy as np
import pytest

from harness import Pair, random_linearisation
from oracle import solvers

pytestmark = pytest.mark.gpu

INVALID_ARG, NOT_CONVERGED, NONFINITE = 1, 4, 6


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def gmres_setup():
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem
    P = Pair("small", 1)
    mat = P.material(kappa=1e-3, p=0.05)
    u, phi, phit = random_linearisation(P, seed=0, u_std=1e-2)
    pb = Problem(P.lm, **mat)
    pb.set_state(dev(P.to_slots(u).T), dev(P.to_slots(phi)), dev(P.to_slots(phit)))
    mg = MG(pb, PFF_F32)
    mg.setup()
    b = np.random.default_rng(9).normal(size=(P.om.nn, 3))
    b[P.om.is_hanging] = 0.0
    return P, pb, mg, P.to_slots(b).T.copy()


def test_gmres_nan_rhs_and_iteration_cap():
    import torch
    from paper_2404_03265_gb300 import gmres
    P, pb, mg, b = gmres_setup()
    bad = b.copy()
    bad[2, np.nonzero((P.lm.slots()[2] & 1) == 1)[0][17]] = np.nan   # one phi entry of a node
    x = torch.zeros((3, P.n_slots), dtype=torch.float64, device="cuda")
    r = gmres(pb, mg, dev(bad), x, rtol=1e-10, maxiter=50, check=False)
    assert r["status"] == NONFINITE and not r["converged"]
    # iteration cap: one Arnoldi step cannot reach 1e-12
    x.zero_()
    r = gmres(pb, mg, dev(b), x, rtol=1e-12, restart=50, maxiter=1, check=False)
    assert r["status"] == NOT_CONVERGED and not r["converged"]
    assert r["iterations"] == 1
    assert np.isfinite(r["initial"]) and r["initial"] > 0
    assert np.isfinite(r["estimate"]) and 0 < r["estimate"] < r["initial"]
    # the context is still usable
    x.zero_()
    r = gmres(pb, mg, dev(b), x, rtol=1e-8, maxiter=400, check=False)
    assert r["status"] == 0 and r["converged"]


def sneddon(P):
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem
    om = P.om
    mat = P.material()
    pb = Problem(P.lm, **mat)
    mg = MG(pb, PFF_F32)
    _, po = solvers.sneddon_initial(om, om.h_min_diag())
    return pb, mg, po


def test_newton_nan_state_and_newton_cap():
    import torch
    from paper_2404_03265_gb300 import newton_step
    P = Pair("small", 1)
    pb, mg, po = sneddon(P)
    ns = P.n_slots
    ps = dev(P.to_slots(po))
    # a NaN in the host-generated state: the first residual is non-finite
    u = torch.zeros((2, ns), dtype=torch.float64, device="cuda")
    phi = ps.clone()
    bad = P.to_slots(po)
    bad[np.nonzero((P.lm.slots()[2] & 1) == 1)[0][40]] = np.nan
    phi_bad = dev(bad)
    act = torch.zeros(ns, dtype=torch.uint8, device="cuda")
    r = newton_step(pb, mg, u, phi_bad, ps, act, check=False)
    assert r["status"] == NONFINITE and not r["converged"]
    # Newton capped at one iteration: the Sneddon step needs several
    u.zero_()
    phi = ps.clone()
    act.zero_()
    r = newton_step(pb, mg, u, phi, ps, act, max_newton=1, check=False)
    assert r["status"] == NOT_CONVERGED and not r["converged"]
    assert r["newton"] == 1
    assert r["gmres_total"] >= 1 and np.isfinite(r["residual"]) and r["residual"] > 0
    # the same problem then solves the step
    u.zero_()
    phi = ps.clone()
    act.zero_()
    r = newton_step(pb, mg, u, phi, ps, act, check=False)
    assert r["status"] == 0 and r["converged"]


def test_invalid_arguments_are_reported():
    import torch
    from paper_2404_03265_gb300 import Problem, _lib
    P = Pair("tiny", 1)
    pb = Problem(P.lm, **P.material())
    ns = P.n_slots
    u, phi, phit = random_linearisation(P, seed=1, u_std=1e-2)
    pb.set_state(dev(P.to_slots(u).T), dev(P.to_slots(phi)), dev(P.to_slots(phit)))
    xu = torch.zeros((2, ns), dtype=torch.float64, device="cuda")
    xp = torch.zeros(ns, dtype=torch.float64, device="cuda")
    yu, yp = torch.zeros_like(xu), torch.zeros_like(xp)
    L = _lib.lib()
    assert L.pff_apply(pb._h, 7, 0, _lib.ptr(xu), _lib.ptr(xp), _lib.ptr(yu), _lib.ptr(yp), None) == INVALID_ARG
    assert b"precision" in L.pff_last_error()
    assert L.pff_apply(pb._h, 0, 0, _lib.ptr(xu), _lib.ptr(xp), _lib.ptr(xu), _lib.ptr(yp), None) == INVALID_ARG
    assert L.pff_set_cell_loop(pb._h, 4) == INVALID_ARG
    assert L.pff_apply(pb._h, 0, 0, _lib.ptr(xu), _lib.ptr(xp), _lib.ptr(yu), _lib.ptr(yp), None) == 0
    from paper_2404_03265_gb300 import MG, PFF_F32
    mg = MG(pb, PFF_F32)
    assert L.pff_mg_set_fused_smoother(mg._h, 2) == INVALID_ARG
    assert L.pff_mg_set_coarse(mg._h, 5) == INVALID_ARG
    assert L.pff_mg_set_fused_smoother(mg._h, 0) == 0
