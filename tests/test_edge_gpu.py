"""Edge cases through the C-ABI, against the oracle where it applies.

* Apply (Q1 and Q2): a uniform mesh without hanging nodes, a mesh of one coarse
  cell (all its boundary nodes Dirichlet), an all-active phase field (phi rows
  are identity rows, exact), and a zero input (exact zero output).  Tolerances as
  in test_apply_gpu.py: 1e-12 (FP64), 1e-5 (FP32).
* Block V-cycle on a mesh of global levels only and on a single-level mesh.
* GMRES with a zero right-hand side; a load step from an already solved state."""
import numpy as np
import pytest

import synthetic as synth
from harness import Pair, oracle_apply, random_active, random_linearisation, rel_err
from test_apply_gpu import TOL, run_lib

pytestmark = pytest.mark.gpu

ONE_CELL = dict(domain=synth.DOMAIN, ncx=1, ncy=1, n_global=0, steps=[])


_pairs = {}


def pair(case, k):
    if (case, k) not in _pairs:
        _pairs[(case, k)] = Pair({"uniform": "table2_0", "one_cell": ONE_CELL}.get(case, "small"), k)
    return _pairs[(case, k)]


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("case", ["uniform", "one_cell", "all_active", "zero_x"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("op", ["jacobian", "transpose"])
def test_apply_edge_cases(case, prec, op, k):
    P = pair(case, k)
    om = P.om
    mat = P.material(kappa=1e-2, p=0.3)
    u, phi, phit = random_linearisation(P, seed=2, u_std=0.1)
    if case == "all_active":
        active = ~om.is_hanging
    else:
        active = random_active(P, seed=5, frac=0.1)
    x = synth.vector(om.X, om.Y, seed=1)
    if case == "zero_x":
        x = np.zeros_like(x)
    if case == "uniform":
        assert not om.is_hanging.any()
    if case == "one_cell":
        assert om.nn == (k + 1) ** 2 and om.dirichlet.sum() == 4 * k
    ref = oracle_apply(P, mat, u, phi, phit, active, x, op=op)
    ys = run_lib(P, mat, u, phi, phit, active, x, prec, op)
    assert np.all(ys[~P.valid] == 0.0)
    y = P.from_slots(ys)
    assert np.all(np.isfinite(y))
    if case == "zero_x":
        assert np.all(y == 0.0)
        return
    if case == "all_active":
        # active phi rows are identity rows, in the apply's precision
        xa = x[active, 2] if prec == "f64" else x[active, 2].astype(np.float32).astype(np.float64)
        assert np.array_equal(y[active, 2], xa)
    inf, two = rel_err(y, ref)
    assert inf < TOL[prec] and two < TOL[prec], (inf, two)


@pytest.mark.parametrize("case", ["uniform", "one_cell"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_vcycle_edge_meshes(case, prec, tol):
    """Block V-cycle parity on a mesh with global levels only, and on a single-level
    mesh (one cell: the V-cycle is the coarse solve; the u block has no interior,
    so z = r on its fixed rows and nothing else)."""
    import torch
    from oracle import mg as omg
    from oracle import operators as ops
    from test_mg_gpu import lib_mg
    P = Pair({"uniform": "table2_0", "one_cell": ONE_CELL}[case], 1)
    om = P.om
    nn = om.nn
    mat = P.material(kappa=1e-3, p=0.05)
    u, phi, phit = random_linearisation(P, seed=0, u_std=1e-2)
    active = np.zeros(nn, bool)
    M = omg.MG(om, ops.Material(**mat), u, phi, phit, active)
    pb, mg = lib_mg(P, mat, u, phi, phit, active, prec)
    rng = np.random.default_rng(3)
    for b, blk, nc in ((0, "uu", 2), (1, "pp", 1)):
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
        assert inf < tol and two < tol, (case, blk, prec, inf, two)


def test_gmres_zero_rhs():
    """GMRES with a zero right-hand side returns x = 0 at once, converged."""
    import torch
    from paper_2404_03265_gb300 import gmres
    from test_mg_gpu import lib_mg
    P = Pair("small", 1)
    mat = P.material()
    u, phi, phit = random_linearisation(P, seed=0, u_std=1e-2)
    pb, mg = lib_mg(P, mat, u, phi, phit, np.zeros(P.om.nn, bool), "f32")
    rhs = torch.zeros((3, P.n_slots), dtype=torch.float64, device="cuda")
    x = torch.full_like(rhs, float("nan"))
    d = gmres(pb, mg, rhs, x)
    torch.cuda.synchronize()
    assert d["converged"] and d["iterations"] == 0
    assert bool((x == 0).all())


def test_newton_already_solved_state():
    """p = 0 and an intact phase field (u = 0, phi = phi_old = 1) make the residual
    of Problem 2 vanish: the load step stops before its first Newton step and
    leaves the state untouched."""
    import torch
    from paper_2404_03265_gb300 import MG, PFF_F32, Problem, newton_step
    P = Pair("small", 1)
    pb = Problem(P.lm, **P.material(p=0.0))
    mg = MG(pb, PFF_F32)
    u = torch.zeros((2, P.n_slots), dtype=torch.float64, device="cuda")
    phi = torch.tensor(P.to_slots(np.ones(P.om.nn)), device="cuda")
    phi_old = phi.clone()
    act = torch.zeros(P.n_slots, dtype=torch.uint8, device="cuda")
    info = newton_step(pb, mg, u, phi, phi_old, act)
    torch.cuda.synchronize()
    assert info["converged"] and info["newton"] == 0, info
    assert bool((u == 0).all()) and bool((phi == phi_old).all()) and int(act.sum()) == 0
