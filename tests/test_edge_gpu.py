"""Edge cases of the constrained Jacobian apply through the C-ABI, against the
oracle: a uniform mesh without hanging nodes, a mesh of one coarse cell (every
node on the Dirichlet boundary), an all-active phase field (phi rows are the
identity), and a zero input (exact zero output).  Tolerances as in
test_apply_gpu.py: 1e-12 (FP64), 1e-5 (FP32)."""
import numpy as np
import pytest

import synthetic as synth
from harness import Pair, oracle_apply, random_active, random_linearisation, rel_err
from test_apply_gpu import TOL, run_lib

pytestmark = pytest.mark.gpu

ONE_CELL = dict(domain=synth.DOMAIN, ncx=1, ncy=1, n_global=0, steps=[])


@pytest.mark.parametrize("case", ["uniform", "one_cell", "all_active", "zero_x"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("op", ["jacobian", "transpose"])
def test_apply_edge_cases(case, prec, op):
    P = Pair({"uniform": "table2_0", "one_cell": ONE_CELL}.get(case, "small"), 1)
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
        assert om.nn == 4 and om.dirichlet.all()
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
