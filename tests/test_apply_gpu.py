"""Parity of the CUDA Jacobian apply (through the C-ABI) with the oracle's
explicitly assembled constrained Jacobian.

Tolerances: 1e-12 relative (FP64 apply), 1e-5 relative (FP32 apply), in the
infinity norm and the 2-norm over all DoFs.
"""
import numpy as np
import pytest

from harness import Pair, oracle_apply, random_active, random_linearisation, rel_err

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
PARAMS = {
    # the workload's material (Table 1, kappa = 1e-10, p = 1e-3) with u ~ N(0, 1e-3)
    "workload": (dict(), 1e-3),
    # every term of the Jacobian of the same order: large p, kappa, u
    "strong": (dict(E=1.7, nu=0.3, Gc=2.0, kappa=1e-2, p=0.4), 0.3),
}

_pairs = {}


def pair(name, k=1):
    if (name, k) not in _pairs:
        _pairs[(name, k)] = Pair(name, k)
    return _pairs[(name, k)]


def run_lib(P, mat, u, phi, phit, active, x, prec, op):
    import torch
    from paper_2404_03265_gb300 import PFF_OP_CONDENSED, PFF_OP_JACOBIAN, PFF_OP_TRANSPOSE, Problem
    dev = torch.device("cuda:0")
    pb = Problem(P.lm, **mat)
    us = torch.tensor(P.to_slots(u).T.copy(), device=dev)
    ps = torch.tensor(P.to_slots(phi), device=dev)
    pts = torch.tensor(P.to_slots(phit), device=dev)
    pb.set_state(us, ps, pts)
    pb.set_active(torch.tensor(P.to_slots(active.astype(np.uint8)), device=dev))
    dt = torch.float64 if prec == "f64" else torch.float32
    xs = P.to_slots(x)
    # garbage in holes and hanging entries must be ignored
    holes = ~P.valid
    xs[holes] = 1e30
    hang = P.slots[(P.slot_F[P.slots] & 4) != 0]
    xs[hang] = 7.0
    xu = torch.tensor(xs[:, :2].T.copy(), device=dev, dtype=dt)
    xp = torch.tensor(xs[:, 2].copy(), device=dev, dtype=dt)
    yu = torch.full_like(xu, float("nan"))
    yp = torch.full_like(xp, float("nan"))
    opc = {"jacobian": PFF_OP_JACOBIAN, "transpose": PFF_OP_TRANSPOSE, "condensed": PFF_OP_CONDENSED}[op]
    pb.apply(xu, xp, yu, yp, op=opc)
    torch.cuda.synchronize()
    ys = np.concatenate([yu.cpu().double().numpy().T, yp.cpu().double().numpy()[:, None]], axis=1)
    return ys


@pytest.mark.parametrize("name", ["tiny", "small", "adjoint"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("op", ["jacobian", "transpose", "condensed"])
@pytest.mark.parametrize("params", ["workload", "strong"])
def test_apply_parity_q1(name, prec, op, params):
    P = pair(name, 1)
    kw, ustd = PARAMS[params]
    mat = P.material(**kw)
    u, phi, phit = random_linearisation(P, seed=0, u_std=ustd)
    active = random_active(P, seed=5, frac=0.05)
    import synthetic as synth
    x = synth.vector(P.om.X, P.om.Y, seed=1)
    ref = oracle_apply(P, mat, u, phi, phit, active, x, op=op)
    ys = run_lib(P, mat, u, phi, phit, active, x, prec, op)
    assert np.all(ys[~P.valid] == 0.0), "holes must be written as zero"
    y = P.from_slots(ys)
    assert np.all(np.isfinite(y))
    assert np.all(y[P.om.is_hanging] == 0.0)
    inf, two = rel_err(y, ref)
    assert inf < TOL[prec] and two < TOL[prec], (inf, two)
