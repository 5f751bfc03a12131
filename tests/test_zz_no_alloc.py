"""pff_apply_noalloc (scratch in a fixed device array of the library) against
pff_apply (scratch in the problem's buffers), both through the C-ABI.

The scratch of one apply is the input resolved on the hanging nodes (Q1) and
the interface partial sums.  Both calls run the same kernels in the same
summation order, so the results agree to the parity tolerances of the apply
(1e-12 FP64, 1e-5 FP32, relative 2-norm); in practice they are bit-identical.
Each case makes two no-alloc calls in a row with different inputs, on meshes
with different scratch sizes and both element degrees, because the fixed array
keeps the previous call's contents.  A further test checks that repeated calls
change neither the device's free memory nor torch's reserved memory.  The file
is collected last so that the first no-alloc call of the process may come
either first (run alone) or after every other GPU test.
"""
import ctypes

import numpy as np
import pytest

import synthetic as synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}   # PFF_F64, PFF_F32

_cases = {}


def case(name, k=1):
    """Mesh, problem with a random state and 10% active phi, and two inputs."""
    if (name, k) in _cases:
        return _cases[(name, k)]
    import torch
    from paper_2404_03265_gb300 import Mesh, Problem
    dev = torch.device("cuda:0")
    m = Mesh.from_recipe(synth.recipe(name)).finalize(k)
    X, Y, F = m.slots()
    valid = np.nonzero((F & 1) == 1)[0]
    ns = len(X)
    xv, yv = X[valid], Y[valid]
    u, phi, phit = synth.linearisation(xv, yv, m.info["x_max"], m.info["y_max"], seed=3)

    def slots(a):
        out = np.zeros((ns,) + a.shape[1:], dtype=a.dtype)
        out[valid] = a
        return out

    h = m.info["h_min"]
    pb = Problem(m, E=1.0, nu=0.2, Gc=1.0, eps=2.0 * h, kappa=1e-2, p=0.1)
    pb.set_state(torch.tensor(slots(u).T.copy(), device=dev), torch.tensor(slots(phi), device=dev),
                 torch.tensor(slots(phit), device=dev))
    rng = np.random.Generator(np.random.PCG64(11))
    pb.set_active(torch.tensor(slots((rng.uniform(size=len(valid)) < 0.1).astype(np.uint8)), device=dev))
    xs = []
    for seed in (5, 6):
        v = slots(synth.vector(xv, yv, seed=seed))
        xs.append((torch.tensor(v[:, :2].T.copy(), device=dev), torch.tensor(v[:, 2].copy(), device=dev)))
    _cases[(name, k)] = (m, pb, xs, ns)
    return _cases[(name, k)]


def call(fn, pb, prec, op, xu, xp, ns):
    import torch
    from paper_2404_03265_gb300 import _lib
    dt = torch.float64 if prec == 0 else torch.float32
    xu, xp = xu.to(dt), xp.to(dt)
    yu = torch.full((2, ns), float("nan"), dtype=dt, device=xu.device)
    yp = torch.full((ns,), float("nan"), dtype=dt, device=xu.device)
    _lib.check(getattr(_lib.lib(), fn)(pb._h, prec, op, _lib.ptr(xu), _lib.ptr(xp), _lib.ptr(yu), _lib.ptr(yp),
                                       _lib.stream_ptr(None)))
    torch.cuda.synchronize()
    return torch.cat([yu.reshape(-1), yp]).double().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("op", [0, 1, 2], ids=["jacobian", "transpose", "condensed"])
@pytest.mark.parametrize("name,k", [("solve", 1), ("small", 1), ("small", 2), ("adjoint", 2)])
def test_noalloc_matches_apply(prec, op, name, k):
    m, pb, xs, ns = case(name, k)
    scratch = m.info["n_partials"] + (m.info["n_hanging"] if k == 1 else 0)
    assert 0 < m.info["n_partials"] and scratch <= 65536
    got = [call("pff_apply_noalloc", pb, prec, op, xu, xp, ns) for xu, xp in xs]   # two in a row
    want = [call("pff_apply", pb, prec, op, xu, xp, ns) for xu, xp in xs]
    for g, w in zip(got, want):
        assert np.all(np.isfinite(g))
        assert rel(g, w) <= TOL[prec], (name, k, rel(g, w))
    assert rel(got[0], got[1]) > 0.1    # the two inputs give different results


def test_noalloc_allocates_nothing():
    """After a first call, further calls leave the device's free memory (driver
    view) and torch's reserved memory unchanged."""
    import torch
    m, pb, xs, ns = case("solve", 1)
    dt = torch.float32
    xu, xp = xs[0][0].to(dt), xs[0][1].to(dt)
    yu = torch.empty((2, ns), dtype=dt, device=xu.device)
    yp = torch.empty((ns,), dtype=dt, device=xu.device)
    from paper_2404_03265_gb300 import _lib

    def go():
        _lib.check(_lib.lib().pff_apply_noalloc(pb._h, 1, 0, _lib.ptr(xu), _lib.ptr(xp), _lib.ptr(yu), _lib.ptr(yp),
                                                _lib.stream_ptr(None)))
    go()
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(5):
        go()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_oversized_mesh():
    import torch
    from paper_2404_03265_gb300 import Mesh, Problem, _lib
    m = Mesh.from_recipe(synth.recipe("large")).finalize(1)
    assert m.info["n_partials"] > 65536
    pb = Problem(m)
    ns = m.info["n_slots"]
    xu = torch.zeros((2, ns), dtype=torch.float64, device="cuda:0")
    xp = torch.zeros(ns, dtype=torch.float64, device="cuda:0")
    yu, yp = torch.zeros_like(xu), torch.zeros_like(xp)
    st = _lib.lib().pff_apply_noalloc(pb._h, 0, 0, _lib.ptr(xu), _lib.ptr(xp), _lib.ptr(yu), _lib.ptr(yp),
                                      _lib.stream_ptr(None))
    assert st == 1   # PFF_ERR_INVALID_ARG
    msg = _lib.lib().pff_last_error().decode()
    assert "65536" in msg and "pff_apply" in msg
