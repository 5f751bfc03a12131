"""Test harness: builds the oracle and the library on the same workload and maps
between the oracle's canonical node order and the library's slot layout.

Mapping is by integer node coordinates only; no arithmetic of the method is
shared.  Inputs come from the top-level module ``synthetic``.
"""
import numpy as np

from oracle import operators as ops
from oracle.mesh import LeafMesh, build_recipe
import synthetic as synth


class Pair:
    """Oracle mesh + library mesh of one recipe and degree, with the node map."""

    def __init__(self, recipe_name, k=1, lib_mesh=True):
        from paper_2404_03265_gb300 import Mesh
        self.recipe = synth.recipe(recipe_name) if isinstance(recipe_name, str) else recipe_name
        self.k = k
        self.om = LeafMesh(build_recipe(self.recipe), k)
        self.lm = Mesh.from_recipe(self.recipe).finalize(k) if lib_mesh else None
        X, Y, F = self.lm.slots()
        self.slot_X, self.slot_Y, self.slot_F = X, Y, F
        valid = (F & 1) == 1
        self.valid = valid
        self.slots = np.nonzero(valid)[0]
        key_l = Y[valid].astype(np.int64) * (self.om.Xmax + 1) + X[valid].astype(np.int64)
        pos = np.searchsorted(self.om.key, key_l)
        assert np.all(self.om.key[np.minimum(pos, self.om.nn - 1)] == key_l), "node sets differ"
        self.onode = pos                     # oracle node of each valid slot
        self.n_slots = len(X)
        assert len(self.slots) == self.om.nn

    # oracle (nn, c) -> library (n_slots, c), holes zero
    def to_slots(self, a):
        a = np.asarray(a)
        out = np.zeros((self.n_slots,) + a.shape[1:], dtype=a.dtype)
        out[self.slots] = a[self.onode]
        return out

    def from_slots(self, s):
        s = np.asarray(s)
        out = np.zeros((self.om.nn,) + s.shape[1:], dtype=s.dtype)
        out[self.onode] = s[self.slots]
        return out

    def material(self, **kw):
        h = self.om.h_min_diag()
        m = dict(E=1.0, nu=0.2, Gc=1.0, eps=2.0 * h, kappa=1e-10, p=1e-3)
        m.update(kw)
        return m


def random_linearisation(pair, seed=0, u_std=1e-3):
    om = pair.om
    u, phi, phit = synth.linearisation(om.X, om.Y, om.Xmax, om.Ymax, seed=seed, u_std=u_std)
    return u, phi, phit


def random_active(pair, seed=5, frac=0.05):
    om = pair.om
    rng = np.random.Generator(np.random.PCG64(seed))
    order = synth.canonical_order(om.X, om.Y)
    a = np.zeros(om.nn, bool)
    a[order] = rng.uniform(size=om.nn) < frac
    a &= ~om.is_hanging
    return a


def oracle_apply(pair, mat, u, phi, phit, active, x, op="jacobian", E_cells=None):
    """y = G~ x (or G~^T x, or M_f C^T G C x) with the oracle; x, y as (nn, 3)."""
    om = pair.om
    st = ops.State(om, u, phi, phit, E_cells)
    G = ops.assemble_jacobian(om, ops.Material(**mat), st)
    nn = om.nn
    v = np.concatenate([x[:, 0], x[:, 1], x[:, 2]])
    if op == "jacobian":
        y = ops.constrained_operator(om, G, active) @ v
    elif op == "transpose":
        y = ops.constrained_operator(om, G, active).T @ v
    elif op == "condensed":
        y = ops.condensed_operator(om, G, active) @ v
    else:
        raise ValueError(op)
    return np.stack([y[:nn], y[nn:2 * nn], y[2 * nn:]], axis=1)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    inf = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
    two = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    return inf, two


# lambda_max parity: the FP64 V-cycle's estimates come from FP64 CG runs (the
# oracle's arithmetic); the FP32 V-cycle's CG applies its level operators (levels
# >= 1) in FP32, which moves lambda by FP32 rounding of the operator
LAMBDA_RTOL = {"f64": 1e-9, "f32": 5e-6}
