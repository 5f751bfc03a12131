"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the method's arithmetic: it only describes the
workload meshes as refinement recipes and draws random fields.  Every field is
drawn in the CANONICAL node order (ascending integer (Y, X)) or canonical cell
order (ascending (level, j, i)), so that two independent implementations that
number nodes differently still receive identical bits: the caller passes its
own integer node coordinates and gets the values back in its own order.

Workloads (the pressurised straight crack of Sec. 4, Omega = (-10, 10)^2):

* ``small``   4x4 coarse, 3 global, 2 box steps |x|<=2, |y|<=1   (Q1 ~4.3k DoFs)
* ``apply``   16x16 coarse, 6 global, 2 box steps                 (Q1 ~4.1M, Q2 ~16.4M DoFs)
* ``solve``   16x16 coarse, 5 global, 7 band steps toward the crack (Q1 ~1.04M DoFs)
* ``adjoint`` 4x4 coarse, 5 global, 2 box steps                   (Q1 ~65k DoFs)
* ``large``   14x14 coarse, 6 global, 9 band steps                 (Q2 ~16.5M DoFs)
* ``table2_0`` 10x10 coarse, 2 global: the unrefined mesh of Table 2 (Q1 5043 DoFs)

A band step refines every leaf that meets |x| <= 1 + 2 h_min, |y| <= 2 h_min,
h_min the diagonal of the finest cell of the final mesh.
"""
import math

import numpy as np

DOMAIN = (-10.0, 10.0, -10.0, 10.0)


def _band(ncx, n_global, n_band):
    side = (DOMAIN[1] - DOMAIN[0]) / (ncx * 2 ** (n_global + n_band))
    hmin = math.sqrt(2.0) * side
    return ("band", -(1.0 + 2.0 * hmin), 1.0 + 2.0 * hmin, -2.0 * hmin, 2.0 * hmin)


def recipe(name):
    """Mesh recipe: dict(domain, ncx, ncy, n_global, steps=[(kind, x0, x1, y0, y1), ...])."""
    box = ("box", -2.0, 2.0, -1.0, 1.0)
    if name == "tiny":
        return dict(domain=DOMAIN, ncx=2, ncy=2, n_global=1, steps=[("box", -5.0, 5.0, -5.0, 5.0), ("box", -2.0, 2.0, -3.0, 1.0)])
    if name == "small":
        return dict(domain=DOMAIN, ncx=4, ncy=4, n_global=3, steps=[box, box])
    if name == "apply":
        return dict(domain=DOMAIN, ncx=16, ncy=16, n_global=6, steps=[box, box])
    if name == "solve":
        return dict(domain=DOMAIN, ncx=16, ncy=16, n_global=5, steps=[_band(16, 5, 7)] * 7)
    if name == "adjoint":
        return dict(domain=DOMAIN, ncx=4, ncy=4, n_global=5, steps=[box, box])
    if name == "large":
        return dict(domain=DOMAIN, ncx=14, ncy=14, n_global=6, steps=[_band(14, 6, 9)] * 9)
    if name == "table2_0":
        return dict(domain=DOMAIN, ncx=10, ncy=10, n_global=2, steps=[])
    if name.startswith("box"):  # box<ncx>_<global>_<steps>: box |x|<=2, |y|<=1 refined <steps> times
        a, b, c = name[3:].split("_")
        return dict(domain=DOMAIN, ncx=int(a), ncy=int(a), n_global=int(b), steps=[box] * int(c))
    if name.startswith("band"):  # band<ncx>_<global>_<steps>, e.g. band4_2_3
        a, b, c = name[4:].split("_")
        ncx, g, s = int(a), int(b), int(c)
        return dict(domain=DOMAIN, ncx=ncx, ncy=ncx, n_global=g, steps=[_band(ncx, g, s)] * s)
    raise KeyError(name)


def material(name="sneddon", h_min=None):
    """Table 1 material with the workload's kappa and PDAS constant."""
    m = dict(E=1.0, nu=0.2, Gc=1.0, p=1e-3, kappa=1e-10, c=1e4)
    if h_min is not None:
        m["eps"] = 2.0 * h_min
    return m


def canonical_order(X, Y):
    """Permutation that lists nodes in ascending (Y, X)."""
    return np.lexsort((np.asarray(X), np.asarray(Y)))


def canonical_cell_order(level, i, j):
    return np.lexsort((np.asarray(i), np.asarray(j), np.asarray(level)))


def _scatter(values_canonical, order):
    out = np.empty_like(values_canonical)
    out[order] = values_canonical
    return out


def linearisation(X, Y, Xmax, Ymax, seed=0, u_std=1e-3):
    """Random linearisation point: phi, phi_tilde ~ U[0,1], u ~ N(0, u_std^2).

    u is set to 0 on boundary nodes (the discrete space has u = 0 there).
    Returns u (n, 2), phi (n,), phi_tilde (n,) in the caller's node order.
    """
    X = np.asarray(X)
    Y = np.asarray(Y)
    n = X.size
    order = canonical_order(X, Y)
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = rng.uniform(0.0, 1.0, n)
    phit = rng.uniform(0.0, 1.0, n)
    u = rng.normal(0.0, u_std, (n, 2))
    Xc, Yc = X[order], Y[order]
    bd = (Xc == 0) | (Xc == Xmax) | (Yc == 0) | (Yc == Ymax)
    u[bd] = 0.0
    return _scatter(u, order), _scatter(phi, order), _scatter(phit, order)


def vector(X, Y, seed=1, ncomp=3):
    """Random input vector ~ N(0, 1), (n, ncomp) in the caller's node order."""
    X = np.asarray(X)
    order = canonical_order(X, Y)
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(0.0, 1.0, (X.size, ncomp))
    return _scatter(v, order)


def cell_modulus(level, i, j, seed=1, sigma_log=0.1):
    """Per-cell Young's modulus, lognormal with mean 1 (mu_log = -sigma^2/2)."""
    order = canonical_cell_order(level, i, j)
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.lognormal(-0.5 * sigma_log ** 2, sigma_log, np.asarray(level).size)
    return _scatter(e, order)


def crack_phi_old(x, y, h_min, half_length=1.0):
    """Initial crack of Sec. 4: phi_old = 0 where |x| <= l0 and |y| <= h_min, else 1."""
    x = np.asarray(x)
    y = np.asarray(y)
    return np.where((np.abs(x) <= half_length) & (np.abs(y) <= h_min), 0.0, 1.0)


def node_xy(X, Y, Xmax, Ymax, domain=DOMAIN):
    """Physical coordinates of integer node positions (x0 + X * (x1 - x0) / Xmax)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return (domain[0] + X * ((domain[1] - domain[0]) / Xmax),
            domain[2] + Y * ((domain[3] - domain[2]) / Ymax))
