"""Pins of the level active sets of the oracle multigrid (oracle/mg.py,
MG.level_active; paper Sec. 3.2, last paragraph: a DoF is inactive on a level
only if all its neighbours are inactive).

The reading under test: a level-l node is active if the leaf node at its
position is active, or, unless l is the node's home level (the coarsest level
among its leaf cells), if its level-l basis function is nonzero at an active
node of level l+1.  The pins:

* construction: the sets equal those built here from the level basis functions
  themselves (1D Lagrange products on the level-l cells, evaluated at level-(l+1)
  node positions), with home levels read off the leaf cells; nothing of the
  oracle's prolongation matrices or node maps is used;
* coverage: every free leaf phi DoF is interior (neither active nor on the
  refinement edge) on its home level, so the V-cycle corrects it;
* consistency: with the active set inside a region of one refinement level, away
  from its edges, every level-interior basis function vanishes at every active
  leaf node, and the V-cycle equals the multiplicative subspace correction on the
  free DoFs (constant coefficients: Galerkin level operators).  No exact identity
  holds when an active node lies within the support of a coarser level function
  whose node is on its home level: that DoF keeps its leaf state there, so its
  level function reaches the active node while the leaf operator does not see it.

Planted mistakes in copies of the rule (no pessimistic coarsening; coarsening on
home levels too; children taken from the wrong level) fail these pins.
"""
import numpy as np
import pytest

from oracle import mg
from oracle import operators as ops
from oracle.mesh import LeafMesh, build_recipe
import synthetic as synth


def lag(k, a, t):
    """1D Lagrange basis polynomial a on the equispaced nodes 0, 1/k, .., 1 at t."""
    v = 1.0
    for m in range(k + 1):
        if m != a:
            v *= (t - m / k) / (a / k - m / k)
    return v


class Geometry:
    """Level node sets, home levels and level basis functions from the quadtree alone."""

    def __init__(self, leaf):
        self.leaf, self.tree, self.k, self.Lf = leaf, leaf.tree, leaf.k, leaf.Lf
        k = self.k
        self.home = {}
        for (l, i, j) in leaf.cells:
            s = 1 << (self.Lf - int(l))
            for b in range(k + 1):
                for a in range(k + 1):
                    p = ((int(i) * k + a) * s, (int(j) * k + b) * s)
                    self.home[p] = min(self.home.get(p, 99), int(l))
        self.hanging = {(int(x), int(y)) for x, y, h in zip(leaf.X, leaf.Y, leaf.is_hanging) if h}

    def nodes(self, l):
        k, s = self.k, 1 << (self.Lf - l)
        pts = set()
        for (i, j) in self.tree.levels[l]:
            for b in range(k + 1):
                for a in range(k + 1):
                    pts.add(((i * k + a) * s, (j * k + b) * s))
        return pts

    def phi(self, l, y, p):
        """Level-l nodal basis function of node y at point p (finest-grid integers)."""
        k, s = self.k, 1 << (self.Lf - l)
        span = k * s
        cells = self.tree.levels[l]
        for i in {p[0] // span, (p[0] - 1) // span}:
            for j in {p[1] // span, (p[1] - 1) // span}:
                if (i, j) not in cells:
                    continue
                tx, ty = (p[0] - i * span) / span, (p[1] - j * span) / span
                if not (0 <= tx <= 1 and 0 <= ty <= 1):
                    continue
                ax, ay = (y[0] - i * span), (y[1] - j * span)
                if ax % s or ay % s or not (0 <= ax // s <= k and 0 <= ay // s <= k):
                    return 0.0     # y is not a node of this cell: its function is 0 on it
                return lag(k, ax // s, tx) * lag(k, ay // s, ty)
        return 0.0

    def expected_active(self, active_pos):
        """Level active sets by the reading, finest to coarsest (sets of positions)."""
        act = {}
        for l in range(self.Lf, -1, -1):
            a = set()
            for y in self.nodes(l):
                if y in active_pos and y not in self.hanging:
                    a.add(y)
                elif l < self.Lf and (y in self.hanging or self.home.get(y) != l):
                    if any(abs(self.phi(l, y, z)) > 1e-14 for z in act[l + 1]):
                        a.add(y)
            act[l] = a
        return act


def setup(k, name, where, seed=4, frac=0.5):
    leaf = LeafMesh(build_recipe(synth.recipe(name)), k)
    x, y = leaf.node_xy()
    rng = np.random.default_rng(seed)
    active = where(x, y) & (rng.uniform(size=leaf.nn) < frac) & ~leaf.is_hanging
    assert active.any()
    mat = ops.Material(E=1.0, nu=0.2, Gc=1.0, eps=0.5, kappa=1e-10, p=1e-3)
    u = np.zeros((leaf.nn, 2))
    phi = np.ones(leaf.nn)
    return leaf, mat, u, phi, active


def positions(lm, mask):
    return {(int(a), int(b)) for a, b in zip(lm.X[mask], lm.Y[mask])}


class NoCoarsening(mg.MG):
    def level_active(self):
        return [self.active_leaf[lm.leaf_node] & ~self.leaf.is_hanging[lm.leaf_node] for lm in self.levels]


class CoarsenOnHome(mg.MG):
    def level_active(self):
        leaf, Lf = self.leaf, self.leaf.Lf
        act = [None] * (Lf + 1)
        for l in range(Lf, -1, -1):
            ln = self.levels[l].leaf_node
            a = self.active_leaf[ln] & ~leaf.is_hanging[ln]
            if l < Lf:
                a = a | ((abs(self.P[l + 1]).T @ act[l + 1].astype(np.float64)) > 0)
            act[l] = a
        return act


class WrongLevel(mg.MG):
    def level_active(self):
        leaf, Lf = self.leaf, self.leaf.Lf
        act = [None] * (Lf + 1)
        for l in range(Lf, -1, -1):
            ln = self.levels[l].leaf_node
            a = self.active_leaf[ln] & ~leaf.is_hanging[ln]
            if 0 < l:     # children taken from the coarser level's leaf state (a misindexed recursion)
                lc = self.levels[l - 1]
                ca = self.active_leaf[lc.leaf_node] & ~leaf.is_hanging[lc.leaf_node]
                home = (self.lmin[ln] == l) & ~leaf.is_hanging[ln]
                a = a | (((abs(self.P[l]) @ ca.astype(np.float64)) > 0) & ~home)
            act[l] = a
        return act


def construction_matches(M, geo, active_pos):
    exp = geo.expected_active(active_pos)
    return all(positions(lm, M.act[l]) == exp[l] for l, lm in enumerate(M.levels))


def coverage_holds(M):
    leaf = M.leaf
    for l, lm in enumerate(M.levels):
        nodes, idx = M.copy_idx[l]
        free = ~M.active_leaf[nodes]
        if np.any(M.act[l][idx[free]] | lm.edge[idx[free]]):
            return False
    return True


def vanishing_holds(M, geo, active_pos):
    for l, lm in enumerate(M.levels):
        interior = ~M.act[l] & ~lm.edge
        for y in positions(lm, interior):
            if any(abs(geo.phi(l, y, z)) > 1e-14 for z in active_pos):
                return False
    return True


def vcycle_error(M, leaf, mat, u, phi, active):
    st = ops.State(leaf, u, phi, phi)
    Gt = ops.constrained_operator(leaf, ops.assemble_jacobian(leaf, mat, st), active)
    nn = leaf.nn
    A = Gt[2 * nn:, 2 * nn:]
    free = ~active & ~leaf.is_hanging
    r = np.random.default_rng(7).normal(size=nn)
    z = M.vcycle("pp", r)
    e = M.msc("pp", A, r)
    return np.abs(z[free] - e[free]).max() / np.abs(e[free]).max()


def inner(x, y):
    return (np.abs(x) <= 0.7) & (np.abs(y) <= 0.3)


def scattered(x, y):
    return np.ones_like(x, dtype=bool)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("name,where", [("small", inner), ("small", scattered), ("band4_2_4", scattered)])
def test_level_active_sets_follow_the_reading(k, name, where):
    leaf, mat, u, phi, active = setup(k, name, where, frac=0.5 if where is inner else 0.1)
    M = mg.MG(leaf, mat, u, phi, phi, active, blocks=("pp",))
    geo = Geometry(leaf)
    act_pos = {(int(a), int(b)) for a, b in zip(leaf.X[active], leaf.Y[active])}
    assert construction_matches(M, geo, act_pos)
    assert coverage_holds(M)


@pytest.mark.parametrize("k", [1, 2])
def test_interior_active_set_keeps_the_subspace_correction(k):
    leaf, mat, u, phi, active = setup(k, "small", inner)
    M = mg.MG(leaf, mat, u, phi, phi, active, blocks=("pp",))
    geo = Geometry(leaf)
    act_pos = {(int(a), int(b)) for a, b in zip(leaf.X[active], leaf.Y[active])}
    assert vanishing_holds(M, geo, act_pos)
    assert vcycle_error(M, leaf, mat, u, phi, active) < 1e-11


@pytest.mark.parametrize("wrong", [NoCoarsening, CoarsenOnHome, WrongLevel])
def test_planted_level_rule_mistakes_fail(wrong):
    """Each planted mistake fails the independent construction, and also one of the
    properties (coverage, vanishing, subspace-correction identity) on its own."""
    k = 1
    construction, properties = True, True
    for name, where, frac in (("small", inner, 0.5), ("band4_2_4", scattered, 0.1)):
        leaf, mat, u, phi, active = setup(k, name, where, frac=frac)
        geo = Geometry(leaf)
        act_pos = {(int(a), int(b)) for a, b in zip(leaf.X[active], leaf.Y[active])}
        M = wrong(leaf, mat, u, phi, phi, active, blocks=("pp",))
        construction = construction and construction_matches(M, geo, act_pos)
        properties = properties and coverage_holds(M)
        if where is inner:
            properties = properties and vanishing_holds(M, geo, act_pos) and \
                vcycle_error(M, leaf, mat, u, phi, active) < 1e-11
    assert not construction
    assert not properties
