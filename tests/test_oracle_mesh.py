"""Pins of the oracle quadtree, nodes and hanging constraints (oracle/mesh.py)."""
import os

import numpy as np
import pytest

from oracle.fe import lagrange1d
from oracle.mesh import LeafMesh, QuadTree, build_recipe
import synthetic as synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table2():
    rows = []
    with open(os.path.join(GOLDEN, "table2.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_table2_unrefined_mesh_dofs():
    """Table 2, first row: h = 0.7071 (cell side 0.5 on (-10,10)^2) has 5043 DoFs = 3 * 41^2."""
    t2 = table2()
    m = LeafMesh(build_recipe(synth.recipe("table2_0")), 1)
    assert 3 * m.nn == int(t2[0, 1])
    assert abs(m.h_min_diag() - t2[0, 0]) < 1e-4
    assert len(m.hanging) == 0


@pytest.mark.parametrize("name,cells,nodes", [("small", 1336, 1431), ("adjoint", 21292, 21667)])
def test_recipe_counts(name, cells, nodes):
    m = LeafMesh(build_recipe(synth.recipe(name)), 1)
    assert len(m.cells) == cells
    assert m.nn == nodes


def _leaf_level_map(tree):
    """Level of the leaf covering each finest-level cell (brute force)."""
    L = tree.finest_level()
    nx, ny = tree.ncx << L, tree.ncy << L
    lev = -np.ones((nx, ny), dtype=int)
    for (l, i, j) in tree.leaves():
        s = 1 << (L - l)
        lev[i * s:(i + 1) * s, j * s:(j + 1) * s] = l
    return lev


@pytest.mark.parametrize("name", ["tiny", "small", "band4_2_4"])
def test_face_balance_and_cover(name):
    tree = build_recipe(synth.recipe(name))
    lev = _leaf_level_map(tree)
    assert (lev >= 0).all()                      # leaves tile the domain
    assert np.abs(np.diff(lev, axis=0)).max() <= 1   # across vertical edges
    assert np.abs(np.diff(lev, axis=1)).max() <= 1   # across horizontal edges
    cells = tree.leaves()
    area = sum(tree.hx(l) * tree.hy(l) for (l, i, j) in cells)
    assert abs(area - 400.0) < 1e-9


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("name", ["tiny", "small"])
def test_constraints_conforming(name, k):
    """Constraint weights sum to one, and a function given by its free nodal values
    (hanging values from C) is continuous across every hanging edge: evaluated from
    the coarse cell and from the fine cells at points of the shared edge."""
    m = LeafMesh(build_recipe(synth.recipe(name)), k)
    assert len(m.hanging) > 0
    for h, plist in m.hanging.items():
        assert abs(sum(w for _, w in plist) - 1.0) < 1e-14
        assert len(plist) == k + 1
    rng = np.random.default_rng(3)
    f = m.C @ rng.normal(size=m.nn)
    # edge points: every cell edge sampled at t; evaluate trace from each cell that owns it
    key = {}
    Lf = m.Lf
    ts = np.array([0.1, 0.3, 0.55, 0.8])
    Lt, _ = lagrange1d(k, ts)
    for c, (l, i, j) in enumerate(m.cells):
        s = 1 << (Lf - l)
        nodes = m.cell_nodes[c].reshape(k + 1, k + 1)  # [b, a]
        edges = {
            ("h", j * s, i * s, (i + 1) * s): nodes[0, :],
            ("h", (j + 1) * s, i * s, (i + 1) * s): nodes[k, :],
            ("v", i * s, j * s, (j + 1) * s): nodes[:, 0],
            ("v", (i + 1) * s, j * s, (j + 1) * s): nodes[:, k],
        }
        for (o, fixc, a0, a1), en in edges.items():
            vals = Lt.T @ f[en]
            pos = a0 + ts * (a1 - a0)
            for p, v in zip(pos, vals):
                key.setdefault((o, fixc, round(p * 64)), []).append(v)
    nshared = 0
    for vs in key.values():
        if len(vs) > 1:
            nshared += 1
            assert max(vs) - min(vs) < 1e-12
    assert nshared > 0
