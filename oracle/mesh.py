"""Quadtree mesh, nodes and hanging-node constraints for the oracle.

Test infrastructure only (see ``oracle/__init__``).

What the paper fixes and what is read into it
---------------------------------------------
* Sec. 4: Omega = (-10, 10)^2 made of coarse quadrilaterals, some global
  refinements and then local refinements (Table 1: 2 global, 0-8 local).  The
  refined region is not stated; meshes here are described by explicit steps
  (global, "centre in box", "cell meets band").
* Sec. 3 / Fig. 1: locally refined quadrilateral meshes with hanging nodes.
  The oracle keeps a 2:1 face balance after every step (at most one level of
  difference across an edge), which gives the usual hanging nodes: for Q1 the
  midpoint of a coarse edge (weights 1/2, 1/2 of the edge ends); for Q2 the
  points at 1/4 and 3/4 of a coarse edge (weights 3/8, 3/4, -1/8 of the coarse
  edge nodes, i.e. the quadratic Lagrange values).
* Problem 1: V = H^1_0 for u (Dirichlet u = 0 on the whole boundary), W = H^1
  for phi (no Dirichlet condition).

Integer coordinates
-------------------
A cell (l, i, j) covers [x0 + i*hx_l, x0 + (i+1)*hx_l] x [...], hx_l =
(x1 - x0) / (ncx * 2**l).  Node positions are integers in units of
h_Lf / k where Lf is the finest level present: cell (l, i, j) has nodes
X = (i*k + a) * 2**(Lf - l), Y = (j*k + b) * 2**(Lf - l), a, b = 0..k.
Canonical node order: ascending (Y, X).  Canonical cell order: ascending
(level, j, i).

Pinned by tests/test_oracle_mesh.py: cell / node counts of the workload
recipes, the Table 2 count 5043 = 3 * 41^2 for the unrefined 40 x 40 mesh,
partition of unity of the constraint weights, conformity of the constrained
space (a function interpolated from the free nodes is continuous across every
hanging edge).
"""
import numpy as np

from .fe import lagrange1d


class QuadTree:
    """All cells of the tree, per level, as Python sets of (i, j)."""

    def __init__(self, x0, x1, y0, y1, ncx, ncy):
        self.x0, self.x1, self.y0, self.y1 = float(x0), float(x1), float(y0), float(y1)
        self.ncx, self.ncy = int(ncx), int(ncy)
        self.levels = [set((i, j) for j in range(self.ncy) for i in range(self.ncx))]

    # -- geometry -------------------------------------------------------
    def hx(self, l):
        return (self.x1 - self.x0) / (self.ncx * 2 ** l)

    def hy(self, l):
        return (self.y1 - self.y0) / (self.ncy * 2 ** l)

    # -- structure ------------------------------------------------------
    def _split(self, l, i, j):
        while len(self.levels) <= l + 1:
            self.levels.append(set())
        s = self.levels[l + 1]
        s.add((2 * i, 2 * j))
        s.add((2 * i + 1, 2 * j))
        s.add((2 * i, 2 * j + 1))
        s.add((2 * i + 1, 2 * j + 1))

    def is_leaf(self, l, i, j):
        return l + 1 >= len(self.levels) or (2 * i, 2 * j) not in self.levels[l + 1]

    def leaves(self):
        """Leaf cells in canonical order (level, j, i) as an int64 array (n, 3)."""
        out = []
        for l, cells in enumerate(self.levels):
            nxt = self.levels[l + 1] if l + 1 < len(self.levels) else set()
            for (i, j) in cells:
                if (2 * i, 2 * j) not in nxt:
                    out.append((l, i, j))
        a = np.array(out, dtype=np.int64).reshape(-1, 3)
        order = np.lexsort((a[:, 1], a[:, 2], a[:, 0]))
        return a[order]

    def finest_level(self):
        L = len(self.levels) - 1
        while L > 0 and not self.levels[L]:
            L -= 1
        return L

    # -- refinement -----------------------------------------------------
    def refine_global(self):
        for (l, i, j) in self.leaves():
            self._split(int(l), int(i), int(j))
        self.balance()

    def refine_marked(self, marks):
        """Refine the given leaves (iterable of (l, i, j)), then 2:1 balance."""
        for (l, i, j) in marks:
            assert self.is_leaf(l, i, j)
            self._split(int(l), int(i), int(j))
        self.balance()

    def refine_box_centres(self, bx0, bx1, by0, by1):
        """Refine every leaf whose centre lies in the closed box."""
        marks = []
        for (l, i, j) in self.leaves():
            hx, hy = self.hx(l), self.hy(l)
            xc = self.x0 + (i + 0.5) * hx
            yc = self.y0 + (j + 0.5) * hy
            if bx0 <= xc <= bx1 and by0 <= yc <= by1:
                marks.append((l, i, j))
        self.refine_marked(marks)

    def refine_band(self, bx0, bx1, by0, by1):
        """Refine every leaf whose closed cell meets the closed box."""
        marks = []
        for (l, i, j) in self.leaves():
            hx, hy = self.hx(l), self.hy(l)
            xa = self.x0 + i * hx
            xb = self.x0 + (i + 1) * hx
            ya = self.y0 + j * hy
            yb = self.y0 + (j + 1) * hy
            if xa <= bx1 and xb >= bx0 and ya <= by1 and yb >= by0:
                marks.append((l, i, j))
        self.refine_marked(marks)

    def balance(self):
        """2:1 face balance: a face neighbour of a level-m cell must exist at level m-1.

        Walks levels from fine to coarse; creating a missing cell refines its
        leaf ancestor down to the needed level (new cells are coarser than m,
        so they are checked when their level is reached).
        """
        for m in range(len(self.levels) - 1, 1, -1):
            nxm, nym = self.ncx << m, self.ncy << m
            for (i, j) in list(self.levels[m]):
                for (ni, nj) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                    if not (0 <= ni < nxm and 0 <= nj < nym):
                        continue
                    pi, pj = ni >> 1, nj >> 1
                    if (pi, pj) not in self.levels[m - 1]:
                        self._ensure(m - 1, pi, pj)

    def _ensure(self, l, i, j):
        chain = []
        while (i, j) not in self.levels[l]:
            chain.append((l, i, j))
            l, i, j = l - 1, i >> 1, j >> 1
        for (cl, ci, cj) in reversed(chain):
            self._split(cl - 1, ci >> 1, cj >> 1)


def build_recipe(recipe):
    """Build a QuadTree from a recipe dict (see synthetic.py)."""
    d = recipe["domain"]
    t = QuadTree(d[0], d[1], d[2], d[3], recipe["ncx"], recipe["ncy"])
    for _ in range(recipe["n_global"]):
        t.refine_global()
    for step in recipe["steps"]:
        kind, box = step[0], step[1:]
        if kind == "box":
            t.refine_box_centres(*box)
        elif kind == "band":
            t.refine_band(*box)
        else:
            raise ValueError(kind)
    return t


class LeafMesh:
    """Q_k nodes, hanging constraints and Dirichlet nodes of the leaf mesh.

    Attributes
    ----------
    cells      (nc, 3) leaf cells (level, i, j), canonical order
    cell_nodes (nc, (k+1)^2) node indices (local index a + (k+1) b)
    X, Y       (nn,) integer node coordinates (units h_Lf / k), canonical order
    hanging    dict node -> list of (parent node, weight)
    dirichlet  (nn,) bool, node on the boundary of Omega
    C          (nn, nn) scipy CSR: x_full = C @ x; identity rows for ordinary
               nodes, weight rows for hanging nodes (column of a hanging node
               is empty, so its own value is ignored)
    """

    def __init__(self, tree, k):
        import scipy.sparse as sp

        self.tree = tree
        self.k = k
        self.Lf = tree.finest_level()
        cells = tree.leaves()
        self.cells = cells
        l, ci, cj = cells[:, 0], cells[:, 1], cells[:, 2]
        s = np.left_shift(1, self.Lf - l)
        nb = (k + 1) ** 2
        Xc = np.empty((len(cells), nb), dtype=np.int64)
        Yc = np.empty((len(cells), nb), dtype=np.int64)
        for b in range(k + 1):
            for a in range(k + 1):
                A = a + (k + 1) * b
                Xc[:, A] = (ci * k + a) * s
                Yc[:, A] = (cj * k + b) * s
        self.Xmax = tree.ncx * k * (1 << self.Lf)
        self.Ymax = tree.ncy * k * (1 << self.Lf)
        key = Yc * (self.Xmax + 1) + Xc
        ukey, inv = np.unique(key.ravel(), return_inverse=True)
        self.key = ukey
        self.cell_nodes = inv.reshape(len(cells), nb)
        self.X = ukey % (self.Xmax + 1)
        self.Y = ukey // (self.Xmax + 1)
        nn = len(ukey)
        self.nn = nn
        self.dirichlet = (self.X == 0) | (self.X == self.Xmax) | (self.Y == 0) | (self.Y == self.Ymax)

        # hanging nodes: candidates strictly inside a leaf edge, between its own nodes
        t_h = (2 * np.arange(k) + 1) / (2.0 * k)
        Lh, _ = lagrange1d(k, t_h)  # Lh[b, a]: weight of edge node b at candidate a
        self.hanging = {}
        coarse = s >= 2
        rows, cols, vals = [], [], []
        for e in range(4):
            for a in range(k):
                half = (2 * a + 1) * s // 2
                if e == 0:   # bottom edge, along x
                    hx_, hy_ = ci * k * s + half, cj * k * s
                    own = [(bb, 0) for bb in range(k + 1)]
                elif e == 1:  # top edge
                    hx_, hy_ = ci * k * s + half, (cj + 1) * k * s
                    own = [(bb, k) for bb in range(k + 1)]
                elif e == 2:  # left edge, along y
                    hx_, hy_ = ci * k * s, cj * k * s + half
                    own = [(0, bb) for bb in range(k + 1)]
                else:         # right edge
                    hx_, hy_ = (ci + 1) * k * s, cj * k * s + half
                    own = [(k, bb) for bb in range(k + 1)]
                hkey = hy_ * (self.Xmax + 1) + hx_
                pos = np.searchsorted(ukey, hkey)
                pos = np.minimum(pos, nn - 1)
                found = coarse & (ukey[pos] == hkey)
                for c in np.nonzero(found)[0]:
                    h = int(pos[c])
                    plist = []
                    for bb, (pa, pb) in enumerate(own):
                        par = int(self.cell_nodes[c, pa + (k + 1) * pb])
                        plist.append((par, float(Lh[bb, a])))
                    assert h not in self.hanging, "hanging node found twice"
                    self.hanging[h] = plist
        # constraint matrix; chains (a parent that is itself hanging) are closed
        # transitively, although 2:1 balanced 2D meshes do not produce them
        def resolve(n):
            if n not in self.hanging:
                return {n: 1.0}
            acc = {}
            for p, w in self.hanging[n]:
                for q, v in resolve(p).items():
                    acc[q] = acc.get(q, 0.0) + w * v
            return acc
        self.hanging_closed = {h: resolve(h) for h in self.hanging}
        is_h = np.zeros(nn, dtype=bool)
        is_h[list(self.hanging.keys())] = True
        self.is_hanging = is_h
        ordinary = np.nonzero(~is_h)[0]
        rows.extend(ordinary.tolist())
        cols.extend(ordinary.tolist())
        vals.extend([1.0] * len(ordinary))
        for h, dct in self.hanging_closed.items():
            for p, w in dct.items():
                if w != 0.0:
                    rows.append(h)
                    cols.append(p)
                    vals.append(w)
        self.C = sp.csr_matrix((vals, (rows, cols)), shape=(nn, nn))

    # -- geometry helpers ----------------------------------------------
    def node_xy(self):
        sx = (self.tree.x1 - self.tree.x0) / self.Xmax
        sy = (self.tree.y1 - self.tree.y0) / self.Ymax
        return self.tree.x0 + self.X * sx, self.tree.y0 + self.Y * sy

    def h_min_diag(self):
        return float(np.hypot(self.tree.hx(self.Lf), self.tree.hy(self.Lf)))
