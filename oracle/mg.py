"""Geometric multigrid with local smoothing for the diagonal blocks (oracle).

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 3.2: the preconditioner applies one V-cycle to each diagonal block
of the Jacobian (u-u and phi-phi); the smoother is Chebyshev-accelerated
Jacobi, needing the inverse diagonal and an estimate of the largest eigenvalue
obtained by conjugate gradients; the smoothing range is [0.08, 1.2] * lambda_max
on the levels above 0; local smoothing acts only on the cells refined to the
current level (no hanging nodes on a level); Dirichlet conditions go to the
levels canonically; a DoF is inactive on a level only if all its neighbours are.

Readings where the paper is silent:
* level mesh l = all cells of refinement level l (leaf or refined); its
  refinement edge E_l = level nodes that touch a leaf cell of level < l;
* level linearisation = injection of the (constraint-resolved) leaf nodal
  values; per-cell modulus of a refined cell = mean of its four children;
* level active set: level-l nodes that coincide with an active leaf node, or
  that are not on their home level (the coarsest level among the node's leaf
  cells; hanging positions have none) and interpolate onto an active node of
  level l+1 (pessimistic coarsening); on its home level a DoF keeps its leaf
  state, since it is smoothed on no other level;
* Chebyshev: textbook three-term recurrence for D^-1 A on [a, b];
  lambda_max: largest Ritz value of 12 steps of Jacobi-preconditioned CG from a
  fixed start vector 1 + 0.01 * (splitmix64(key) mod 1000) / 1000;
* coarse level: direct FP64 solve (the paper iterates there);
* V-cycle bookkeeping: leaf defect copied to the coarsest level on which the
  node is interior; down sweep smooths, forms the defect on interior AND edge
  rows (edge rows: the finer-level contributions restricted there so far minus
  the operator row), restricts; up sweep prolongates onto all level nodes and
  post-smooths with the same polynomial; the result is read back on the same
  levels.  With Galerkin level operators this is exactly the multiplicative
  subspace correction over the level spaces V_l^0 (pinned by
  tests/test_oracle_mg.py against that definition computed independently).

Pinned: Chebyshev error polynomial on a diagonal operator; Ritz value bounds;
V-cycle == multiplicative subspace correction (constant coefficients), also
with an active set inside a single-level region; the level active sets ==
their construction from level basis functions evaluated geometrically, every
free leaf DoF interior on its home level, and every level-interior function
zero on the active leaf nodes in that setting;
symmetry of the V-cycle; the variable-coefficient level blocks == the Jacobian
blocks of a uniform mesh built on its own (own numbering and coordinates) with
the same nodal values: of the whole level on globally refined levels, and of
the level's cells within their bounding rectangle on locally refined ones; the
prolongation reproduces every x^a y^b with a, b <= k exactly.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import operators as ops
from .fe import lagrange1d

M64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on a Python int."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def lanczos_start(gx, gy):
    """Deterministic start vector entry for level-grid node (gx, gy)."""
    h = splitmix64((int(gx) << 32) | int(gy))
    return 1.0 + 0.01 * (h % 1000) / 1000.0


class LevelMesh:
    """All cells of one refinement level, with the attributes operators.* read."""

    def __init__(self, leaf, level):
        tree, k, Lf = leaf.tree, leaf.k, leaf.Lf
        self.tree, self.k, self.Lf, self.level = tree, k, Lf, level
        cl = sorted(tree.levels[level], key=lambda c: (c[1], c[0]))
        self.cells = np.array([(level, i, j) for (i, j) in cl], dtype=np.int64).reshape(-1, 3)
        s = 1 << (Lf - level)
        self.s = s
        nb = (k + 1) ** 2
        Xc = np.empty((len(cl), nb), dtype=np.int64)
        Yc = np.empty((len(cl), nb), dtype=np.int64)
        ci, cj = self.cells[:, 1], self.cells[:, 2]
        for b in range(k + 1):
            for a in range(k + 1):
                Xc[:, a + (k + 1) * b] = (ci * k + a) * s
                Yc[:, a + (k + 1) * b] = (cj * k + b) * s
        self.Xmax, self.Ymax = leaf.Xmax, leaf.Ymax
        key = Yc * (self.Xmax + 1) + Xc
        ukey, inv = np.unique(key.ravel(), return_inverse=True)
        self.key = ukey
        self.cell_nodes = inv.reshape(len(cl), nb)
        self.X = ukey % (self.Xmax + 1)
        self.Y = ukey // (self.Xmax + 1)
        self.nn = len(ukey)
        self.C = sp.identity(self.nn, format="csr")
        self.dirichlet = (self.X == 0) | (self.X == self.Xmax) | (self.Y == 0) | (self.Y == self.Ymax)
        # refinement edge: a level-l cell whose closure holds the node is missing
        cellset = tree.levels[level]
        nx, ny = tree.ncx << level, tree.ncy << level
        gx, gy = self.X // s, self.Y // s
        self.gx, self.gy = gx, gy
        edge = np.zeros(self.nn, dtype=bool)
        for n in range(self.nn):
            cx = [gx[n] // k - 1, gx[n] // k] if gx[n] % k == 0 else [gx[n] // k]
            cy = [gy[n] // k - 1, gy[n] // k] if gy[n] % k == 0 else [gy[n] // k]
            for a in cx:
                for b in cy:
                    if 0 <= a < nx and 0 <= b < ny and (a, b) not in cellset:
                        edge[n] = True
        self.edge = edge

    def find(self, X, Y):
        kk = np.asarray(Y, dtype=np.int64) * (self.Xmax + 1) + np.asarray(X, dtype=np.int64)
        pos = np.searchsorted(self.key, kk)
        pos = np.minimum(pos, self.nn - 1)
        ok = self.key[pos] == kk
        return np.where(ok, pos, -1)


def level_cell_modulus(leaf, E_leaf, level_mesh):
    """Per-cell modulus on a level: leaf value, or mean of the four children."""
    tree = leaf.tree
    val = {}
    for c, (l, i, j) in enumerate(leaf.cells):
        val[(int(l), int(i), int(j))] = float(E_leaf[c])
    for l in range(len(tree.levels) - 2, -1, -1):
        for (i, j) in tree.levels[l]:
            if (l, i, j) not in val:
                val[(l, i, j)] = 0.25 * sum(val[(l + 1, 2 * i + a, 2 * j + b)] for a in (0, 1) for b in (0, 1))
    return np.array([val[(int(l), int(i), int(j))] for (l, i, j) in level_mesh.cells])


def prolongation(fine, coarse):
    """Nodal interpolation of the coarse Q_k field at the fine level nodes (CSR, fine x coarse)."""
    k = fine.k
    span = k * coarse.s   # coarse cell width in finest node units
    nxc = fine.tree.ncx << coarse.level
    nyc = fine.tree.ncy << coarse.level
    rows, cols, vals = [], [], []
    for n in range(fine.nn):
        X, Y = int(fine.X[n]), int(fine.Y[n])
        cx = min(X // span, nxc - 1)
        cy = min(Y // span, nyc - 1)
        tx = (X - cx * span) / span
        ty = (Y - cy * span) / span
        Lx, _ = lagrange1d(k, np.array([tx]))
        Ly, _ = lagrange1d(k, np.array([ty]))
        for b in range(k + 1):
            for a in range(k + 1):
                w = Lx[a, 0] * Ly[b, 0]
                if abs(w) < 1e-15:
                    continue
                cn = coarse.find((cx * k + a) * coarse.s, (cy * k + b) * coarse.s)
                assert cn >= 0
                rows.append(n)
                cols.append(int(cn))
                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.nn, coarse.nn))


def block_matrices(lm, mat, st):
    """Assembled level blocks A_uu (2N x 2N, index comp*N + node) and A_pp (N x N)."""
    nn = lm.nn
    G = ops.assemble_jacobian(lm, mat, st)
    Auu = G[:2 * nn, :2 * nn].tocsr()
    App = G[2 * nn:, 2 * nn:].tocsr()
    return Auu, App


def chebyshev(apply_A, dinv, d, lam, degree, lo=0.08, hi=1.2, x0=None):
    """Chebyshev-Jacobi smoothing of A x = d on [lo*lam, hi*lam] for D^-1 A.

    Textbook three-term recurrence: theta = (b+a)/2, delta = (b-a)/2,
    sigma = theta/delta; x1 = x0 + D^-1 r0 / theta; then
    rho_j = 1/(2 sigma - rho_{j-1}), x_{j+1} = x_j + rho_j rho_{j-1} (x_j - x_{j-1})
    + (2 rho_j / delta) D^-1 (d - A x_j).  `degree` applications of D^-1.
    """
    a, b = lo * lam, hi * lam
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    x = np.zeros_like(d) if x0 is None else x0.copy()
    r = d - apply_A(x) if x0 is not None else d.copy()
    x_prev = x.copy()
    x = x + dinv * r / theta
    rho = 1.0 / sigma
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        r = d - apply_A(x)
        x_new = x + rho_new * rho * (x - x_prev) + (2.0 * rho_new / delta) * dinv * r
        x_prev, x = x, x_new
        rho = rho_new
    return x


def ritz_extremes_cg(apply_A, dinv, b, steps=12):
    """(smallest, largest) Ritz value of `steps` Jacobi-preconditioned CG steps from residual b."""
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    if rz <= 0:
        return 0.0, 0.0
    for _ in range(steps):
        q = apply_A(p)
        pq = float(p @ q)
        if pq <= 0:
            break
        alpha = rz / pq
        r = r - alpha * q
        z = dinv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        if rz_new <= 1e-300:
            break
        p = z + beta * p
        rz = rz_new
    m = len(alphas)
    if m == 0:
        return 0.0, 0.0
    diag = np.array([1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0) for j in range(m)])
    off = np.array([np.sqrt(betas[j]) / alphas[j] for j in range(m - 1)])
    ev = sla.eigh_tridiagonal(diag, off, eigvals_only=True)
    return float(ev.min()), float(ev.max())


def coarse_chebyshev_degree(a, b, tol=1e-3, cap=64):
    """Smallest degree m with 1 / T_m((b + a) / (b - a)) <= tol (Chebyshev error bound on [a, b])."""
    sigma = (b + a) / (b - a)
    for m in range(1, cap + 1):
        if 1.0 / np.cosh(m * np.arccosh(sigma)) <= tol:
            return m
    return cap


def lambda_max_cg(apply_A, dinv, b, steps=12):
    """Largest Ritz value of `steps` Jacobi-preconditioned CG steps from residual b."""
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    if rz <= 0:
        return 0.0
    for _ in range(steps):
        q = apply_A(p)
        pq = float(p @ q)
        if pq <= 0:
            break
        alpha = rz / pq
        r = r - alpha * q
        z = dinv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        if rz_new <= 1e-300:
            break
        p = z + beta * p
        rz = rz_new
    m = len(alphas)
    if m == 0:
        return 0.0
    diag = np.array([1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0) for j in range(m)])
    off = np.array([np.sqrt(betas[j]) / alphas[j] for j in range(m - 1)])
    ev = sla.eigh_tridiagonal(diag, off, eigvals_only=True)
    return float(ev.max())


class Block:
    """One diagonal block (u-u: ncomp 2, phi-phi: ncomp 1) on one level."""

    def __init__(self, lm, A, fixed_nodes, ncomp):
        self.lm, self.A, self.ncomp = lm, A, ncomp
        nn = lm.nn
        fixed = np.tile(fixed_nodes, ncomp)
        edge = np.tile(lm.edge, ncomp)
        self.fixed = fixed
        self.edge = edge
        self.interior = ~fixed & ~edge
        dg = A.diagonal()
        self.dinv = np.where(self.interior, 1.0 / np.where(dg != 0, dg, 1.0), 0.0)
        self.free_mask = (~fixed).astype(np.float64)

    def apply(self, x):
        """A x with fixed columns masked; fixed rows 0."""
        return self.free_mask * (self.A @ (self.free_mask * x))


class MG:
    """Block-diagonal local-smoothing V-cycles at a linearisation point."""

    def __init__(self, leaf, mat, u, phi, phit, active, E_cells=None, degree=3, lanczos_steps=12,
                 smooth=(0.08, 1.2), blocks=("uu", "pp"), coarse="direct"):
        """coarse: "direct" (dense Cholesky of the level-0 block) or "chebyshev" (Sec. 3.2:
        Chebyshev-Jacobi on level 0 over [0.9 lambda_min, 1.2 lambda_max] of the Ritz values of the
        same CG run, degree from coarse_chebyshev_degree)."""
        self.leaf, self.mat, self.degree, self.smooth = leaf, mat, degree, smooth
        self.coarse = coarse
        Lf = leaf.Lf
        C = leaf.C
        uf = np.stack([C @ u[:, 0], C @ u[:, 1]], 1)
        pf, ptf = C @ phi, C @ phit
        self.active_leaf = np.asarray(active, dtype=bool)
        self.levels = [LevelMesh(leaf, l) for l in range(Lf + 1)]
        self.P = [None] + [prolongation(self.levels[l], self.levels[l - 1]) for l in range(1, Lf + 1)]
        # level linearisation: injection of leaf nodal values
        lin = []
        for lm in self.levels:
            ln = np.searchsorted(leaf.key, lm.key)
            assert np.all(leaf.key[ln] == lm.key)
            lm.leaf_node = ln
            Ec = None if E_cells is None else level_cell_modulus(leaf, E_cells, lm)
            lin.append(ops.State(lm, uf[ln], pf[ln], ptf[ln], Ec))
        # copy map: leaf node -> coarsest level among its leaf cells ("home" level)
        lmin = np.full(leaf.nn, 10 ** 6)
        for c, (l, i, j) in enumerate(leaf.cells):
            lmin[leaf.cell_nodes[c]] = np.minimum(lmin[leaf.cell_nodes[c]], l)
        self.lmin = lmin
        self.act = self.level_active()
        self.copy_idx = {}
        for l, lm in enumerate(self.levels):
            nodes = np.nonzero((lmin == l) & ~leaf.is_hanging)[0]
            idx = lm.find(leaf.X[nodes], leaf.Y[nodes])
            assert np.all(idx >= 0)
            self.copy_idx[l] = (nodes, idx)
        # blocks per level
        self.B = {}
        for name in blocks:
            bl = []
            for l, lm in enumerate(self.levels):
                Auu, App = block_matrices(lm, mat, lin[l])
                if name == "uu":
                    bl.append(Block(lm, Auu, lm.dirichlet, 2))
                else:
                    bl.append(Block(lm, App, self.act[l], 1))
            for l, blk in enumerate(bl):
                if l == 0:
                    blk.lam = None
                    continue
                lm = blk.lm
                start = np.array([lanczos_start(gx, gy) for gx, gy in zip(lm.gx // 1, lm.gy // 1)])
                # level-grid coordinates in units of h_l / k
                start = np.tile(start, blk.ncomp) * blk.interior
                blk.lam = lambda_max_cg(blk.apply, blk.dinv, start, lanczos_steps) if blk.interior.any() else 0.0
            # coarse solve on interior DoFs of level 0 (E_0 is empty)
            b0 = bl[0]
            if coarse == "chebyshev":
                lm = b0.lm
                start = np.array([lanczos_start(gx, gy) for gx, gy in zip(lm.gx // 1, lm.gy // 1)])
                start = np.tile(start, b0.ncomp) * b0.interior
                lo, hi = ritz_extremes_cg(b0.apply, b0.dinv, start, lanczos_steps) if b0.interior.any() \
                    else (0.0, 0.0)
                b0.cheb = (0.9 * lo, 1.2 * hi, coarse_chebyshev_degree(0.9 * lo, 1.2 * hi) if hi > 0 else 0)
            I0 = np.nonzero(b0.interior)[0]
            b0.I0 = I0
            b0.A0 = b0.A[I0][:, I0].toarray() if len(I0) else np.zeros((0, 0))
            b0.cho = sla.cho_factor(b0.A0) if len(I0) else None
            self.B[name] = bl

    def level_active(self):
        """Level active sets of the phi block (Sec. 3.2, last paragraph), finest to
        coarsest: a level node is active if the leaf node at its position is
        active, or -- unless this level is the node's home level -- if it
        interpolates onto an active node of the next finer level (pessimistic
        coarsening).  On its home level a DoF keeps its own leaf state, else it
        would be smoothed on no level at all.  Hanging positions have no home."""
        leaf = self.leaf
        Lf = leaf.Lf
        act = [None] * (Lf + 1)
        for l in range(Lf, -1, -1):
            lm = self.levels[l]
            ln = lm.leaf_node
            a = self.active_leaf[ln] & ~leaf.is_hanging[ln]
            if l < Lf:
                Pf = self.P[l + 1]   # fine(l+1) x coarse(l)
                child_active = (abs(Pf).T @ act[l + 1].astype(np.float64)) > 0
                home = (self.lmin[ln] == l) & ~leaf.is_hanging[ln]
                a = a | (child_active & ~home)
            act[l] = a
        return act

    # ---- level helpers
    def _P(self, l, ncomp):
        P = self.P[l]
        return sp.block_diag([P] * ncomp, format="csr") if ncomp > 1 else P

    def _smooth(self, blk, d):
        if blk.lam is None or blk.lam <= 0:
            return np.zeros_like(d)
        return chebyshev(blk.apply, blk.dinv, d, blk.lam, self.degree, self.smooth[0], self.smooth[1])

    def vcycle(self, name, r):
        """z = MG(r) for block name ('uu': r of length 2 nn, 'pp': nn)."""
        leaf = self.leaf
        bl = self.B[name]
        nc = bl[0].ncomp
        nn = leaf.nn
        L = len(bl) - 1
        if name == "uu":
            free_leaf = ~leaf.dirichlet & ~leaf.is_hanging
        else:
            free_leaf = ~self.active_leaf & ~leaf.is_hanging
        d = [np.zeros(nc * blk.lm.nn) for blk in bl]
        for l in range(L + 1):
            nodes, idx = self.copy_idx[l]
            keep = free_leaf[nodes]
            for c in range(nc):
                d[l][c * bl[l].lm.nn + idx[keep]] = r[c * nn + nodes[keep]]
        x = [None] * (L + 1)
        for l in range(L, 0, -1):
            blk = bl[l]
            x[l] = self._smooth(blk, d[l])
            t = d[l] - blk.apply(x[l])
            t[blk.fixed] = 0.0
            d[l - 1] = d[l - 1] + self._P(l, nc).T @ t
            d[l - 1][bl[l - 1].fixed] = 0.0
        b0 = bl[0]
        x0 = np.zeros(nc * b0.lm.nn)
        if self.coarse == "chebyshev":
            a, b, m = b0.cheb
            if m > 0:
                x0 = chebyshev(b0.apply, b0.dinv, d[0], 1.0, m, a, b)
        elif len(b0.I0):
            x0[b0.I0] = sla.cho_solve(b0.cho, d[0][b0.I0])
        x[0] = x0
        for l in range(1, L + 1):
            blk = bl[l]
            x[l] = x[l] + self._P(l, nc) @ x[l - 1]
            x[l][blk.fixed] = 0.0
            res = d[l] - blk.apply(x[l])
            x[l] = x[l] + self._smooth(blk, res)
        z = np.zeros(nc * nn)
        for l in range(L + 1):
            nodes, idx = self.copy_idx[l]
            keep = free_leaf[nodes]
            for c in range(nc):
                z[c * nn + nodes[keep]] = x[l][c * bl[l].lm.nn + idx[keep]]
        fixed_leaf = ~free_leaf & ~leaf.is_hanging
        for c in range(nc):
            z[c * nn + np.nonzero(fixed_leaf)[0]] = r[c * nn + np.nonzero(fixed_leaf)[0]]
        return z

    # ---- independent reference: multiplicative subspace correction
    def interpolation_to_leaf(self, l):
        """R_l: level-l interior DoFs -> leaf free DoFs (values of the level function at leaf nodes)."""
        leaf, lm = self.leaf, self.levels[l]
        k = leaf.k
        span = k * lm.s
        cellset = leaf.tree.levels[l]
        rows, cols, vals = [], [], []
        seen = set()
        for n in range(leaf.nn):
            if leaf.is_hanging[n]:
                continue
            X, Y = int(leaf.X[n]), int(leaf.Y[n])
            cx, cy = X // span, Y // span
            cands = [(cx, cy), (cx - 1, cy), (cx, cy - 1), (cx - 1, cy - 1)]
            for (a0, b0) in cands:
                if (a0, b0) not in cellset:
                    continue
                tx, ty = (X - a0 * span) / span, (Y - b0 * span) / span
                if not (0 <= tx <= 1 and 0 <= ty <= 1):
                    continue
                Lx, _ = lagrange1d(k, np.array([tx]))
                Ly, _ = lagrange1d(k, np.array([ty]))
                for b in range(k + 1):
                    for a in range(k + 1):
                        w = Lx[a, 0] * Ly[b, 0]
                        if abs(w) < 1e-15:
                            continue
                        ln = int(lm.find((a0 * k + a) * lm.s, (b0 * k + b) * lm.s))
                        if (n, ln) in seen:
                            continue
                        seen.add((n, ln))
                        rows.append(n)
                        cols.append(ln)
                        vals.append(w)
                break
        return sp.csr_matrix((vals, (rows, cols)), shape=(leaf.nn, lm.nn))

    def msc(self, name, A_leaf, r):
        """Multiplicative subspace correction over V_L^0, ..., V_0^0 (Galerkin level
        operators R^T A R), Chebyshev smoothing with the same D and lambda, exact
        coarse solve, symmetric sweep.  A_leaf: the leaf block on free DoFs
        (rows/cols of fixed and hanging DoFs zero)."""
        leaf = self.leaf
        bl = self.B[name]
        nc = bl[0].ncomp
        L = len(bl) - 1
        R = []
        for l in range(L + 1):
            Rl = self.interpolation_to_leaf(l)
            Rl = sp.block_diag([Rl] * nc, format="csr") if nc > 1 else Rl
            Rl = Rl[:, np.nonzero(bl[l].interior)[0]]
            R.append(Rl)
        if name == "uu":
            free = np.tile(~leaf.dirichlet & ~leaf.is_hanging, 2)
        else:
            free = ~self.active_leaf & ~leaf.is_hanging
        Fm = sp.diags(free.astype(np.float64))
        A = (Fm @ A_leaf @ Fm).tocsr()
        b = r * free
        e = np.zeros_like(b)

        def smooth(l, res):
            Rl = R[l]
            Ag = (Rl.T @ A @ Rl).tocsr()
            dinv = bl[l].dinv[np.nonzero(bl[l].interior)[0]]
            if bl[l].lam is None or bl[l].lam <= 0 or Rl.shape[1] == 0:
                return np.zeros(Rl.shape[0])
            c = chebyshev(lambda v: Ag @ v, dinv, Rl.T @ res, bl[l].lam, self.degree, self.smooth[0],
                          self.smooth[1])
            return Rl @ c

        for l in range(L, 0, -1):
            e = e + smooth(l, b - A @ e)
        R0 = R[0]
        A0 = (R0.T @ A @ R0).toarray()
        if A0.size:
            e = e + R0 @ np.linalg.solve(A0, R0.T @ (b - A @ e))
        for l in range(1, L + 1):
            e = e + smooth(l, b - A @ e)
        return e
