"""Residual, Jacobian and constrained Newton system, assembled explicitly (FP64).

Test infrastructure only (see ``oracle/__init__``).

Degrees of freedom: global index ``comp * nn + node`` with comp 0, 1 the two
displacement components and comp 2 the phase field (block order u_x | u_y | phi).

Definitions followed (paper sections / equations):

* Constitutive law, Problem 1: sigma(u) = 2 mu e(u) + lambda tr(e(u)) I,
  e(u) = (grad u + grad u^T) / 2; plane strain Lame constants from E, nu
  (mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 - 2 nu)); Table 1 lists
  mu = 0.42, lambda = 0.28 for E = 1, nu = 0.2, which is plane strain).
  A per-cell modulus E_K scales both Lame constants.
* Degradation, Problem 1: g(phi) = (1 - kappa) phi^2 + kappa, evaluated at the
  linearised phase field phi_tilde (Sec. 2, linearised u-equation).
* Residual form A(U)(Psi), Problem 2, with sigma^+ read as sigma and the
  G_c / l term carrying the sign that makes the Jacobian of Sec. 3.1 its exact
  derivative:
      A_u(psi)   = (g(phi~) sigma(u), e(psi)) + (phi~^2 p, div psi)
      A_phi(psi) = (1-kappa)(phi sigma(u):e(u), psi) + 2 p (phi div u, psi)
                   - (G_c / l)(1 - phi, psi) + G_c l (grad phi, grad psi)
  The Newton right-hand side is R = -A(U) (Sec. 3.1).
* Jacobian A'(U)(dU, Psi), Sec. 3.1, all four terms:
      (g(phi~) sigma(du), e(psi_u))
    + (1-kappa)(dphi sigma(u):e(u) + 2 phi sigma(du):e(u), psi_phi)
    + 2 p (dphi div u + phi div du, psi_phi)
    + G_c ((1/l)(dphi, psi_phi) + l (grad dphi, grad psi_phi))
  The u-rows do not depend on dphi: the matrix is block lower triangular
  (Sec. 3.2).
* Constrained system G~ (Sec. 3.2, three kinds of constraints):
  hanging nodes eliminated through x_full = C x (their own entries ignored on
  input, zero rows on output, contributions condensed onto the parents);
  Dirichlet u DoFs (Problem 1, V = H^1_0) and active phi DoFs (Algorithm 2)
  become identity rows and columns:
      G~ = M_f C^T G C M_f + I_fixed,   M_f = diag(free DoFs).
* Lumped mass B_ii = integral of the constrained phi basis function i
  (the matrix B of the active-set rule, Algorithm 2).
* TCV = integral of u . grad phi over Omega (Sec. 4).

Quadrature: (k+1)^2 Gauss points per leaf cell on every term.

Pinned by tests/test_oracle_operators.py: closed-form elastic energy of linear
fields, rigid modes, patch test with hanging nodes, pure-elasticity limit
(R == 0 at u = 0, phi = 1), closed-form sum rules of every term of A for
linear fields (exact domain integrals of the weak form at linear test fields),
Table 1's Lame constants, central-difference Jacobian of the residual (cubic
in U, Richardson-extrapolated), block triangular / symmetric diagonal blocks,
TCV of an exactly represented field.
"""
import numpy as np
import scipy.sparse as sp

from .fe import CellTables


class Material:
    def __init__(self, E=1.0, nu=0.2, Gc=1.0, eps=1.0, kappa=1e-10, p=1e-3):
        self.E, self.nu, self.Gc, self.eps, self.kappa, self.p = E, nu, Gc, eps, kappa, p
        # Lame constants for unit modulus; scaled by E (or the cell's E_K)
        self.mu1 = 1.0 / (2.0 * (1.0 + nu))
        self.lam1 = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))

    @property
    def mu(self):
        return self.E * self.mu1

    @property
    def lam(self):
        return self.E * self.lam1


class State:
    """Linearisation point.  Hanging entries are overwritten by their
    constraint (x_full = C x) before any use."""

    def __init__(self, mesh, u, phi, phit, E_cells=None):
        C = mesh.C
        self.u = np.stack([C @ u[:, 0], C @ u[:, 1]], axis=1)
        self.phi = C @ phi
        self.phit = C @ phit
        self.E_cells = None if E_cells is None else np.asarray(E_cells, dtype=np.float64)


def level_groups(mesh, cell_idx=None):
    """Leaf cells grouped by level: list of (level, indices)."""
    lv = mesh.cells[:, 0]
    idx = np.arange(len(lv)) if cell_idx is None else np.asarray(cell_idx)
    out = []
    for l in np.unique(lv[idx]):
        out.append((int(l), idx[lv[idx] == l]))
    return out


def _basis_strain(T):
    """e(N_A e_i) and unit-modulus sigma(N_A e_i) per quadrature point.

    Ebas[q, A, i, m, n] = (delta_mi dN_A/dx_n + delta_ni dN_A/dx_m) / 2.
    """
    nq, nb, _ = T.dN.shape
    Eb = np.zeros((nq, nb, 2, 2, 2))
    for i in range(2):
        for m in range(2):
            for n in range(2):
                Eb[:, :, i, m, n] = 0.5 * ((m == i) * T.dN[:, :, n] + (n == i) * T.dN[:, :, m])
    return Eb


def _sigma(e, mu, lam):
    """sigma = 2 mu e + lam tr(e) I on arrays [..., 2, 2]."""
    tr = e[..., 0, 0] + e[..., 1, 1]
    s = 2.0 * mu * e
    s[..., 0, 0] += lam * tr
    s[..., 1, 1] += lam * tr
    return s


class _CellData:
    """Quadrature-point values of the linearisation on a group of same-level cells."""

    def __init__(self, mesh, mat, st, level, idx):
        k = mesh.k
        tr = mesh.tree
        T = CellTables(k, tr.hx(level), tr.hy(level))
        self.T = T
        cn = mesh.cell_nodes[idx]
        self.cn = cn
        uc = st.u[cn]                     # (c, A, i)
        self.uq = np.einsum('qa,cai->cqi', T.N, uc)
        self.gu = np.einsum('qad,cai->cqid', T.dN, uc)   # grad u: [i][d] = du_i/dx_d
        self.phiq = np.einsum('qa,ca->cq', T.N, st.phi[cn])
        self.gphi = np.einsum('qad,ca->cqd', T.dN, st.phi[cn])
        self.phitq = np.einsum('qa,ca->cq', T.N, st.phit[cn])
        self.Ec = np.full(len(idx), mat.E) if st.E_cells is None else st.E_cells[idx]
        eu = 0.5 * (self.gu + np.swapaxes(self.gu, -1, -2))
        self.eu = eu
        self.sig_u = self.Ec[:, None, None, None] * _sigma(eu, mat.mu1, mat.lam1)
        self.sig_e = np.einsum('cqmn,cqmn->cq', self.sig_u, eu)
        self.divu = self.gu[:, :, 0, 0] + self.gu[:, :, 1, 1]
        self.g = (1.0 - mat.kappa) * self.phitq ** 2 + mat.kappa


def element_jacobian(mesh, mat, st, level, idx):
    """Element matrices (uu, phi-u, phi-phi blocks) of A'(U) on same-level cells."""
    d = _CellData(mesh, mat, st, level, idx)
    T = d.T
    Eb = _basis_strain(T)
    Sb1 = _sigma(Eb, mat.mu1, mat.lam1)
    W = T.JxW
    # (g sigma(du), e(psi))
    Kuu = np.einsum('cq,q,qbjmn,qaimn->caibj', d.g * d.Ec[:, None], W, Sb1, Eb)
    # (1-kappa) 2 phi sigma(du):e(u) psi + 2 p phi div(du) psi
    sig_du_e_u = d.Ec[:, None, None, None] * np.einsum('qbjmn,cqmn->cqbj', Sb1, d.eu)
    div_du = T.dN  # div(N_B e_j) = dN_B/dx_j  -> [q, B, j]
    coef = (1.0 - mat.kappa) * 2.0 * d.phiq[:, :, None, None] * sig_du_e_u \
        + 2.0 * mat.p * d.phiq[:, :, None, None] * div_du[None]
    Kpu = np.einsum('q,qa,cqbj->cabj', W, T.N, coef)
    # dphi ((1-kappa) sigma(u):e(u) + 2 p div u + G_c / l) psi + G_c l grad dphi . grad psi
    m = (1.0 - mat.kappa) * d.sig_e + 2.0 * mat.p * d.divu + mat.Gc / mat.eps
    Kpp = np.einsum('cq,q,qa,qb->cab', m, W, T.N, T.N) \
        + mat.Gc * mat.eps * np.einsum('q,qad,qbd->ab', W, T.dN, T.dN)[None]
    return d.cn, Kuu, Kpu, Kpp


def assemble_jacobian(mesh, mat, st, cell_idx=None):
    """Unconstrained global Jacobian G (3 nn x 3 nn CSR), hanging nodes as ordinary vertices."""
    nn = mesh.nn
    rows, cols, vals = [], [], []
    for level, idx in level_groups(mesh, cell_idx):
        cn, Kuu, Kpu, Kpp = element_jacobian(mesh, mat, st, level, idx)
        nb = cn.shape[1]
        for i in range(2):
            for j in range(2):
                r = (i * nn + cn)[:, :, None].repeat(nb, 2)
                c = (j * nn + cn)[:, None, :].repeat(nb, 1)
                rows.append(r.ravel()); cols.append(c.ravel()); vals.append(Kuu[:, :, i, :, j].ravel())
        for j in range(2):
            r = (2 * nn + cn)[:, :, None].repeat(nb, 2)
            c = (j * nn + cn)[:, None, :].repeat(nb, 1)
            rows.append(r.ravel()); cols.append(c.ravel()); vals.append(Kpu[:, :, :, j].ravel())
        r = (2 * nn + cn)[:, :, None].repeat(nb, 2)
        c = (2 * nn + cn)[:, None, :].repeat(nb, 1)
        rows.append(r.ravel()); cols.append(c.ravel()); vals.append(Kpp.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(3 * nn, 3 * nn))


def residual_form(mesh, mat, st):
    """A(U)(Psi) for every basis function Psi, unconstrained (3 nn)."""
    nn = mesh.nn
    out = np.zeros(3 * nn)
    for level, idx in level_groups(mesh):
        d = _CellData(mesh, mat, st, level, idx)
        T = d.T
        W = T.JxW
        Eb = _basis_strain(T)
        Au = np.einsum('q,cq,cqmn,qaimn->cai', W, d.g, d.sig_u, Eb) \
            + np.einsum('q,cq,qai->cai', W, d.phitq ** 2 * mat.p, T.dN)
        val = (1.0 - mat.kappa) * d.phiq * d.sig_e + 2.0 * mat.p * d.phiq * d.divu \
            - (mat.Gc / mat.eps) * (1.0 - d.phiq)
        Ap = np.einsum('q,cq,qa->ca', W, val, T.N) \
            + mat.Gc * mat.eps * np.einsum('q,cqd,qad->ca', W, d.gphi, T.dN)
        for i in range(2):
            np.add.at(out, i * nn + d.cn, Au[:, :, i])
        np.add.at(out, 2 * nn + d.cn, Ap)
    return out


def lumped_mass(mesh):
    """B_ii = integral of the constrained (condensed) phi basis function i; 0 on hanging nodes."""
    b = np.zeros(mesh.nn)
    for level, idx in level_groups(mesh):
        T = CellTables(mesh.k, mesh.tree.hx(level), mesh.tree.hy(level))
        np.add.at(b, mesh.cell_nodes[idx], np.einsum('q,qa->a', T.JxW, T.N)[None, :].repeat(len(idx), 0))
    return mesh.C.T @ b


def tcv(mesh, st):
    """Total crack volume: integral of u . grad phi (Gauss rule on leaf cells)."""
    tot = 0.0
    for level, idx in level_groups(mesh):
        T = CellTables(mesh.k, mesh.tree.hx(level), mesh.tree.hy(level))
        cn = mesh.cell_nodes[idx]
        uq = np.einsum('qa,cai->cqi', T.N, st.u[cn])
        gp = np.einsum('qad,ca->cqd', T.dN, st.phi[cn])
        tot += float(np.einsum('q,cqi,cqi->', T.JxW, uq, gp))
    return tot


# ---------------------------------------------------------------- constraints
def fixed_dofs(mesh, active):
    """Dirichlet u DoFs and active phi DoFs (bool, 3 nn)."""
    nn = mesh.nn
    f = np.zeros(3 * nn, dtype=bool)
    f[:nn] = mesh.dirichlet
    f[nn:2 * nn] = mesh.dirichlet
    f[2 * nn:] = np.asarray(active, dtype=bool)
    return f


def free_dofs(mesh, active):
    hang = np.tile(mesh.is_hanging, 3)
    return ~fixed_dofs(mesh, active) & ~hang


def C3(mesh):
    return sp.block_diag([mesh.C, mesh.C, mesh.C], format='csr')


def constrained_operator(mesh, G, active):
    """G~ = M_f C^T G C M_f + I_fixed (3 nn x 3 nn CSR)."""
    C = C3(mesh)
    fr = free_dofs(mesh, active).astype(np.float64)
    fx = fixed_dofs(mesh, active).astype(np.float64)
    Mf = sp.diags(fr)
    return (Mf @ C.T @ G @ C @ Mf + sp.diags(fx)).tocsr()


def condensed_operator(mesh, G, active):
    """M_f C^T G C: constrained rows, unmasked columns (for inhomogeneous constraints)."""
    C = C3(mesh)
    Mf = sp.diags(free_dofs(mesh, active).astype(np.float64))
    return (Mf @ C.T @ G @ C).tocsr()


def condense(mesh, r):
    """C^T r on a 3 nn vector (hanging entries condensed onto parents, then 0)."""
    return C3(mesh).T @ r


def distribute(mesh, x):
    """x_full = C x: hanging entries from their parents."""
    return C3(mesh) @ x


def cod(mesh, st, xs):
    """COD(x) = integral over y of u . grad phi along the vertical line at x (Sec. 4)
    for every x in xs: the (k+1)-point Gauss rule in y on each leaf cell the line
    crosses.  A cell [x0, x0 + hx) contains x when x0 <= x < x0 + hx, with
    x0 = domain x0 + i hx in FP64; a line on a vertical cell edge takes the cells
    to its right."""
    from .fe import gauss01, lagrange1d
    tr = mesh.tree
    k = mesh.k
    eta, w = gauss01(k + 1)
    Le, dLe = lagrange1d(k, eta)            # (k+1, nq) in y
    xs = np.asarray(xs, dtype=np.float64)
    out = np.zeros(len(xs))
    for level, idx in level_groups(mesh):
        hx, hy = tr.hx(level), tr.hy(level)
        x0 = tr.x0 + mesh.cells[idx, 1] * hx
        for n, x in enumerate(xs):
            sel = np.nonzero((x0 <= x) & (x < x0 + hx))[0]
            for c in sel:
                t = (x - x0[c]) / hx
                Lx, dLx = lagrange1d(k, [t])
                cn = mesh.cell_nodes[idx[c]].reshape(k + 1, k + 1)   # [b][a]
                ux, uy, ph = st.u[cn, 0], st.u[cn, 1], st.phi[cn]
                tot = 0.0
                for q in range(k + 1):
                    Nab = Le[:, q][:, None] * Lx[:, 0][None, :]          # [b][a]
                    dxab = Le[:, q][:, None] * dLx[:, 0][None, :] / hx
                    dyab = dLe[:, q][:, None] * Lx[:, 0][None, :] / hy
                    tot += w[q] * ((Nab * ux).sum() * (dxab * ph).sum() + (Nab * uy).sum() * (dyab * ph).sum())
                out[n] += hy * tot
    return out
