"""Adjoint gradient of the total crack volume of one load step (FP64, explicit).

Test infrastructure only (see ``oracle/__init__``).

Quantity of interest: J(U) = TCV = integral of u . grad phi (Sec. 4), at the
converged state U of a load step of Algorithm 2.  Parameters: the pressure p,
the fracture toughness G_c (Problem 1) and a per-cell Young's modulus E_K
(sigma = E_K sigma_1, sigma_1 the unit-modulus stress).

At convergence the free DoFs F (not Dirichlet, not active, not hanging) satisfy
[C^T A(U; theta)]_F = 0, the fixed ones are independent of theta (u = 0 on the
boundary, phi = phi_old on the active set, phi_tilde = phi_old), hanging values
follow their parents (U = C U_c).  With K = C^T G C, G = dA/dU the Jacobian of
Sec. 3.1:

    K_FF^T lambda_F = [C^T dJ/dU]_F,      dJ/dtheta = -lambda_F . [C^T dA/dtheta]_F

The derivatives of the residual form with respect to the parameters follow from
A (Problem 2, sigma^+ read as sigma):

    dA_u/dp   = (phi~^2, div psi)            dA_phi/dp  = 2 (phi div u, psi)
    dA_u/dGc  = 0                            dA_phi/dGc = -(1/l)(1 - phi, psi) + l (grad phi, grad psi)
    dA_u/dE_K = (g(phi~) sigma_1(u), e(psi))_K
    dA_phi/dE_K = (1 - kappa)(phi sigma_1(u) : e(u), psi)_K

Pinned by tests/test_oracle_adjoint.py: the TCV gradient and the parameter
derivatives against central differences of ``operators.tcv`` and
``operators.residual_form`` (both exact: J is bilinear in (u, phi), A is linear
in p, G_c and E_K), and the adjoint gradient against central differences of
converged load steps (relative step 1e-6).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import operators as ops
from .fe import CellTables


def tcv_gradient(mesh, st):
    """dJ/dU (3 nn, block order u_x | u_y | phi) at the state st, unconstrained."""
    nn = mesh.nn
    out = np.zeros(3 * nn)
    for level, idx in ops.level_groups(mesh):
        T = CellTables(mesh.k, mesh.tree.hx(level), mesh.tree.hy(level))
        cn = mesh.cell_nodes[idx]
        uq = np.einsum('qa,cai->cqi', T.N, st.u[cn])
        gp = np.einsum('qad,ca->cqd', T.dN, st.phi[cn])
        du = np.einsum('q,qa,cqi->cai', T.JxW, T.N, gp)       # integral of N_A d(phi)/dx_i
        dphi = np.einsum('q,cqd,qad->ca', T.JxW, uq, T.dN)    # integral of u . grad N_A
        for i in range(2):
            np.add.at(out, i * nn + cn, du[:, :, i])
        np.add.at(out, 2 * nn + cn, dphi)
    return out


def residual_param_derivatives(mesh, mat, st):
    """dA/dp (3 nn), dA/dG_c (3 nn) and dA/dE (3 nn x n_cells CSR), unconstrained."""
    nn = mesh.nn
    ncell = len(mesh.cells)
    d_p = np.zeros(3 * nn)
    d_gc = np.zeros(3 * nn)
    rows, cols, vals = [], [], []
    for level, idx in ops.level_groups(mesh):
        d = ops._CellData(mesh, mat, st, level, idx)
        T = d.T
        W = T.JxW
        Eb = ops._basis_strain(T)
        sig1 = ops._sigma(d.eu, mat.mu1, mat.lam1)
        se1 = np.einsum('cqmn,cqmn->cq', sig1, d.eu)
        au_e = np.einsum('q,cq,cqmn,qaimn->cai', W, d.g, sig1, Eb)
        ap_e = np.einsum('q,cq,qa->ca', W, (1.0 - mat.kappa) * d.phiq * se1, T.N)
        au_p = np.einsum('q,cq,qai->cai', W, d.phitq ** 2, T.dN)
        ap_p = np.einsum('q,cq,qa->ca', W, 2.0 * d.phiq * d.divu, T.N)
        ap_g = np.einsum('q,cq,qa->ca', W, -(1.0 - d.phiq) / mat.eps, T.N) \
            + mat.eps * np.einsum('q,cqd,qad->ca', W, d.gphi, T.dN)
        cn = d.cn
        for i in range(2):
            np.add.at(d_p, i * nn + cn, au_p[:, :, i])
            rows.append((i * nn + cn).ravel())
            cols.append(np.repeat(idx, cn.shape[1]))
            vals.append(au_e[:, :, i].ravel())
        np.add.at(d_p, 2 * nn + cn, ap_p)
        np.add.at(d_gc, 2 * nn + cn, ap_g)
        rows.append((2 * nn + cn).ravel())
        cols.append(np.repeat(idx, cn.shape[1]))
        vals.append(ap_e.ravel())
    d_e = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(3 * nn, ncell))
    return d_p, d_gc, d_e


def tcv_adjoint(mesh, mat, st, active):
    """dJ/dp, dJ/dG_c and dJ/dE_K (n_cells) at a converged load-step state.

    Returns dict(p, Gc, E, lam) with lam the adjoint (3 nn, zero off F)."""
    nn = mesh.nn
    G = ops.assemble_jacobian(mesh, mat, st)
    C = ops.C3(mesh)
    K = (C.T @ G @ C).tocsc()
    f = np.nonzero(ops.free_dofs(mesh, active))[0]
    b = (C.T @ tcv_gradient(mesh, st))[f]
    lam_f = spla.spsolve(K[f][:, f].T.tocsc(), b)
    d_p, d_gc, d_e = residual_param_derivatives(mesh, mat, st)
    lam = np.zeros(3 * nn)
    lam[f] = lam_f
    g_p = -float(lam_f @ (C.T @ d_p)[f])
    g_gc = -float(lam_f @ (C.T @ d_gc)[f])
    g_e = -np.asarray((C.T @ d_e)[f].T @ lam_f).ravel()
    return dict(p=g_p, Gc=g_gc, E=g_e, lam=lam)


def param_vjp(mesh, mat, st, w):
    """w . dR/dtheta with R = -A and w taken through C (x_full = C w):
    returns (g_p, g_Gc, g_E (n_cells)).  With w = lambda this is dJ/dtheta."""
    C = ops.C3(mesh)
    d_p, d_gc, d_e = residual_param_derivatives(mesh, mat, st)
    wf = C @ w
    return -float(wf @ d_p), -float(wf @ d_gc), -np.asarray(d_e.T @ wf).ravel()
