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

Several load steps (``tcv_adjoint_steps``): phi^(n-1) is phi_tilde and the
obstacle of step n, so the adjoint of step n passes a phi-sensitivity to step
n - 1 through (dA/dphi_tilde)^T (``phit_vjp``) and through the active rows.

Pinned by tests/test_oracle_adjoint.py: the TCV gradient and the parameter
derivatives against central differences of ``operators.tcv`` and
``operators.residual_form`` (both exact: J is bilinear in (u, phi), A is linear
in p, G_c and E_K), phit_vjp against central differences of the residual form
in phi_tilde (quadratic: exact), and the one- and several-step adjoint
gradients against central differences of converged load steps (relative step
1e-6).
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


def phit_vjp(mesh, mat, st, w):
    """C^T (dA/dphi_tilde)^T (C w): phi-vector (nn).  A depends on phi_tilde through
    g(phi~) = (1-kappa) phi~^2 + kappa and phi~^2 p in the u-equation (Problem 2):
        (dA_u/dphi~ [psi], w_u) = (psi, 2 phi~ [(1-kappa) sigma(u) : e(w_u) + p div w_u])."""
    nn = mesh.nn
    C = ops.C3(mesh)
    wf = C @ w
    wu = np.stack([wf[:nn], wf[nn:2 * nn]], 1)
    out = np.zeros(nn)
    for level, idx in ops.level_groups(mesh):
        d = ops._CellData(mesh, mat, st, level, idx)
        T = d.T
        gw = np.einsum('qad,cai->cqid', T.dN, wu[d.cn])        # grad w_u: [i][d]
        ew = 0.5 * (gw + np.swapaxes(gw, -1, -2))
        sw = np.einsum('cqmn,cqmn->cq', d.sig_u, ew)
        divw = gw[:, :, 0, 0] + gw[:, :, 1, 1]
        val = 2.0 * d.phitq * ((1.0 - mat.kappa) * sw + mat.p * divw)
        np.add.at(out, d.cn, np.einsum('q,cq,qa->ca', T.JxW, val, T.N))
    return mesh.C.T @ out


def extrapolated_phit(phis, n):
    """phi_tilde of step n >= 2 by linear extrapolation in the step index, clipped
    to [0, 1] (the reading of Sec. 2's "extrapolation"; oracle/solvers.extrapolate_phi
    restated here so that this module keeps its own arithmetic), and the mask chi
    of its nodes strictly inside (0, 1), where its derivatives in phi^(n-1) and
    phi^(n-2) are 2 and -1 (0 where the clip acts)."""
    raw = 2.0 * phis[n - 1] - phis[n - 2]
    return np.clip(raw, 0.0, 1.0), ((raw > 0.0) & (raw < 1.0)).astype(np.float64)


def tcv_adjoint_steps(mesh, mats, us, phis, actives, E_cells=None, extrapolate=False):
    """Gradient of J = TCV(U^N) after N load steps (Algorithm 2, phi_tilde and the
    obstacle of step n are phi^(n-1)) with respect to each step's pressure p_n,
    G_c and E_K.

    extrapolate: phi_tilde of step n >= 2 is clip(2 phi^(n-1) - phi^(n-2), 0, 1)
    instead (step 1 keeps phi^0; the obstacle stays phi^(n-1)).  The phi_tilde
    sensitivity v^n = C^T (dA/dphi~)^T C M_f mu^n then reaches step n-1 as
    -2 chi v^n and step n-2 as +chi v^n (chi: the unclipped nodes); what reaches
    phi^0 is dropped (the initial state does not depend on the parameters).

    mats[n-1]: Material of step n; us[n], phis[n]: converged state of step n
    (n = 0: the initial state, u = 0 and phi = phi^0, independent of the
    parameters); actives[n-1]: final active set of step n.

    Step n: free rows [C^T A(U^n; phi~ = phi^(n-1))]_F = 0, active rows
    phi^n - phi^(n-1) = 0.  Its Jacobian in U^n is [[K_FF, K_FA], [0, I]] with
    K = C^T G C (the free rows still see the active values).  Backwards:
        K_FF^T mu_F = gbar_F,  mu_A = gbar_A - K_FA^T mu_F,
        gbar^N = C^T dJ/dU^N (Dirichlet rows 0),
        gbar^(n-1) = (0, 0, -C^T (dA/dphi~)^T C M_f mu^n + mu^n on the active rows of step n),
        dJ/dtheta = sum_n (C M_f mu^n) . dR_n/dtheta,  R = -A.
    """
    nn = mesh.nn
    N = len(mats)
    C = ops.C3(mesh)

    def phit_of(n):
        if extrapolate and n >= 2:
            return extrapolated_phit(phis, n)
        return phis[n - 1], None

    st = ops.State(mesh, us[N], phis[N], phit_of(N)[0], E_cells)
    gbar = C.T @ tcv_gradient(mesh, st)
    gbar[:nn][mesh.dirichlet] = 0.0
    gbar[nn:2 * nn][mesh.dirichlet] = 0.0
    g_p = np.zeros(N)
    g_gc = 0.0
    g_e = np.zeros(len(mesh.cells))
    pend = None   # phi sensitivity from step n + 1 that reaches step n - 1
    for n in range(N, 0, -1):
        mat = mats[n - 1]
        act = np.asarray(actives[n - 1], bool)
        phit, chi = phit_of(n)
        st = ops.State(mesh, us[n], phis[n], phit, E_cells)
        K = (C.T @ ops.assemble_jacobian(mesh, mat, st) @ C).tocsc()
        free = ops.free_dofs(mesh, act)
        fixed = ops.fixed_dofs(mesh, act)
        f = np.nonzero(free)[0]
        mu = np.zeros(3 * nn)
        mu[f] = spla.spsolve(K[f][:, f].T.tocsc(), gbar[f])
        fx = np.nonzero(fixed)[0]
        mu[fx] = gbar[fx] - K[f][:, fx].T @ mu[f]
        wf = mu * free
        a, b, c = param_vjp(mesh, mat, st, wf)
        g_p[n - 1] = a
        g_gc += b
        g_e += c
        if n > 1:
            v = phit_vjp(mesh, mat, st, wf)
            gbar = np.zeros(3 * nn)
            gbar[2 * nn:] = -v if chi is None else -2.0 * chi * v
            gbar[2 * nn:][act] += mu[2 * nn:][act]
            if pend is not None:
                gbar[2 * nn:] += pend
            pend = chi * v if (chi is not None and n - 2 >= 1) else None
    return dict(p=g_p, Gc=g_gc, E=g_e)
