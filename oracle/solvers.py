"""GMRES and the Newton / primal-dual active set load step (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

* GMRES (Sec. 1 and Sec. 3.2): left-preconditioned, P^-1 G~ dU = P^-1 R~, with
  the block-diagonal preconditioner P^-1 = diag(MG(G~uu), MG(G~phiphi)).
  Reading where the paper is silent: x0 = 0, restart 50, classical
  Gram-Schmidt with one re-orthogonalisation, Givens rotations, stop when the
  preconditioned residual estimate drops below rtol times its initial value.
* Load step, Algorithm 2 (with Algorithm 1): per Newton iteration k
    1. residual R = -A(U^k) (condensed onto free DoFs),
    2. active set A^k = { i : R_i / B_ii + c (phi_i - phi_i^old) > 0 }
       (B = lumped mass, strict >, hanging nodes never active),
    3. stop if A^k = A^{k-1} and ||R~(U^k)|| <= max(tol * ||R~(U^{n,0})||, atol)
       (atol = 1e-13 lets an already solved state, e.g. phi = 1, stop),
    4. Newton update with the inhomogeneous constraint dphi = phi_old - phi on
       A^k: G~ dU = R~ - M_f C^T G C dU0, identity rows on fixed DoFs,
    5. hanging entries of dU from their constraint,
    6. line search U + omega^(l-1) dU, l = 1..l_max, accept the first trial whose
       ||R~|| (same active set) is below the current one (else the last trial).
  R~ is the Newton residual: R on free rows, phi_old - phi on active rows, 0 on
  Dirichlet and hanging rows.  phi_tilde = phi_old = phi^{n-1} for the step
  unless a phi_tilde is given (e.g. extrapolate_phi of the two previous steps).

Pinned by tests/test_oracle_solvers.py: GMRES against a dense solve, KKT
conditions at convergence, the pure-elasticity limit, and the Sneddon crack
volume against its closed form with errors of the size Table 2 reports.
"""
import numpy as np
import scipy.sparse as sp

from . import mg as mgmod
from . import operators as ops


def gmres(apply_A, apply_M, b, rtol=1e-6, restart=50, maxiter=500):
    """Left-preconditioned restarted GMRES; returns (x, iterations, final estimate, initial)."""
    n = b.size
    x = np.zeros(n)
    r = apply_M(b)
    beta0 = np.linalg.norm(r)
    if beta0 == 0.0:
        return x, 0, 0.0, 0.0
    target = rtol * beta0
    it = 0
    beta = beta0
    while it < maxiter:
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        conv = False
        for j in range(restart):
            w = apply_M(apply_A(V[j]))
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) <= target or hn == 0.0 or it >= maxiter:
                conv = abs(g[j + 1]) <= target or hn == 0.0
                break
            V[j + 1] = w / hn
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        if conv:
            return x, it, abs(g[j_done]), beta0
        r = apply_M(b - apply_A(x))
        beta = np.linalg.norm(r)
    return x, it, beta, beta0


def newton_residual(mesh, R, active, phi, phi_old):
    """R~: R on free rows, phi_old - phi on active phi rows, 0 on Dirichlet / hanging rows."""
    nn = mesh.nn
    res = R * ops.free_dofs(mesh, active)
    a = np.nonzero(active)[0]
    res[2 * nn + a] = phi_old[a] - phi[a]
    return res


def active_set(mesh, R, B, phi, phi_old, c):
    """A = { i : R_phi,i / B_ii + c (phi_i - phi_old_i) > 0 }, never on hanging nodes.

    c <= 0 selects the per-DoF constant of Sec. 2, c_i = 2 |lambda_i / (phi_i - phi_old_i)|,
    for which c_i (phi_i - phi_old_i) = 2 |lambda_i| sign(phi_i - phi_old_i) (0 where phi_i = phi_old_i)."""
    nn = mesh.nn
    ok = ~mesh.is_hanging
    lam = np.zeros(nn)
    lam[ok] = R[2 * nn:][ok] / B[ok]
    d = phi - phi_old
    if c > 0:
        ind = lam + c * d
    else:
        ind = lam + np.where(d > 0, 2.0 * np.abs(lam), np.where(d < 0, -2.0 * np.abs(lam), 0.0))
    return (ind > 0) & ok, ind


class StepInfo:
    def __init__(self):
        self.newton = 0
        self.gmres = []
        self.res = []
        self.active_sizes = []
        self.linesearch_failed = 0
        self.converged = False
        self.margin = None


def load_step(mesh, mat, c, u, phi, phi_old, active_prev=None, E_cells=None, tol=1e-8, gmres_rtol=1e-6,
              restart=50, gmres_maxiter=500, max_newton=100, ls_max=10, omega=0.5, mg_kw=None, atol=1e-13,
              phi_tilde=None):
    """One load step of Algorithm 2; returns (u, phi, active, info).  phi_tilde: the
    linearised phase field of the u-equation (Sec. 2), phi_old when None."""
    nn = mesh.nn
    mg_kw = mg_kw or {}
    phit = phi_old.copy() if phi_tilde is None else np.asarray(phi_tilde, dtype=np.float64).copy()
    B = ops.lumped_mass(mesh)
    C = mesh.C
    u = np.stack([C @ u[:, 0], C @ u[:, 1]], 1)
    phi = C @ phi
    A_prev = np.zeros(nn, bool) if active_prev is None else np.asarray(active_prev, bool).copy()
    info = StepInfo()
    r0 = None
    for k in range(max_newton + 1):
        st = ops.State(mesh, u, phi, phit, E_cells)
        R = ops.condense(mesh, -ops.residual_form(mesh, mat, st))
        act, ind = active_set(mesh, R, B, phi, phi_old, c)
        res = newton_residual(mesh, R, act, phi, phi_old)
        nres = np.linalg.norm(res)
        if r0 is None:
            r0 = nres
        info.res.append(nres)
        info.active_sizes.append(int(act.sum()))
        if np.array_equal(act, A_prev) and nres <= max(tol * r0, atol):
            info.converged = True
            info.margin = float(np.abs(ind[~mesh.is_hanging]).min())
            return u, phi, act, info
        if k == max_newton:
            break
        G = ops.assemble_jacobian(mesh, mat, st)
        Gt = ops.constrained_operator(mesh, G, act)
        Gc = ops.condensed_operator(mesh, G, act)
        dU0 = np.zeros(3 * nn)
        a = np.nonzero(act)[0]
        dU0[2 * nn + a] = phi_old[a] - phi[a]
        rhs = (R - Gc @ dU0) * ops.free_dofs(mesh, act) + dU0
        M = mgmod.MG(mesh, mat, u, phi, phit, act, E_cells=E_cells, **mg_kw)

        def prec(r):
            return np.concatenate([M.vcycle("uu", r[:2 * nn]), M.vcycle("pp", r[2 * nn:])])

        dU, its, _, _ = gmres(lambda v: Gt @ v, prec, rhs, rtol=gmres_rtol, restart=restart, maxiter=gmres_maxiter)
        info.gmres.append(its)
        dU = ops.distribute(mesh, dU)
        du, dp = np.stack([dU[:nn], dU[nn:2 * nn]], 1), dU[2 * nn:]
        accepted = False
        for l in range(1, ls_max + 1):
            w = omega ** (l - 1)
            ut, pt = u + w * du, phi + w * dp
            stt = ops.State(mesh, ut, pt, phit, E_cells)
            Rt = ops.condense(mesh, -ops.residual_form(mesh, mat, stt))
            if np.linalg.norm(newton_residual(mesh, Rt, act, pt, phi_old)) < nres:
                accepted = True
                break
        if not accepted:
            info.linesearch_failed += 1
        u, phi = ut, pt
        A_prev = act
        info.newton = k + 1
    return u, phi, A_prev, info


def extrapolate_phi(phi_prev, phi_prev2):
    """phi_tilde of load step n by extrapolation from the two previous steps (Sec. 2:
    the u-equation's degradation uses phi_tilde, "the old incremental step solution
    or an extrapolation").  Reading: linear extrapolation in the step index, which
    is exact for equidistant load steps on which phi changes linearly, clipped to
    the phase field's range [0, 1]: clip(2 phi^(n-1) - phi^(n-2), 0, 1) per node."""
    return np.clip(2.0 * np.asarray(phi_prev, dtype=np.float64) - np.asarray(phi_prev2, dtype=np.float64), 0.0, 1.0)


def sneddon_initial(mesh, h_min):
    """Initial crack phi_old (|x| <= 1, |y| <= h_min) and u = 0 (Sec. 4)."""
    import synthetic as synth
    x, y = mesh.node_xy()
    phi_old = synth.crack_phi_old(x, y, h_min)
    return np.zeros((mesh.nn, 2)), phi_old
