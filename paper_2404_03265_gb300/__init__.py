"""GB300-native hot path of the matrix-free, GMG-preconditioned Newton-GMRES
phase-field fracture solver of Kolditz & Wick (arXiv 2404.03265).

The compute path is ``libpff.so`` (hand-written CUDA for sm_103a behind the
C-ABI of ``include/pff.h``).  ``Mesh`` and ``Problem`` below only marshal
arguments; torch supplies device memory and streams.
"""
import numpy as np

from . import _lib
from ._lib import (PFF_F32, PFF_F64, PFF_OP_CONDENSED, PFF_OP_JACOBIAN, PFF_OP_TRANSPOSE, PFF_PHIT_EXTRAPOLATED,
                   PFF_PHIT_PREVIOUS, PffError)


class Mesh:
    """Quadtree mesh with 2:1 balance (libpff host side)."""

    def __init__(self, x0, x1, y0, y1, ncx, ncy):
        L = _lib.lib()
        h = _lib.ctypes.c_void_p()
        _lib.check(L.pff_mesh_create(x0, x1, y0, y1, ncx, ncy, _lib.ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_recipe(cls, rec):
        d = rec["domain"]
        m = cls(d[0], d[1], d[2], d[3], rec["ncx"], rec["ncy"])
        m.refine_global(rec["n_global"])
        for step in rec["steps"]:
            m.refine_box(0 if step[0] == "box" else 1, *step[1:])
        return m

    def refine_global(self, times=1):
        _lib.check(_lib.lib().pff_mesh_refine_global(self._h, times))

    def refine_box(self, rule, bx0, bx1, by0, by1):
        _lib.check(_lib.lib().pff_mesh_refine_box(self._h, rule, bx0, bx1, by0, by1))

    def refine_marked(self, marks):
        m = np.ascontiguousarray(marks, dtype=np.uint8)
        _lib.check(_lib.lib().pff_mesh_refine_marked(self._h, _lib.ptr(m), m.size))

    def n_leaves(self):
        n = _lib.ctypes.c_int64()
        _lib.check(_lib.lib().pff_mesh_n_leaves(self._h, _lib.ctypes.byref(n)))
        return n.value

    def finalize(self, fe_degree=1):
        _lib.check(_lib.lib().pff_mesh_finalize(self._h, fe_degree))
        self.info = self.get_info()
        return self

    def get_info(self):
        inf = _lib.MeshInfo()
        _lib.check(_lib.lib().pff_mesh_info_get(self._h, _lib.ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def slots(self):
        n = self.info["n_slots"]
        X = np.empty(n, np.int32)
        Y = np.empty(n, np.int32)
        F = np.empty(n, np.uint8)
        _lib.check(_lib.lib().pff_mesh_slots(self._h, _lib.ptr(X), _lib.ptr(Y), _lib.ptr(F)))
        return X, Y, F

    def leaf_cells(self):
        n = self.info["n_leaf_cells"]
        a = np.empty((n, 3), np.int32)
        _lib.check(_lib.lib().pff_mesh_leaf_cells(self._h, _lib.ptr(a)))
        return a

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lib().pff_mesh_destroy(h)
            self._h = None


class Problem:
    """Parameters bound to a mesh; owns the linearisation and constraint masks on the GPU."""

    def __init__(self, mesh, E=1.0, nu=0.2, Gc=1.0, eps=1.0, kappa=1e-10, p=1e-3, c=1e4):
        self.mesh = mesh
        prm = _lib.Params(E, nu, Gc, eps, kappa, p, c)
        h = _lib.ctypes.c_void_p()
        _lib.check(_lib.lib().pff_problem_create(mesh._h, _lib.ctypes.byref(prm), _lib.ctypes.byref(h)))
        self._h = h
        self.n_slots = mesh.info["n_slots"]
        self.params = dict(E=E, nu=nu, Gc=Gc, eps=eps, kappa=kappa, p=p, c=c)

    def set_state(self, u, phi, phit, stream=None):
        """u: float64 (2, n_slots) (u_x block, u_y block), phi, phit: float64 (n_slots,) CUDA tensors."""
        _lib.check(_lib.lib().pff_set_state(self._h, _lib.ptr(u), _lib.ptr(phi), _lib.ptr(phit),
                                            _lib.stream_ptr(stream)))

    def set_active(self, active, stream=None):
        _lib.check(_lib.lib().pff_set_active(self._h, _lib.ptr(active), _lib.stream_ptr(stream)))

    def apply(self, xu, xp, yu, yp, op=PFF_OP_JACOBIAN, stream=None):
        import torch
        prec = PFF_F64 if xu.dtype == torch.float64 else PFF_F32
        _lib.check(_lib.lib().pff_apply(self._h, prec, op, _lib.ptr(xu), _lib.ptr(xp), _lib.ptr(yu),
                                        _lib.ptr(yp), _lib.stream_ptr(stream)))

    def active_set(self, R, phi, phi_old, active, stream=None):
        """Algorithm 2's active set from the condensed residual R (3, n_slots); active updated in place.
        Returns (n_changed, n_active, margin)."""
        nc, na, mg_ = _lib.ctypes.c_int64(), _lib.ctypes.c_int64(), _lib.ctypes.c_double()
        _lib.check(_lib.lib().pff_active_set(self._h, _lib.ptr(R), _lib.ptr(phi), _lib.ptr(phi_old), _lib.ptr(active),
                                             _lib.ctypes.byref(nc), _lib.ctypes.byref(na), _lib.ctypes.byref(mg_),
                                             _lib.stream_ptr(stream)))
        return nc.value, na.value, mg_.value

    def extrapolate_phi(self, phi_prev, phi_prev2, phi_tilde, stream=None):
        """phi_tilde = clip(2 phi_prev - phi_prev2, 0, 1) on the device (float64 (n_slots,) tensors)."""
        _lib.check(_lib.lib().pff_extrapolate_phi(self._h, _lib.ptr(phi_prev), _lib.ptr(phi_prev2),
                                                  _lib.ptr(phi_tilde), _lib.stream_ptr(stream)))

    def set_cell_loop(self, strip_half_rows):
        """Q1 cell-loop strip half-height: 15, 5, 1, or 0 (by mesh size)."""
        _lib.check(_lib.lib().pff_set_cell_loop(self._h, strip_half_rows))

    def set_pressure(self, p):
        _lib.check(_lib.lib().pff_set_pressure(self._h, p))
        self.params["p"] = p

    def set_params(self, **kw):
        """Update parameters (E, nu, Gc, eps, kappa, p, c); later calls use them."""
        self.params.update(kw)
        q = self.params
        prm = _lib.Params(q["E"], q["nu"], q["Gc"], q["eps"], q["kappa"], q["p"], q["c"])
        _lib.check(_lib.lib().pff_set_params(self._h, _lib.ctypes.byref(prm)))

    def set_cell_modulus(self, E_cells, stream=None):
        """Per-cell Young's modulus (float64 device tensor in leaf_cells() order), or None."""
        _lib.check(_lib.lib().pff_set_cell_modulus(self._h, None if E_cells is None else _lib.ptr(E_cells),
                                                   _lib.stream_ptr(stream)))

    def tcv_gradient(self, u, phi, g, stream=None):
        """g = M_f C^T dJ/dU of J = TCV (g: float64 (3, n_slots))."""
        _lib.check(_lib.lib().pff_tcv_gradient(self._h, _lib.ptr(u), _lib.ptr(phi), _lib.ptr(g),
                                               _lib.stream_ptr(stream)))

    def param_vjp(self, w, gE=None, stream=None):
        """(C M_f w) . dR/dtheta at the current state: returns (g_p, g_Gc); fills gE (per leaf cell)."""
        out = np.zeros(2)
        _lib.check(_lib.lib().pff_param_vjp(self._h, _lib.ptr(w), None if gE is None else _lib.ptr(gE),
                                            _lib.ptr(out), _lib.stream_ptr(stream)))
        return float(out[0]), float(out[1])

    def residual(self, u, phi, phit, R, stream=None):
        """R (3, n_slots) float64 = -A(U) condensed, Dirichlet rows 0."""
        _lib.check(_lib.lib().pff_residual(self._h, _lib.ptr(u), _lib.ptr(phi), _lib.ptr(phit), _lib.ptr(R),
                                           _lib.stream_ptr(stream)))

    def lumped_mass(self, B, stream=None):
        _lib.check(_lib.lib().pff_lumped_mass(self._h, _lib.ptr(B), _lib.stream_ptr(stream)))

    def tcv(self, u, phi, stream=None):
        out = _lib.ctypes.c_double()
        _lib.check(_lib.lib().pff_tcv(self._h, _lib.ptr(u), _lib.ptr(phi), _lib.ctypes.byref(out),
                                      _lib.stream_ptr(stream)))
        return out.value

    def cod(self, u, phi, xs, stream=None):
        """COD(x) = integral over y of u . grad phi along the vertical lines x = xs (Sec. 4)."""
        xs = np.ascontiguousarray(xs, dtype=np.float64)
        out = np.zeros(len(xs))
        _lib.check(_lib.lib().pff_cod(self._h, _lib.ptr(u), _lib.ptr(phi), _lib.ptr(xs), len(xs), _lib.ptr(out),
                                      _lib.stream_ptr(stream)))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lib().pff_problem_destroy(h)
            self._h = None


class MG:
    """Block-diagonal GMG preconditioner (u-u block 0, phi-phi block 1) of a Problem."""

    def __init__(self, problem, precision=PFF_F32, coarse="direct"):
        """coarse: "direct" (FP64 solve of the level-0 block) or "chebyshev" (Sec. 3.2)."""
        self.problem = problem
        h = _lib.ctypes.c_void_p()
        _lib.check(_lib.lib().pff_mg_create(problem._h, precision, _lib.ctypes.byref(h)))
        self._h = h
        if coarse != "direct":
            _lib.check(_lib.lib().pff_mg_set_coarse(self._h, {"chebyshev": 1}[coarse]))
        self.n_levels = problem.mesh.info["finest_level"] + 1

    def setup(self, stream=None):
        _lib.check(_lib.lib().pff_mg_setup(self._h, _lib.stream_ptr(stream)))

    def set_fused_smoother(self, on):
        """Chebyshev steps as the stores of the level applies (True, the default)
        or as separate kernels (False)."""
        _lib.check(_lib.lib().pff_mg_set_fused_smoother(self._h, 1 if on else 0))

    def vcycle(self, block, r, z, stream=None):
        """z = MG(r); block 0: r, z float64 (2, n_slots); block 1: (n_slots,)."""
        _lib.check(_lib.lib().pff_vcycle(self._h, block, _lib.ptr(r), _lib.ptr(z), _lib.stream_ptr(stream)))

    def inverse_diagonal(self, level, block, stream=None):
        """(dinv (ncomp * n_slots_l,) float64 device tensor, X, Y level-slot coordinates)."""
        import torch
        n = _lib.ctypes.c_int64()
        _lib.check(_lib.lib().pff_inverse_diagonal(self._h, level, block, None, None, None, 0,
                                                   _lib.ctypes.byref(n), _lib.stream_ptr(stream)))
        ns = n.value // (2 if block == 0 else 1)
        out = torch.empty(n.value, dtype=torch.float64, device="cuda")
        X = np.empty(ns, np.int32)
        Y = np.empty(ns, np.int32)
        _lib.check(_lib.lib().pff_inverse_diagonal(self._h, level, block, _lib.ptr(out), _lib.ptr(X), _lib.ptr(Y),
                                                   n.value, None, _lib.stream_ptr(stream)))
        return out, X, Y

    def lam(self, block):
        out = np.zeros(self.n_levels)
        _lib.check(_lib.lib().pff_mg_lambda(self._h, block, _lib.ptr(out), self.n_levels))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lib().pff_mg_destroy(h)
            self._h = None


def gmres(problem, mg, rhs, x, rtol=1e-6, restart=50, maxiter=500, transpose=False, stream=None, check=True):
    """Left-preconditioned GMRES on the constrained Jacobian (full vectors (3, n_slots) float64)."""
    info = _lib.SolveInfo()
    st = _lib.lib().pff_gmres_solve(problem._h, mg._h, int(transpose), _lib.ptr(rhs), _lib.ptr(x), rtol, restart,
                                    maxiter, _lib.ctypes.byref(info), _lib.stream_ptr(stream))
    d = dict(iterations=info.gmres_total, converged=bool(info.converged), initial=info.residual0,
             estimate=info.residual, status=st, time_apply=info.time_gmres_apply,
             time_vcycle=info.time_gmres_vcycle, time_orth=info.time_gmres_orth)
    if check:
        _lib.check(st)
    return d


def newton_step(problem, mg, u, phi, phi_old, active, tol=1e-8, atol=1e-13, gmres_rtol=1e-6, omega=0.5,
                restart=50, gmres_maxiter=500, max_newton=100, ls_max=10, matvec=PFF_F64, phi_tilde=None,
                stream=None, check=True):
    """One load step of Algorithm 2 (u (2, n_slots), phi, phi_old (n_slots,) float64; active uint8).
    matvec: precision of the Jacobian applies inside GMRES (PFF_F64 or PFF_F32); phi_tilde: the
    linearised phase field of the u-equation (device tensor), phi_old when None."""
    o = _lib.NewtonOpts(tol, atol, gmres_rtol, omega, restart, gmres_maxiter, max_newton, ls_max, matvec, 0,
                        None if phi_tilde is None else _lib.ptr(phi_tilde))
    info = _lib.SolveInfo()
    st = _lib.lib().pff_newton_pdas_step(problem._h, mg._h, _lib.ptr(u), _lib.ptr(phi), _lib.ptr(phi_old),
                                         _lib.ptr(active), _lib.ctypes.byref(o), _lib.ctypes.byref(info),
                                         _lib.stream_ptr(stream))
    d = info.to_dict()
    d["status"] = st
    if check:
        _lib.check(st)
    return d


def tcv_adjoint(problem, mg, u, phi, phi_old, active, gE=None, rtol=1e-10, restart=50, maxiter=2000, stream=None,
                check=True):
    """dJ/dp, dJ/dG_c (and dJ/dE_K into gE) of J = TCV at a converged load step, by one
    adjoint solve with the transposed constrained Jacobian."""
    out = np.zeros(2)
    info = _lib.SolveInfo()
    st = _lib.lib().pff_tcv_adjoint(problem._h, mg._h, _lib.ptr(u), _lib.ptr(phi), _lib.ptr(phi_old),
                                    _lib.ptr(active), rtol, restart, maxiter, None if gE is None else _lib.ptr(gE),
                                    _lib.ptr(out), _lib.ctypes.byref(info), _lib.stream_ptr(stream))
    if check:
        _lib.check(st)
    return dict(p=float(out[0]), Gc=float(out[1]), iterations=info.gmres_total, converged=bool(info.converged),
                status=st)


def tcv_adjoint_steps(problem, mg, us, phis, actives, ps, gE=None, extrapolated=False, rtol=1e-10, restart=50,
                      maxiter=2000, stream=None, check=True):
    """dJ/dp_k (k = 1..N), dJ/dG_c (and dJ/dE_K into gE) of J = TCV after N load steps.

    us, phis: N + 1 converged states (index 0 the initial state) as device tensors
    (u (2, n_slots), phi (n_slots,) float64); actives: N uint8 device tensors;
    ps: the N pressures; extrapolated: the steps k >= 2 were solved with
    phi_tilde = clip(2 phi^(k-1) - phi^(k-2), 0, 1) (Problem.extrapolate_phi), else
    with phi_tilde = phi^(k-1)."""
    N = len(ps)
    assert len(us) == N + 1 and len(phis) == N + 1 and len(actives) == N
    VP = _lib.ctypes.c_void_p
    ua = (VP * (N + 1))(*[_lib.ptr(t) for t in us])
    pa = (VP * (N + 1))(*[_lib.ptr(t) for t in phis])
    aa = (VP * N)(*[_lib.ptr(t) for t in actives])
    p_host = np.ascontiguousarray(ps, dtype=np.float64)
    gp = np.zeros(N)
    ggc = np.zeros(1)
    info = _lib.SolveInfo()
    mode = _lib.PFF_PHIT_EXTRAPOLATED if extrapolated else _lib.PFF_PHIT_PREVIOUS
    st = _lib.lib().pff_tcv_adjoint_steps(problem._h, mg._h, N, ua, pa, aa, _lib.ptr(p_host), mode, rtol, restart,
                                          maxiter, None if gE is None else _lib.ptr(gE), _lib.ptr(gp), _lib.ptr(ggc),
                                          _lib.ctypes.byref(info), _lib.stream_ptr(stream))
    if check:
        _lib.check(st)
    return dict(p=gp, Gc=float(ggc[0]), gmres_total=info.gmres_total, gmres_max=info.gmres_max,
                converged=bool(info.converged), status=st)
