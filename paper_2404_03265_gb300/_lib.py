"""ctypes binding of libpff (include/pff.h): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module converts
Python / torch arguments into plain pointers and sizes.  If ``libpff.so`` has
not been built the import of the binding fails loudly (there is no fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.environ.get("PFF_LIBPATH") or os.path.join(HERE, "libpff.so")

PFF_OK = 0
PFF_F64, PFF_F32 = 0, 1
PFF_OP_JACOBIAN, PFF_OP_TRANSPOSE, PFF_OP_CONDENSED = 0, 1, 2
PFF_PHIT_PREVIOUS, PFF_PHIT_EXTRAPOLATED = 0, 1
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "GMRES_BREAKDOWN",
                6: "NONFINITE", 7: "LINESEARCH", 8: "TIMEOUT", 9: "STATE"}


class PffError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libpff %s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("n_leaf_cells", ctypes.c_int64),
                ("n_hanging", ctypes.c_int64), ("n_partials", ctypes.c_int64), ("n_bricks", ctypes.c_int64),
                ("n_irregular", ctypes.c_int64), ("x_max", ctypes.c_int64), ("y_max", ctypes.c_int64),
                ("h_min", ctypes.c_double), ("fe_degree", ctypes.c_int32), ("finest_level", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("Gc", ctypes.c_double), ("eps", ctypes.c_double),
                ("kappa", ctypes.c_double), ("p", ctypes.c_double), ("c", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("newton_iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("linesearch_failures", ctypes.c_int32), ("gmres_total", ctypes.c_int32),
                ("gmres_max", ctypes.c_int32), ("pad", ctypes.c_int32), ("active_size", ctypes.c_int64),
                ("residual0", ctypes.c_double), ("residual", ctypes.c_double), ("margin", ctypes.c_double),
                ("gmres_per_newton", ctypes.c_int32 * 128), ("residual_history", ctypes.c_double * 129),
                ("time_mg_setup", ctypes.c_double), ("time_gmres", ctypes.c_double),
                ("time_gmres_apply", ctypes.c_double), ("time_gmres_vcycle", ctypes.c_double),
                ("time_gmres_orth", ctypes.c_double)]

    def to_dict(self):
        n = self.newton_iterations
        return dict(newton=n, converged=bool(self.converged), linesearch_failures=self.linesearch_failures,
                    gmres_total=self.gmres_total, gmres_max=self.gmres_max, active_size=self.active_size,
                    residual0=self.residual0, residual=self.residual, margin=self.margin,
                    gmres=list(self.gmres_per_newton[:min(n, 128)]),
                    residual_history=list(self.residual_history[:min(n + 1, 129)]),
                    time_mg_setup=self.time_mg_setup, time_gmres=self.time_gmres,
                    time_gmres_apply=self.time_gmres_apply, time_gmres_vcycle=self.time_gmres_vcycle,
                    time_gmres_orth=self.time_gmres_orth)


class NewtonOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("atol", ctypes.c_double), ("gmres_rtol", ctypes.c_double),
                ("omega", ctypes.c_double), ("restart", ctypes.c_int32), ("gmres_maxiter", ctypes.c_int32),
                ("max_newton", ctypes.c_int32), ("ls_max", ctypes.c_int32), ("matvec_precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("phi_tilde", ctypes.c_void_p)]


_lib = None

# (name, restype, argtypes)
_P = ctypes.c_void_p
_SIGS = [
    ("pff_last_error", ctypes.c_char_p, []),
    ("pff_mesh_create", ctypes.c_int32, [ctypes.c_double] * 4 + [ctypes.c_int32] * 2 + [ctypes.POINTER(_P)]),
    ("pff_mesh_refine_global", ctypes.c_int32, [_P, ctypes.c_int32]),
    ("pff_mesh_refine_box", ctypes.c_int32, [_P, ctypes.c_int32] + [ctypes.c_double] * 4),
    ("pff_mesh_refine_marked", ctypes.c_int32, [_P, _P, ctypes.c_int64]),
    ("pff_mesh_n_leaves", ctypes.c_int32, [_P, ctypes.POINTER(ctypes.c_int64)]),
    ("pff_mesh_finalize", ctypes.c_int32, [_P, ctypes.c_int32]),
    ("pff_mesh_info_get", ctypes.c_int32, [_P, ctypes.POINTER(MeshInfo)]),
    ("pff_mesh_slots", ctypes.c_int32, [_P, _P, _P, _P]),
    ("pff_mesh_leaf_cells", ctypes.c_int32, [_P, _P]),
    ("pff_mesh_destroy", None, [_P]),
    ("pff_problem_create", ctypes.c_int32, [_P, ctypes.POINTER(Params), ctypes.POINTER(_P)]),
    ("pff_problem_destroy", None, [_P]),
    ("pff_set_state", ctypes.c_int32, [_P, _P, _P, _P, _P]),
    ("pff_set_active", ctypes.c_int32, [_P, _P, _P]),
    ("pff_apply", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P]),
    ("pff_apply_noalloc", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P]),
    ("pff_mg_create", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    ("pff_mg_setup", ctypes.c_int32, [_P, _P]),
    ("pff_mg_set_coarse", ctypes.c_int32, [_P, ctypes.c_int32]),
    ("pff_mg_set_fused_smoother", ctypes.c_int32, [_P, ctypes.c_int32]),
    ("pff_vcycle", ctypes.c_int32, [_P, ctypes.c_int32, _P, _P, _P]),
    ("pff_mg_lambda", ctypes.c_int32, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    ("pff_mg_destroy", None, [_P]),
    ("pff_set_pressure", ctypes.c_int32, [_P, ctypes.c_double]),
    ("pff_set_cell_loop", ctypes.c_int32, [_P, ctypes.c_int32]),
    ("pff_extrapolate_phi", ctypes.c_int32, [_P, _P, _P, _P, _P]),
    ("pff_residual", ctypes.c_int32, [_P, _P, _P, _P, _P, _P]),
    ("pff_lumped_mass", ctypes.c_int32, [_P, _P, _P]),
    ("pff_tcv", ctypes.c_int32, [_P, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    ("pff_cod", ctypes.c_int32, [_P, _P, _P, _P, ctypes.c_int32, _P, _P]),
    ("pff_gmres_solve", ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P, ctypes.c_double, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.POINTER(SolveInfo), _P]),
    ("pff_newton_pdas_step", ctypes.c_int32, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(NewtonOpts),
                                              ctypes.POINTER(SolveInfo), _P]),
    ("pff_set_cell_modulus", ctypes.c_int32, [_P, _P, _P]),
    ("pff_set_params", ctypes.c_int32, [_P, ctypes.POINTER(Params)]),
    ("pff_tcv_gradient", ctypes.c_int32, [_P, _P, _P, _P, _P]),
    ("pff_param_vjp", ctypes.c_int32, [_P, _P, _P, _P, _P]),
    ("pff_tcv_adjoint", ctypes.c_int32, [_P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                         _P, _P, ctypes.POINTER(SolveInfo), _P]),
    ("pff_active_set", ctypes.c_int32, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double), _P]),
    ("pff_inverse_diagonal", ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_int64), _P]),
    ("pff_tcv_adjoint_steps", ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32,
                                               ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                               ctypes.POINTER(SolveInfo), _P]),
]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise ImportError("libpff.so is not built: run `python -c \"import __graft_entry__ as g; g.build()\"`")
        L = ctypes.CDLL(LIBPATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return [s[0] for s in _SIGS]


def check(status):
    if status != PFF_OK:
        raise PffError(status, lib().pff_last_error().decode())


def ptr(t):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream
