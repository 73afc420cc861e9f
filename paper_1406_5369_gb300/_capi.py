"""ctypes declarations of the C ABI in include/mg.h, include/mg_cc.h and
include/mg_cd.h (argument marshalling only).

Loading fails loudly if libmg.so has not been built: there is no fallback
implementation of any operation in Python.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmg.so")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ENOCONV, MG_ETIMEOUT = range(6)
STATUS_NAMES = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ENOCONV",
                5: "MG_ETIMEOUT"}
MG_RBGS, MG_JACOBI = 0, 1
MG_FP64, MG_FP32_DC, MG_BF16_DC = 0, 1, 2
MG_FIELD_U, MG_FIELD_F, MG_FIELD_R = 0, 1, 2
(MG_KERNEL_PRESMOOTH, MG_KERNEL_POSTSMOOTH, MG_KERNEL_COARSE, MG_KERNEL_OUTER, MG_KERNEL_NORM, MG_KERNEL_OTHER,
 MG_KERNEL_POSTPRE) = range(7)


class mg_const_stencil(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double)]


class mg_boundary(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dirichlet_values", ctypes.c_void_p)]


class mg_options(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("omega", ctypes.c_double), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("coarsest_n", ctypes.c_int), ("maxit", ctypes.c_int),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("fuse", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("inner_cycles", ctypes.c_int), ("exact_outer", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("tile_max_n", ctypes.c_int), ("fuse_depth", ctypes.c_int),
                ("join_cycles", ctypes.c_int), ("cluster_max_n", ctypes.c_int), ("canary", ctypes.c_int)]


class mg_cc_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("c", ctypes.c_double * 3),
                ("sigma", ctypes.c_double), ("bc", ctypes.c_int), ("smoother", ctypes.c_int),
                ("omega", ctypes.c_double), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("coarsest_n", ctypes.c_int), ("maxit", ctypes.c_int), ("stream", ctypes.c_void_p)]


MG_CC_NEUMANN, MG_CC_DIRICHLET = 0, 1


class mg_cd_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("tau", ctypes.c_double), ("theta", ctypes.c_double),
                ("kappa", ctypes.c_double), ("smoother", ctypes.c_int), ("omega", ctypes.c_double),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("maxit", ctypes.c_int), ("stream", ctypes.c_void_p)]


MG_CD_U, MG_CD_F, MG_CD_R, MG_CD_GX, MG_CD_GY = range(5)

# name -> (restype, argtypes); every function declared in include/mg.h, mg_cc.h and mg_cd.h.
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "mg_default_options": (None, [ctypes.POINTER(mg_options)]),
    "mg_workspace_bytes": (ctypes.c_size_t, [_I, _I, _I, ctypes.POINTER(mg_options)]),
    "mg_create": (_I, [_I, _I, ctypes.POINTER(mg_const_stencil), _P, ctypes.POINTER(mg_boundary),
                       ctypes.POINTER(mg_options), _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "mg_destroy": (_I, [_P]),
    "mg_check_canaries": (_I, [_P, ctypes.POINTER(_I)]),
    "mg_num_levels": (_I, [_P]),
    "mg_level_size": (_I, [_P, _I]),
    "mg_set_rhs": (_I, [_P, _P]),
    "mg_set_solution": (_I, [_P, _P]),
    "mg_get_solution": (_I, [_P, _P]),
    "mg_set_field": (_I, [_P, _I, _I, _P]),
    "mg_get_field": (_I, [_P, _I, _I, _P]),
    "mg_smooth": (_I, [_P, _I, _I]),
    "mg_residual": (_I, [_P, _I]),
    "mg_restrict": (_I, [_P, _I]),
    "mg_prolongate": (_I, [_P, _I]),
    "mg_coarse_solve": (_I, [_P]),
    "mg_vcycle": (_I, [_P]),
    "mg_residual_norm": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "mg_solve": (_I, [_P, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "mg_kernel_launches": (ctypes.c_ulonglong, [_P]),
    "mg_set_timing": (_I, [_P, _I]),
    "mg_get_timing": (_I, [_P, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_ulonglong)]),
    "mg_reset_timing": (_I, [_P]),
    "mg_residual_norm_noalloc": (_I, [_I, _I, ctypes.POINTER(mg_const_stencil), _P, _P,
                                      ctypes.POINTER(_D), _P]),
    "mg_solve_sequence": (_I, [_P, _P, _P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, ctypes.POINTER(_I),
                               ctypes.POINTER(_D)]),
    "mg_batch_workspace_bytes": (ctypes.c_size_t, [_I]),
    "mg_batch_create": (_I, [_I, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "mg_batch_destroy": (_I, [_P]),
    "mg_batch_add": (_I, [_P, _P, ctypes.POINTER(_I)]),
    "mg_batch_remove": (_I, [_P, _I]),
    "mg_batch_step": (_I, [_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_D)]),
    "mg_batch_step_async": (_I, [_P, ctypes.POINTER(_I), _I]),
    "mg_batch_step_wait": (_I, [_P, ctypes.POINTER(_D)]),
    "mg_batch_solve": (_I, [_P, ctypes.POINTER(_D), _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "mg_batch_launches": (ctypes.c_ulonglong, [_P]),
    "mg_batch_set_inner_cycles": (_I, [_P, _I]),
    "mg_batch_set_tile_rows": (_I, [_P, _I]),
    "mg_batch_set_capture": (_I, [_P, _I]),
    "mg_batch_solve_profile": (_I, [_P, ctypes.POINTER(_D)]),
    "mg_batch_set_timing": (_I, [_P, _I]),
    "mg_batch_get_timing": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(_D)]),
    "mg_batch_reset_timing": (_I, [_P]),
    "mg_last_error": (ctypes.c_char_p, []),
    "mg_cc_default_params": (None, [ctypes.POINTER(mg_cc_params)]),
    "mg_cc_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(mg_cc_params)]),
    "mg_cc_create": (_I, [ctypes.POINTER(mg_cc_params), _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "mg_cc_destroy": (_I, [_P]),
    "mg_cc_num_levels": (_I, [_P]),
    "mg_cc_level_size": (_I, [_P, _I]),
    "mg_cc_set_field": (_I, [_P, _I, _I, _P]),
    "mg_cc_get_field": (_I, [_P, _I, _I, _P]),
    "mg_cc_smooth": (_I, [_P, _I, _I]),
    "mg_cc_residual": (_I, [_P, _I]),
    "mg_cc_restrict": (_I, [_P, _I]),
    "mg_cc_prolongate": (_I, [_P, _I]),
    "mg_cc_coarse_solve": (_I, [_P]),
    "mg_cc_vcycle": (_I, [_P]),
    "mg_cc_residual_norm": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "mg_cc_solve": (_I, [_P, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "mg_cd_default_params": (None, [ctypes.POINTER(mg_cd_params)]),
    "mg_cd_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(mg_cd_params)]),
    "mg_cd_create": (_I, [ctypes.POINTER(mg_cd_params), _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "mg_cd_destroy": (_I, [_P]),
    "mg_cd_num_levels": (_I, [_P]),
    "mg_cd_level_size": (_I, [_P, _I]),
    "mg_cd_set_field": (_I, [_P, _I, _I, _P]),
    "mg_cd_get_field": (_I, [_P, _I, _I, _P]),
    "mg_cd_begin_step": (_I, [_P, _P]),
    "mg_cd_smooth": (_I, [_P, _I, _I]),
    "mg_cd_residual": (_I, [_P, _I]),
    "mg_cd_restrict": (_I, [_P, _I]),
    "mg_cd_prolongate": (_I, [_P, _I]),
    "mg_cd_coarse_solve": (_I, [_P]),
    "mg_cd_vcycle": (_I, [_P]),
    "mg_cd_residual_norm": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "mg_cd_solve": (_I, [_P, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "mg_cd_time_step": (_I, [_P, _P, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
}

_lib = None


class MGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH):
    """Loads libmg.so and declares every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmg.so not built at {path}; run __graft_entry__.build() "
                          "or python -m paper_1406_5369_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != MG_OK:
        raise MGError(status, load().mg_last_error().decode(errors="replace"))
    return status
