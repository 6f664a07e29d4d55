"""ctypes declarations of the C ABI in include/lbm.h (argument marshalling only).

Every function of the header is exposed under the same name. Loading fails loudly if the
in-tree liblbm.so has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = range(7)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
                4: "LBM_EUNSTABLE", 5: "LBM_ETIMEOUT", 6: "LBM_ESTATE"}
LBM_BC_PERIODIC, LBM_BC_ZG, LBM_BC_NRBC = 0, 1, 2
LBM_NRBC_PNR_LODI, LBM_NRBC_CBC_RELAX = 0, 1
LBM_FP64, LBM_FP32_DEV = 0, 1
LBM_TOTALS_NOALLOC_MAX_N = 1 << 28


class lbm_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int)]


class lbm_sigma_profile(C.Structure):
    _fields_ = [("sigma_max", C.c_double), ("power", C.c_int), ("split", C.c_int)]


class lbm_bc_params(C.Structure):
    _fields_ = [("edge", C.c_int * 4), ("beta", C.c_double), ("relax_sign", C.c_double),
                ("rho0", C.c_double), ("u0x", C.c_double), ("u0y", C.c_double),
                ("T0", C.c_double), ("use_pml_widths", C.c_int), ("pml_widths", C.c_int * 4),
                ("pml_source", C.c_int), ("periodic_y", C.c_int), ("pml_grad", C.c_int)]


_dp = C.POINTER(C.c_double)
_ctx = C.c_void_p

# name -> (restype, argtypes); mirrors include/lbm.h
PROTOTYPES = {
    "lbm_create": (C.c_int, [C.POINTER(lbm_grid), C.c_int, C.c_double, C.c_int,
                             C.POINTER(lbm_sigma_profile), C.c_int, C.POINTER(lbm_bc_params),
                             C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_init": (C.c_int, [_ctx, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "lbm_step": (C.c_int, [_ctx, C.c_int]),
    "lbm_sync": (C.c_int, [_ctx]),
    "lbm_moments": (C.c_int, [_ctx, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_int]),
    "lbm_reduce": (C.c_int, [_ctx, _dp]),
    "lbm_error_sums": (C.c_int, [_ctx, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, _dp]),
    "lbm_lattice_info": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp, _dp]),
    "lbm_geometry": (C.c_int, [_ctx, C.POINTER(C.c_int64)]),
    "lbm_debug_check_guards": (C.c_int, [_ctx, C.POINTER(C.c_int)]),
    "lbm_export_populations": (C.c_int, [_ctx, _dp]),
    "lbm_import_populations": (C.c_int, [_ctx, _dp]),
    "lbm_checkpoint_size": (C.c_int, [_ctx, C.POINTER(C.c_size_t)]),
    "lbm_checkpoint": (C.c_int, [_ctx, C.c_void_p, C.c_size_t]),
    "lbm_restore": (C.c_int, [_ctx, C.c_void_p, C.c_size_t]),
    "lbm_profile_enable": (C.c_int, [_ctx, C.c_int]),
    "lbm_profile_read": (C.c_int, [_ctx, _dp, C.POINTER(C.c_int)]),
    "lbm_estimate_bytes": (C.c_int, [C.POINTER(lbm_grid), C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.POINTER(C.c_size_t)]),
    "lbm_estimate_bytes_bc": (C.c_int, [C.POINTER(lbm_grid), C.c_int, C.c_int,
                                        C.POINTER(lbm_sigma_profile), C.c_int,
                                        C.POINTER(lbm_bc_params), C.c_int,
                                        C.POINTER(C.c_size_t)]),
    "lbm_export_pull_index": (C.c_int, [_ctx, C.c_void_p]),
    "lbm_export_site_class": (C.c_int, [_ctx, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_peak_fma": (C.c_int, [C.c_int, _dp, _dp, C.c_void_p]),
    "lbm_batch_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_batch_set": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.c_int]),
    "lbm_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_batch_destroy": (C.c_int, [C.c_void_p]),
    "lbm_batch_tile": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "lbm_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int)]),
    "lbm_totals_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [_ctx]),
    "lbm_destroy": (C.c_int, [_ctx]),
}

_lib = None


def lib():
    """Load liblbm.so and declare every prototype. Raises if the library is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is not built; run `python -m paper_2504_20169_gb300.build` "
                "(no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
