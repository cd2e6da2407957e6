"""ctypes view of include/ps.h.  Loading only; no arithmetic lives here."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libps.so")

PS_OK = 0
PS_ERR_INVALID_ARG = 1
PS_ERR_CUDA = 2
PS_ERR_WORKSPACE = 3
PS_ERR_UNSUPPORTED = 4
PS_ERR_TIMEOUT = 5
PS_ERR_DEVICE_STATUS = 6

PS_F32, PS_BF16, PS_F16, PS_F64, PS_F32X4, PS_BF16X4, PS_F16X4 = 0, 1, 2, 3, 4, 5, 6

PS_DEV_OK = 0
PS_DEV_NONFINITE_POS = 1
PS_DEV_TIMEOUT = 2
PS_DEV_BAD_BINS = 3


class PsGrid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("L", ctypes.c_double * 3)]


class PsBatchField(ctypes.Structure):
    _fields_ = [("field", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("scale", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_D = ctypes.c_double
_GP = ctypes.POINTER(PsGrid)

# name -> (restype, argtypes); mirrors include/ps.h
SIGNATURES = {
    "ps_last_error": (ctypes.c_char_p, []),
    "ps_version": (ctypes.c_char_p, []),
    "ps_coef_row_pitch": (_I64, [_I, _I]),
    "ps_tune_set": (_I, [ctypes.c_char_p, _I64]),
    "ps_tune_get": (_I64, [ctypes.c_char_p]),
    "ps_status_clear": (_I, [_P, _P]),
    "ps_status_read": (_I, [_P, _P, _P]),
    "ps_spline_coeffs_workspace_size": (_SZ, [_GP, _I, _I]),
    "ps_spline_coeffs": (_I, [_GP, _I, _I, _P, _I, _P, _P, _P, _SZ, _P]),
    "ps_spline_truncated_workspace_size": (_SZ, [_GP, _I]),
    "ps_spline_coeffs_truncated": (_I, [_GP, _I, _P, _I, _P, _P, _SZ, _P]),
    "ps_bin_workspace_size": (_SZ, [_GP, _P, _I64]),
    "ps_bin_particles": (_I, [_GP, _P, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "ps_bin_particles_noalloc": (_I, [_GP, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "ps_interp": (_I, [_GP, _I, _I, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ps_interp_backward": (_I, [_GP, _I, _I, _P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "ps_interp_hessian": (_I, [_GP, _I, _I, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "ps_lagrangian_accel": (_I, [_GP, _I, _P, _P, _P, _P, _D, _I64, _P, _P, _P, _P, _P, _P,
                                _P, _P]),
    "ps_batch_plan": (_I, [_I, _GP, _P, _I, _P, ctypes.c_char_p, _P]),
    "ps_batch_workspace_size": (_SZ, [_P]),
    "ps_batch_num_particles": (_I64, [_P]),
    "ps_batch_particle_base": (_I64, [_P, _I]),
    "ps_batch_run": (_I, [_P, _P, _I, _P, _P, _P, _I, _D, _I, _P, _SZ, _P, _P]),
    "ps_plan_destroy": (None, [_P]),
    "ps_rk2_workspace_size": (_SZ, [_GP, _P, _I64]),
    "ps_rk2_step": (_I, [_GP, _I, _P, _P, _P, _P, _I64, _P, _P, _P, _D, _P, _I, _P, _P, _SZ,
                         _P, _P]),
    "ps_rk2_sort": (_I, [_GP, _P, _I64, _P, _P, _I, _P, _P, _P, _P, _SZ, _P, _P]),
}

_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libps.so (building it with nvcc first if it is missing or stale).
    Raises if the library cannot be built or loaded: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libps.so not found at {LIB_PATH}; run "
                               "python -m paper_2005_13193_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return list(SIGNATURES)
