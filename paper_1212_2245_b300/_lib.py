"""ctypes declarations of the libdeblur C ABI (include/libdeblur.h)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdeblur.so")

c_int, c_float, c_void_p, c_size_t, c_char_p = (ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_char_p)


class DbPsf(ctypes.Structure):
    _fields_ = [("kh", c_int), ("kw", c_int), ("kind", c_int), ("taps", c_void_p)]


class DbParams(ctypes.Structure):
    _fields_ = [("K", c_float), ("alpha", c_float), ("eps_phi", c_float), ("eps_psi", c_float),
                ("pos_floor", c_float), ("phi_robust", c_int), ("psi_tv", c_int), ("conv", c_int)]


DB_PSF_GENERAL, DB_PSF_BOX = 0, 1
DB_CONV_CLAMP, DB_CONV_PERIODIC = 0, 1
SCHED_AUTO, SCHED_FUSED, SCHED_SPLIT, SCHED_FLOW, SCHED_CLUSTER = 0, 1, 2, 3, 4
RF_LOG1P, RF_LUT = 0, 1
NOALLOC_SCRATCH_BYTES = 32 << 20  # DB_NOALLOC_SCRATCH_BYTES
FLAG_TAPS, FLAG_NONFINITE, FLAG_TIMEOUT, FLAG_BOX = 0x1, 0x2, 0x4, 0x8

class DbImageDesc(ctypes.Structure):
    _fields_ = [("f", c_void_p), ("u", c_void_p), ("H", c_int), ("W", c_int), ("ld", c_int),
                ("psf", DbPsf), ("p", DbParams)]


P_PSF = ctypes.POINTER(DbPsf)
P_PAR = ctypes.POINTER(DbParams)

# name -> (restype, argtypes); every symbol declared in include/libdeblur.h
SIGNATURES = {
    "db_workspace_bytes": (c_size_t, [c_int, c_int, P_PSF, P_PAR]),
    "db_wiener": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, P_PSF, P_PAR, c_void_p, c_size_t,
                          c_void_p, c_void_p]),
    "db_rrl_iterate": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, P_PSF, P_PAR, c_int, c_void_p,
                               c_int, c_void_p, c_size_t, c_void_p, c_void_p]),
    "db_deblur": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, P_PSF, P_PAR, c_int, c_void_p,
                          c_size_t, c_void_p, c_void_p]),
    "db_workspace_bytes_n": (c_size_t, [c_int, c_int, c_int, P_PSF, P_PAR]),
    "db_deblur_n": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, ctypes.c_longlong, P_PSF, P_PAR, c_int,
                            c_void_p, c_int, c_void_p, c_size_t, c_void_p, c_void_p]),
    "db_rrl_iterate_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, P_PSF, P_PAR, c_int,
                                       c_void_p, c_void_p]),
    "db_batch_workspace_bytes": (c_size_t, [ctypes.POINTER(DbImageDesc), c_int, c_int]),
    "db_batch_create": (c_int, [ctypes.POINTER(DbImageDesc), c_int, c_int, c_void_p, c_size_t, c_void_p,
                                c_void_p, ctypes.POINTER(c_void_p)]),
    "db_batch_run": (c_int, [c_void_p, c_void_p, c_void_p]),
    "db_batch_destroy": (None, [c_void_p]),
    "db_batch_autotune": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                  ctypes.POINTER(c_int)]),
    "db_deblur_batch": (c_int, [ctypes.POINTER(DbImageDesc), c_int, c_int, c_void_p, c_size_t, c_void_p,
                                c_void_p]),
    "db_batch_stream_workspace_bytes": (c_size_t, [ctypes.POINTER(DbImageDesc), c_int, c_int, c_int]),
    "db_batch_stream_create": (c_int, [ctypes.POINTER(DbImageDesc), c_int, c_int, c_int, c_void_p, c_size_t,
                                       c_void_p, c_void_p, ctypes.POINTER(c_void_p)]),
    "db_batch_stream_run_host": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_void_p,
                                         c_void_p]),
    "db_batch_stream_parts": (c_int, [c_void_p]),
    "db_batch_stream_destroy": (None, [c_void_p]),
    "db_set_spin_limit": (c_int, [ctypes.c_longlong]),
    "db_set_batch_order": (c_int, [c_int]),
    "db_set_tma": (c_int, [c_int]),
    "db_backward_workspace_bytes": (c_size_t, [c_int, c_int, c_int, P_PSF, c_int]),
    "db_rrl_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, P_PSF, P_PAR, c_int, c_int,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "db_plan_create": (c_int, [c_int, c_int, c_int, P_PSF, P_PAR, c_int, c_void_p, c_size_t, c_void_p, c_void_p,
                               ctypes.POINTER(c_void_p)]),
    "db_plan_run": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "db_plan_run_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "db_plan_destroy": (None, [c_void_p]),
    "db_plan_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                 ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "db_host_alloc": (c_int, [c_size_t, ctypes.POINTER(c_void_p)]),
    "db_host_free": (None, [c_void_p]),
    "db_status_string": (c_char_p, [c_int]),
    "db_status_from_flags": (c_int, [c_int]),
    "db_version": (c_char_p, []),
    "db_launch_count": (ctypes.c_longlong, []),
    "db_set_schedule": (c_int, [c_int]),
    "db_set_one_axis_min": (c_int, [c_int]),
    "db_set_dense_min": (c_int, [c_int]),
    "db_set_fft_tiles": (c_int, [c_int]),
    "db_set_rf_eval": (c_int, [c_int]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libdeblur.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdeblur.so not built at {LIB_PATH}; run `python -m paper_1212_2245_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
