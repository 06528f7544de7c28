"""ctypes loader for libfmm.so (the C ABI in include/fmm.h).

The library is built in-tree by build.py.  There is no fallback: if the
shared object is missing and cannot be built, loading raises."""
import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_i64 = ctypes.c_int64
c_p = ctypes.c_void_p


class PlanInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("K", ctypes.c_int), ("N", ctypes.c_int), ("R", ctypes.c_int),
                ("levels", ctypes.c_int), ("flags", ctypes.c_uint),
                ("leaves", c_i64), ("nnz_a_terms", c_i64), ("nnz_b_terms", c_i64),
                ("nnz_c_terms", c_i64), ("max_a_terms", ctypes.c_int),
                ("max_b_terms", ctypes.c_int), ("max_c_terms", ctypes.c_int)]


def _declare(L):
    st = ctypes.c_int
    L.fmm_plan_create.argtypes = [ctypes.POINTER(c_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, c_p, c_p, c_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_uint]
    L.fmm_plan_create.restype = st
    L.fmm_plan_load.argtypes = [ctypes.POINTER(c_p), ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                ctypes.c_uint]
    L.fmm_plan_load.restype = st
    L.fmm_plan_destroy.argtypes = [c_p]
    L.fmm_plan_destroy.restype = None
    L.fmm_plan_set_tile.argtypes = [c_p, ctypes.c_int]
    L.fmm_plan_set_tile.restype = st
    L.fmm_plan_info.argtypes = [c_p, ctypes.POINTER(PlanInfo)]
    L.fmm_plan_info.restype = st
    L.fmm_plan_leaf_terms.argtypes = [c_p, ctypes.c_int, c_p, c_p, c_p, c_p, c_i64]
    L.fmm_plan_leaf_terms.restype = st
    L.fmm_workspace_size.argtypes = [c_p, c_i64, c_i64, c_i64, ctypes.POINTER(ctypes.c_size_t)]
    L.fmm_workspace_size.restype = st
    L.fmm_gemm.argtypes = [c_p, c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64, c_i64, c_i64, c_p,
                           ctypes.c_size_t, c_p]
    L.fmm_gemm.restype = st
    L.fmm_classical_gemm.argtypes = [c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64, c_i64, c_i64, c_p]
    L.fmm_classical_gemm.restype = st
    L.fmm_host_workspace_size.argtypes = [c_p, c_i64, c_i64, c_i64, ctypes.POINTER(ctypes.c_size_t)]
    L.fmm_host_workspace_size.restype = st
    L.fmm_set_host_pipeline.argtypes = [ctypes.c_int, ctypes.c_int]
    L.fmm_set_host_pipeline.restype = st
    L.fmm_gemm_host.argtypes = [c_p, c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64, c_i64, c_i64,
                                c_p, ctypes.c_size_t, c_p]
    L.fmm_gemm_host.restype = st
    L.fmm_gemm_noalloc.argtypes = [c_p, c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64, c_i64, c_i64, c_p]
    L.fmm_gemm_noalloc.restype = st
    L.fmm_workspace_size_batched.argtypes = [c_p, c_i64, c_i64, c_i64, c_i64, ctypes.POINTER(ctypes.c_size_t)]
    L.fmm_workspace_size_batched.restype = st
    L.fmm_gemm_batched.argtypes = [c_p, c_i64, c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64, c_i64, c_i64,
                                   c_p, ctypes.c_size_t, c_p]
    L.fmm_gemm_batched.restype = st
    L.fmm_plan_prepare.argtypes = [c_p]
    L.fmm_plan_prepare.restype = st
    L.fmm_plan_set_moduli.argtypes = [c_p, ctypes.c_int]
    L.fmm_plan_set_moduli.restype = st
    L.fmm_check_device_error.argtypes = []
    L.fmm_check_device_error.restype = st
    L.fmm_last_launch_count.argtypes = []
    L.fmm_last_launch_count.restype = ctypes.c_int
    L.fmm_timing_enable.argtypes = [ctypes.c_int]
    L.fmm_timing_enable.restype = st
    L.fmm_timing_leaf_ms.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    L.fmm_timing_leaf_ms.restype = st
    L.fmm_gemm_grouped.argtypes = [c_i64, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p]
    L.fmm_gemm_grouped.restype = st
    L.fmm_set_wait_limit.argtypes = [ctypes.c_uint64]
    L.fmm_set_wait_limit.restype = st
    L.fmm_selftest_wait_timeout.argtypes = [ctypes.c_int, ctypes.c_uint64, c_p]
    L.fmm_selftest_wait_timeout.restype = st
    L.fmm_status_string.argtypes = [ctypes.c_int]
    L.fmm_status_string.restype = ctypes.c_char_p


def path():
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            if _build.stale():
                _build.build()
            L = ctypes.CDLL(_build.LIB)
            _declare(L)
            _lib = L
    return _lib
