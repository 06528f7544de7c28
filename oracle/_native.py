"""Build and load the oracle's C part (classical.c) with gcc.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py)."""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "classical.c")
_LIB = os.path.join(_HERE, "_classical.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile classical.c -> _classical.so (plain C, -O2, OpenMP, no
    fast-math and no FMA contraction, so each product and sum rounds once)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I = ctypes.c_int64
            L.oracle_gemm_f64.argtypes = [P, I, P, I, P, I, I, I, I]
            L.oracle_gemm_ld.argtypes = [P, I, P, I, P, I, I, I, I]
            L.oracle_gemm_entries.argtypes = [P, I, P, I, I, P, P, I, P, P]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(a):
    if a.dtype != np.float64 or a.ndim != 2 or a.strides[1] != 8:
        raise ValueError("oracle expects 2-D float64 arrays with unit column stride")


def gemm(A, B, precision="f64"):
    """Classical product C = A B (Section 2.1) in FP64 or long double."""
    _check(A)
    _check(B)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    C = np.empty((m, n), np.float64)
    f = lib().oracle_gemm_f64 if precision == "f64" else lib().oracle_gemm_ld
    f(_ptr(A), A.strides[0] // 8, _ptr(B), B.strides[0] // 8, _ptr(C), n, m, k, n)
    return C


def gemm_entries(A, B, rows, cols):
    """(fp64, long double) values of selected entries of A B, one dot
    product each."""
    _check(A)
    _check(B)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    k = A.shape[1]
    o64 = np.empty(len(rows))
    old = np.empty(len(rows))
    lib().oracle_gemm_entries(_ptr(A), A.strides[0] // 8, _ptr(B), B.strides[0] // 8, k,
                              _ptr(rows), _ptr(cols), len(rows), _ptr(o64), _ptr(old))
    return o64, old


def num_threads():
    return lib().oracle_num_threads()


def set_threads(n):
    lib().oracle_set_threads(int(n))
