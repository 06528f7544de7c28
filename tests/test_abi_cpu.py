"""CPU-side checks of the C ABI: the library builds, loads and exports every
declared symbol; plan creation validates exactly; the unrolled plan equals
the oracle's independent unrolling; argument errors are caught on the host
before any launch."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import _lib
from oracle import tensor
from tests import _golden_io as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ALGS = sorted(glob.glob(os.path.join(fmm.ALGORITHM_DIR, "*.fmm")))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    names = declared_functions()
    assert "fmm_gemm" in names and "fmm_plan_create" in names
    for name in names:
        assert hasattr(L, name), name


def test_status_strings():
    L = _lib.lib()
    for st in range(0, -7, -1):
        s = L.fmm_status_string(st).decode()
        assert s and s != "unknown status"


def _factors_from_file(path):
    M, K, N, R, U, V, W = tensor.load_fmm(path)
    return M, K, N, tensor.to_float(U), tensor.to_float(V), tensor.to_float(W)


def test_printed_strassen_rejected():
    M, K, N, R, U, V, W = tensor.parse_fmm(G.read_text("strassen_printed_factors.txt"))
    with pytest.raises(fmm.FmmError) as ei:
        fmm.Plan(factors=(M, K, N, tensor.to_float(U), tensor.to_float(V), tensor.to_float(W)))
    assert ei.value.status == fmm.FMM_ERR_INVALID_ALGORITHM


@pytest.mark.parametrize("path", ALGS)
def test_plan_accepts_shipped_algorithms(path):
    p = fmm.Plan(path, levels=1)
    inf = p.info()
    M, K, N, R, U, V, W = tensor.load_fmm(path)
    assert (inf["M"], inf["K"], inf["N"], inf["R"], inf["leaves"]) == (M, K, N, R, R)
    assert inf["nnz_a_terms"] == tensor.nnz(U)
    assert inf["nnz_b_terms"] == tensor.nnz(V)
    assert inf["nnz_c_terms"] == tensor.nnz(W)


def _compare_unrolling(path, levels):
    M, K, N, R, U, V, W = tensor.load_fmm(path)
    flat = tensor.flatten(M, K, N, U, V, W, levels)
    p = fmm.Plan(path, levels=levels)
    Q = (K ** levels, N ** levels, N ** levels)
    for which in range(3):
        ptr, row, col, coef = p.leaf_terms(which)
        F = flat[which]
        ncols = Q[which]
        # the library lists each leaf's blocks in ascending (row, col); the
        # oracle's matrix holds them by row-order vec index
        for r in range(R ** levels):
            got = [(int(row[t]), int(col[t]), float(coef[t])) for t in range(ptr[r], ptr[r + 1])]
            want = [(i // ncols, i % ncols, float(F[i][r])) for i in range(len(F)) if F[i][r] != 0]
            assert got == sorted(want), (which, r)


@pytest.mark.parametrize("path", ALGS)
@pytest.mark.parametrize("levels", [1, 2])
def test_unrolling_matches_oracle(path, levels):
    _compare_unrolling(path, levels)


def test_unrolling_matches_oracle_strassen_l3():
    _compare_unrolling(os.path.join(fmm.ALGORITHM_DIR, "strassen_222_7.fmm"), 3)


def test_plan_argument_errors():
    L = _lib.lib()
    h = ctypes.c_void_p()
    U = np.zeros((4, 7))
    st = L.fmm_plan_create(ctypes.byref(h), 2, 2, 2, 7, U.ctypes.data, None, U.ctypes.data, 1, 0, 3)
    assert st == fmm.FMM_ERR_ARG
    st = L.fmm_plan_create(ctypes.byref(h), 2, 2, 2, 7, U.ctypes.data, U.ctypes.data, U.ctypes.data, 9, 0, 3)
    assert st == fmm.FMM_ERR_ARG
    st = L.fmm_plan_create(ctypes.byref(h), 2, 2, 2, 7, U.ctypes.data, U.ctypes.data, U.ctypes.data, 1, 0, 1 << 9)
    assert st == fmm.FMM_ERR_ARG
    st = L.fmm_plan_load(ctypes.byref(h), b"/nonexistent/file.fmm", 1, 0, 3)
    assert st == fmm.FMM_ERR_ARG


def test_non_dyadic_file_unsupported(tmp_path):
    text = open(os.path.join(fmm.ALGORITHM_DIR, "strassen_222_7.fmm")).read()
    bad = text.replace("1 0 1 0 1 -1 0\n", "1/3 0 1 0 1 -1 0\n", 1)
    p = tmp_path / "bad.fmm"
    p.write_text(bad)
    with pytest.raises(fmm.FmmError) as ei:
        fmm.Plan(str(p))
    assert ei.value.status == fmm.FMM_ERR_UNSUPPORTED


def test_scaled_algorithm_accepted():
    # Prop 2.3 diagonal scaling (D_x D_y D_z = I) keeps an algorithm exact;
    # the library's check must accept it, and reject a broken scaling
    M, K, N, U, V, W = _factors_from_file(os.path.join(fmm.ALGORITHM_DIR, "strassen_222_7.fmm"))
    d = np.array([2.0, 0.5, 1.0, -1.0, 4.0, 1.0, 0.25])
    fmm.Plan(factors=(M, K, N, U * d, V / d, W))
    with pytest.raises(fmm.FmmError):
        fmm.Plan(factors=(M, K, N, U * d, V, W))


def test_workspace_sizes():
    p = fmm.Plan("strassen_222_7", levels=1, flags=fmm.FLAGS_DEFAULT)
    assert p.workspace_size(512, 512, 512) == 0
    p = fmm.Plan("strassen_222_7", levels=1, flags=0)
    # write-once: 5 S slots + 5 T slots of 256^2, 7 products of 256^2
    assert p.workspace_size(512, 512, 512) == (5 + 5 + 7) * 256 * 256 * 8
    p = fmm.Plan("strassen_222_7", levels=2, flags=fmm.FLAG_FUSED_ST)
    assert p.workspace_size(1024, 1024, 1024) == 49 * 256 * 256 * 8
    # level by level: every level's S, T and products are kept
    p = fmm.Plan("strassen_222_7", levels=2, flags=fmm.FLAG_LEVELWISE)
    per_operand = 7 * 512 * 512 * 8 + 49 * 256 * 256 * 8
    assert p.workspace_size(1024, 1024, 1024) == 3 * per_operand
    p = fmm.Plan("strassen_222_7", levels=2, flags=fmm.FLAG_LEVELWISE | fmm.FLAG_FUSED_W)
    assert p.workspace_size(1024, 1024, 1024) == 2 * per_operand


def test_gemm_argument_errors_before_launch():
    L = _lib.lib()
    p = fmm.Plan("strassen_222_7", levels=1)
    buf = (ctypes.c_double * 64)()
    a = ctypes.addressof(buf)
    # null pointers, bad sizes, short leading dimensions, misalignment, aliasing
    cases = [
        (None, 4, a, 4, a + 256, 4, 4, 4, 4),
        (a, 4, a + 128, 4, a + 256, 4, 0, 4, 4),
        (a, 3, a + 128, 4, a + 256, 4, 4, 4, 4),
        (a + 4, 4, a + 128, 4, a + 256, 4, 4, 4, 4),
        (a, 4, a + 128, 4, a + 8, 4, 4, 4, 4),
    ]
    for A, lda, B, ldb, C, ldc, m, k, n in cases:
        st = L.fmm_gemm(p.handle, A, lda, B, ldb, C, ldc, m, k, n, None, 0, None)
        assert st == fmm.FMM_ERR_ARG
        st = L.fmm_classical_gemm(A, lda, B, ldb, C, ldc, m, k, n, None)
        assert st == fmm.FMM_ERR_ARG
    st = L.fmm_gemm(None, a, 4, a + 128, 4, a + 256, 4, 4, 4, 4, None, 0, None)
    assert st == fmm.FMM_ERR_ARG


def test_host_pipeline_argument_errors():
    L = _lib.lib()
    for bands, gemm_bands in [(-1, 0), (0, -1), (65, 0), (0, 65)]:
        assert L.fmm_set_host_pipeline(bands, gemm_bands) == fmm.FMM_ERR_ARG
    assert L.fmm_set_host_pipeline(64, 64) == fmm.FMM_OK
    assert L.fmm_set_host_pipeline(0, 0) == fmm.FMM_OK


def test_write_once_workspace_too_small_is_reported():
    L = _lib.lib()
    p = fmm.Plan("strassen_222_7", levels=1, flags=0)
    buf = (ctypes.c_double * 64)()
    a = ctypes.addressof(buf)
    st = L.fmm_gemm(p.handle, a, 2, a + 64, 2, a + 128, 2, 2, 2, 2, None, 0, None)
    assert st == fmm.FMM_ERR_NO_MEMORY


def test_emulated_and_tf32_workspace_layouts():
    # the documented layouts, region by region (256-byte aligned)
    al = lambda x: (x + 255) // 256 * 256
    n = 8192
    # Strassen 1 level, 12 moduli: exponents, 7 x 12 bf16 planes per operand
    # (4096 x 4096, k padded to 64), 7 x 12 int8 product planes (rows padded to 16)
    p = fmm.Plan("strassen_222_7", levels=1, precision="ozaki_bf16", moduli=12)
    want = al(n * 4) * 2 + 2 * al(7 * 12 * 4096 * 4096 * 2) + al(7 * 12 * 4096 * 4096)
    assert p.workspace_size(n, n, n) == want == 7046496256
    # the host entry point adds device copies of A, B and C in front
    assert fmm.host_workspace_size(p, n, n, n) == 3 * al(n * n * 8) + want
    # no level: the classical emulated product, 12 planes per operand
    p0 = fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16", moduli=12)
    assert p0.workspace_size(n, n, n) == al(n * 4) * 2 + 2 * al(12 * n * n * 2) + al(12 * n * n)
    # TF32 operands in FP32 with k padded to 32; the FP32-accurate variant triples k
    kpad = 1024
    assert fmm.Plan("strassen_222_7", levels=0, precision="tf32").workspace_size(1000, 1000, 1000) == \
        2 * al(1000 * kpad * 4)
    assert fmm.Plan("strassen_222_7", levels=0, precision="fp32").workspace_size(1000, 1000, 1000) == \
        2 * al(1000 * 3 * kpad * 4)


def test_wait_limit_argument_errors():
    # checked on the host, no GPU involved
    L = _lib.lib()
    assert L.fmm_set_wait_limit(0) == fmm.FMM_ERR_ARG
    assert L.fmm_set_wait_limit(2_000_000_000) == fmm.FMM_OK
    assert L.fmm_selftest_wait_timeout(2, 1000, None) == fmm.FMM_ERR_ARG
    assert L.fmm_selftest_wait_timeout(0, 0, None) == fmm.FMM_ERR_ARG
