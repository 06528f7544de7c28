"""Pins of the oracle's recursive fast multiply: exact on integers for
every shipped algorithm and depth, L = 0 is the classical product, and the
peeled fringe is handled (Sections 3.1, 3.5)."""
import glob
import os

import numpy as np
import pytest

import oracle
from oracle import fastmm, norms, tensor

ALG = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1409_2908_gb300", "algorithms")


def _alg(name):
    M, K, N, R, U, V, W = tensor.load_fmm(os.path.join(ALG, name))
    return M, K, N, tensor.to_float(U), tensor.to_float(V), tensor.to_float(W)


ALGS = sorted(os.path.basename(p) for p in glob.glob(os.path.join(ALG, "*.fmm")))


@pytest.mark.parametrize("name", ALGS)
@pytest.mark.parametrize("levels", [1, 2])
def test_integer_exact_with_peeling(name, levels):
    M, K, N, U, V, W = _alg(name)
    rng = np.random.default_rng(levels)
    m, k, n = M ** levels * 3 + 1, K ** levels * 2 + 1, N ** levels * 3 + 2
    A = rng.integers(-4, 5, (m, k)).astype(np.float64)
    B = rng.integers(-4, 5, (k, n)).astype(np.float64)
    C = fastmm.fast_mm(A, B, M, K, N, U, V, W, levels)
    assert np.array_equal(C, oracle.gemm(A, B))


def test_levels0_is_classical():
    M, K, N, U, V, W = _alg("strassen_222_7.fmm")
    rng = np.random.default_rng(0)
    A = rng.uniform(-1, 1, (33, 17))
    B = rng.uniform(-1, 1, (17, 9))
    assert np.array_equal(fastmm.fast_mm(A, B, M, K, N, U, V, W, 0), oracle.gemm(A, B))


def test_strassen_random_error_small():
    M, K, N, U, V, W = _alg("strassen_222_7.fmm")
    rng = np.random.default_rng(1)
    A = rng.uniform(-1, 1, (256, 256))
    B = rng.uniform(-1, 1, (256, 256))
    C = oracle.gemm(A, B)
    for L in (1, 2, 3):
        e = norms.rel_frobenius(fastmm.fast_mm(A, B, M, K, N, U, V, W, L), C)
        assert e < 1e-13


def test_broken_w_gives_wrong_product():
    M, K, N, U, V, W = _alg("strassen_222_7.fmm")
    W = W.copy()
    W[3, 5] = 0.0
    A = np.arange(16.0).reshape(4, 4)
    B = np.eye(4)
    assert not np.array_equal(fastmm.fast_mm(A, B, M, K, N, U, V, W, 1), A)
