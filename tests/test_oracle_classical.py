"""Pins of the oracle's classical product (classical.c) against exact
integer arithmetic, closed forms and the classical error bound."""
import numpy as np
import pytest

import oracle
from oracle import norms


@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (5, 7, 3), (64, 33, 17), (130, 257, 66)])
def test_integer_inputs_exact(m, k, n):
    rng = np.random.default_rng(m * 1000 + k)
    A = rng.integers(-4, 5, size=(m, k))
    B = rng.integers(-4, 5, size=(k, n))
    C = oracle.gemm(A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(C, (A @ B).astype(np.float64))


def test_closed_forms():
    k = 37
    A = np.ones((4, k))
    B = np.ones((k, 5))
    assert np.all(oracle.gemm(A, B) == k)
    B = np.random.default_rng(1).uniform(-1, 1, (6, 9))
    assert np.array_equal(oracle.gemm(np.eye(6), B), B)


def test_leading_dimensions_respected():
    rng = np.random.default_rng(3)
    big = rng.integers(-3, 4, size=(20, 30)).astype(np.float64)
    A = big[2:9, 1:12]
    B = big[5:16, 3:20]
    assert np.array_equal(oracle.gemm(A, B), A @ B)


def test_random_within_classical_bound():
    rng = np.random.default_rng(11)
    m, k, n = 96, 300, 80
    A = rng.uniform(-1, 1, (m, k))
    B = rng.uniform(-1, 1, (k, n))
    C64 = oracle.gemm(A, B)
    Cld = oracle.gemm(A, B, precision="ld")
    bound = norms.gamma(k) * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C64 - Cld) <= bound + 1e-300)


def test_entries_match_full_product():
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (40, 50))
    B = rng.uniform(-1, 1, (50, 30))
    C = oracle.gemm(A, B)
    rows = rng.integers(0, 40, 25)
    cols = rng.integers(0, 30, 25)
    e64, eld = oracle.gemm_entries(A, B, rows, cols)
    assert np.array_equal(e64, C[rows, cols])
    assert np.all(np.abs(eld - e64) <= norms.gamma(50) * 50)


def test_error_norms():
    C = np.array([[3.0, 4.0]])
    assert norms.rel_frobenius(C, C) == 0.0
    assert norms.rel_frobenius(C + np.array([[0.0, 0.5]]), C) == pytest.approx(0.1)
    A = np.full((1, 2), 2.0)
    B = np.full((2, 2), 0.5)
    assert norms.rel_max(C + 1.0, C, A, B) == pytest.approx(1.0 / 2.0)
