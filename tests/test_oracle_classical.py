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


def test_long_double_accumulator_keeps_what_fp64_loses():
    # 2^53 + 1 + 1 - 2^53 = 2 exactly; an FP64 accumulator rounds 2^53 + 1 back
    # to 2^53 (ties to even) and returns 0.  The wide variant must return 2: a
    # double accumulator in oracle_gemm_ld fails here.
    big = 2.0 ** 53
    A = np.array([[big, 1.0, 1.0, -big]])
    B = np.ones((4, 1))
    assert oracle.gemm(A, B)[0, 0] == 0.0          # the FP64 loop loses the ones
    assert oracle.gemm(A, B, precision="ld")[0, 0] == 2.0
    _, eld = oracle.gemm_entries(A, B, [0], [0])
    assert eld[0] == 2.0


def test_long_double_products_are_formed_wide():
    # (1 + 2^-30)^2 = 1 + 2^-29 + 2^-60: the 2^-60 term needs 61 significant
    # bits, so a product rounded to FP64 before the wide sum loses it and the
    # entry comes out 0 instead of 2^-60.
    a = 1.0 + 2.0 ** -30
    A = np.array([[a, -(1.0 + 2.0 ** -29)]])
    B = np.array([[a], [1.0]])
    assert oracle.gemm(A, B)[0, 0] == 0.0
    assert oracle.gemm(A, B, precision="ld")[0, 0] == 2.0 ** -60
    _, eld = oracle.gemm_entries(A, B, [0], [0])
    assert eld[0] == 2.0 ** -60


def test_gamma_closed_form():
    # gamma_n = n u / (1 - n u) with u = 2^-53 (unit roundoff of round to
    # nearest in FP64) equals n / (2^53 - n) exactly; gamma_1 = u / (1 - u).
    from fractions import Fraction
    for n in (1, 2, 3, 1000, 16384, 2 ** 20):
        want = Fraction(n, 2 ** 53 - n)
        assert abs(Fraction(norms.gamma(n)) - want) <= want * Fraction(1, 2 ** 52)
    assert norms.gamma(1) == pytest.approx(2.0 ** -53, rel=1e-15)
    # a unit roundoff of 2^-52 (machine epsilon) would double every bound
    assert norms.gamma(1000) < 1000 * 2.0 ** -52 * 0.75
