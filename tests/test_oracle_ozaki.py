"""Pins of the emulated-FP64 oracle (CRT over small moduli) against exact
arithmetic and closed forms."""
import math

import numpy as np
import pytest

import oracle
from oracle import ozaki


def test_moduli_pairwise_coprime_and_small():
    m = ozaki.MODULI
    for i in range(len(m)):
        assert m[i] <= 256
        for j in range(i):
            assert math.gcd(m[i], m[j]) == 1


def test_balanced_residue_range():
    for p in (256, 255, 193):
        vals = {ozaki.balanced(x, p) for x in range(-1000, 1000)}
        assert min(vals) >= -(p // 2) and max(vals) <= (p - 1) // 2 + (p % 2 == 0) * 0
        assert len(vals) == p
        assert all((ozaki.balanced(x, p) - x) % p == 0 for x in range(-300, 300))


def test_crt_reconstructs_integers():
    mods = ozaki.moduli(6)
    P = math.prod(mods)
    rng = np.random.default_rng(0)
    for x in [0, 1, -1, P // 2 - 1, -(P // 2)] + [int(v) for v in rng.integers(-2**40, 2**40, 20)]:
        assert ozaki.crt([ozaki.balanced(x, p) for p in mods], mods) == x


def test_beta_keeps_product_below_half_modulus():
    for n in (8, 12, 15, 18):
        for k in (64, 1000, 16384):
            b = ozaki.beta_bits(n, k)
            P = math.prod(ozaki.moduli(n))
            assert 2 * k * (2 ** b) ** 2 < P
            if b < 62:   # maximal: one more bit would break the bound
                assert 2 * k * (2 ** (b + 1)) ** 2 >= P


def test_residue_product_matches_exact_product():
    rng = np.random.default_rng(1)
    A = rng.uniform(-1, 1, (7, 33))
    B = rng.uniform(-1, 1, (33, 5))
    beta = ozaki.beta_bits(12, 33)
    Ai, _ = ozaki.scale_rows(A, beta)
    Bi, _ = ozaki.scale_cols(B, beta)
    Z = ozaki.exact_product(Ai, Bi)
    for p in ozaki.moduli(12):
        zp = ozaki.residue_product(Ai, Bi, p)
        want = np.vectorize(lambda x: ozaki.balanced(int(x), p))(Z)
        assert np.array_equal(zp, want.astype(np.int64))
    # and the residues reconstruct Z
    res = [ozaki.residue_product(Ai, Bi, p) for p in ozaki.moduli(12)]
    for i in range(7):
        for j in range(5):
            assert ozaki.crt([r[i, j] for r in res], ozaki.moduli(12)) == Z[i, j]


def test_scaling_is_exact_for_short_integers():
    # integer inputs whose rows fit in beta bits are not truncated, so the
    # emulation reproduces the exact product
    rng = np.random.default_rng(2)
    A = rng.integers(-4, 5, (9, 40)).astype(np.float64)
    B = rng.integers(-4, 5, (40, 11)).astype(np.float64)
    assert np.array_equal(ozaki.emulated_gemm(A, B, 12), A @ B)


@pytest.mark.parametrize("n", [8, 12, 15])
def test_error_within_truncation_bound(n):
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (12, 64))
    B = rng.uniform(-1, 1, (64, 10))
    C = ozaki.emulated_gemm(A, B, n)
    Cl = oracle.gemm(A, B, precision="ld")
    beta = ozaki.beta_bits(n, 64)
    # |dA_ij| <= 2^(1-beta) max_j |A_ij| (likewise B): first-order bound
    ra = np.abs(A).max(axis=1, keepdims=True) * 2.0 ** (1 - beta)
    rb = np.abs(B).max(axis=0, keepdims=True) * 2.0 ** (1 - beta)
    colsum_b = np.abs(B).sum(axis=0, keepdims=True)
    rowsum_a = np.abs(A).sum(axis=1, keepdims=True)
    bound = ra * colsum_b + rowsum_a * rb + 64 * ra * rb + 4 * 2.0 ** -53 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - Cl) <= bound)


def test_subnormal_rows_and_columns_scale_exactly():
    # a row (and a column) of small multiples of the least subnormal 2^-1074:
    # its exponent comes from frexp, and the scaled integers are exact, so the
    # emulation reproduces the exact product (every value here is a small
    # integer times a power of two, exact in FP64)
    rng = np.random.default_rng(4)
    tiny = 2.0 ** -1074
    A = rng.integers(-4, 5, (6, 30)).astype(np.float64)
    B = rng.integers(-4, 5, (30, 5)).astype(np.float64)
    A[2] = rng.integers(-9, 10, 30) * tiny
    B[:, 3] = rng.integers(-9, 10, 30) * 2.0 ** 900
    assert np.all(np.abs(A[2]) < 2.0 ** -1022) and np.any(A[2] != 0)
    C = ozaki.emulated_gemm(A, B, 12)
    assert np.array_equal(C, A @ B)
    assert np.any(C[2] != 0)
