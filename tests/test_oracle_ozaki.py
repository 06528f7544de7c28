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
    # integer inputs whose rows fit in beta bits scale to integers exactly (no
    # rounding), so the emulation reproduces the exact product
    rng = np.random.default_rng(2)
    A = rng.integers(-4, 5, (9, 40)).astype(np.float64)
    B = rng.integers(-4, 5, (40, 11)).astype(np.float64)
    assert np.array_equal(ozaki.emulated_gemm(A, B, 12), A @ B)


def test_round_half_away_against_exact_rationals():
    # brute force against exact rational rounding (floor(|y| + 1/2), sign
    # restored) on ties, near-ties and values over many binades
    from fractions import Fraction
    rng = np.random.default_rng(7)
    ties = [0.5, -0.5, 1.5, -1.5, 2.5, -2.5, 2.0 ** 51 + 0.5, -(2.0 ** 40 + 0.5), 0.0, -0.0]
    near = [0.49999999999999994, -0.49999999999999994, 2.5 - 2 ** -51, 1.0 - 2 ** -53]
    rand = list(rng.uniform(-1, 1, 200) * 2.0 ** rng.integers(-3, 60, 200))
    ys = np.array(ties + near + rand)
    got = ozaki.round_half_away(ys)
    for y, g in zip(ys, got):
        a = Fraction(abs(float(y)))
        want = (a + Fraction(1, 2)).__floor__()
        assert g == (-want if y < 0 else want), y
    assert list(ozaki.round_half_away(np.array([0.5, 2.5, -2.5]))) == [1.0, 3.0, -3.0]


def test_scaled_entries_round_to_nearest():
    # |A_ij 2^s_i - A'_ij| <= 1/2 (truncation would leave errors up to 1), and
    # |A'_ij| <= 2^beta, with the row maximum mapped into [2^(beta-1), 2^beta]
    rng = np.random.default_rng(8)
    A = rng.uniform(-1, 1, (20, 50)) * 2.0 ** rng.integers(-30, 30, (20, 1))
    beta = 20
    Ai, s = ozaki.scale_rows(A, beta)
    exact = np.ldexp(A, s[:, None])      # exact: powers of two, no underflow here
    assert np.all(np.abs(exact - Ai) <= 0.5)
    assert np.max(np.abs(exact - Ai)) > 0.45   # the bound is reached, not slack
    assert np.all(np.abs(Ai) <= 2 ** beta)
    mx = np.abs(Ai).max(axis=1)
    assert np.all((mx >= 2 ** (beta - 1)) & (mx <= 2 ** beta))
    # a row maximum just below 2^(e+1) rounds up to exactly 2^beta
    Ai2, _ = ozaki.scale_rows(np.array([[2.0 - 2.0 ** -40, 0.25]]), beta)
    assert Ai2[0, 0] == 2 ** beta


@pytest.mark.parametrize("n", [8, 12, 15])
def test_error_within_rounding_bound(n):
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (12, 64))
    B = rng.uniform(-1, 1, (64, 10))
    C = ozaki.emulated_gemm(A, B, n)
    Cl = oracle.gemm(A, B, precision="ld")
    beta = ozaki.beta_bits(n, 64)
    # |dA_ij| <= 2^-beta max_j |A_ij| (likewise B): rounding to nearest moves
    # each scaled entry by at most 1/2, and 2^-s_i <= 2^(1-beta) max_j |A_ij|
    ra = np.abs(A).max(axis=1, keepdims=True) * 2.0 ** (-beta)
    rb = np.abs(B).max(axis=0, keepdims=True) * 2.0 ** (-beta)
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


@pytest.mark.parametrize("kind,n", [("uniform", 12), ("uniform", 14), ("loguniform", 13)])
def test_emulated_entries_match_full_emulation(kind, n):
    from paper_1409_2908_gb300 import synth
    A, B = synth.operands(37, 90, 29, 9, kind=kind)
    C = ozaki.emulated_gemm(A, B, n)
    rng = np.random.default_rng(10)
    rows = rng.integers(0, 37, 60)
    cols = rng.integers(0, 29, 60)
    assert np.array_equal(ozaki.emulated_entries(A, B, rows, cols, n), C[rows, cols])
