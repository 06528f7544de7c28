"""Pins of the oracle's tensor code against what the paper prints and what
the mathematics fixes (Section 2.2, Eq. 2, Props 2.1-2.2)."""
import glob
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import tensor
from tests import _golden_io as G

ALG = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1409_2908_gb300", "algorithms")


def test_tensor_222_matches_printed_slices():
    # Section 2.2.2 prints the four frontal slices of the <2,2,2> tensor
    T = tensor.matmul_tensor(2, 2, 2)
    slices = G.tensor_slices("matmul_tensor_222_slices.txt")
    assert len(slices) == 4
    for k, S in enumerate(slices):
        assert T[:, :, k].tolist() == S


@pytest.mark.parametrize("M,K,N", [(1, 1, 1), (2, 3, 4), (3, 2, 3), (4, 2, 4), (3, 3, 3), (4, 2, 3)])
def test_tensor_is_the_bilinear_map_of_matmul(M, K, N):
    # T x1 vec(A) x2 vec(B) = vec(AB) for all A, B (Section 2.2.2); checked
    # on integer matrices, where every quantity is exact
    T = tensor.matmul_tensor(M, K, N)
    assert T.shape == (M * K, K * N, M * N)
    assert int(T.sum()) == M * K * N
    rng = np.random.default_rng(7)
    for _ in range(3):
        A = rng.integers(-5, 6, size=(M, K))
        B = rng.integers(-5, 6, size=(K, N))
        z = np.einsum("ijq,i,j->q", T, A.reshape(-1), B.reshape(-1))
        assert z.tolist() == (A @ B).reshape(-1).tolist()


def test_strassen_text_formulas_are_exact():
    U, V, W = G.formulas_to_factors("strassen_text_formulas.txt")
    assert tensor.brent_violations(2, 2, 2, U, V, W) == []


def test_classical_formulas_are_exact_rank8():
    U, V, W = G.formulas_to_factors("classical_222_formulas.txt")
    assert len(U[0]) == 8
    assert tensor.brent_violations(2, 2, 2, U, V, W) == []


def test_printed_strassen_w_is_rejected():
    # the W printed in Section 2.2.2 disagrees with the formulas; the exact
    # check must find it wrong (14 of the 64 Brent equations fail)
    M, K, N, R, U, V, W = tensor.parse_fmm(G.read_text("strassen_printed_factors.txt"))
    bad = tensor.brent_violations(M, K, N, U, V, W)
    assert len(bad) == 14
    # the printed U and V agree with the written-out S_r and T_r
    Ut, Vt, Wt = G.formulas_to_factors("strassen_text_formulas.txt")
    assert U == Ut and V == Vt and W != Wt


def test_strassen_file_matches_text():
    M, K, N, R, U, V, W = tensor.load_fmm(os.path.join(ALG, "strassen_222_7.fmm"))
    Ut, Vt, Wt = G.formulas_to_factors("strassen_text_formulas.txt")
    assert (M, K, N, R) == (2, 2, 2, 7)
    assert (U, V, W) == (Ut, Vt, Wt)


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(ALG, "*.fmm"))))
def test_every_shipped_algorithm_is_exact(path):
    M, K, N, R, U, V, W = tensor.load_fmm(path)
    assert tensor.brent_violations(M, K, N, U, V, W) == []
    # dyadic coefficients only: integer inputs stay exact on the fast path
    for F in (U, V, W):
        for row in F:
            for v in row:
                d = v.denominator
                assert d & (d - 1) == 0


def _strassen():
    return tensor.load_fmm(os.path.join(ALG, "strassen_222_7.fmm"))


@pytest.mark.parametrize("mutation", ["drop_term", "flip_sign", "swap_w_rows", "transpose_u"])
def test_brent_check_detects_plausible_mistakes(mutation):
    M, K, N, R, U, V, W = _strassen()
    U = [row[:] for row in U]
    W = [row[:] for row in W]
    if mutation == "drop_term":
        W[0][3] = Fraction(0)
    elif mutation == "flip_sign":
        U[3][6] = -U[3][6]
    elif mutation == "swap_w_rows":
        W[1], W[2] = W[2], W[1]
    elif mutation == "transpose_u":
        U[1], U[2] = U[2], U[1]
    assert tensor.brent_violations(M, K, N, U, V, W) != []


def test_classical_algorithm_generic_is_exact():
    for M, K, N in [(2, 3, 4), (3, 2, 3), (4, 2, 4)]:
        U, V, W = tensor.classical_algorithm(M, K, N)
        assert tensor.is_exact_algorithm(M, K, N, U, V, W)


def test_perm_matrix_transposes_vec():
    A = np.arange(12).reshape(3, 4)
    P = np.array(tensor.perm_matrix(3, 4))
    assert (P @ A.reshape(-1)).tolist() == A.T.reshape(-1).tolist()


@pytest.mark.parametrize("which", ["prop21", "prop22"])
def test_props_keep_exactness(which):
    # Props 2.1 and 2.2 map an algorithm for <M,K,N> to one for <N,K,M> and
    # <N,M,K>; applied to a non-square classical decomposition and to Strassen
    for M, K, N, U, V, W in [(2, 3, 4, *tensor.classical_algorithm(2, 3, 4)),
                             (2, 2, 2, *_strassen()[4:])]:
        out = getattr(tensor, which)(M, K, N, U, V, W)
        M2, K2, N2 = out[:3]
        if which == "prop21":
            assert (M2, K2, N2) == (N, K, M)
        else:
            assert (M2, K2, N2) == (N, M, K)
        assert tensor.is_exact_algorithm(*out)


def test_prop21_without_w_permutation_fails():
    U, V, W = tensor.classical_algorithm(2, 3, 4)
    N2, K2, M2, U2, V2, W2 = tensor.prop21(2, 3, 4, U, V, W)
    assert not tensor.is_exact_algorithm(N2, K2, M2, U2, V2, W)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_flattened_strassen_is_exact(levels):
    M, K, N, R, U, V, W = _strassen()
    Uf, Vf, Wf = tensor.flatten(M, K, N, U, V, W, levels)
    assert len(Uf[0]) == R ** levels
    assert tensor.is_exact_algorithm(M ** levels, K ** levels, N ** levels, Uf, Vf, Wf)


def test_flatten_one_level_is_identity():
    M, K, N, R, U, V, W = _strassen()
    assert tensor.flatten(M, K, N, U, V, W, 1) == (U, V, W)


def test_flattened_nonsquare_is_exact():
    U, V, W = tensor.classical_algorithm(2, 1, 3)
    Uf, Vf, Wf = tensor.flatten(2, 1, 3, U, V, W, 2)
    assert tensor.is_exact_algorithm(4, 1, 9, Uf, Vf, Wf)


def test_flatten_with_wrong_block_order_fails():
    # a plausible mistake in the block-index map (K used where M belongs)
    # must break exactness for a non-square base case
    U, V, W = tensor.classical_algorithm(2, 3, 1)
    Uf, Vf, Wf = tensor.flatten(2, 3, 1, U, V, W, 2)
    # permute rows of Uf as if row and column digits were interleaved wrongly
    rows = len(Uf)
    bad = [Uf[(i * 7) % rows] for i in range(rows)]
    assert not tensor.is_exact_algorithm(4, 9, 1, bad, Vf, Wf)
