"""Oracle: the matrix-multiplication tensor, exact checks of the Brent
equations, L-level flattening, and the permutations of Props 2.1 and 2.2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Everything here is exact: coefficients are ``fractions.Fraction``; the Brent
check scales each factor matrix to integers by the least common multiple of
its denominators and compares integer sums, so no floating point is involved.
"""
from fractions import Fraction
from math import lcm
import itertools

import numpy as np


# ---------------------------------------------------------------- file format
def parse_fmm(text):
    """Parse the text form of an algorithm: a '#' comment, a line 'M K N R',
    then blocks 'U', 'V', 'W' with MK, KN, MN rows of R rationals (p or p/q).
    Rows follow the row-order vectorisation of A, B, C (Section 2.2.2)."""
    lines = [ln.split("#", 1)[0].strip() for ln in text.splitlines()]
    lines = [ln for ln in lines if ln]
    M, K, N, R = (int(t) for t in lines[0].split())
    out = {}
    pos = 1
    for name, rows in (("U", M * K), ("V", K * N), ("W", M * N)):
        if lines[pos] != name:
            raise ValueError(f"expected block {name}, got {lines[pos]!r}")
        pos += 1
        mat = []
        for _ in range(rows):
            vals = [Fraction(t) for t in lines[pos].split()]
            if len(vals) != R:
                raise ValueError(f"row of {name} has {len(vals)} entries, expected {R}")
            mat.append(vals)
            pos += 1
        out[name] = mat
    return M, K, N, R, out["U"], out["V"], out["W"]


def load_fmm(path):
    with open(path) as fh:
        return parse_fmm(fh.read())


# ------------------------------------------------------------- the tensor T
def matmul_tensor(M, K, N):
    """The <M,K,N> tensor of Section 2.2.2: dims MK x KN x MN, entry 1 exactly
    when (1-indexed i, j, k)
        (i-1) mod K = floor((j-1)/N),
        (j-1) mod N = (k-1) mod N,
        floor((i-1)/K) = floor((k-1)/N),
    returned as a dense 0/1 integer array indexed from 0."""
    T = np.zeros((M * K, K * N, M * N), dtype=np.int64)
    for i in range(1, M * K + 1):
        for j in range(1, K * N + 1):
            for k in range(1, M * N + 1):
                if ((i - 1) % K == (j - 1) // N
                        and (j - 1) % N == (k - 1) % N
                        and (i - 1) // K == (k - 1) // N):
                    T[i - 1, j - 1, k - 1] = 1
    return T


def _to_int_matrix(F):
    """Integer matrix G and scale d with F = G / d exactly."""
    d = 1
    for row in F:
        for v in row:
            d = lcm(d, Fraction(v).denominator)
    G = np.array([[int(Fraction(v) * d) for v in row] for row in F], dtype=object)
    return G, d


def brent_violations(M, K, N, U, V, W, limit=None):
    """List of (i, j, q, lhs) where Eq. (2),
        T_ijq = sum_r u_ir v_jr w_qr,
    fails; lhs is the exact rational value of the sum.  Empty list <=> the
    factor matrices are an exact algorithm for <M,K,N>."""
    R = len(U[0])
    T = matmul_tensor(M, K, N)
    Gu, du = _to_int_matrix(U)
    Gv, dv = _to_int_matrix(V)
    Gw, dw = _to_int_matrix(W)
    scale = du * dv * dw
    I, J, Q = M * K, K * N, M * N
    acc = {}
    # sparse accumulation over the nonzeros of each rank-one term
    for r in range(R):
        iu = [(i, Gu[i, r]) for i in range(I) if Gu[i, r] != 0]
        jv = [(j, Gv[j, r]) for j in range(J) if Gv[j, r] != 0]
        qw = [(q, Gw[q, r]) for q in range(Q) if Gw[q, r] != 0]
        for (i, a), (j, b), (q, c) in itertools.product(iu, jv, qw):
            acc[(i, j, q)] = acc.get((i, j, q), 0) + a * b * c
    bad = []
    keys = set(acc) | {tuple(int(t) for t in idx) for idx in zip(*np.nonzero(T))}
    for key in sorted(keys):
        lhs = acc.get(key, 0)
        if lhs != int(T[key]) * scale:
            bad.append((*key, Fraction(lhs, scale)))
            if limit is not None and len(bad) >= limit:
                break
    return bad


def is_exact_algorithm(M, K, N, U, V, W):
    return not brent_violations(M, K, N, U, V, W, limit=1)


# ------------------------------------------------------------ recursion
def flatten(M, K, N, U, V, W, levels):
    """Factor matrices of L = ``levels`` recursive steps viewed as one base
    case <M^L, K^L, N^L; R^L> (the recursion of Section 3.1 unrolled).

    Leaf r = (r_1, ..., r_L), r_1 the outermost step, has index
    sum_l r_l R^(L-l).  A block of A at step l is (a_l, b_l) with
    i_l = a_l K + b_l; after L steps the block sits in row
    sum_l a_l M^(L-l) and column sum_l b_l K^(L-l) of the M^L x K^L grid of
    blocks, and its coefficient in S_r is prod_l U[i_l, r_l] (the same for
    B with V and for C with W)."""
    R = len(U[0])

    def one(F, P, Q):
        rows = (P ** levels) * (Q ** levels)
        out = [[Fraction(0)] * (R ** levels) for _ in range(rows)]
        for rs in itertools.product(range(R), repeat=levels):
            r = 0
            for rl in rs:
                r = r * R + rl
            for idx in itertools.product(range(P * Q), repeat=levels):
                coef = Fraction(1)
                for il, rl in zip(idx, rs):
                    coef *= F[il][rl]
                    if coef == 0:
                        break
                if coef == 0:
                    continue
                row = col = 0
                for il in idx:
                    row = row * P + il // Q
                    col = col * Q + il % Q
                out[row * (Q ** levels) + col][r] = coef
        return out

    return one(U, M, K), one(V, K, N), one(W, M, N)


# --------------------------------------------------------- Props 2.1, 2.2
def perm_matrix(I, J):
    """P_{IxJ}: P vec(A) = vec(A^T) for an I x J matrix A (row-order vec)."""
    P = [[0] * (I * J) for _ in range(I * J)]
    for i in range(I):
        for j in range(J):
            P[j * I + i][i * J + j] = 1
    return P


def _matmul(P, F):
    return [[sum((Fraction(P[a][b]) * F[b][r] for b in range(len(F)) if P[a][b]), Fraction(0))
             for r in range(len(F[0]))] for a in range(len(P))]


def prop21(M, K, N, U, V, W):
    """Prop 2.1: [[P_{KxN} V, P_{MxK} U, P_{MxN} W]] computes <N,K,M>."""
    return (N, K, M, _matmul(perm_matrix(K, N), V), _matmul(perm_matrix(M, K), U),
            _matmul(perm_matrix(M, N), W))


def prop22(M, K, N, U, V, W):
    """Prop 2.2: [[P_{MxN} W, U, P_{KxN} V]] computes <N,M,K>."""
    return (N, M, K, _matmul(perm_matrix(M, N), W), [row[:] for row in U],
            _matmul(perm_matrix(K, N), V))


def classical_algorithm(M, K, N):
    """The rank-MKN decomposition of the classical algorithm (one product
    A_ab B_bc per term, Section 2.1 for <2,2,2>)."""
    R = M * K * N
    U = [[Fraction(0)] * R for _ in range(M * K)]
    V = [[Fraction(0)] * R for _ in range(K * N)]
    W = [[Fraction(0)] * R for _ in range(M * N)]
    r = 0
    for a in range(M):
        for b in range(K):
            for c in range(N):
                U[a * K + b][r] = Fraction(1)
                V[b * N + c][r] = Fraction(1)
                W[a * N + c][r] = Fraction(1)
                r += 1
    return U, V, W


def nnz(F):
    return sum(1 for row in F for v in row if v != 0)


def to_float(F):
    return np.array([[float(v) for v in row] for row in F], dtype=np.float64)
