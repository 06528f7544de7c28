"""Oracle: recursive fast matrix multiplication on the CPU, level by level
with write-once additions (Sections 3.1 and 3.2), for debugging and for
cross-checking rounding behaviour.  It is NOT the parity target: the parity
target is the classical product (classical.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reading of Section 3.5 (dynamic peeling): the core m' x k' x n' with m' the
largest multiple of M^L not above m (likewise k', n') goes through the fast
recursion; the fringe is added with classical products:
    C[:m', :n'] += A[:m', k':] B[k':, :n']
    C[m':, :]    = A[m':, :] B
    C[:m', n':]  = A[:m', :] B[:, n']
"""
import numpy as np

from . import _native


def _classical(A, B):
    return _native.gemm(np.ascontiguousarray(A), np.ascontiguousarray(B))


def _fast_core(A, B, M, K, N, Uf, Vf, Wf, levels):
    if levels == 0:
        return _classical(A, B)
    m, k = A.shape
    n = B.shape[1]
    mb, kb, nb = m // M, k // K, n // N
    R = Uf.shape[1]
    Ablk = [A[a * mb:(a + 1) * mb, b * kb:(b + 1) * kb] for a in range(M) for b in range(K)]
    Bblk = [B[b * kb:(b + 1) * kb, c * nb:(c + 1) * nb] for b in range(K) for c in range(N)]
    Ms = []
    for r in range(R):
        # S_r = sum_i U_ir A_i and T_r = sum_j V_jr B_j, each written once
        S = np.zeros((mb, kb))
        for i in range(M * K):
            if Uf[i, r] != 0:
                S += Uf[i, r] * Ablk[i]
        T = np.zeros((kb, nb))
        for j in range(K * N):
            if Vf[j, r] != 0:
                T += Vf[j, r] * Bblk[j]
        Ms.append(_fast_core(S, T, M, K, N, Uf, Vf, Wf, levels - 1))
    C = np.zeros((m, n))
    for q in range(M * N):
        a, c = divmod(q, N)
        blk = np.zeros((mb, nb))
        for r in range(R):
            if Wf[q, r] != 0:
                blk += Wf[q, r] * Ms[r]
        C[a * mb:(a + 1) * mb, c * nb:(c + 1) * nb] = blk
    return C


def fast_mm(A, B, M, K, N, Uf, Vf, Wf, levels):
    """C = A B by ``levels`` recursive steps of the base case [[U,V,W]]
    (float64 factor matrices), classical products at the leaves."""
    m, k = A.shape
    n = B.shape[1]
    mm_, kk, nn = M ** levels, K ** levels, N ** levels
    mp, kp, np_ = (m // mm_) * mm_, (k // kk) * kk, (n // nn) * nn
    C = np.zeros((m, n))
    if mp and kp and np_:
        C[:mp, :np_] = _fast_core(A[:mp, :kp], B[:kp, :np_], M, K, N, Uf, Vf, Wf, levels)
    if kp < k and mp and np_:
        C[:mp, :np_] += _classical(A[:mp, kp:], B[kp:, :np_])
    if mp < m:
        C[mp:, :] = _classical(A[mp:, :], B)
    if np_ < n and mp:
        C[:mp, np_:] = _classical(A[:mp, :], B[:, np_:])
    return C
