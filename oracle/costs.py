"""Oracle: the paper's closed-form cost models.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from math import log


def flops_classical_rec(N):
    """F_C by its recurrence (Section 2.1): F_C(1) = 1,
    F_C(N) = 8 F_C(N/2) + 4 (N/2)^2 for N a power of two."""
    return 1 if N == 1 else 8 * flops_classical_rec(N // 2) + 4 * (N // 2) ** 2


def flops_classical(N):
    """Closed form F_C(N) = 2 N^3 - N^2 (Section 2.1)."""
    return 2 * N ** 3 - N ** 2


def flops_strassen_rec(N):
    """Strassen's flop recurrence (Section 2.1) read as F_S(1) = 1,
    F_S(N) = 7 F_S(N/2) + 18 (N/2)^2 (the recursive calls are Strassen too;
    that is the reading whose solution is the printed closed form)."""
    return 1 if N == 1 else 7 * flops_strassen_rec(N // 2) + 18 * (N // 2) ** 2


def flops_strassen(N):
    """Closed form F_S(N) = 7 N^(log2 7) - 6 N^2, exact for N = 2^j."""
    j = N.bit_length() - 1
    return 7 * 7 ** j - 6 * N * N


def additions(M, K, N, R, nnz_u, nnz_v, nnz_w):
    """Block additions of one recursive step: (nnz U - R) + (nnz V - R) +
    (nnz W - MN) (Strassen: 5 + 5 + 8 = 18)."""
    return (nnz_u - R) + (nnz_v - R) + (nnz_w - M * N)


def pairwise_traffic(M, N, R, nnz_uvw):
    """(block reads, block writes) of pairwise daxpy additions (Section 3.2)."""
    return 2 * nnz_uvw - 2 * R - M * N, nnz_uvw


def write_once_traffic(M, N, R, nnz_uvw):
    """(block reads, max block writes) of write-once additions (Section 3.2)."""
    return nnz_uvw, 2 * R + M * N


def streaming_traffic(M, K, N, R):
    """(block reads, max block writes) of streaming additions (Section 3.2)."""
    return M * K + K * N + R, 2 * R + M * N


def bfs_memory_factor(M, N, R):
    """Extra memory per BFS level for the M_r, relative to C (Section 4.2)."""
    return R / (M * N)


def speedup_per_step(M, K, N, R):
    """Multiplication speedup per recursive step, MKN/R - 1 (Table 1)."""
    return M * K * N / R - 1


def leaf_flops(m, k, n, M, K, N, R, levels):
    """Flops of the R^L leaf products of an m x k x n core:
    2 m k n (R / MKN)^L."""
    return 2 * m * k * n * (R / (M * K * N)) ** levels


def omega(base, R):
    """Exponent of a square <b,b,b;R> algorithm: log_b R (e.g. the composed
    <54,54,54> of Section 5.2 with R = 40^3 gives 3 log_54 40)."""
    return log(R) / log(base)
