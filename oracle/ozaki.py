"""Oracle for the emulated-FP64 precision variant: an exact integer product
through the Chinese remainder theorem over small moduli (the "Ozaki-style"
slicing of the precision variants; the paper itself has no such variant and
recommends lower precision as the honest alternative to approximate
algorithms, Section 5).  This module states the definition the GPU path
implements, in plain integer arithmetic.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definition (our reading, fixed here):
  * beta = the largest width (at most 62) with k 2^(2 beta + 1) < P, P the
    product of the moduli: then |A'B'| < P/2 is guaranteed;
  * row exponents s_i = beta - 1 - floor(log2 max_j |A_ij|) (0 for a zero row),
    A'_ij = round(A_ij 2^s_i), to the nearest integer with ties away from
    zero, so |A'_ij| <= 2^beta; column exponents t_j and B'_ij likewise;
  * Z = A' B' exactly (integers); residues Z mod p for each modulus p are what
    the tensor cores compute, from balanced residues A' mod p and B' mod p;
  * C_ij = Z_ij 2^(-s_i - t_j).
"""
import math

import numpy as np

# pairwise coprime moduli <= 256, largest first (balanced residues fit in
# [-128, 127], exactly representable in bfloat16)
MODULI = (256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193,
          191, 181, 179, 173)


def moduli(n):
    if not 1 <= n <= len(MODULI):
        raise ValueError("unsupported number of moduli")
    return MODULI[:n]


def beta_bits(n, k):
    """Largest beta (at most 62) with k 2^(2 beta + 1) < P, i.e. every
    |A'B'| <= k (2^beta)^2 stays below P/2."""
    P = math.prod(moduli(n))
    beta = 62
    while beta > 0 and k * 2 ** (2 * beta + 1) >= P:
        beta -= 1
    return beta


def balanced(x, p):
    """Representative of x mod p in [-floor(p/2), ceil(p/2) - 1]."""
    r = x % p
    return r - p if r >= (p + 1) // 2 else r


def round_half_away(y):
    """Nearest integer to each entry of y, ties away from zero.  Exact: for
    |y| >= 1 the fraction |y| - floor(|y|) is computed without rounding, and
    below 1 the answer is 0 or 1 by comparison with 1/2."""
    a = np.abs(y)
    f = np.floor(a)
    r = f + (a - f >= 0.5)
    return np.where(y < 0, -r, r)


def scale_rows(A, beta):
    """(A' as int64, exponents s) with A'_ij = round(A_ij 2^s_i), ties away
    from zero (2^s_i is a power of two, so A_ij 2^s_i itself is exact wherever
    it is at least 2^-1022; anything smaller rounds to 0 either way)."""
    A = np.asarray(A, np.float64)
    s = np.zeros(A.shape[0], np.int64)
    out = np.zeros(A.shape, np.int64)
    for i in range(A.shape[0]):
        mx = float(np.max(np.abs(A[i]))) if A.shape[1] else 0.0
        if mx == 0.0:
            continue
        e = math.frexp(mx)[1] - 1          # floor(log2 mx)
        s[i] = beta - 1 - e
        out[i] = round_half_away(np.ldexp(A[i], int(s[i]))).astype(np.int64)
    return out, s


def scale_cols(B, beta):
    Bt, t = scale_rows(np.asarray(B).T, beta)
    return Bt.T.copy(), t


def residue_product(Ai, Bi, p):
    """Balanced residues of (A' B') mod p, from balanced residues of A', B'."""
    ra = np.vectorize(lambda x: balanced(int(x), p))(Ai).astype(np.int64)
    rb = np.vectorize(lambda x: balanced(int(x), p))(Bi).astype(np.int64)
    z = ra @ rb                       # |z| <= k * 2^14: exact in int64
    return np.vectorize(lambda x: balanced(int(x), p))(z).astype(np.int64)


def crt(residues, mods):
    """The unique integer in [-P/2, P/2) congruent to each residue."""
    P = math.prod(mods)
    x = 0
    for r, p in zip(residues, mods):
        Mp = P // p
        x += int(r) * Mp * pow(Mp, -1, p)
    x %= P
    return x - P if x >= P // 2 else x


def exact_product(Ai, Bi):
    """A' B' with Python integers (object arithmetic)."""
    Ao = Ai.astype(object)
    Bo = Bi.astype(object)
    return Ao.dot(Bo)


def emulated_gemm(A, B, n_moduli):
    """C = Z 2^(-s_i - t_j), Z = A'B' exact, rounded once to FP64."""
    k = A.shape[1]
    beta = beta_bits(n_moduli, k)
    Ai, s = scale_rows(A, beta)
    Bi, t = scale_cols(B, beta)
    Z = exact_product(Ai, Bi)
    C = np.empty(Z.shape)
    for i in range(Z.shape[0]):
        for j in range(Z.shape[1]):
            C[i, j] = math.ldexp(float(Z[i, j]), -int(s[i]) - int(t[j]))
    return C


def emulated_entries(A, B, rows, cols, n_moduli):
    """Entries (rows[t], cols[t]) of emulated_gemm(A, B, n_moduli), each from
    its own row of A and column of B: the row exponent depends only on the
    row and the column exponent only on the column, so this is the same
    definition evaluated one entry at a time (for sampling full-size
    products)."""
    k = A.shape[1]
    beta = beta_bits(n_moduli, k)
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    ur, ri = np.unique(rows, return_inverse=True)
    uc, ci = np.unique(cols, return_inverse=True)
    Ai, s = scale_rows(np.asarray(A)[ur], beta)
    Bi, t = scale_cols(np.asarray(B)[:, uc], beta)
    arows = [list(map(int, Ai[i])) for i in range(len(ur))]
    bcols = [list(map(int, Bi[:, j])) for j in range(len(uc))]
    out = np.empty(len(rows))
    for e, (i, j) in enumerate(zip(ri, ci)):
        z = sum(a * b for a, b in zip(arows[i], bcols[j]))
        out[e] = math.ldexp(float(z), -int(s[i]) - int(t[j]))
    return out
