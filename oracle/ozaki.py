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
    A'_ij = trunc(A_ij 2^s_i); column exponents t_j and B'_ij likewise;
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


def scale_rows(A, beta):
    """(A' as int64, exponents s) with A'_ij = trunc(A_ij 2^s_i)."""
    A = np.asarray(A, np.float64)
    s = np.zeros(A.shape[0], np.int64)
    out = np.zeros(A.shape, np.int64)
    for i in range(A.shape[0]):
        mx = float(np.max(np.abs(A[i]))) if A.shape[1] else 0.0
        if mx == 0.0:
            continue
        e = math.frexp(mx)[1] - 1          # floor(log2 mx)
        s[i] = beta - 1 - e
        out[i] = np.trunc(np.ldexp(A[i], int(s[i]))).astype(np.int64)
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
