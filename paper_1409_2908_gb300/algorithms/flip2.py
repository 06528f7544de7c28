"""Offline search for exact base cases <M,K,N;R>: flip-graph walk over GF(2)
followed by a Hensel lift of the found scheme to exact small rationals.

Section 2.3 frames the search as finding a rank-R decomposition of the matmul
tensor and recovering discrete coefficients.  Here the discrete structure
comes first, by the flip-graph method of Kauers and Moosbauer ("Flip graphs
for matrix multiplication", 2022; plus transitions from their follow-up work),
implemented here from its published description: a random walk over schemes modulo 2 (a flip rewrites two terms
sharing a factor, x(y1)(z1) + x(y2)(z2) = x(y1+y2)(z1) + x(y2)(z1+z2) mod 2;
a reduction merges two terms sharing two factors; terms with a zero factor
vanish) from the classical scheme until the rank is R.  The scheme is then
lifted from GF(2) to the 2-adic integers (Hensel lifting: one linear solve
over GF(2) per bit) and each coefficient is read back as a small rational by
rational reconstruction; the result is checked exactly against Eq. (2).

For larger cases (<4,2,4;26>) the walk runs in C (flipwalk.c, compiled with
gcc on first use): it adds plus transitions that split two terms into three,
so isolated rank-R schemes can be left, and emits the sparsest rank-R scheme
of each window; every emitted scheme is lifted and the sparsest one with
dyadic coefficients is written.

Usage: python -m paper_1409_2908_gb300.algorithms.flip2 M K N R [--workers W] [--out FILE]
       python -m paper_1409_2908_gb300.algorithms.flip2 M K N R --c-walker [--seconds S]
"""
import argparse
import multiprocessing as mp
import os
import random
import sys
import time

import numpy as np


def classical(M, K, N):
    t = []
    for a in range(M):
        for b in range(K):
            for c in range(N):
                t.append([1 << (a * K + b), 1 << (b * N + c), 1 << (a * N + c)])
    return t


def reduce_mod2(terms):
    changed = True
    while changed:
        changed = False
        terms = [t for t in terms if t[0] and t[1] and t[2]]
        seen = {}
        for idx, t in enumerate(terms):
            for keep in range(3):
                o1, o2 = [m for m in range(3) if m != keep]
                key = (keep, t[o1], t[o2])
                if key in seen:
                    j = seen[key]
                    terms[j][keep] ^= t[keep]
                    terms.pop(idx)
                    changed = True
                    break
                seen[key] = idx
            if changed:
                break
    return terms


def walk_mod2(M, K, N, R, seed, max_steps, plateau):
    rng = random.Random(seed)
    terms = reduce_mod2(classical(M, K, N))
    since = 0
    for step in range(max_steps):
        groups = {}
        for idx, t in enumerate(terms):
            for mode in range(3):
                groups.setdefault((mode, t[mode]), []).append(idx)
        pairs = [(k[0], v) for k, v in groups.items() if len(v) >= 2]
        if not pairs:
            terms = reduce_mod2(classical(M, K, N))
            continue
        mode, members = rng.choice(pairs)
        i, j = rng.sample(members, 2)
        p, q = [m for m in range(3) if m != mode]
        if rng.random() < 0.5:
            p, q = q, p
        terms[i][p] ^= terms[j][p]
        terms[j][q] ^= terms[i][q]
        n0 = len(terms)
        terms = reduce_mod2(terms)
        since = 0 if len(terms) < n0 else since + 1
        if len(terms) <= R:
            return terms, step
        if since > plateau:
            terms = reduce_mod2(classical(M, K, N))
            since = 0
    return None, max_steps


def _gf2_solver(rows, n):
    """Gauss-Jordan elimination over GF(2) of a system given as row bitmasks;
    returns solve(rhs_bits) -> solution bitmask (free variables 0) or None."""
    rows = list(rows)
    P = len(rows)
    ops = [1 << i for i in range(P)]
    pivots = []
    r = 0
    for c in range(n):
        sel = next((i for i in range(r, P) if (rows[i] >> c) & 1), None)
        if sel is None:
            continue
        rows[r], rows[sel] = rows[sel], rows[r]
        ops[r], ops[sel] = ops[sel], ops[r]
        for i in range(P):
            if i != r and (rows[i] >> c) & 1:
                rows[i] ^= rows[r]
                ops[i] ^= ops[r]
        pivots.append(c)
        r += 1
        if r == P:
            break

    def solve(rhs):
        x = 0
        for i in range(P):
            b = bin(ops[i] & rhs).count("1") & 1
            if i < len(pivots):
                if b:
                    x |= 1 << pivots[i]
            elif b:
                return None
        return x

    return solve


def lift(M, K, N, terms, bits=40):
    """Hensel-lift a GF(2) scheme to the 2-adic integers and read off small
    rationals.  With x = x0 + 2 x1 + ..., each step solves J(x0) d = -F(x)/2^k
    over GF(2) (J = Jacobian of the Brent equations, which mod 2 depends only
    on x0) and adds 2^k d; after `bits` steps every entry is recovered by
    rational reconstruction.  Returns (U, V, W) as Fractions or None."""
    from fractions import Fraction
    from . import search as S
    R = len(terms)
    prob = S.Problem(M, K, N, R)
    I, J, Q = prob.I, prob.J, prob.Q
    sizes = (I, J, Q)
    offs = (0, prob.nU, prob.nU + prob.nV)
    x0 = np.zeros(prob.n)
    for mode in range(3):
        for r, t in enumerate(terms):
            for i in range(sizes[mode]):
                if (t[mode] >> i) & 1:
                    x0[offs[mode] + i * R + r] = 1.0
    Jm = prob.jacobian(x0).astype(np.int64) % 2
    n = prob.n
    solve = _gf2_solver([int("".join(str(int(b)) for b in row[::-1]), 2) for row in Jm], n)
    T = prob.T.astype(np.int64).astype(object).ravel()
    x = [int(v) for v in x0]

    def residual(x):
        U = np.array(x[:prob.nU], dtype=object).reshape(I, R)
        V = np.array(x[prob.nU:prob.nU + prob.nV], dtype=object).reshape(J, R)
        W = np.array(x[prob.nU + prob.nV:], dtype=object).reshape(Q, R)
        out = np.zeros((I, J, Q), dtype=object)
        for r in range(R):
            out += np.multiply.outer(np.multiply.outer(U[:, r], V[:, r]), W[:, r])
        return out.ravel() - T

    mod = 1
    for _ in range(1, bits):
        mod *= 2
        f = residual(x)
        rhs = 0
        for i, v in enumerate(f):
            if (-(v // mod)) % 2:
                rhs |= 1 << i
        d = solve(rhs)
        if d is None:
            return None
        for c in range(n):
            if (d >> c) & 1:
                x[c] += mod
    modK = 2 ** bits
    bound = 2 ** (bits // 2 - 1)
    vals = []
    for v in x:
        r0, r1 = modK, v % modK
        s0, s1 = 0, 1
        while r1 > bound:
            q = r0 // r1
            r0, r1 = r1, r0 - q * r1
            s0, s1 = s1, s0 - q * s1
        if s1 == 0 or abs(s1) > bound:
            return None
        vals.append(Fraction(r1, s1))
    xs = np.array([float(v) for v in vals])
    return S.exact_check(prob, xs)


def attempt(args):
    M, K, N, R, seed, steps, plateau = args
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    terms, info = walk_mod2(M, K, N, R, seed, steps, plateau)
    if terms is None:
        return seed, None, "no mod-2 scheme"
    # not every mod-2 scheme lifts; keep flipping at rank R and retry the lift
    # (a short lift favours small coefficients, a long one general rationals)
    rng = random.Random(seed + 1)
    for tries in range(40):
        for bits in (8, 40):
            ex = lift(M, K, N, terms, bits=bits)
            if ex is not None:
                return seed, ex, f"mod-2 rank {len(terms)} after {info} steps, lifted (try {tries})"
        for _ in range(2000):
            groups = {}
            for idx, t in enumerate(terms):
                for mode in range(3):
                    groups.setdefault((mode, t[mode]), []).append(idx)
            pairs = [(k[0], v) for k, v in groups.items() if len(v) >= 2]
            if not pairs:
                break
            mode, members = rng.choice(pairs)
            i, j = rng.sample(members, 2)
            p_, q_ = [m for m in range(3) if m != mode]
            if rng.random() < 0.5:
                p_, q_ = q_, p_
            terms[i][p_] ^= terms[j][p_]
            terms[j][q_] ^= terms[i][q_]
            terms = reduce_mod2(terms)
    return seed, None, f"mod-2 rank {len(terms)} after {info} steps, lift failed"


def _c_walker_bin():
    import subprocess
    import tempfile
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flipwalk.c")
    out = os.path.join(tempfile.gettempdir(), f"flipwalk_{os.getpid()}")
    subprocess.run(["gcc", "-O2", "-o", out, src], check=True)
    return out


def c_walk(M, K, N, R, seeds, seconds, windows=100000, gap=50):
    """Run the C walker on several seeds in parallel for `seconds` and lift
    every emitted scheme; returns the sparsest exact dyadic (U, V, W)."""
    import subprocess
    from .search import nnz
    exe = _c_walker_bin()
    procs = [subprocess.Popen(["timeout", str(seconds), exe, str(M), str(K), str(N), str(R), str(s),
                               str(10 ** 12), "200000", str(windows), str(gap)],
                              stdout=subprocess.PIPE, text=True) for s in seeds]
    lines = []
    for p in procs:
        lines += p.communicate()[0].splitlines()
    os.unlink(exe)

    def weight(line):
        return sum(bin(int(x, 16)).count("1") for x in line.replace(";", " ").split())

    best = None
    for line in sorted(set(lines), key=weight)[:60]:
        terms = [[int(x, 16) for x in t.split()] for t in line.split(";")]
        for bits in (8, 40):
            ex = lift(M, K, N, [list(t) for t in terms], bits=bits)
            if ex is not None:
                break
        if ex is None:
            continue
        dyadic = all((v.denominator & (v.denominator - 1)) == 0 for F in ex for row in F for v in row)
        tot = sum(nnz(F) for F in ex)
        if dyadic and (best is None or tot < best[0]):
            best = (tot, ex)
    return best


def main():
    from .search import write_fmm, nnz
    ap = argparse.ArgumentParser()
    for k in ("M", "K", "N", "R"):
        ap.add_argument(k, type=int)
    ap.add_argument("--workers", type=int, default=max(1, os.cpu_count() - 1))
    ap.add_argument("--seeds", type=int, default=100000)
    ap.add_argument("--steps", type=int, default=3_000_000)
    ap.add_argument("--plateau", type=int, default=200_000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--c-walker", action="store_true", help="walk in C with plus transitions")
    ap.add_argument("--seconds", type=int, default=300)
    a = ap.parse_args()
    if a.c_walker:
        best = c_walk(a.M, a.K, a.N, a.R, range(1, a.workers + 1), a.seconds)
        if best is None:
            return 1
        tot, (Uf, Vf, Wf) = best
        out = a.out or f"fmm_{a.M}{a.K}{a.N}_{a.R}.fmm"
        write_fmm(out, a.M, a.K, a.N, a.R, Uf, Vf, Wf,
                  f"found by a GF(2) flip-graph walk with plus transitions and Hensel lifting, nnz {tot}")
        print("wrote", out, "nnz", tot)
        return 0
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    t0 = time.time()
    jobs = [(a.M, a.K, a.N, a.R, s, a.steps, a.plateau) for s in range(a.seeds)]
    with mp.get_context("spawn").Pool(a.workers) as pool:
        for seed, ex, info in pool.imap_unordered(attempt, jobs):
            print(f"[{time.time()-t0:8.1f}s] seed {seed}: {info}", flush=True)
            if ex is None:
                continue
            Uf, Vf, Wf = ex
            tot = nnz(Uf) + nnz(Vf) + nnz(Wf)
            out = a.out or f"fmm_{a.M}{a.K}{a.N}_{a.R}.fmm"
            write_fmm(out, a.M, a.K, a.N, a.R, Uf, Vf, Wf,
                      f"found by a GF(2) flip-graph walk and Hensel lifting (seed {seed}), nnz {tot}")
            print("wrote", out, flush=True)
            pool.terminate()
            return 0
    return 1


if __name__ == "__main__":
    sys.exit(main())
