"""Offline discrete search for exact integer base cases <M,K,N;R>.

A second route to the factor matrices of Section 2.3, complementary to the
numerical search in ``search.py``: a random walk over exact schemes with
coefficients in {-1, 0, 1}.  It starts from the classical decomposition
(rank MKN, one rank-one term per scalar product a_ab*b_bc) and applies two
moves that keep the sum of rank-one terms equal to the matmul tensor:

* flip: two terms sharing one factor x,
      x(y1)(z1) + x(y2)(z2) = x(y1 + y2)(z1) + x(y2)(z2 - z1),
  rewrites both terms without changing the rank;
* reduction: two terms sharing two factors merge into one,
      x(y)(z1) + x(y)(z2) = x(y)(z1 + z2),
  and a term with a zero factor is dropped.

Flips whose result leaves {-1,0,1} are rejected, so every scheme on the walk
is exact with integer coefficients (which keeps integer inputs bit-exact on
the fast path).  The walk restarts after a plateau.  Every result is checked
against Eq. (2) before it is written.

Usage: python -m paper_1409_2908_gb300.algorithms.flipsearch M K N R [--workers W] [--out FILE]
"""
import argparse
import multiprocessing as mp
import os
import random
import sys
import time


def classical_scheme(M, K, N):
    terms = []
    for a in range(M):
        for b in range(K):
            for c in range(N):
                u = [0] * (M * K)
                v = [0] * (K * N)
                w = [0] * (M * N)
                u[a * K + b] = 1
                v[b * N + c] = 1
                w[a * N + c] = 1
                terms.append([tuple(u), tuple(v), tuple(w)])
    return terms


def canon(vec):
    """(sign, canonical) with the first nonzero entry of canonical positive."""
    for e in vec:
        if e != 0:
            if e > 0:
                return 1, vec
            return -1, tuple(-x for x in vec)
    return 0, vec


def bounded(vec):
    return all(-1 <= e <= 1 for e in vec)


def add(x, y, s=1):
    return tuple(a + s * b for a, b in zip(x, y))


def is_zero(x):
    return not any(x)


def reduce_scheme(terms):
    """Apply reductions until none applies; returns the new term list."""
    changed = True
    while changed:
        changed = False
        terms = [t for t in terms if not (is_zero(t[0]) or is_zero(t[1]) or is_zero(t[2]))]
        seen = {}
        for idx, t in enumerate(terms):
            sa, ca = canon(t[0])
            sb, cb = canon(t[1])
            sc, cc = canon(t[2])
            for keep, key, sgn in ((2, (0, ca, 1, cb), sa * sb), (1, (0, ca, 2, cc), sa * sc), (0, (1, cb, 2, cc), sb * sc)):
                if key in seen:
                    j, sj, kj = seen[key]
                    if kj != keep:
                        continue
                    # terms j and idx share the two factors other than `keep`
                    # up to signs; fold idx into j on factor `keep`
                    tj = terms[j]
                    s = sgn * sj
                    merged = add(tj[keep], t[keep], s)
                    if not bounded(merged):
                        continue
                    newt = list(tj)
                    newt[keep] = merged
                    terms[j] = newt
                    terms.pop(idx)
                    changed = True
                    break
                seen[key] = (idx, sgn, keep)
            if changed:
                break
    return terms


def flip_once(terms, rng):
    """One random flip between two terms sharing a factor (up to sign)."""
    groups = {}
    for idx, t in enumerate(terms):
        for mode in range(3):
            s, c = canon(t[mode])
            groups.setdefault((mode, c), []).append((idx, s))
    pairs = [g for g in groups.items() if len(g[1]) >= 2]
    if not pairs:
        return False
    for _ in range(8):
        (mode, _c), members = rng.choice(pairs)
        (i, si), (j, sj) = rng.sample(members, 2)
        others = [m for m in range(3) if m != mode]
        rng.shuffle(others)
        p, q = others
        ti, tj = list(terms[i]), list(terms[j])
        # make x_j == x_i by moving the sign into factor q of term j
        if si != sj:
            tj[mode] = ti[mode]
            tj[q] = tuple(-e for e in tj[q])
        sign = rng.choice((1, -1))
        # x(yi)(zi) + x(yj)(zj) = x(yi + s*yj)(zi) + x(yj)(zj - s*zi)
        yi = add(ti[p], tj[p], sign)
        zj = add(tj[q], ti[q], -sign)
        if not (bounded(yi) and bounded(zj)):
            continue
        ti[p] = yi
        tj[q] = zj
        terms[i], terms[j] = ti, tj
        return True
    return False


def check(terms, M, K, N):
    T = {}
    for a in range(M):
        for b in range(K):
            for c in range(N):
                T[(a * K + b, b * N + c, a * N + c)] = 1
    acc = {}
    for u, v, w in terms:
        for i, x in enumerate(u):
            if not x:
                continue
            for j, y in enumerate(v):
                if not y:
                    continue
                for q, z in enumerate(w):
                    if z:
                        acc[(i, j, q)] = acc.get((i, j, q), 0) + x * y * z
    acc = {k: v for k, v in acc.items() if v != 0}
    return acc == T


def walk(args):
    M, K, N, R, seed, max_steps, plateau = args
    rng = random.Random(seed)
    terms = reduce_scheme(classical_scheme(M, K, N))
    best = len(terms)
    since = 0
    for step in range(max_steps):
        if not flip_once(terms, rng):
            terms = reduce_scheme(classical_scheme(M, K, N))
            continue
        n0 = len(terms)
        terms = reduce_scheme(terms)
        if len(terms) < n0:
            since = 0
        else:
            since += 1
        if len(terms) < best:
            best = len(terms)
        if len(terms) <= R:
            return seed, terms, step
        if since > plateau:
            terms = reduce_scheme(classical_scheme(M, K, N))
            since = 0
    return seed, None, best


def write_fmm(path, M, K, N, terms, note):
    R = len(terms)
    with open(path, "w") as fh:
        fh.write(f"# <{M},{K},{N};{R}> {note}\n")
        fh.write(f"{M} {K} {N} {R}\n")
        for name, mode, rows in (("U", 0, M * K), ("V", 1, K * N), ("W", 2, M * N)):
            fh.write(f"{name}\n")
            for i in range(rows):
                fh.write(" ".join(str(t[mode][i]) for t in terms) + "\n")


def main():
    ap = argparse.ArgumentParser()
    for k in ("M", "K", "N", "R"):
        ap.add_argument(k, type=int)
    ap.add_argument("--workers", type=int, default=max(1, os.cpu_count() - 1))
    ap.add_argument("--seeds", type=int, default=10000)
    ap.add_argument("--steps", type=int, default=2_000_000)
    ap.add_argument("--plateau", type=int, default=50_000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    t0 = time.time()
    jobs = [(a.M, a.K, a.N, a.R, s, a.steps, a.plateau) for s in range(a.seeds)]
    with mp.get_context("spawn").Pool(a.workers) as pool:
        for seed, terms, info in pool.imap_unordered(walk, jobs):
            if terms is None:
                print(f"[{time.time()-t0:8.1f}s] seed {seed}: best rank {info}", flush=True)
                continue
            ok = check(terms, a.M, a.K, a.N)
            nnz = sum(1 for t in terms for f in t for e in f if e)
            print(f"[{time.time()-t0:8.1f}s] seed {seed}: rank {len(terms)} after {info} steps, exact={ok}, nnz={nnz}", flush=True)
            if ok:
                out = a.out or f"fmm_{a.M}{a.K}{a.N}_{len(terms)}.fmm"
                write_fmm(out, a.M, a.K, a.N, terms,
                          f"found by the flip-graph walk (seed {seed}), coefficients in {{-1,0,1}}, nnz {nnz}")
                print("wrote", out, flush=True)
                pool.terminate()
                return 0
    return 1


if __name__ == "__main__":
    sys.exit(main())
