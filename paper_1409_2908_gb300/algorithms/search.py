"""Offline search for exact bilinear base cases <M,K,N;R> (Section 2.3, "Numerical search").

The paper finds low-rank decompositions [[U,V,W]] of the matrix-multiplication
tensor numerically (alternating/least-squares iterations from many random
starts, with regularisation) and then drives the numerical solution to exact
discrete values.  This tool follows that recipe with a damped Gauss-Newton
(Levenberg-Marquardt) solver over all three factors at once, then a greedy
fix-and-resolve discretisation onto the dyadic set {0, +-1, +-1/2, +-2}:

  1. random start -> damped least squares until the Brent residual is ~0;
  2. use the diagonal-scaling freedom (Prop. 2.3) to put a +-1 at the
     largest entry of every u_r and v_r;
  3. repeatedly fix the free entry nearest to an allowed value and re-solve
     for the rest; an entry whose fix makes the residual unrecoverable is
     released and that value is banned for it;
  4. when every entry is fixed, check Eq. (2) in exact rational arithmetic.

It is offline tooling: nothing on the GPU path imports it.  A found algorithm
is written as a text ``.fmm`` file (format in ``fmm_format.py``).

Usage: python -m paper_1409_2908_gb300.algorithms.search M K N R [--seeds S] [--workers W] [--out FILE]
"""
import argparse
import itertools
import multiprocessing as mp
import os
import sys
import time
from fractions import Fraction

import numpy as np

ALLOWED = (0.0, 1.0, -1.0, 0.5, -0.5, 2.0, -2.0)


def mm_tensor(M, K, N):
    """Matmul tensor of <M,K,N> in row-order vec: A_ab*B_bc contributes to C_ac."""
    T = np.zeros((M * K, K * N, M * N))
    for a in range(M):
        for b in range(K):
            for c in range(N):
                T[a * K + b, b * N + c, a * N + c] = 1.0
    return T


class Problem:
    def __init__(self, M, K, N, R):
        self.M, self.K, self.N, self.R = M, K, N, R
        self.T = mm_tensor(M, K, N)
        self.I, self.J, self.Q = self.T.shape
        self.nU, self.nV, self.nW = self.I * R, self.J * R, self.Q * R
        self.n = self.nU + self.nV + self.nW

    def split(self, x):
        R = self.R
        U = x[: self.nU].reshape(self.I, R)
        V = x[self.nU: self.nU + self.nV].reshape(self.J, R)
        W = x[self.nU + self.nV:].reshape(self.Q, R)
        return U, V, W

    def residual(self, x):
        U, V, W = self.split(x)
        return (np.einsum("ir,jr,qr->ijq", U, V, W) - self.T).ravel()

    def jacobian(self, x):
        U, V, W = self.split(x)
        I, J, Q, R = self.I, self.J, self.Q, self.R
        out = np.zeros((I, J, Q, self.n))
        # d r_ijq / d U[i,r] = V[j,r] W[q,r]  (and cyclically for V, W)
        VW = np.einsum("jr,qr->jqr", V, W)
        UW = np.einsum("ir,qr->iqr", U, W)
        UV = np.einsum("ir,jr->ijr", U, V)
        for i in range(I):
            out[i, :, :, i * R:(i + 1) * R] = VW
        for j in range(J):
            out[:, j, :, self.nU + j * R:self.nU + (j + 1) * R] = UW
        for q in range(Q):
            out[:, :, q, self.nU + self.nV + q * R:self.nU + self.nV + (q + 1) * R] = UV
        return out.reshape(I * J * Q, self.n)


def lm(prob, x, free, iters=400, tol=1e-13, mu=1e-3, reg=0.0):
    """Levenberg-Marquardt on the free coordinates; returns (x, |F|)."""
    x = x.copy()
    f = prob.residual(x)
    cost = f @ f + reg * (x[free] @ x[free])
    for _ in range(iters):
        if cost < tol * tol and reg == 0.0:
            break
        Jm = prob.jacobian(x)[:, free]
        g = Jm.T @ f + reg * x[free]
        H = Jm.T @ Jm
        H[np.diag_indices_from(H)] += reg
        while True:
            A = H.copy()
            A[np.diag_indices_from(A)] += mu * (1.0 + np.diag(H))
            try:
                step = np.linalg.solve(A, -g)
            except np.linalg.LinAlgError:
                mu *= 10
                continue
            xn = x.copy()
            xn[free] += step
            fn = prob.residual(xn)
            cn = fn @ fn + reg * (xn[free] @ xn[free])
            if cn < cost:
                x, f, cost = xn, fn, cn
                mu = max(mu / 3.0, 1e-12)
                break
            mu *= 4.0
            if mu > 1e12:
                return x, float(np.sqrt(f @ f))
    return x, float(np.sqrt(f @ f))


def normalise(prob, x):
    U, V, W = (m.copy() for m in prob.split(x))
    for r in range(prob.R):
        su = U[np.argmax(np.abs(U[:, r])), r]
        sv = V[np.argmax(np.abs(V[:, r])), r]
        if su != 0 and sv != 0:
            U[:, r] /= su
            V[:, r] /= sv
            W[:, r] *= su * sv
    return np.concatenate([U.ravel(), V.ravel(), W.ravel()])


def _try_fix(prob, x, fixed, idx, value, iters=120):
    """Fix x[idx]=value and re-solve the free entries; None if the residual
    cannot be brought back to ~0."""
    x_try = x.copy()
    x_try[idx] = value
    fixed[idx] = True
    still = np.flatnonzero(~fixed)
    if len(still):
        x_new, res = lm(prob, x_try, still, iters=iters)
    else:
        x_new, res = x_try, float(np.linalg.norm(prob.residual(x_try)))
    if res < 1e-10:
        return x_new
    fixed[idx] = False
    return None


def sparsify(prob, x, fixed, rng):
    """Phase A: drive as many entries as possible to exactly zero, smallest
    magnitude first (discrete solutions are mostly zeros)."""
    tried = np.zeros(prob.n, bool)
    while True:
        cand = np.flatnonzero(~fixed & ~tried)
        if not len(cand):
            return x
        idx = cand[np.argmin(np.abs(x[cand]))]
        tried[idx] = True
        got = _try_fix(prob, x, fixed, idx, 0.0)
        if got is not None:
            x = got
            tried[:] = fixed  # a new zero can make earlier failures feasible


def discretise(prob, x, rng, log=None, max_fail=600):
    """Alternate zero-fixing (sparsify) with fixing one entry to +-1 (then
    +-2, +-1/2 as fallbacks), nearest-in-ratio first, re-solving each time."""
    return discretise_from(prob, x, np.zeros(prob.n, bool), rng, max_fail=max_fail)


def discretise_from(prob, x, fixed, rng, max_fail=600):
    """discretise() with the entries flagged in ``fixed`` already final."""
    n = prob.n
    x = sparsify(prob, x, fixed, rng)
    x = normalise(prob, x)
    x, res = lm(prob, x, np.flatnonzero(~fixed), iters=100)
    if res > 1e-10:
        return None
    banned = [set() for _ in range(n)]
    fails = 0
    while not fixed.all():
        free = np.flatnonzero(~fixed)
        # snap whatever is already discrete
        snapped = False
        for idx in free:
            for v in ALLOWED:
                if abs(x[idx] - v) < 1e-9:
                    x[idx] = v
                    fixed[idx] = True
                    snapped = True
                    break
        if snapped:
            continue
        best = None
        for stage in ((1.0,), (2.0, 0.5)):
            cands = []
            for idx in free:
                for mag in stage:
                    v = mag * (1.0 if x[idx] > 0 else -1.0)
                    if v in banned[idx]:
                        continue
                    cands.append((abs(np.log(abs(x[idx]) / mag)) if x[idx] != 0 else np.inf, idx, v))
            if cands:
                best = min(cands)
                break
        if best is None or not np.isfinite(best[0]):
            return None
        _, idx, v = best
        got = _try_fix(prob, x, fixed, idx, v)
        if got is None:
            banned[idx].add(v)
            fails += 1
            if fails > max_fail:
                return None
            continue
        x = sparsify(prob, got, fixed, rng)
    return x


def exact_check(prob, x):
    U, V, W = prob.split(x)
    Uf = [[Fraction(v).limit_denominator(64) for v in row] for row in U]
    Vf = [[Fraction(v).limit_denominator(64) for v in row] for row in V]
    Wf = [[Fraction(v).limit_denominator(64) for v in row] for row in W]
    R = prob.R
    for i in range(prob.I):
        for j in range(prob.J):
            for q in range(prob.Q):
                s = sum(Uf[i][r] * Vf[j][r] * Wf[q][r] for r in range(R))
                if s != int(prob.T[i, j, q]):
                    return None
    return Uf, Vf, Wf


def attempt(args):
    M, K, N, R, seed = args
    prob = Problem(M, K, N, R)
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal(prob.n) * 0.5
    free = np.arange(prob.n)
    # regularised phase then plain phase (the paper adds regularisation to
    # fight ill-conditioning)
    x, _ = lm(prob, x0, free, iters=40, reg=1e-3)
    x, res = lm(prob, x, free, iters=1500)
    if res > 1e-10:
        return seed, None, res
    x = normalise(prob, x)
    x, res = lm(prob, x, free, iters=200)
    if res > 1e-10:
        return seed, None, res
    xd = discretise(prob, x, rng)
    if xd is None:
        return seed, None, -1.0
    ex = exact_check(prob, xd)
    if ex is None:
        return seed, None, -2.0
    return seed, ex, 0.0


def write_fmm(path, M, K, N, R, Uf, Vf, Wf, note):
    def fmt(v):
        return str(v.numerator) if v.denominator == 1 else f"{v.numerator}/{v.denominator}"
    with open(path, "w") as fh:
        fh.write(f"# <{M},{K},{N};{R}> {note}\n")
        fh.write(f"{M} {K} {N} {R}\n")
        for name, F in (("U", Uf), ("V", Vf), ("W", Wf)):
            fh.write(f"{name}\n")
            for row in F:
                fh.write(" ".join(fmt(v) for v in row) + "\n")


def nnz(F):
    return sum(1 for row in F for v in row if v != 0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("M", type=int)
    ap.add_argument("K", type=int)
    ap.add_argument("N", type=int)
    ap.add_argument("R", type=int)
    ap.add_argument("--seeds", type=int, default=200)
    ap.add_argument("--seed0", type=int, default=0)
    ap.add_argument("--workers", type=int, default=max(1, os.cpu_count() - 1))
    ap.add_argument("--out", default=None)
    ap.add_argument("--keep", type=int, default=3, help="stop after this many exact solutions")
    a = ap.parse_args()
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    jobs = [(a.M, a.K, a.N, a.R, s) for s in range(a.seed0, a.seed0 + a.seeds)]
    found = []
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.workers) as pool:
        for seed, ex, res in pool.imap_unordered(attempt, jobs):
            tag = "EXACT" if ex is not None else f"fail({res:.2e})"
            print(f"[{time.time()-t0:7.1f}s] seed {seed}: {tag}", flush=True)
            if ex is not None:
                Uf, Vf, Wf = ex
                tot = nnz(Uf) + nnz(Vf) + nnz(Wf)
                print(f"   nnz U {nnz(Uf)} V {nnz(Vf)} W {nnz(Wf)} total {tot}", flush=True)
                found.append((tot, seed, ex))
                if len(found) >= a.keep:
                    pool.terminate()
                    break
    if not found:
        print("no exact solution found")
        return 1
    found.sort(key=lambda t: t[0])
    tot, seed, (Uf, Vf, Wf) = found[0]
    out = a.out or f"fmm_{a.M}{a.K}{a.N}_{a.R}.fmm"
    write_fmm(out, a.M, a.K, a.N, a.R, Uf, Vf, Wf,
              f"found by the damped least-squares search (seed {seed}), nnz {tot}")
    print("wrote", out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
