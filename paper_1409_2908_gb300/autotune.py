"""Autotuner: for a product shape (m, k, n) and an accuracy target, pick the
base case, the number of recursive levels, the execution scheme, the leaf
tile and the leaf precision.

The paper's rule for recursion (Section 3.4) is the model prior: a recursive
step only pays while its sub-products stay on the flat part of the classical
GEMM's performance curve, and the best algorithm depends on the shape
(Section 5: algorithms that "match the shape" win on rectangular products).
Here the classical curve is the library's own classical GEMM measured on this
GPU, the model ranks every (algorithm, levels, scheme, precision) candidate,
and the few best candidates are timed on the real shape; the fastest that
meets the accuracy target is kept (per shape, in memory and optionally in a
JSON file).

Nothing here computes the product: every candidate runs through the C ABI.
"""
import functools
import glob
import json
import math
import os
from dataclasses import asdict, dataclass

import paper_1409_2908_gb300 as fmm

# measured on GB300 (benchmark runs at 8192^3), used only to rank candidates:
# the classical FP64 DFMA GEMM, the residue GEMM, and the emulated path's
# memory passes as achieved bytes per second
FP64_TFLOPS = 1.22
TC_TFLOPS = 1850.0                   # residue GEMM (tcgen05, bf16 residues)
SPLIT_GBS = 3900.0                   # fused scaling + residues + first level
LEVEL_GBS = 2200.0                   # later levels of S/T and W on int8 residues
CRT_PS_PER_ELEM_MOD = 0.98           # CRT per output element and modulus (L = 0)
W_TERM_FACTOR = 0.1                  # extra CRT cost per additional W term of an output block
LAUNCH_US = 4.0                      # per kernel launch (6 launches for the emulated path)
NUM_SMS = 152
HBM_GBS = 6700.0
TF32_TFLOPS = {"tf32": 850.0, "fp32": 550.0}   # leaf launch, TF32 work per second (fp32: 3 products)
# e_F against the FP64 oracle on uniform data at 16384^3, per recursion level
# (0, 1, 2: tf32 2.6e-4, 5.6e-4, 1.2e-3; fp32 3.7e-6, 3.9e-6, 4.3e-6), used
# with a factor 2 of slack to admit the two precisions
TF32_ERR = {"tf32": (3e-4, 2.0), "fp32": (4e-6, 1.1)}   # (e_F at 0 levels, growth per level)


def _transpose_case(M, K, N, U, V, W):
    """<M,K,N;R> -> <N,K,M;R> from C^T = B^T A^T (Section 2.3, Prop. 2.1):
    the new A is B^T (block (c,b) = B_bc^T), the new B is A^T and the new C
    is C^T, and each product (S_r T_r)^T = T_r^T S_r^T keeps its index r."""
    import numpy as np
    R = U.shape[1]
    U2, V2, W2 = np.zeros((N * K, R)), np.zeros((K * M, R)), np.zeros((N * M, R))
    for b in range(K):
        for c in range(N):
            U2[c * K + b] = V[b * N + c]
    for a in range(M):
        for b in range(K):
            V2[b * M + a] = U[a * K + b]
        for c in range(N):
            W2[c * M + a] = W[a * N + c]
    return N, K, M, U2, V2, W2


def _cycle_case(M, K, N, U, V, W):
    """<M,K,N;R> -> <K,N,M;R> by the cyclic symmetry of the matmul tensor
    (Section 2.3, Prop. 2.2): sum_r U_(a,b)r V_(b,c)r W_(a,c)r is unchanged
    when the roles rotate, so [[V, W', U']] with W' indexed (c,a) and U'
    indexed (b,a) is an exact <K,N,M> algorithm."""
    import numpy as np
    R = U.shape[1]
    V2, W2 = np.zeros((N * M, R)), np.zeros((K * M, R))
    for a in range(M):
        for c in range(N):
            V2[c * M + a] = W[a * N + c]
        for b in range(K):
            W2[b * M + a] = U[a * K + b]
    return K, N, M, V.copy(), V2, W2


PERMS = ("", "c", "cc", "t", "tc", "tcc")   # identity, cycles, transpose then cycles


def permuted_factors(name, perm):
    """(M, K, N, U, V, W) of a shipped base case under a permutation of its
    dimensions: "c" cycles <M,K,N> to <K,N,M>, "t" transposes it to <N,K,M>;
    the six strings of PERMS give every ordering of (M, K, N).  Every result
    is checked exactly by fmm_plan_create when a plan is built from it."""
    from . import algorithm_factors
    f = algorithm_factors(name)
    for op in perm:
        f = _transpose_case(*f) if op == "t" else _cycle_case(*f)
    return f


_FACTORS = {}


def _factors(name, perm):
    key = (name, perm)
    if key not in _FACTORS:
        _FACTORS[key] = permuted_factors(name, perm)
    return _FACTORS[key]


@dataclass(frozen=True)
class Choice:
    algorithm: str            # algorithm file name (levels 0: the classical product)
    levels: int
    flags: int
    precision: str            # "fp64", "ozaki_bf16", "tf32" or "fp32"
    moduli: int = 15
    tile: str = "auto"        # leaf tile (FP64 leaf GEMM tiles; 128x128 narrows the tensor-core tiles)
    model_ms: float = 0.0
    measured_ms: float = -1.0
    perm: str = ""            # permutation of the base case (PERMS)
    measured_err: float = -1.0   # e_F of the chosen moduli against a 16-moduli product (emulated)

    @property
    def label(self):
        p = f"[{self.perm}]" if self.perm else ""
        m = f" x{self.moduli}" if self.precision == "ozaki_bf16" else ""
        return f"{self.algorithm}{p} L{self.levels} {self.precision}{m} tile {self.tile}"

    def plan(self):
        mod = self.moduli if self.precision == "ozaki_bf16" else None
        if self.perm and self.levels > 0:
            return fmm.Plan(levels=self.levels, flags=self.flags, precision=self.precision, tile=self.tile,
                            factors=_factors(self.algorithm, self.perm), moduli=mod)
        return fmm.Plan(self.algorithm, levels=self.levels, flags=self.flags,
                        precision=self.precision, tile=self.tile, moduli=mod)


_ALGS = None


def algorithms():
    """Shipped base cases: name -> (M, K, N, R) (read once)."""
    global _ALGS
    if _ALGS is not None:
        return _ALGS
    out = {}
    for path in sorted(glob.glob(os.path.join(fmm.ALGORITHM_DIR, "*.fmm"))):
        with open(path) as fh:
            lines = [ln.split("#", 1)[0].strip() for ln in fh]
        M, K, N, R = (int(t) for t in next(ln for ln in lines if ln).split())
        out[os.path.basename(path)[:-4]] = (M, K, N, R)
    _ALGS = out
    return out


def cases():
    """Every base case with its permutations: (name, perm) -> (M, K, N, R),
    one entry per distinct (M, K, N) of each shipped algorithm."""
    out = {}
    for name, (M, K, N, R) in algorithms().items():
        seen = set()
        for perm in PERMS:
            dims = (M, K, N)
            for op in perm:
                a, b, c = dims
                dims = (c, b, a) if op == "t" else (b, c, a)
            if dims in seen:
                continue
            seen.add(dims)
            out[(name, perm)] = dims + (R,)
    return out


MODULI = (256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193)
_PRODUCTS = tuple(math.prod(MODULI[:n]) for n in range(len(MODULI) + 1))


def beta_for(n, k):
    """Width of the scaled integers with n moduli (the library's rule: the
    largest beta <= 62 with k 2^(2 beta + 1) < P).  k 2^e < P holds exactly
    when 2^e <= (P - 1) div k, so 2 beta + 1 <= bitlength((P - 1) div k) - 1."""
    e = ((_PRODUCTS[n] - 1) // int(k)).bit_length() - 1
    return max(0, min(62, (e - 1) // 2))


@functools.lru_cache(maxsize=4096)
def moduli_for(tol, k):
    """Fewest moduli whose rounding error 2^-beta (with a factor 2 of slack;
    the e_F measured on uniform data is about 0.9 x 2^-beta once the scaled
    operands are rounded to nearest) meets the relative tolerance: the prior
    that measured trials then correct."""
    for n in range(6, 17):
        if 2 * 2.0 ** (-beta_for(n, k)) <= tol:
            return n
    return None


def classical_efficiency(m, n, tile=128, tile_n=None, planes=1):
    """Fraction of the peak a grouped launch of `planes` products of m x n
    reaches: tile fill (the classical curve is flat above one tile on this
    GPU; below it the padded tile wastes work) times wave quantisation over
    the SMs."""
    tile_n = tile_n or tile
    tm, tn = math.ceil(m / tile), math.ceil(n / tile_n)
    fill = (m * n) / (tm * tile * tn * tile_n)
    tiles = tm * tn * planes
    waves = tiles / (math.ceil(tiles / NUM_SMS) * NUM_SMS)
    return max(fill * waves, 0.02)


# relative speed of each FP64 leaf tile per flop (the 128 x 128 tile runs at
# 97 % of the DFMA ceiling; smaller tiles pay more shared-memory traffic)
FP64_TILES = {"128x128": (128, 128, 1.0), "128x64": (128, 64, 0.95), "64x128": (64, 128, 0.95),
              "96x96": (96, 96, 0.93), "64x64": (64, 64, 0.85), "32x32": (32, 32, 0.6)}
# tensor-core tiles: 128 x 256 ("auto" where the leaves are at least 256 wide)
# or 128 x 128 ("128x128"), relative speed per flop
TC_TILES = {"auto": 1.0, "128x128": 0.92}
FUSED_BLOCKS = (1, 4, 6, 8, 9)   # block grids with a fused first-level split in the library


class Autotuner:
    def __init__(self, tol=1e-11, precisions=("fp64", "ozaki_bf16"), max_levels=3,
                 trials=3, cache_file=None, measure=True, permutations=True):
        self.tol = tol
        self.precisions = tuple(precisions)
        self.max_levels = max_levels
        self.trials = trials
        self.cache_file = cache_file
        self.measure = measure
        self.permutations = permutations
        # model rates (this GPU's measured defaults; calibrate() re-measures them)
        self.fp64_tflops = FP64_TFLOPS
        self.tc_tflops = TC_TFLOPS
        self.pass_scale = 1.0        # measured / modelled time of the emulated path's passes
        self._cache = {}
        self._plans = {}
        if cache_file and os.path.exists(cache_file):
            with open(cache_file) as fh:
                for key, d in json.load(fh).items():
                    self._cache[key] = Choice(**d)

    # ----------------------------------------------------------- model
    def _cases(self):
        """(name, perm, (M, K, N, R), W nonzeros) of every case searched."""
        if getattr(self, "_case_list", None) is None:
            allc = cases() if self.permutations else {(nm, ""): b for nm, b in algorithms().items()}
            self._case_list = [(nm, pm, b, self._w_terms(nm, pm)) for (nm, pm), b in allc.items()]
        return self._case_list

    def _space(self, m, k, n):
        """(lower bound ms, name, perm, base, levels, precision, moduli) of
        every admissible candidate: each shipped base case and (with
        permutations) each ordering of its dimensions (Section 2.3), at
        0..max_levels levels, every listed leaf precision.  The bound is the
        model time with every efficiency factor set to 1 (the leaf products
        at the precision's full rate; the emulated path's passes, CRT and
        launches as modelled; the classical fringe): no model time can be
        lower."""
        out = []
        nmod = moduli_for(self.tol, k) if "ozaki_bf16" in self.precisions else None
        rate = {"fp64": self.fp64_tflops, "ozaki_bf16": self.tc_tflops / (nmod or 1), **TF32_TFLOPS}
        for prec in self.precisions:
            if prec == "ozaki_bf16" and nmod is None:
                continue
            if prec in TF32_ERR and 2 * TF32_ERR[prec][0] > self.tol:
                continue
            work = 3.0 if prec == "fp32" else 1.0
            entries = [("strassen_222_7", "", (2, 2, 2, 7), 0, 1)]
            for name, perm, base, wt in self._cases():
                M, K, N, R = base
                for L in range(1, self.max_levels + 1):
                    if min(m // M ** L, k // K ** L, n // N ** L) < 64 or R ** L > 20000:
                        break
                    if prec == "ozaki_bf16" and R ** L * nmod > 65535:
                        break
                    entries.append((name, perm, base, L, wt))
            for name, perm, base, L, wt in entries:
                M, K, N, R = base
                sm, sk, sn = M ** L, K ** L, N ** L
                mp, kp, np_ = (m // sm) * sm, (k // sk) * sk, (n // sn) * sn
                lb = (2.0 * (R / (M * K * N)) ** L * mp * kp * np_ * work / (rate[prec] * 1e12)
                      + 2.0 * (m * n * k - mp * np_ * kp) / (self.fp64_tflops * 1e12))
                out.append((1e3 * lb, name, perm, base, L, prec, nmod, (mp, kp, np_, wt)))
        out.sort(key=lambda e: e[0])
        return out

    def _bound(self, e):
        """The tighter bound of a _space entry: its leaf and fringe bound plus,
        for the emulated path, the modelled passes."""
        lb, name, perm, base, L, prec, nmod, (mp, kp, np_, wt) = e
        if prec == "ozaki_bf16":
            M, K, N, R = base
            lb += 1e3 * self._emulated_passes(mp, kp, np_, M, K, N, R, L, nmod, wt)
        return lb

    def _emulated_passes(self, mp, kp, np_, M, K, N, R, L, nmod, wterms):
        """Seconds of the emulated path's passes besides the residue GEMM
        (exponents, the fused first level, later levels, W + CRT, launches)."""
        grow_a = R / (M * K) if L else 1.0
        grow_b = R / (K * N) if L else 1.0
        width = 2 if L <= 1 else 1
        t = (mp * kp + kp * np_) * 8 * 2 / (HBM_GBS * 1e9)
        t += (mp * kp * (8 + grow_a * nmod * width) + kp * np_ * (8 + grow_b * nmod * width)) / (SPLIT_GBS * 1e9)
        if L and (M * K not in FUSED_BLOCKS or K * N not in FUSED_BLOCKS):
            # no fused first level for this block grid: a residue pass first
            t += (mp * kp + kp * np_) * (8 + 2 * nmod) / (LEVEL_GBS * 1e9)
        for l in range(2, L + 1):
            w = 2 if l == L else 1
            ml, kl, nl = mp // M ** l, kp // K ** l, np_ // N ** l
            t += R ** l * (ml * kl + kl * nl) * nmod * (2 + w) / (LEVEL_GBS * 1e9)
            t += R ** (l - 1) * M * N * ml * nl * nmod * 3 / (LEVEL_GBS * 1e9)
        terms = (wterms / (M * N)) if L else 1.0
        t += mp * np_ * nmod * CRT_PS_PER_ELEM_MOD * 1e-12 * (1.0 + W_TERM_FACTOR * (terms - 1.0))
        t += (6 + 3 * max(L - 1, 0)) * LAUNCH_US * 1e-6
        return t * self.pass_scale

    def candidates(self, m, k, n):
        """Every admissible candidate with its model time (ms), best first,
        with the leaf tile the model prefers."""
        out = [self._model(m, k, n, name, perm, base, L, prec, nmod)
               for _, name, perm, base, L, prec, nmod, _ in self._space(m, k, n)]
        # FP64 error grows with depth; drop plans that cannot meet the target
        out = [c for c in out if c is not None]
        out.sort(key=lambda c: c.model_ms)
        return out

    def _levels(self):
        """The recursive cases as arrays (computed once): for each (case, L),
        L >= 1, in increasing rho^L (rho = R / (M K N), the fraction of the
        classical flops one level keeps): rho^L, M^L, K^L, N^L, R^L and the
        coefficients of the emulated passes' model time (seconds before the
        pass scale) as a + b nmod per unit of the block areas mp kp, kp np and
        mp np, plus a constant (the launches)."""
        if getattr(self, "_level_tab", None) is None:
            import numpy as np
            rows, info = [], []
            for name, perm, base, wt in self._cases():
                M, K, N, R = base
                for L in range(1, self.max_levels + 1):
                    if R ** L > 20000:
                        break
                    rows.append([(R / (M * K * N)) ** L, M ** L, K ** L, N ** L, R ** L]
                                + self._pass_coeffs(M, K, N, R, L, wt))
                    info.append((name, perm, base, L, wt))
            order = sorted(range(len(rows)), key=lambda i: rows[i][0])
            self._level_tab = (np.array([rows[i] for i in order], dtype=np.float64).reshape(-1, 12),
                               [info[i] for i in order])
            # per depth L: the least rho^L and the least of each pass
            # coefficient over the cases (a bound for every case of that depth)
            self._level_min = {}
            for L in range(1, self.max_levels + 1):
                sel = [r for r, inf in zip(rows, info) if inf[3] == L]
                if sel:
                    self._level_min[L] = [min(r[0] for r in sel)] + [min(r[5 + j] for r in sel) for j in range(7)]
        return self._level_tab

    def _recursion_excluded(self, m, k, n, precs, rate, work, nmod, limit):
        """True when no recursive candidate can beat `limit` (ms), by a bound
        over all cases of each depth at once: rho^L is at least its least
        value at that depth, the leaves and fringe cost at least
        2 rho^L m k n min(work / leaf rate, 1 / FP64 rate), and an admissible
        case (leaves at least 64 on a side) peels at most 1/64 of each
        dimension, so every block area is at least (63/64)^2 of the full one
        and the emulated passes at least the least coefficients times those
        areas."""
        self._levels()
        flops = 2.0 * m * k * n
        q2 = (63.0 / 64.0) ** 2
        for L, (rho, amk, bmk, akn, bkn, amn, bmn, c) in self._level_min.items():
            for prec in precs:
                lb = rho * flops * min(work[prec] / (rate[prec] * 1e12), 1.0 / (self.fp64_tflops * 1e12))
                if prec == "ozaki_bf16":
                    lb += self.pass_scale * (q2 * ((amk + bmk * nmod) * m * k + (akn + bkn * nmod) * k * n
                                                   + (amn + bmn * nmod) * m * n) + c)
                if 1e3 * lb <= limit:
                    return False
        return True

    @staticmethod
    def _pass_coeffs(M, K, N, R, L, wterms):
        """_emulated_passes as a linear form (L >= 1): [a_mk, b_mk, a_kn, b_kn,
        a_mn, b_mn, c], time = sum_x (a_x + b_x nmod) area_x + c."""
        ga, gb = R / (M * K), R / (K * N)
        width = 2 if L <= 1 else 1
        H, S, V = HBM_GBS * 1e9, SPLIT_GBS * 1e9, LEVEL_GBS * 1e9
        a_mk = a_kn = 16.0 / H + 8.0 / S
        b_mk, b_kn = ga * width / S, gb * width / S
        if M * K not in FUSED_BLOCKS or K * N not in FUSED_BLOCKS:
            a_mk += 8.0 / V
            a_kn += 8.0 / V
            b_mk += 2.0 / V
            b_kn += 2.0 / V
        b_mn = 0.0
        for l in range(2, L + 1):
            w = 2 if l == L else 1
            b_mk += R ** l * (2 + w) / ((M * K) ** l * V)
            b_kn += R ** l * (2 + w) / ((K * N) ** l * V)
            b_mn += R ** (l - 1) * M * N * 3 / ((M * N) ** l * V)
        b_mn += CRT_PS_PER_ELEM_MOD * 1e-12 * (1.0 + W_TERM_FACTOR * (wterms / (M * N) - 1.0))
        c = (6 + 3 * (L - 1)) * LAUNCH_US * 1e-6
        return [a_mk, b_mk, a_kn, b_kn, 0.0, b_mn, c]

    def _recursive_bounds(self, m, k, n, precs, rate, work, nmod, limit=float("inf")):
        """(bound ms, index into the level table, precision) of every
        admissible recursive candidate whose bound is at most `limit`, in
        increasing bound: the _space bound plus, for the emulated path, the
        modelled passes (the same numbers as _bound), computed for all cases
        at once."""
        import numpy as np
        tab, _ = self._levels()
        if not len(tab):
            return []
        rho, sm, sk, sn, RL = tab[:, 0], tab[:, 1], tab[:, 2], tab[:, 3], tab[:, 4]
        mb, kb, nb = m // sm, k // sk, n // sn
        ok = np.minimum(np.minimum(mb, kb), nb) >= 64
        mp, kp, np_ = mb * sm, kb * sk, nb * sn
        core = mp * kp * np_
        fringe = 2.0 * (float(m) * n * k - core) / (self.fp64_tflops * 1e12)
        out = []
        for prec in precs:
            lb = 1e3 * (2.0 * rho * core * work[prec] / (rate[prec] * 1e12) + fringe)
            mask = ok
            if prec == "ozaki_bf16":
                mask = ok & (RL * nmod <= 65535)
                c = tab[:, 5:]
                t = ((c[:, 0] + c[:, 1] * nmod) * mp * kp + (c[:, 2] + c[:, 3] * nmod) * kp * np_
                     + (c[:, 4] + c[:, 5] * nmod) * mp * np_ + c[:, 6])
                lb = lb + 1e3 * t * self.pass_scale
            out += [(float(lb[i]), int(i), prec) for i in np.nonzero(mask & (lb <= limit))[0]]
        out.sort(key=lambda e: e[0])
        return out

    def best_candidates(self, m, k, n, count=1):
        """The `count` candidates of least model time, found by branch and
        bound (the same model times as candidates()[:count], at a fraction of
        the work): the classical candidates are modelled first; the recursive
        ones are taken in increasing order of their _space + pass bound
        (computed for all of them at once) and modelled until the bound
        exceeds the count-th best model time so far."""
        nmod = moduli_for(self.tol, k) if "ozaki_bf16" in self.precisions else None
        rate = {"fp64": self.fp64_tflops, "ozaki_bf16": self.tc_tflops / (nmod or 1), **TF32_TFLOPS}
        precs = []
        for prec in self.precisions:
            if prec == "ozaki_bf16" and nmod is None:
                continue
            if prec in TF32_ERR and 2 * TF32_ERR[prec][0] > self.tol:
                continue
            precs.append(prec)
        work = {p: (3.0 if p == "fp32" else 1.0) for p in precs}
        best = []

        def add(c):
            if c is not None:
                best.append(c)
                best.sort(key=lambda c: c.model_ms)
                del best[count:]

        for prec in precs:
            add(self._model(m, k, n, "strassen_222_7", "", (2, 2, 2, 7), 0, prec, nmod))
        _, info = self._levels()
        limit = best[count - 1].model_ms if len(best) >= count else float("inf")
        if self._recursion_excluded(m, k, n, precs, rate, work, nmod, limit):
            return best
        for lb, i, prec in self._recursive_bounds(m, k, n, precs, rate, work, nmod, limit):
            if len(best) >= count and lb > best[count - 1].model_ms:
                break
            name, perm, base, L, _ = info[i]
            add(self._model(m, k, n, name, perm, base, L, prec, nmod))
        return best

    def _model(self, m, k, n, name, perm, base, L, prec, nmod):
        M, K, N, R = base
        if prec == "fp64" and L > 0 and self.tol < 1e-13 * (2.0 ** L):
            return None
        if prec in TF32_ERR and 2 * TF32_ERR[prec][0] * TF32_ERR[prec][1] ** L > self.tol:
            return None
        sm, sk, sn = M ** L, K ** L, N ** L
        mp, kp, np_ = (m // sm) * sm, (k // sk) * sk, (n // sn) * sn
        mL, kL, nL = mp // sm, kp // sk, np_ // sn
        leaves = R ** L
        fringe = 2.0 * (m * n * k - mp * np_ * kp)
        tile = "auto"
        if prec == "fp64":
            leaf_flops = 2.0 * leaves * mL * kL * nL
            best = None
            for tname, (bm, bn, speed) in FP64_TILES.items():
                tt = leaf_flops / (self.fp64_tflops * 1e12 * speed * classical_efficiency(mL, nL, bm, bn, leaves))
                if best is None or tt < best[0]:
                    best = (tt, tname)
            t, tile = best
            # level-by-level additions: bytes moved per level
            adds = 0.0
            for l in range(1, L + 1):
                adds += R ** l * ((mp // M ** l) * (kp // K ** l) + (kp // K ** l) * (np_ // N ** l)
                                  + (mp // M ** l) * (np_ // N ** l)) * 8 * 3
            t += adds / (HBM_GBS * 1e9)
            flags = fmm.FLAG_LEVELWISE if L > 0 else fmm.FLAGS_DEFAULT
        elif prec in TF32_ERR:
            # leaves on the TF32 tensor path; S/T and W level by level in FP64
            split = 3 if prec == "fp32" else 1
            kpad = -(-kL // 32) * 32
            best = None
            for tname, speed in TC_TILES.items():
                tile_n = 256 if (nL >= 256 and split == 1 and tname == "auto") else 128
                tt = 2.0 * leaves * mL * kpad * split * nL / (
                    TF32_TFLOPS[prec] * 1e12 * speed * classical_efficiency(mL, nL, 128, tile_n, leaves))
                if best is None or tt < best[0]:
                    best = (tt, tname)
            t, tile = best
            adds = 0.0
            if L == 1 and M * K in FUSED_BLOCKS and K * N in FUSED_BLOCKS and R <= 64:
                # the level fused with the conversion: each operand read once,
                # the leaves' TF32 operands written; FP32 products, W in FP32
                t += (8 * (mp * kp + kp * np_) + 4 * split * leaves * (mL + nL) * kpad) / (HBM_GBS * 1e9)
                adds = R * mL * nL * 4 * 2 + mp * np_ * 8
            else:
                # FP64 operands to TF32 (8 bytes in, 4 split bytes out per element)
                t += leaves * (mL * kL + kL * nL) * (8 + 4 * split) / (HBM_GBS * 1e9)
                for l in range(1, L + 1):
                    adds += R ** l * ((mp // M ** l) * (kp // K ** l) + (kp // K ** l) * (np_ // N ** l)
                                      + (mp // M ** l) * (np_ // N ** l)) * 8 * 3
            t += adds / (HBM_GBS * 1e9)
            t += (3 + 3 * L) * LAUNCH_US * 1e-6
            flags = fmm.FLAG_LEVELWISE if L > 0 else fmm.FLAGS_DEFAULT
        else:
            kpad = -(-kL // 64) * 64
            best = None
            for tname, speed in TC_TILES.items():
                tile_n = 256 if (nL >= 256 and tname == "auto") else 128
                tt = 2.0 * leaves * nmod * mL * kpad * nL / (
                    self.tc_tflops * 1e12 * speed * classical_efficiency(mL, nL, 128, tile_n, leaves * nmod))
                if best is None or tt < best[0]:
                    best = (tt, tname)
            t, tile = best
            t += self._emulated_passes(mp, kp, np_, M, K, N, R, L, nmod,
                                       self._w_terms(name, perm) if L else M * N)
            flags = fmm.FLAGS_DEFAULT
        t += fringe / (self.fp64_tflops * 1e12)
        return Choice(name, L, flags, prec, nmod or 15, tile, 1e3 * t, perm=perm if L else "")

    def _w_terms(self, name, perm=""):
        """Nonzeros of the (permuted) base case's W (terms of the top-level W
        combination)."""
        if not hasattr(self, "_wnnz"):
            self._wnnz = {}
        if (name, perm) not in self._wnnz:
            self._wnnz[(name, perm)] = int((_factors(name, perm)[5] != 0).sum())
        return self._wnnz[(name, perm)]

    # ----------------------------------------------------------- calibration
    def calibrate(self, size=4096, nmod=12):
        """Re-measure the model's rates on this GPU: the classical FP64 GEMM
        (flops per second at size/2), the residue GEMM (the leaf launch of a
        classical emulated product at `size`, timed with the library's event
        pair) and the emulated path's other passes (the rest of that product,
        as a scale on their modelled time).  Clears the choice cache; returns
        the rates."""
        import torch
        n2 = size // 2
        A = torch.rand((n2, n2), dtype=torch.float64, device="cuda")
        fmm.classical_gemm(A, A)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fmm.classical_gemm(A, A)
        e1.record()
        e1.synchronize()
        self.fp64_tflops = 2.0 * n2 ** 3 / e0.elapsed_time(e1) / 1e9
        B = torch.rand((size, size), dtype=torch.float64, device="cuda")
        p = fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16", moduli=nmod)
        ws = torch.empty(p.workspace_size(size, size, size), dtype=torch.uint8, device="cuda")
        C = torch.empty_like(B)
        fmm.gemm(p, B, B, C=C, workspace=ws)
        torch.cuda.synchronize()
        fmm.timing_enable(True)
        e0.record()
        for _ in range(3):
            fmm.gemm(p, B, B, C=C, workspace=ws)
        e1.record()
        e1.synchronize()
        leaf_ms, leaf_n = fmm.timing_leaf_ms()
        fmm.timing_enable(False)
        step = e0.elapsed_time(e1) / 3
        leaf = leaf_ms / max(leaf_n, 1)
        kpad = -(-size // 64) * 64
        self.tc_tflops = 2.0 * nmod * size * kpad * size * classical_efficiency(size, size, 128, 256, nmod) ** -1 \
            / leaf / 1e9
        modelled = self._emulated_passes(size, size, size, 1, 1, 1, 1, 0, nmod, 1) / self.pass_scale
        self.pass_scale = max(step - leaf, 1e-3) * 1e-3 / modelled
        self._cache.clear()
        del A, B, C, ws
        return {"fp64_tflops": self.fp64_tflops, "tc_tflops": self.tc_tflops, "pass_scale": self.pass_scale}

    # ----------------------------------------------------------- choice
    def choose(self, m, k, n):
        """The choice for (m, k, n).  Without measurement: the model's best.
        With measurement: the model's best few, each checked for accuracy
        against a 16-moduli emulated classical product on random uniform
        operands of the shape (the emulated candidates' moduli count moved up
        or down until its measured e_F meets the target with the fewest
        moduli), then timed (median of three calls); the fastest kept."""
        m, k, n = int(m), int(k), int(n)   # numpy integers would overflow the exact bounds
        key = f"{m}x{k}x{n}:{self.tol:g}:{','.join(self.precisions)}"
        c = self._cache.get(key)
        if c is not None:
            return c
        cands = self.best_candidates(m, k, n, max(1, self.trials if self.measure else 1))
        best = cands[0]
        if self.measure and self.trials > 0:
            import torch
            A = torch.rand((m, k), dtype=torch.float64, device="cuda") * 2 - 1
            B = torch.rand((k, n), dtype=torch.float64, device="cuda") * 2 - 1
            ref = self._run(Choice("strassen_222_7", 0, fmm.FLAGS_DEFAULT, "ozaki_bf16", 16), A, B)
            timed = []
            for c in cands[:self.trials]:
                c2 = self._fit_accuracy(c, A, B, ref)
                if c2 is not None:
                    timed.append(self._time(c2, A, B))
            if timed:
                best = min(timed, key=lambda c: c.measured_ms)
            del A, B, ref
        self._cache[key] = best
        if self.cache_file:
            with open(self.cache_file, "w") as fh:
                json.dump({k_: asdict(v) for k_, v in self._cache.items()}, fh, indent=1)
        return best

    def plan(self, m, k, n):
        c = self.choose(m, k, n)
        key = (c.algorithm, c.perm, c.levels, c.flags, c.precision, c.moduli, c.tile)
        if key not in self._plans:
            self._plans[key] = c.plan()
        return self._plans[key]

    @staticmethod
    def _run(c, A, B, plan=None):
        import torch
        p = plan or c.plan()
        m, k = A.shape
        n = B.shape[1]
        C = torch.empty((m, n), dtype=torch.float64, device="cuda")
        wsz = p.workspace_size(m, k, n)
        ws = torch.empty(wsz, dtype=torch.uint8, device="cuda") if wsz else None
        fmm.gemm(p, A, B, C=C, workspace=ws)
        torch.cuda.synchronize()
        return C

    @staticmethod
    def _err(C, ref):
        import torch
        return float(torch.linalg.norm(C - ref) / torch.linalg.norm(ref))

    def _fit_accuracy(self, c, A, B, ref):
        """The candidate with its measured e_F, or None if it misses the
        target; emulated candidates get the fewest moduli (<= 16) that meet it."""
        if c.precision != "ozaki_bf16":
            e = self._err(self._run(c, A, B), ref)
            return Choice(**{**asdict(c), "measured_err": e}) if e <= self.tol else None
        nm = c.moduli
        e = self._err(self._run(Choice(**{**asdict(c), "moduli": nm}), A, B), ref)
        while e > self.tol and nm < 16:
            nm += 1
            e = self._err(self._run(Choice(**{**asdict(c), "moduli": nm}), A, B), ref)
        if e > self.tol:
            return None
        while nm > 3:
            e2 = self._err(self._run(Choice(**{**asdict(c), "moduli": nm - 1}), A, B), ref)
            if e2 > self.tol:
                break
            nm, e = nm - 1, e2
        return Choice(**{**asdict(c), "moduli": nm, "measured_err": e})

    def _time(self, c, A, B, reps=3):
        """Median of `reps` timed calls after one untimed call."""
        import statistics
        import torch
        p = c.plan()
        m, k = A.shape
        n = B.shape[1]
        C = torch.empty((m, n), dtype=torch.float64, device="cuda")
        wsz = p.workspace_size(m, k, n)
        ws = torch.empty(wsz, dtype=torch.uint8, device="cuda") if wsz else None
        fmm.gemm(p, A, B, C=C, workspace=ws)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fmm.gemm(p, A, B, C=C, workspace=ws)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return Choice(**{**asdict(c), "measured_ms": statistics.median(times)})
