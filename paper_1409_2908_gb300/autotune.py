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


@dataclass(frozen=True)
class Choice:
    algorithm: str            # algorithm file name (levels 0: the classical product)
    levels: int
    flags: int
    precision: str            # "fp64", "ozaki_bf16", "tf32" or "fp32"
    moduli: int = 15
    tile: str = "auto"
    model_ms: float = 0.0
    measured_ms: float = -1.0

    def plan(self):
        return fmm.Plan(self.algorithm, levels=self.levels, flags=self.flags,
                        precision=self.precision, tile=self.tile,
                        moduli=self.moduli if self.precision == "ozaki_bf16" else None)


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


def moduli_for(tol, k):
    """Fewest moduli whose truncation error 2^(1-beta) (with a factor 4 of
    slack; measured e_F on uniform data is about 0.9 x 2^(1-beta)) meets the
    relative tolerance."""
    for n in range(6, 17):
        P = 1
        for p in (256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193)[:n]:
            P *= p
        beta = 62
        while beta > 0 and k * 2 ** (2 * beta + 1) >= P:
            beta -= 1
        if 4 * 2.0 ** (1 - beta) <= tol:
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


class Autotuner:
    def __init__(self, tol=1e-11, precisions=("fp64", "ozaki_bf16"), max_levels=3,
                 trials=3, cache_file=None, measure=True):
        self.tol = tol
        self.precisions = tuple(precisions)
        self.max_levels = max_levels
        self.trials = trials
        self.cache_file = cache_file
        self.measure = measure
        self._cache = {}
        self._plans = {}
        if cache_file and os.path.exists(cache_file):
            with open(cache_file) as fh:
                for key, d in json.load(fh).items():
                    self._cache[key] = Choice(**d)

    # ----------------------------------------------------------- model
    def candidates(self, m, k, n):
        """Every admissible candidate with its model time (ms), best first."""
        out = []
        algs = algorithms()
        nmod = moduli_for(self.tol, k) if "ozaki_bf16" in self.precisions else None
        emulated = "ozaki_bf16" in self.precisions and nmod is not None
        for prec in self.precisions:
            if prec == "ozaki_bf16" and nmod is None:
                continue
            if prec in TF32_ERR and 2 * TF32_ERR[prec][0] > self.tol:
                continue
            # the DFMA pipe is ~1/100 of the emulated rate: FP64 plans only
            # compete on products too small for the tensor-core path to fill
            if prec == "fp64" and emulated and min(m, k, n) >= 64:
                continue
            out.append(self._model(m, k, n, "strassen_222_7", (2, 2, 2, 7), 0, prec, nmod))
            for name, base in algs.items():
                M, K, N, R = base
                for L in range(1, self.max_levels + 1):
                    mL, kL, nL = m // M ** L, k // K ** L, n // N ** L
                    if min(mL, kL, nL) < 64 or R ** L > 20000:
                        break
                    if prec == "ozaki_bf16" and R ** L * nmod > 65535:
                        break
                    out.append(self._model(m, k, n, name, base, L, prec, nmod))
        # FP64 error grows with depth; drop plans that cannot meet the target
        out = [c for c in out if c is not None]
        out.sort(key=lambda c: c.model_ms)
        return out

    def _model(self, m, k, n, name, base, L, prec, nmod):
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
        if prec == "fp64":
            leaf_flops = 2.0 * leaves * mL * kL * nL
            t = leaf_flops / (FP64_TFLOPS * 1e12 * classical_efficiency(mL, nL))
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
            tile_n = 256 if (nL >= 256 and split == 1) else 128
            t = 2.0 * leaves * mL * kpad * split * nL / (
                TF32_TFLOPS[prec] * 1e12 * classical_efficiency(mL, nL, 128, tile_n, leaves))
            # FP64 operands to TF32 (8 bytes in, 4 split bytes out per element)
            t += leaves * (mL * kL + kL * nL) * (8 + 4 * split) / (HBM_GBS * 1e9)
            adds = 0.0
            for l in range(1, L + 1):
                adds += R ** l * ((mp // M ** l) * (kp // K ** l) + (kp // K ** l) * (np_ // N ** l)
                                  + (mp // M ** l) * (np_ // N ** l)) * 8 * 3
            t += adds / (HBM_GBS * 1e9)
            t += (3 + 3 * L) * LAUNCH_US * 1e-6
            flags = fmm.FLAG_LEVELWISE if L > 0 else fmm.FLAGS_DEFAULT
        else:
            kpad = -(-kL // 64) * 64
            t = 2.0 * leaves * nmod * mL * kpad * nL / (
                TC_TFLOPS * 1e12 * classical_efficiency(mL, nL, 128, 256 if nL >= 256 else 128, leaves * nmod))
            # exponents, then the fused first level: FP64 in, R/(MK) residue
            # planes out per operand element (bfloat16 when it is the last level)
            grow_a = R / (M * K) if L else 1.0
            grow_b = R / (K * N) if L else 1.0
            width = 2 if L <= 1 else 1
            t += (mp * kp + kp * np_) * 8 * 2 / (HBM_GBS * 1e9)
            t += (mp * kp * (8 + grow_a * nmod * width) + kp * np_ * (8 + grow_b * nmod * width)) / (SPLIT_GBS * 1e9)
            for l in range(2, L + 1):
                w = 2 if l == L else 1
                ml, kl, nl = mp // M ** l, kp // K ** l, np_ // N ** l
                t += R ** l * (ml * kl + kl * nl) * nmod * (2 + w) / (LEVEL_GBS * 1e9)
                t += R ** (l - 1) * M * N * ml * nl * nmod * 3 / (LEVEL_GBS * 1e9)
            terms = (self._w_terms(name) / (M * N)) if L else 1.0
            t += mp * np_ * nmod * CRT_PS_PER_ELEM_MOD * 1e-12 * (1.0 + W_TERM_FACTOR * (terms - 1.0))
            t += (6 + 3 * max(L - 1, 0)) * LAUNCH_US * 1e-6
            flags = fmm.FLAGS_DEFAULT
        t += fringe / (FP64_TFLOPS * 1e12)
        return Choice(name, L, flags, prec, nmod or 15, "auto", 1e3 * t)

    def _w_terms(self, name):
        """Nonzeros of the base case's W (terms of the top-level W combination)."""
        if not hasattr(self, "_wnnz"):
            self._wnnz = {}
        if name not in self._wnnz:
            from . import algorithm_factors
            self._wnnz[name] = int((algorithm_factors(name)[5] != 0).sum())
        return self._wnnz[name]

    # ----------------------------------------------------------- choice
    def choose(self, m, k, n):
        key = f"{m}x{k}x{n}:{self.tol:g}:{','.join(self.precisions)}"
        if key in self._cache:
            return self._cache[key]
        cands = self.candidates(m, k, n)
        best = cands[0]
        if self.measure and self.trials > 1:
            timed = [self._time(c, m, k, n) for c in cands[:self.trials]]
            best = min(timed, key=lambda c: c.measured_ms)
        self._cache[key] = best
        if self.cache_file:
            with open(self.cache_file, "w") as fh:
                json.dump({k_: asdict(v) for k_, v in self._cache.items()}, fh, indent=1)
        return best

    def plan(self, m, k, n):
        c = self.choose(m, k, n)
        key = (c.algorithm, c.levels, c.flags, c.precision, c.moduli, c.tile)
        if key not in self._plans:
            self._plans[key] = c.plan()
        return self._plans[key]

    def _time(self, c, m, k, n):
        import torch
        p = c.plan()
        A = torch.rand((m, k), dtype=torch.float64, device="cuda") * 2 - 1
        B = torch.rand((k, n), dtype=torch.float64, device="cuda") * 2 - 1
        C = torch.empty((m, n), dtype=torch.float64, device="cuda")
        wsz = p.workspace_size(m, k, n)
        ws = torch.empty(wsz, dtype=torch.uint8, device="cuda") if wsz else None
        fmm.gemm(p, A, B, C=C, workspace=ws)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fmm.gemm(p, A, B, C=C, workspace=ws)
        e1.record()
        e1.synchronize()
        return Choice(**{**asdict(c), "measured_ms": e0.elapsed_time(e1)})
