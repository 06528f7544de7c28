"""GPU parity of the emulated-FP64 precision variant (tensor-core residue
products + CRT) against the oracle: exact on integer inputs (the scaled
operands need no rounding, so the CRT rebuilds A B exactly), within the
rounding bound and equal to the oracle's own emulation on random inputs,
and combined with the fast recursion."""
import numpy as np
import pytest

import oracle
from oracle import norms, ozaki
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def run(plan, A, B):
    import torch
    C = fmm.gemm(plan, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    fmm.check_device_error()
    return C.cpu().numpy()


@pytest.mark.parametrize("m,k,n", [(128, 64, 128), (1, 1, 1), (200, 300, 100), (257, 1100, 129), (96, 2048, 300)])
def test_classical_emulated_integer_exact(m, k, n):
    p = fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16")
    A, B = synth.operands(m, k, n, 41, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


@pytest.mark.parametrize("nmod", [15, 12, 8])
@pytest.mark.parametrize("m,k,n", [(130, 200, 70), (256, 1500, 256)])
def test_classical_emulated_matches_oracle_emulation(nmod, m, k, n):
    p = fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16", moduli=nmod)
    A, B = synth.operands(m, k, n, 42)
    C = run(p, A, B)
    Coz = ozaki.emulated_gemm(A, B, nmod)
    # same scaled integers, the exact integer product, one correct rounding
    assert np.array_equal(C, Coz)
    e = norms.rel_frobenius(C, oracle.gemm(A, B, precision="ld"))
    assert e <= (1e-14 if nmod == 15 else 1e-7 if nmod == 12 else 1e-2)


def test_classical_emulated_loguniform():
    p = fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16", moduli=16)
    A, B = synth.operands(128, 512, 128, 43, kind="loguniform")
    assert np.array_equal(run(p, A, B), ozaki.emulated_gemm(A, B, 16))


EMUL = {"residue_space": fmm.FLAGS_DEFAULT, "per_leaf": fmm.FLAGS_DEFAULT | fmm.FLAG_LEAF_EMULATION}


@pytest.mark.parametrize("mode", list(EMUL))
@pytest.mark.parametrize("name,levels", [("strassen_222_7", 1), ("strassen_222_7", 2), ("fmm_323_15", 1),
                                         ("fmm_423_20", 1), ("fmm_333_23", 1), ("strassen_222_7", 3),
                                         ("winograd_222_7", 1), ("winograd_222_7", 2)])
def test_fast_emulated_integer_exact(name, levels, mode):
    p = fmm.Plan(name, levels=levels, precision="ozaki_bf16", flags=EMUL[mode])
    A, B = synth.operands(261, 517, 259, 44, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 1), ("strassen_222_7", 2), ("fmm_333_23", 1),
                                         ("fmm_323_15", 2), ("winograd_222_7", 1)])
def test_fast_residue_space_equals_classical_emulation(name, levels):
    # the recursion over Z/pZ computes the same integer A'B' as the classical
    # emulation, so on the peeled core the two agree bit for bit
    M, K, N = {"strassen_222_7": (2, 2, 2), "fmm_333_23": (3, 3, 3), "fmm_323_15": (3, 2, 3),
               "winograd_222_7": (2, 2, 2)}[name]
    m, k, n = M ** levels * 70, K ** levels * 150, N ** levels * 60
    A, B = synth.operands(m, k, n, 46)
    fast = run(fmm.Plan(name, levels=levels, precision="ozaki_bf16"), A, B)
    classical = run(fmm.Plan(name, levels=0, precision="ozaki_bf16"), A, B)
    assert np.array_equal(fast, classical)
    assert np.array_equal(fast, ozaki.emulated_gemm(A, B, 15))


@pytest.mark.parametrize("mode", list(EMUL))
@pytest.mark.parametrize("name,levels", [("strassen_222_7", 2), ("fmm_333_23", 1)])
def test_fast_emulated_uniform(name, levels, mode):
    p = fmm.Plan(name, levels=levels, precision="ozaki_bf16", flags=EMUL[mode])
    A, B = synth.operands(300, 700, 290, 45)
    e = norms.rel_frobenius(run(p, A, B), oracle.gemm(A, B))
    assert e <= 1e-13


@pytest.mark.parametrize("nmod", [12, 13, 14, 16, 9])
@pytest.mark.parametrize("name,levels", [("strassen_222_7", 1), ("fmm_424_26", 1), ("strassen_222_7", 2)])
def test_fast_emulated_every_moduli_count(name, levels, nmod):
    # each moduli count has its own compiled W + CRT instance and its own limb
    # layout in the split; all must give the oracle's emulation bit for bit
    M, K, N = {"strassen_222_7": (2, 2, 2), "fmm_424_26": (4, 2, 4)}[name]
    m, k, n = M ** levels * 40, K ** levels * 200, N ** levels * 40
    A, B = synth.operands(m, k, n, 47)
    p = fmm.Plan(name, levels=levels, precision="ozaki_bf16", moduli=nmod)
    assert np.array_equal(run(p, A, B), ozaki.emulated_gemm(A, B, nmod))
    Ai, Bi = synth.operands(m + 3, k + 1, n + 2, 48, kind="integer")
    assert np.array_equal(run(p, Ai, Bi), oracle.gemm(Ai, Bi))


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 1), ("fmm_333_23", 1)])
def test_fast_emulated_loguniform(name, levels):
    # magnitudes over eight decades: the per-row and per-column exponents keep
    # the scaled integers full; the result is the oracle's emulation exactly
    M, K, N = {"strassen_222_7": (2, 2, 2), "fmm_333_23": (3, 3, 3)}[name]
    A, B = synth.operands(M * 90, K * 200, N * 80, 49, kind="loguniform")
    p = fmm.Plan(name, levels=levels, precision="ozaki_bf16", moduli=16)
    assert np.array_equal(run(p, A, B), ozaki.emulated_gemm(A, B, 16))


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 0), ("strassen_222_7", 1), ("fmm_424_26", 1)])
def test_emulated_zero_and_subnormal_rows_and_columns(name, levels):
    # row and column exponents on their special cases: all-zero and all
    # negative-zero rows/columns (exponent 0), rows/columns whose largest
    # entry is subnormal (the exact FP64 fallback), subnormal entries under a
    # normal maximum (truncated away); magnitudes keep every result normal
    rng = np.random.default_rng(50)
    m, k, n = 256, 320, 192
    A = rng.uniform(-1, 1, (m, k)) * 1e140
    B = rng.uniform(-1, 1, (k, n)) * 1e140
    A[3] = 0.0
    A[5] = rng.uniform(-1, 1, k) * 1e-310
    A[7] = rng.uniform(-1, 1, k) * 1e-310
    A[7, 10] = 0.5e140
    A[9] = -0.0
    B[:, 4] = 0.0
    B[:, 6] = rng.uniform(-1, 1, k) * 1e-310
    B[:, 8] = rng.uniform(-1, 1, k) * 1e-310
    B[11, 8] = -0.25e140
    B[:, 12] = -0.0
    assert np.all(np.abs(A[5]) < 2.3e-308) and np.any(A[5] != 0)
    p = fmm.Plan(name, levels=levels, precision="ozaki_bf16", moduli=13)
    C = run(p, A, B)
    assert np.array_equal(C, ozaki.emulated_gemm(A, B, 13))
    assert np.all(C[3] == 0) and np.all(C[:, 4] == 0)
    assert np.all(np.isfinite(C))


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 0), ("strassen_222_7", 1), ("fmm_424_26", 1)])
def test_emulated_rounding_ties(name, levels):
    # entries whose scaled values are exact half-integers (ties): the scaling
    # rounds them away from zero, as the oracle's emulation does
    rng = np.random.default_rng(51)
    M, K, N = {"strassen_222_7": (2, 2, 2), "fmm_424_26": (4, 2, 4)}[name]
    m, k, n = (M ** levels) * 64, (K ** levels) * 128, (N ** levels) * 48
    nmod = 12
    beta = ozaki.beta_bits(nmod, k)
    ulp = 2.0 ** -(beta - 1)        # rows and columns with maximum in [1, 2)
    A = (rng.integers(-5000, 5000, (m, k)) + 0.5) * ulp
    B = (rng.integers(-5000, 5000, (k, n)) + 0.5) * ulp
    A[:, 0] = 1.5
    B[0, :] = -1.25
    A[1::3] += rng.uniform(-1, 1, (len(range(1, m, 3)), k)) * 1e-9
    assert np.all(np.abs(A).max(axis=1) < 2) and np.all(np.abs(B).max(axis=0) < 2)
    p = fmm.Plan(name, levels=levels, precision="ozaki_bf16", moduli=nmod)
    assert np.array_equal(run(p, A, B), ozaki.emulated_gemm(A, B, nmod))


def test_longest_supported_k():
    # k_L = 65536 is the longest k the emulated product takes (the drain's
    # int32 sums); integer inputs stay exact and random ones equal the
    # oracle's emulation; one more is refused before anything is enqueued
    import torch
    p = fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16", moduli=14)
    A, B = synth.operands(40, 65536, 24, 43, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))
    A, B = synth.operands(40, 65536, 24, 44)
    assert np.array_equal(run(p, A, B), ozaki.emulated_gemm(A, B, 14))
    A = torch.zeros((8, 65537), dtype=torch.float64, device="cuda")
    B = torch.zeros((65537, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(fmm.FmmError) as ei:
        fmm.gemm(p, A, B)
    assert ei.value.status == fmm.FMM_ERR_UNSUPPORTED
