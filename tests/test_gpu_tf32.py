"""The TF32 precision variants (tensor-core leaf products with operands
rounded to TF32, and the FP32-accurate variant summing three TF32 pair
products): exact on small integer inputs (they are representable in TF32 and
every partial sum is exact in FP32), and within their rounding bounds of the
FP64 oracle on random inputs, alone and under the fast recursion."""
import numpy as np
import pytest

import oracle
from oracle import norms
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


@pytest.mark.parametrize("name,levels,shape", [("strassen_222_7", 0, (200, 300, 130)),
                                               ("strassen_222_7", 0, (1, 1, 1)),
                                               ("strassen_222_7", 1, (257, 515, 259)),
                                               ("strassen_222_7", 2, (300, 260, 290)),
                                               ("fmm_323_15", 1, (301, 200, 303)),
                                               # one level fused with the conversion: block grids of 8 and 9
                                               ("fmm_424_26", 1, (516, 202, 390)),
                                               ("fmm_333_23", 1, (301, 330, 299))])
def test_tf32_integer_exact(name, levels, shape):
    p = fmm.Plan(name, levels=levels, precision="tf32")
    A, B = synth.operands(*shape, 61, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 0), ("strassen_222_7", 1), ("strassen_222_7", 2)])
def test_tf32_uniform_within_rounding_bound(name, levels):
    p = fmm.Plan(name, levels=levels, precision="tf32")
    m, k, n = 256, 1024, 192
    A, B = synth.operands(m, k, n, 62)
    C = run(p, A, B)
    ref = oracle.gemm(A, B)
    if levels == 0:
        # each operand rounded to 11 significant bits, FP32 accumulation
        bound = (2.0 ** -10 + k * 2.0 ** -23) * (np.abs(A) @ np.abs(B))
        assert np.all(np.abs(C - ref) <= bound)
    assert norms.rel_frobenius(C, ref) <= 2e-3


# FP32-accurate leaves: each operand split into a TF32 pair (hi, lo), three
# pair products summed in one tensor-core product over a tripled k

@pytest.mark.parametrize("name,levels,shape", [("strassen_222_7", 0, (200, 300, 130)),
                                               ("strassen_222_7", 0, (1, 1, 1)),
                                               ("strassen_222_7", 1, (257, 515, 259)),
                                               ("winograd_222_7", 2, (300, 260, 290)),
                                               ("fmm_323_15", 1, (301, 200, 303)),
                                               ("fmm_424_26", 1, (516, 202, 390)),
                                               ("fmm_333_23", 1, (301, 330, 299))])
def test_fp32_integer_exact(name, levels, shape):
    # small integers are their own hi part (lo = 0) and every sum is exact in FP32
    p = fmm.Plan(name, levels=levels, precision="fp32")
    A, B = synth.operands(*shape, 63, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 0), ("strassen_222_7", 1), ("strassen_222_7", 2)])
def test_fp32_uniform_within_rounding_bound(name, levels):
    m, k, n = 256, 1024, 192
    A, B = synth.operands(m, k, n, 64)
    ref = oracle.gemm(A, B)
    C = run(fmm.Plan(name, levels=levels, precision="fp32"), A, B)
    if levels == 0:
        # operands to FP32 (2^-24), the pair keeps 22 bits of it (2^-22 per
        # operand), lo x lo dropped (2^-22), FP32 accumulation over 3k terms
        # (one unit in the last place per addition, as for TF32 above)
        bound = (4 * 2.0 ** -22 + 3 * k * 2.0 ** -23) * (np.abs(A) @ np.abs(B))
        assert np.all(np.abs(C - ref) <= bound)
    # the tensor core sums chunks of 512 k (x3) in FP32, the chunks are added
    # on the CUDA cores with round to nearest (over the whole tripled k in
    # TMEM the error reached 1.06e-5 here and 1.7e-4 at k = 16384)
    e = norms.rel_frobenius(C, ref)
    assert e <= 3e-5
    # and an order of magnitude more accurate than one TF32 product
    e_tf = norms.rel_frobenius(run(fmm.Plan(name, levels=levels, precision="tf32"), A, B), ref)
    assert e * 10 < e_tf


def test_fp32_loguniform():
    # magnitudes over eight decades: relative accuracy per element, not per norm
    A, B = synth.operands(128, 512, 96, 65, kind="loguniform")
    C = run(fmm.Plan("strassen_222_7", levels=1, precision="fp32"), A, B)
    ref = oracle.gemm(A, B)
    assert np.all(np.abs(C - ref) <= (1e-5 + 512 * 2.0 ** -22) * (np.abs(A) @ np.abs(B)))


@pytest.mark.parametrize("precision", ["tf32", "fp32"])
def test_fused_level_with_non_integer_coefficients(precision):
    # Strassen with U doubled and W halved (still exact: every product doubles
    # and its weight halves): the fused level forms S in FP32 with the
    # coefficient 2, the W pass in FP64 with 1/2; small integers stay exact
    M, K, N, U, V, W = fmm.algorithm_factors("strassen_222_7")
    p = fmm.Plan(factors=(M, K, N, 2.0 * U, V, 0.5 * W), levels=1, precision=precision)
    A, B = synth.operands(258, 260, 262, 66, kind="integer")
    assert np.array_equal(run(p, A, B), oracle.gemm(A, B))


@pytest.mark.parametrize("precision", ["tf32", "fp32"])
def test_host_entry_point_tf32_family(precision):
    # fmm_gemm_host with TF32-family leaves (no overlap: the path waits for
    # all inputs) gives the device entry point's result bit for bit
    import torch
    p = fmm.Plan("strassen_222_7", levels=1, precision=precision)
    m, k, n = 1030, 770, 900
    A, B = synth.operands(m, k, n, 67)
    Cd = run(p, A, B)
    ws = torch.empty(fmm.host_workspace_size(p, m, k, n), dtype=torch.uint8, device="cuda")
    Ah, Bh = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    Ch = torch.zeros((m, n), dtype=torch.float64).pin_memory()
    for _ in range(2):
        fmm.gemm_host(p, Ah, Bh, Ch, ws)
        assert np.array_equal(Ch.numpy(), Cd)
        Ch.zero_()
    fmm.check_device_error()
