"""The autotuner's measured path on the GPU: candidates ranked by the model,
the best few checked for accuracy against a 16-moduli emulated product and
timed (median of three calls); the chosen plan must meet the target against
the oracle on fresh inputs of the shape.  Also: plans built from permuted
base cases (Section 2.3's permutations) compute the exact product."""
import numpy as np
import pytest

import oracle
from oracle import norms
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import autotune, synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,tol", [((1536, 1536, 1536), 1e-11), ((2048, 512, 1024), 1e-11),
                                       ((1536, 1536, 1536), 5e-15)])
def test_measured_choice_meets_target(shape, tol):
    import torch
    m, k, n = shape
    t = autotune.Autotuner(tol=tol, measure=True, trials=3)
    c = t.choose(m, k, n)
    assert c.measured_ms > 0 and 0 <= c.measured_err <= tol
    A, B = synth.operands(m, k, n, 90)
    C = fmm.gemm(t.plan(m, k, n), to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    fmm.check_device_error()
    assert norms.rel_frobenius(C.cpu().numpy(), oracle.gemm(A, B)) <= tol
    # cached: the same choice without another measurement
    assert t.choose(m, k, n) is c


@pytest.mark.parametrize("name,perm,precision", [("fmm_423_20", "c", "fp64"), ("fmm_423_20", "tc", "ozaki_bf16"),
                                                 ("fmm_424_26", "c", "ozaki_bf16"), ("fmm_323_15", "t", "fp64")])
def test_permuted_plans_exact_on_integers(name, perm, precision):
    import torch
    M, K, N, U, V, W = autotune.permuted_factors(name, perm)
    p = fmm.Plan(levels=1, factors=(M, K, N, U, V, W), precision=precision)
    A, B = synth.operands(M * 61 + 1, K * 70 + 2, N * 53 + 1, 91, kind="integer")
    C = fmm.gemm(p, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))


def test_narrow_tensor_tiles_same_result():
    # the 128 x 128 tensor-core tile gives the same integers as 128 x 256
    import torch
    A, B = synth.operands(512, 640, 768, 92)
    out = []
    for tile in ("auto", "128x128"):
        p = fmm.Plan("strassen_222_7", levels=1, precision="ozaki_bf16", moduli=14, tile=tile)
        out.append(fmm.gemm(p, to_dev(A), to_dev(B)).cpu().numpy())
        pt = fmm.Plan("strassen_222_7", levels=1, precision="tf32", tile=tile)
        out.append(fmm.gemm(pt, to_dev(A), to_dev(B)).cpu().numpy())
    torch.cuda.synchronize()
    assert np.array_equal(out[0], out[2])
    assert np.allclose(out[1], out[3], rtol=0, atol=1e-3 * np.abs(out[1]).max())


def test_calibration_measures_this_gpu():
    # the model's rates re-measured: the classical DFMA GEMM, the residue GEMM
    # and the emulated passes, each within a factor two of the defaults
    t = autotune.Autotuner(tol=1e-11, measure=False)
    r = t.calibrate(size=2048, nmod=12)
    assert 0.5 * autotune.FP64_TFLOPS < r["fp64_tflops"] < 2 * autotune.FP64_TFLOPS
    assert 0.5 * autotune.TC_TFLOPS < r["tc_tflops"] < 2 * autotune.TC_TFLOPS
    assert 0.25 < r["pass_scale"] < 4.0
    c = t.choose(3000, 3000, 3000)
    assert c.model_ms > 0
