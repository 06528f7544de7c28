"""The TF32 precision variant (tensor-core leaf products with operands rounded
to TF32): exact on small integer inputs (they are representable in TF32 and
every partial sum is exact in FP32), and within the TF32 rounding bound of
the FP64 oracle on random inputs, alone and under the fast recursion."""
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
                                               ("fmm_323_15", 1, (301, 200, 303))])
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
