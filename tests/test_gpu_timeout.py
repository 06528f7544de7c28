"""The bounded waits of the tensor-core kernels: a wait that nothing
completes runs out after its time limit, the kernel returns, the error flag
reads as FMM_ERR_TIMEOUT, and the context stays usable for correct products
afterwards.  The wait is made to run out by launching one CTA whose load and
MMA threads issue nothing (no copy or MMA is outstanding when it gives up);
nothing here faults or hangs the GPU."""
import time

import numpy as np
import pytest

import oracle
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", [0, 1])
def test_wait_runs_out_and_context_survives(kernel):
    import torch
    fmm.check_device_error()                      # clean flag to start from
    t0 = time.perf_counter()
    st = fmm.selftest_wait_timeout(kernel, 2_000_000)   # 2 ms limit
    dt = time.perf_counter() - t0
    assert st == fmm.FMM_ERR_TIMEOUT
    assert dt < 5.0                               # the limit, not an endless wait
    fmm.check_device_error()                      # read and cleared by the self-test
    # the context is intact: an emulated product and a TF32 one are still right
    A, B = synth.operands(200, 300, 260, 81, kind="integer")
    for prec in ("ozaki_bf16", "tf32"):
        C = fmm.gemm(fmm.Plan("strassen_222_7", levels=1, precision=prec), to_dev(A), to_dev(B))
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))
    fmm.check_device_error()


def test_wait_limit_setting():
    with pytest.raises(fmm.FmmError):
        fmm.set_wait_limit(0)
    fmm.set_wait_limit(500_000_000)
    try:
        A, B = synth.operands(256, 512, 256, 82, kind="integer")
        C = fmm.gemm(fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16"), to_dev(A), to_dev(B))
        fmm.check_device_error()
        assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))
    finally:
        fmm.set_wait_limit(2_000_000_000)
