"""fmm_gemm_noalloc: the entry point for programs that cannot allocate device
memory when they need a product, because another allocator (a framework's
caching allocator, or a pool sized at start-up) already holds the device
memory, or because their hot path may not call the CUDA allocator at all.  It
keeps its only scratch, the leaf products, in a fixed file-scope device array
and reads the plan's lists from the plan's own device copy.

Checked through the C ABI on two calls in a row with different inputs (the
array keeps the previous call's contents): against the oracle (bit-exact on
integer inputs, e_F <= 1e-11 on uniform[-1,1] inputs) and against fmm_gemm
with the same plan.  Sizes beyond the array, and a plan whose lists are not on
the device yet, are rejected before anything runs.  Collected last so that a
run stopping at the first failure has run every other test first; it also
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

TOL_F = 1e-11
SCRATCH = 32 * 1024 * 1024


def _noalloc(plan, A, B, C, stream):
    L = _lib.lib()
    return L.fmm_gemm_noalloc(plan.handle, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                              ctypes.c_void_p(B.data_ptr()), B.stride(0),
                              ctypes.c_void_p(C.data_ptr()), C.stride(0),
                              A.shape[0], A.shape[1], B.shape[1],
                              ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("name,levels,shape", [
    ("strassen_222_7", 1, (515, 513, 517)),
    ("strassen_222_7", 2, (400, 388, 396)),
    ("fmm_323_15", 1, (301, 202, 303)),
])
def test_noalloc_matches_oracle_and_fmm_gemm_two_calls(name, levels, shape):
    import torch
    m, k, n = shape
    plan = fmm.Plan(name, levels=levels)
    plan.prepare()
    stream = torch.cuda.current_stream()
    for call, (seed, kind) in enumerate([(31, "integer"), (32, "uniform")]):
        A, B = synth.operands(m, k, n, seed, kind=kind)
        want = oracle.gemm(A, B)
        Ad = torch.from_numpy(A).cuda()
        Bd = torch.from_numpy(B).cuda()
        C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(plan, Ad, Bd, C, stream)
        assert st == fmm.FMM_OK, (call, st)
        assert fmm.last_launch_count() >= 2
        C_ref = fmm.gemm(plan, Ad, Bd)
        torch.cuda.synchronize()
        got, ref = C.cpu().numpy(), C_ref.cpu().numpy()
        if kind == "integer":
            assert np.array_equal(got, want), call
            assert np.array_equal(got, ref), call
        else:
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL_F, call
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL_F, call


def test_noalloc_rejects_problems_beyond_the_scratch():
    import torch
    plan = fmm.Plan("strassen_222_7", levels=1)
    plan.prepare()
    m = k = n = 2048            # 7 leaf products of 1024^2 doubles = 56 MiB > 32 MiB
    assert 7 * (m // 2) * (n // 2) * 8 > SCRATCH
    Ad = torch.zeros((m, k), dtype=torch.float64, device="cuda")
    Bd = torch.zeros((k, n), dtype=torch.float64, device="cuda")
    C = torch.full((m, n), 5.0, dtype=torch.float64, device="cuda")
    st = _noalloc(plan, Ad, Bd, C, torch.cuda.current_stream())
    assert st == fmm.FMM_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert bool((C == 5.0).all())   # nothing was enqueued


def test_noalloc_needs_the_plan_on_the_device():
    import torch
    plan = fmm.Plan("strassen_222_7", levels=1)    # not prepared: its lists are host-only
    Ad = torch.ones((64, 64), dtype=torch.float64, device="cuda")
    Bd = torch.ones((64, 64), dtype=torch.float64, device="cuda")
    C = torch.full((64, 64), 5.0, dtype=torch.float64, device="cuda")
    assert _noalloc(plan, Ad, Bd, C, torch.cuda.current_stream()) == fmm.FMM_ERR_ARG
    torch.cuda.synchronize()
    assert bool((C == 5.0).all())
    plan.prepare()
    assert _noalloc(plan, Ad, Bd, C, torch.cuda.current_stream()) == fmm.FMM_OK
    torch.cuda.synchronize()
    assert bool((C == 64.0).all())
