"""Emulated FP64 with S' formed inside the tensor-core GEMM
(FMM_FLAG_TC_FUSED_S): converter warps combine the int8 residues of A' into
the fp16 operand in tensor memory.  The same integers as the ordinary path,
so the result must be bit-identical to it and to the oracle's emulation, on
ragged shapes (k blocks that end inside a 64-wide k-block, partial row and
column tiles), for base cases with one- and two-term S', and for base cases
the fused kernel does not take (they fall back, still exact)."""
import numpy as np
import pytest

import oracle
from oracle import ozaki
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

FUSED = fmm.FLAGS_DEFAULT | fmm.FLAG_TC_FUSED_S


def run(plan, A, B):
    import torch
    C = fmm.gemm(plan, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    fmm.check_device_error()
    return C.cpu().numpy()


@pytest.mark.parametrize("name,levels,shape,nmod", [
    ("strassen_222_7", 0, (300, 336, 250), 14),      # k = 336: the last k-block holds 16 of 64
    ("strassen_222_7", 0, (129, 64, 385), 12),
    ("strassen_222_7", 1, (514, 416, 390), 14),      # k_L = 208
    ("strassen_222_7", 1, (1024, 1024, 1024), 13),
    ("fmm_323_15", 1, (390, 192, 579), 14),
    ("winograd_222_7", 1, (260, 256, 260), 12),      # three-term S': falls back
    ("fmm_424_26", 1, (512, 256, 512), 14),
])
def test_fused_s_matches_ordinary_path_and_oracle(name, levels, shape, nmod):
    A, B = synth.operands(*shape, 101)
    fused = run(fmm.Plan(name, levels=levels, precision="ozaki_bf16", moduli=nmod, flags=FUSED), A, B)
    plain = run(fmm.Plan(name, levels=levels, precision="ozaki_bf16", moduli=nmod), A, B)
    assert np.array_equal(fused, plain)
    assert np.array_equal(fused, ozaki.emulated_gemm(A, B, nmod))


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 0), ("strassen_222_7", 1), ("fmm_323_15", 1)])
def test_fused_s_integer_exact(name, levels):
    A, B = synth.operands(385, 448, 321, 102, kind="integer")
    assert np.array_equal(run(fmm.Plan(name, levels=levels, precision="ozaki_bf16", flags=FUSED), A, B),
                          oracle.gemm(A, B))


def test_fused_s_full_size_sampled():
    # the benchmark's 8192^3 workload with 14 moduli, sampled against the
    # oracle's per-entry emulation
    import torch
    m = k = n = 8192
    A, B = synth.operands(m, k, n, 1410)
    p = fmm.Plan("strassen_222_7", levels=1, precision="ozaki_bf16", moduli=14, flags=FUSED)
    C = fmm.gemm(p, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    fmm.check_device_error()
    rows, cols = synth.sample_indices(m, n, 256, 103)
    got = C[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    assert np.array_equal(got, ozaki.emulated_entries(A, B, rows, cols, 14))


@pytest.mark.parametrize("k", [32768, 32832])
def test_fused_s_k_boundary(k):
    # k_L up to 32768 takes the fused kernel (its drain sums stay below the
    # final reduction's shift); beyond, the plan falls back to the ordinary
    # path: the same integers either way
    A, B = synth.operands(48, k, 40, 104)
    fused = run(fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16", moduli=14, flags=FUSED), A, B)
    assert np.array_equal(fused, ozaki.emulated_gemm(A, B, 14))
