"""fmm_gemm_grouped: products of different shapes and plans issued together,
the emulated products' residue GEMMs sharing grouped tensor-core launches.
Each result must be bit-identical to fmm_gemm's for that product alone, and
match the oracle (bit-exact on integer inputs)."""
import numpy as np
import pytest

import oracle
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _case(count, seed, kind="uniform"):
    rng = np.random.default_rng(seed)
    plans, As, Bs = [], [], []
    for i in range(count):
        m, k, n = (int(x) for x in rng.integers(60, 700, 3))
        name, L = [("strassen_222_7", 0), ("strassen_222_7", 1), ("fmm_323_15", 1), ("winograd_222_7", 1)][i % 4]
        nmod = [12, 14, 13][i % 3]
        tile = "128x128" if i % 5 == 4 else "auto"
        plans.append(fmm.Plan(name, levels=L, precision="ozaki_bf16", moduli=nmod, tile=tile))
        A, B = synth.operands(m, k, n, seed * 100 + i, kind=kind)
        As.append(A)
        Bs.append(B)
    return plans, As, Bs


@pytest.mark.parametrize("count", [1, 5, 11])
def test_grouped_equals_alone(count):
    import torch
    plans, As, Bs = _case(count, 7 + count)
    Cs = fmm.gemm_grouped(plans, [to_dev(a) for a in As], [to_dev(b) for b in Bs])
    torch.cuda.synchronize()
    fmm.check_device_error()
    if count > 1:
        # grouped residue GEMMs: fewer launches than the products issued one by one
        grouped_launches = fmm.last_launch_count()
        alone_launches = 0
    for p, A, B, C in zip(plans, As, Bs, Cs):
        alone = fmm.gemm(p, to_dev(A), to_dev(B))
        torch.cuda.synchronize()
        if count > 1:
            alone_launches += fmm.last_launch_count()
        assert torch.equal(C, alone)
    if count > 1:
        assert grouped_launches < alone_launches


def test_grouped_integer_exact_and_mixed_precisions():
    import torch
    plans, As, Bs = _case(6, 21, kind="integer")
    # an FP64 plan and a TF32 plan in the mix run as fmm_gemm would
    plans[1] = fmm.Plan("strassen_222_7", levels=1)
    plans[2] = fmm.Plan("strassen_222_7", levels=1, precision="tf32")
    Cs = fmm.gemm_grouped(plans, [to_dev(a) for a in As], [to_dev(b) for b in Bs])
    torch.cuda.synchronize()
    for A, B, C in zip(As, Bs, Cs):
        assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))


def test_grouped_rejects_overlapping_outputs():
    import torch
    p = fmm.Plan("strassen_222_7", levels=0, precision="ozaki_bf16")
    A = torch.ones((64, 64), dtype=torch.float64, device="cuda")
    C = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(fmm.FmmError):
        fmm.gemm_grouped([p, p], [A, A], [A, A], Cs=[C, C])
