"""The three addition schemes of Section 3.2 for the level-by-level passes:
write-once (each child from all its terms), streaming (each parent element
read once, written into every child) and pairwise (one pass per term).  They
do the same additions in the same order, so the product is the same to the
bit on random inputs, and bit-exact against the oracle on integer inputs."""
import numpy as np
import pytest

import oracle
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

SCHEMES = {"write_once": fmm.FLAG_LEVELWISE, "streaming": fmm.FLAG_LEVELWISE | fmm.FLAG_STREAMING,
           "pairwise": fmm.FLAG_LEVELWISE | fmm.FLAG_PAIRWISE}


def run(plan, A, B):
    import torch
    C = fmm.gemm(plan, to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    return C.cpu().numpy()


@pytest.mark.parametrize("name,levels", [("strassen_222_7", 1), ("strassen_222_7", 2), ("fmm_424_26", 2),
                                         ("fmm_423_20", 1), ("fmm_333_23", 2), ("winograd_222_7", 3)])
def test_schemes_give_the_same_bits(name, levels):
    M, K, N = {"strassen_222_7": (2, 2, 2), "fmm_424_26": (4, 2, 4), "fmm_423_20": (4, 2, 3),
               "fmm_333_23": (3, 3, 3), "winograd_222_7": (2, 2, 2)}[name]
    shape = (M ** levels * 37 + 1, K ** levels * 41 + 2, N ** levels * 29 + 3)
    A, B = synth.operands(*shape, 95)
    out = {sc: run(fmm.Plan(name, levels=levels, flags=f), A, B) for sc, f in SCHEMES.items()}
    assert np.array_equal(out["streaming"], out["write_once"])
    assert np.array_equal(out["pairwise"], out["write_once"])
    Ai, Bi = synth.operands(*shape, 96, kind="integer")
    ref = oracle.gemm(Ai, Bi)
    for f in SCHEMES.values():
        assert np.array_equal(run(fmm.Plan(name, levels=levels, flags=f), Ai, Bi), ref)


def test_streaming_with_tf32_leaves():
    A, B = synth.operands(260, 300, 280, 97)
    a = run(fmm.Plan("strassen_222_7", levels=2, precision="tf32", flags=SCHEMES["streaming"]), A, B)
    b = run(fmm.Plan("strassen_222_7", levels=2, precision="tf32", flags=SCHEMES["write_once"]), A, B)
    assert np.array_equal(a, b)


def test_streaming_and_pairwise_exclusive():
    with pytest.raises(fmm.FmmError):
        fmm.Plan("strassen_222_7", levels=1, flags=fmm.FLAG_STREAMING | fmm.FLAG_PAIRWISE)
