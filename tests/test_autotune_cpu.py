"""CPU checks of the autotuner's candidate model (no timing)."""
import pytest

from paper_1409_2908_gb300 import autotune


def test_candidates_cover_algorithms_levels_precisions():
    t = autotune.Autotuner(tol=1e-11, precisions=("fp64",), measure=False)
    cands = t.candidates(8192, 8192, 8192)
    names = {(c.algorithm, c.levels, c.precision) for c in cands}
    assert ("strassen_222_7", 0, "fp64") in names
    assert ("strassen_222_7", 3, "fp64") in names
    assert cands == sorted(cands, key=lambda c: c.model_ms)
    t = autotune.Autotuner(tol=1e-11, measure=False)
    cands = t.candidates(8192, 8192, 8192)
    assert any(c.precision == "ozaki_bf16" and c.levels >= 1 for c in cands)
    assert any(c.precision == "ozaki_bf16" and c.levels == 0 for c in cands)
    # with the emulated variant available, FP64 plans only compete on tiny products
    assert all(c.precision == "ozaki_bf16" for c in cands)
    assert any(c.precision == "fp64" for c in t.candidates(40, 3000, 40))


def test_recursion_stops_when_leaves_get_small():
    # the paper's cutoff: no step whose sub-products fall below the flat part
    t = autotune.Autotuner(tol=1e-11, precisions=("fp64",), measure=False)
    for c in t.candidates(256, 256, 256):
        M = autotune.algorithms()[c.algorithm][0] if c.levels else 1
        assert 256 // M ** c.levels >= 64


def test_shape_matching_prefers_rank_k_algorithms():
    # an outer-product shape (k small) favours a base case with small K
    t = autotune.Autotuner(tol=1e-11, precisions=("fp64",), measure=False)
    best = t.choose(16384, 2048, 16384)
    assert best.levels >= 1


def test_moduli_for_tolerance():
    assert autotune.moduli_for(1e-11, 8192) <= 15
    assert autotune.moduli_for(1e-6, 8192) < autotune.moduli_for(1e-14, 8192)
    assert autotune.moduli_for(1e-30, 8192) is None


def test_strict_tolerance_drops_deep_fp64_plans():
    t = autotune.Autotuner(tol=1e-14, precisions=("fp64",), measure=False)
    assert all(c.levels <= 1 for c in t.candidates(4096, 4096, 4096))


def test_tf32_and_fp32_admitted_by_tolerance():
    precs = ("tf32", "fp32", "ozaki_bf16")
    # a loose target admits TF32 (classical; one level doubles its error) and FP32 at any depth
    loose = autotune.Autotuner(tol=1e-3, precisions=precs, measure=False).candidates(8192, 8192, 8192)
    kinds = {(c.precision, c.levels) for c in loose}
    assert ("tf32", 0) in kinds and ("tf32", 1) not in kinds
    assert ("fp32", 0) in kinds and ("fp32", 2) in kinds
    # TF32 does the least work per product: it leads the loose target
    assert loose[0].precision == "tf32"
    # an FP32-level target keeps FP32, drops TF32
    mid = autotune.Autotuner(tol=2e-5, precisions=precs, measure=False).candidates(8192, 8192, 8192)
    assert {c.precision for c in mid} == {"fp32", "ozaki_bf16"}
    # an FP64-level target leaves only the emulated FP64 plans
    strict = autotune.Autotuner(tol=1e-11, precisions=precs, measure=False).candidates(8192, 8192, 8192)
    assert {c.precision for c in strict} == {"ozaki_bf16"}


def test_choice_plans_carry_moduli_only_for_emulated_fp64():
    c = autotune.Choice("strassen_222_7", 1, 0, "tf32")
    assert c.plan().precision == "tf32"
    c = autotune.Choice("strassen_222_7", 0, 0, "fp32")
    assert c.plan().precision == "fp32"
