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
    # with the emulated variant available it leads; the native FP64 plans stay
    # in the ranking (an FP64-only tuner reaches them)
    assert cands[0].precision == "ozaki_bf16"
    assert any(c.precision == "fp64" and c.levels >= 1 for c in cands)
    assert any(c.precision == "fp64" for c in t.candidates(40, 3000, 40))
    best = autotune.Autotuner(tol=1e-11, precisions=("fp64",), measure=False).choose(8192, 8192, 8192)
    assert best.precision == "fp64" and best.levels >= 1


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


def test_permuted_base_cases_are_exact():
    # every ordering of every shipped base case (Section 2.3's permutations)
    # passes the oracle's exact Brent check and the library's plan check
    import numpy as np
    from fractions import Fraction
    import paper_1409_2908_gb300 as fmm
    from oracle import tensor
    for name in autotune.algorithms():
        M0, K0, N0 = autotune.algorithms()[name][:3]
        shapes = set()
        for perm in autotune.PERMS:
            M, K, N, U, V, W = autotune.permuted_factors(name, perm)
            shapes.add((M, K, N))
            F = [[[Fraction(float(x)) for x in row] for row in X] for X in (U, V, W)]
            assert tensor.brent_violations(M, K, N, *F) == [], (name, perm)
            fmm.Plan(levels=1, factors=(M, K, N, U, V, W))
        assert shapes == {(M0, K0, N0), (K0, N0, M0), (N0, M0, K0), (N0, K0, M0), (K0, M0, N0), (M0, N0, K0)}


def test_permutations_reach_shape_matched_cases():
    # tall-skinny m >> k = n: orderings of <4,2,3> with the 4 on m are candidates
    t = autotune.Autotuner(tol=1e-11, precisions=("fp64",), measure=False)
    cands = t.candidates(16384, 2048, 2048)
    dims = {autotune.cases()[(c.algorithm, c.perm)][:3] for c in cands if c.levels >= 1}
    assert (4, 3, 2) in dims and (4, 2, 3) in dims
    assert any(c.perm for c in cands)


def test_fp64_tile_follows_leaf_size():
    t = autotune.Autotuner(tol=1e-11, precisions=("fp64",), measure=False, permutations=False)
    big = [c for c in t.candidates(8192, 8192, 8192) if c.levels == 1 and c.algorithm == "strassen_222_7"][0]
    assert big.tile == "128x128"
    small = [c for c in t.candidates(192, 4096, 192) if c.levels == 1 and c.algorithm == "strassen_222_7"][0]
    assert small.tile in ("96x96", "64x64", "32x32")


@pytest.mark.parametrize("shape", [(8192, 8192, 8192), (16384, 2048, 2048), (300, 5000, 700), (256, 256, 8000)])
@pytest.mark.parametrize("precs", [("fp64", "ozaki_bf16"), ("fp64",), ("tf32", "fp32", "ozaki_bf16")])
def test_branch_and_bound_finds_the_model_optimum(shape, precs):
    t = autotune.Autotuner(tol=1e-11 if "tf32" not in precs else 1e-3, precisions=precs, measure=False)
    full = t.candidates(*shape)
    for count in (1, 3):
        got = t.best_candidates(*shape, count)
        assert [c.model_ms for c in got] == [c.model_ms for c in full[:count]]


def test_fast_search_matches_the_full_ranking_on_the_serving_mix():
    # the pruned search (vectorised bounds, per-depth exclusion) returns the
    # model optimum of the full ranking on shapes of the serving mix
    from paper_1409_2908_gb300 import serve
    for precs in (("fp64", "ozaki_bf16"), ("fp64",)):
        t = autotune.Autotuner(tol=1e-11, precisions=precs, measure=False)
        for m, k, n in serve.request_shapes(150, seed=77):
            m, k, n = int(m), int(k), int(n)
            full = t.candidates(m, k, n)
            got = t.best_candidates(m, k, n, 2)
            assert [c.model_ms for c in got] == [c.model_ms for c in full[:2]], (m, k, n)


def test_vectorised_bounds_equal_the_scalar_bounds():
    t = autotune.Autotuner(tol=1e-11, measure=False)
    m, k, n = 6000, 5000, 7000
    nmod = autotune.moduli_for(t.tol, k)
    rate = {"fp64": t.fp64_tflops, "ozaki_bf16": t.tc_tflops / nmod}
    work = {"fp64": 1.0, "ozaki_bf16": 1.0}
    _, info = t._levels()
    vec = {(info[i][0], info[i][1], info[i][3], p): lb
           for lb, i, p in t._recursive_bounds(m, k, n, ("fp64", "ozaki_bf16"), rate, work, nmod)}
    scal = {(e[1], e[2], e[4], e[5]): t._bound(e) for e in t._space(m, k, n) if e[4] > 0}
    assert vec.keys() == scal.keys()
    for key in vec:
        assert abs(vec[key] - scal[key]) <= 1e-9 * scal[key]


def test_beta_rule_matches_the_oracle():
    # the tuner's closed form (one integer division) against the oracle's
    # definition of beta, for every moduli count and k across 1..2^40
    from oracle import ozaki
    ks = list(range(1, 3000)) + [2 ** e + d for e in range(11, 41) for d in (-1, 0, 1)] + [6912, 8191, 16384, 65536]
    for n in range(6, 17):
        assert autotune.MODULI[:n] == tuple(ozaki.moduli(n))
        for k in ks:
            assert autotune.beta_for(n, k) == ozaki.beta_bits(n, k), (n, k)
