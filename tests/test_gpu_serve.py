"""The serving loop: continuous batching of mixed-shape requests, grouped by
plan into captured CUDA graphs on several streams.  Each result must be the
same alone and in the mix (the plans are deterministic, so bit for bit), and
agree with the CPU oracle."""
import numpy as np
import pytest

import oracle
from oracle import norms
import paper_1409_2908_gb300 as fmm
from paper_1409_2908_gb300 import autotune, serve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precisions,group_shapes", [(("fp64",), False), (("ozaki_bf16",), False),
                                                    (("ozaki_bf16",), True)])
@pytest.mark.parametrize("use_graphs", [True, False])
def test_results_same_alone_and_in_the_mix(precisions, use_graphs, group_shapes):
    import torch
    tuner = autotune.Autotuner(tol=1e-11, precisions=precisions, measure=False)
    # grouping across shapes takes the small products (whose residue GEMM
    # underfills the GPU) that wait together: let them arrive at once
    reqs = serve.poisson_requests(18, rate_per_s=1e6 if group_shapes else 2000.0, lo=128,
                                  hi=400 if group_shapes else 700, seed=7)
    # repeat a few shapes so that graphs are replayed
    for i in range(6):
        r = reqs[i]
        reqs.append(serve.Request(100 + i, r.A.clone(), r.B.clone(), r.arrival + 0.002))
    srv = serve.Server(tuner, memory_budget_bytes=1 << 30, slots=3, use_graphs=use_graphs,
                       group_shapes=group_shapes)
    stats = srv.run(reqs)
    if group_shapes:
        # requests of different shapes went out together in grouped calls
        assert stats["grouped_calls"] >= 1 and stats["mean_group_size"] > 1
    torch.cuda.synchronize()
    assert stats["requests"] == len(reqs)
    assert stats["p50_ms"] is not None and stats["p99_ms"] >= stats["p50_ms"]
    if use_graphs:
        # the six repeated shapes are replayed from captured graphs
        assert stats["graphs_captured"] >= 1 and stats["graph_replays"] >= 6
    for r in reqs:
        m, k, n = r.shape
        plan = tuner.plan(m, k, n)
        alone = fmm.gemm(plan, r.A, r.B)
        torch.cuda.synchronize()
        assert torch.equal(alone, r.C), r.rid
    for r in reqs[:4]:
        A, B = r.A.cpu().numpy(), r.B.cpu().numpy()
        assert norms.rel_frobenius(r.C.cpu().numpy(), oracle.gemm(A, B)) <= 1e-11


def test_admission_respects_memory_budget():
    import torch
    tuner = autotune.Autotuner(tol=1e-11, precisions=("fp64",), measure=False)
    reqs = serve.poisson_requests(8, rate_per_s=1e6, lo=512, hi=513, seed=3)
    # room for about one request at a time: all arrive at once, none is lost
    one = 8 * 513 * 513 + tuner.plan(512, 512, 512).workspace_size(513, 513, 513)
    srv = serve.Server(tuner, memory_budget_bytes=int(1.5 * one), slots=4, use_graphs=False)
    stats = srv.run(reqs)
    assert stats["requests"] == 8
    assert stats["max_inflight_groups"] >= 1
    assert srv.used == 0
