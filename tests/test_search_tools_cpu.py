"""The offline base-case search (Section 2.3): the C flip-graph walker finds
rank-7 schemes for <2,2,2> modulo 2, and Hensel lifting turns them into
exact integer schemes, checked here by the oracle's exact Brent check (the
tool's own check is not trusted for this)."""
import shutil

import numpy as np
import pytest

from oracle import tensor
from paper_1409_2908_gb300.algorithms import flip2


@pytest.mark.skipif(shutil.which("gcc") is None or shutil.which("timeout") is None,
                    reason="needs gcc and timeout")
def test_c_walker_finds_an_exact_strassen_rank_scheme():
    best = flip2.c_walk(2, 2, 2, 7, seeds=[1, 2], seconds=3, windows=50, gap=20)
    assert best is not None
    total, (U, V, W) = best
    U, V, W = (np.array([[float(x) for x in row] for row in F]) for F in (U, V, W))
    assert U.shape == (4, 7) and V.shape == (4, 7) and W.shape == (4, 7)
    assert not tensor.brent_violations(2, 2, 2, U, V, W)
    # the sparsest rank-7 schemes have Strassen's 36 nonzeros
    assert total == int((U != 0).sum() + (V != 0).sum() + (W != 0).sum()) >= 36


def test_lift_rejects_a_scheme_that_is_not_one_mod_2():
    # the classical scheme with one term dropped is no scheme at all: nothing to lift
    terms = flip2.classical(2, 2, 2)[:-1]
    assert flip2.lift(2, 2, 2, [list(t) for t in terms], bits=8) is None
