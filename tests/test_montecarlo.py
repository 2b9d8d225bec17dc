"""The Monte Carlo estimate of Section 5.3: rank selection of partial squares
against the oracle's enumeration, the estimate made exact by an exhaustive
sample, and a seeded sample against a known total."""
import os

import numpy as np
import pytest

import dls_inputs
import oracle
from oracle import orders

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
D, V = 1, 2
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.mark.parametrize("n,flags,k", [(6, D, 14), (7, D, 12), (8, D | V, 10), (6, 0, 13)])
def test_rank_selection_matches_enumeration(dls, n, flags, k):
    from paper_1709_02599_gb300 import montecarlo
    vs = bool(flags & V)
    o_order = orders.row_major(n, vsym=vs)[:k]
    first = np.array([orders.identity(n, vs)], np.uint8)
    every, _ = oracle.extend(n, flags, o_order, first, k)   # lexicographic
    total = len(every)
    r = np.concatenate([[0, 1, total // 2, total - 1], dls_inputs.ranks(total, 60, seed=n + k)])
    order_k = dls.fill_order(n, flags, dls.ORDER_ROW_MAJOR)[:k]
    got, n_k = montecarlo.select_by_rank(n, flags, order_k, r)
    assert n_k == total
    assert (got == every[r]).all()
    with pytest.raises(ValueError):
        montecarlo.select_by_rank(n, flags, order_k, [total])


def test_exhaustive_sample_gives_the_exact_total(dls, golden):
    # every k-cell partial square once: N^k x mean = the number of squares
    from paper_1709_02599_gb300 import montecarlo
    n, k = 6, 14
    order_k = dls.fill_order(n, D, dls.ORDER_ROW_MAJOR)[:k]
    _, n_k = montecarlo.select_by_rank(n, D, order_k, [0])
    res = montecarlo.estimate(n, D, k, np.arange(n_k))
    assert res["n_k"] == n_k
    assert int(res["completions"].sum()) * 720 == golden["dls_total_6"]
    assert round(res["estimate"]) == golden["dls_total_6"] // 720
    # each sampled completion count against the oracle
    full = [tuple(map(int, c)) for c in dls.order_complete(n, D, order_k, k, dls.ORDER_HEURISTIC)]
    o_every, _ = oracle.extend(n, D, orders.row_major(n)[:k],
                               np.array([orders.identity(n)], np.uint8), k)
    ref, _ = oracle.count_many(n, D, full, o_every)
    assert (res["completions"] == ref).all()


@pytest.mark.slow
def test_seeded_sample_estimates_order8_total(dls, golden):
    # Section 5.3's estimator on order 8, where Section 5.1 gives the exact
    # count (7 447 587 840 squares with row 0 fixed): 400 uniform ranks of the
    # 16-cell row-major partial squares
    from paper_1709_02599_gb300 import montecarlo
    n, k, m = 8, 16, 400
    order_k = dls.fill_order(n, D, dls.ORDER_ROW_MAJOR)[:k]
    _, n_k = montecarlo.select_by_rank(n, D, order_k, [0])
    res = montecarlo.estimate(n, D, k, dls_inputs.ranks(n_k, m, seed=8))
    exact = golden["dls8_row0_fixed"]
    assert res["stderr"] > 0
    assert abs(res["estimate"] - exact) < 4.5 * res["stderr"]
    # a few completion counts against the oracle
    full = [tuple(map(int, c)) for c in dls.order_complete(n, D, order_k, k, dls.ORDER_HEURISTIC)]
    ref, _ = oracle.count_many(n, D, full, res["samples"][:6], threads=THREADS)
    assert (res["completions"][:6] == ref).all()
