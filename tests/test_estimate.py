"""CPU tests of dls_estimate_nodes, the random-descent size estimate the
serving path uses to decide how finely a job is split (D. E. Knuth,
"Estimating the efficiency of backtrack programs", 1975; not a method of
the paper).

The estimate is unbiased for the number of values the search places after
the prefix, which is the oracle's exact `nodes`. So over many seeds the mean
estimate must lie within a few standard errors of that count. Where only the
last cell is left, the descent has no choice to make, and the estimate must
equal the count exactly."""
import numpy as np
import pytest

import oracle
from oracle import brute

D, V = 1, 2


def _seed_estimates(dls, n, flags, order, prefix, seeds, probes):
    return np.array([dls.estimate_nodes(n, flags, order, prefix, seed=s, probes=probes)
                     for s in range(seeds)])


@pytest.mark.parametrize("n,flags,depth", [(6, D, 6), (7, D, 12), (8, D | V, 8)])
def test_mean_estimate_matches_exact_nodes(dls, n, flags, depth):
    order = dls.fill_order(n, flags, dls.ORDER_HEURISTIC)
    row0 = np.arange(n // 2 if flags & V else n, dtype=np.uint8)[None]
    pref, _ = dls.extend_prefixes(n, flags, order, row0, depth)
    assert len(pref) > 0
    # a few prefixes spread over the split, each against its own exact count
    for prefix in pref[np.unique(np.linspace(0, len(pref) - 1, 3).astype(int))]:
        _, exact = oracle.count(n, flags, order, prefix)
        est = _seed_estimates(dls, n, flags, order, prefix, seeds=200, probes=1024)
        mean = est.mean()
        se = est.std(ddof=1) / np.sqrt(len(est))
        if exact == 0:
            assert np.all(est == 0.0)
            continue
        # the test must be able to see a bias of a few percent
        assert se < 0.03 * exact, (se, exact)
        assert abs(mean - exact) <= 5.0 * se, (mean, exact, se)


def test_one_cell_left_is_exact(dls):
    n = 5
    order = dls.fill_order(n, D, dls.ORDER_HEURISTIC)
    row0 = np.arange(n, dtype=np.uint8)[None]
    pref, _ = dls.extend_prefixes(n, D, order, row0, len(order) - 1)
    assert len(pref) > 0
    _, nodes = oracle.count_many(n, D, order, pref)
    got = [dls.estimate_nodes(n, D, order, p, seed=7, probes=3) for p in pref]
    assert got == [float(x) for x in nodes]
    assert sum(got) > 0


def test_deterministic_and_degenerate_cases(dls):
    n = 7
    order = dls.fill_order(n, D, dls.ORDER_HEURISTIC)
    prefix = np.arange(n, dtype=np.uint8)
    a = dls.estimate_nodes(n, D, order, prefix, seed=3, probes=32)
    assert a == dls.estimate_nodes(n, D, order, prefix, seed=3, probes=32)
    assert a != dls.estimate_nodes(n, D, order, prefix, seed=4, probes=32)
    assert a > 0
    # an invalid prefix (a repeated value in row 0) has no search below it
    bad = prefix.copy()
    bad[1] = bad[0]
    assert dls.estimate_nodes(n, D, order, bad, seed=3, probes=32) == 0.0
    # a full square: nothing is placed after it
    full = brute.squares(5, diagonal=True, row0=list(range(5)))[0]
    o5 = dls.fill_order(5, D, dls.ORDER_ROW_MAJOR)
    vals = np.array([full[i][j] for i, j in o5], np.uint8)
    assert dls.estimate_nodes(5, D, o5, vals, probes=4) == 0.0
    # odd order with vertical symmetry: no squares, no search
    o = dls.fill_order(7, D | V, dls.ORDER_HEURISTIC)
    assert dls.estimate_nodes(7, D | V, o, np.zeros(0, np.uint8), probes=4) == 0.0


def test_argument_errors(dls):
    from paper_1709_02599_gb300 import DlsError
    order = dls.fill_order(6, D, dls.ORDER_HEURISTIC)
    with pytest.raises(DlsError):
        dls.estimate_nodes(6, D, order, np.arange(6, dtype=np.uint8), probes=0)
    with pytest.raises(DlsError):
        dls.estimate_nodes(6, D, order, np.zeros(len(order) + 1, np.uint8))
    with pytest.raises(DlsError):
        dls.estimate_nodes(6, 8, order, np.arange(6, dtype=np.uint8))
    with pytest.raises(DlsError):
        dls.estimate_nodes(33, D, order, np.arange(6, dtype=np.uint8))
