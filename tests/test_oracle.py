"""Pins for the oracle: values it must reproduce that do not come from itself.

* brute force (row-permutation lister, oracle/brute.py) on orders 4..6,
  whole-square counts and per-prefix counts;
* known totals 48 / 960 / 92160 and the paper's printed hourglass count;
* invariants the mathematics fixes: independence of the fill order, of the
  symbols of row 0, transposition, the multipliers, sums over prefix splits.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import brute, orders

D = oracle.DIAGONAL
V = oracle.VSYM


def _full_count(n, flags, order=None, row0=None):
    vs = bool(flags & V)
    if order is None:
        order = orders.md_ad_rows(n, vsym=vs)
    if row0 is None:
        row0 = orders.identity(n, vsym=vs)
    return oracle.count(n, flags, order, row0)[0]


@pytest.mark.parametrize("n", [4, 5, 6])
def test_brute_force_dls_row0_fixed(n):
    sq = brute.squares(n, diagonal=True, row0=list(range(n)))
    assert _full_count(n, D) == len(sq)


@pytest.mark.parametrize("n", [4, 5])
def test_brute_force_free_row0(n):
    # no prefix at all: every square of the order
    for flags, diag in ((D, True), (0, False)):
        sq = brute.squares(n, diagonal=diag, row0=None)
        got = oracle.count(n, flags, orders.row_major(n), [])[0]
        assert got == len(sq)


@pytest.mark.parametrize("n", [4, 5])
def test_brute_force_latin_row0_fixed(n):
    sq = brute.squares(n, diagonal=False, row0=list(range(n)))
    assert _full_count(n, 0) == len(sq)


@pytest.mark.parametrize("n", [4, 6])
def test_brute_force_vsym(n):
    sq = brute.squares(n, diagonal=True, vsym=True, row0=list(range(n)))
    assert _full_count(n, D | V) == len(sq)
    # vertically symmetric squares are diagonal squares too
    assert len(sq) <= _full_count(n, D)


@pytest.mark.parametrize("n", [4, 6])
def test_vsym_multiplier_by_brute_force(n):
    free = brute.squares(n, diagonal=True, vsym=True, row0=None)
    assert len(free) == _full_count(n, D | V) * oracle.multiplier(n, D | V)


@pytest.mark.parametrize("n", [4, 5])
def test_dls_multiplier_by_brute_force(n):
    free = brute.squares(n, diagonal=True, row0=None)
    assert len(free) == _full_count(n, D) * oracle.multiplier(n, D)


@pytest.mark.parametrize("n", [3, 5, 7])
def test_vsym_odd_order_is_empty(n):
    assert _full_count(n, D | V) == 0
    assert len(brute.squares(min(n, 5), True, True, row0=None)) == 0


def test_known_totals(golden):
    for n in (4, 5, 6):
        assert _full_count(n, D) * oracle.multiplier(n, D) == golden["dls_total_%d" % n]


def test_hourglass_count_order8(golden):
    # Section 4.2: hourglass designs of order 8 (row 0 identity, both
    # diagonals, last row); the hourglass order lists exactly those cells first
    n = 8
    ho = orders.hourglass(n)
    cells = set()
    for i in range(n):
        cells |= {(0, i), (i, i), (i, n - 1 - i), (n - 1, i)}
    part = ho[:len(cells)]
    assert set(part) == cells
    assert oracle.count(n, D, part, orders.identity(n))[0] == golden["hourglass8"]


@pytest.mark.parametrize("n", [5, 6])
def test_fill_order_invariance(n):
    ref = _full_count(n, D)
    rng = np.random.default_rng(n)
    for order in (orders.row_major(n), orders.hourglass(n)):
        assert _full_count(n, D, order) == ref
    rest = [c for c in orders.row_major(n) if c[0] != 0]
    for _ in range(3):
        perm = rng.permutation(len(rest))
        order = orders.row0(n) + [rest[k] for k in perm]
        assert _full_count(n, D, order) == ref


def test_relabel_invariance_of_row0():
    # any permutation as row 0 gives the same count (the symbols can be renamed)
    n = 5
    ref = _full_count(n, D)
    for p in itertools.permutations(range(n)):
        assert _full_count(n, D, row0=list(p)) == ref


def test_transpose_invariance():
    # transposing keeps both diagonals, so fixing column 0 counts the same
    n = 6
    order = [(i, 0) for i in range(n)] + [c for c in orders.row_major(n) if c[1] != 0]
    assert oracle.count(n, D, order, list(range(n)))[0] == _full_count(n, D)


@pytest.mark.parametrize("n,flags", [(5, D), (6, D), (6, D | V), (5, 0)])
def test_per_prefix_counts_against_brute_force(n, flags):
    vs = bool(flags & V)
    sq = brute.squares(n, diagonal=bool(flags & D), vsym=vs, row0=list(range(n)))
    order = orders.md_ad_rows(n, vsym=vs)
    base = np.array([orders.identity(n, vs)], np.uint8)
    r0 = len(base[0])
    for depth in range(r0, len(order) + 1, 3):
        pre, _ = oracle.extend(n, flags, order, base, depth)
        # every full square is counted exactly once across the prefixes
        cnt, _ = oracle.count_many(n, flags, order, pre)
        assert int(cnt.sum()) == len(sq)
        for k in range(0, len(pre), max(1, len(pre) // 25)):
            cells = order[:depth]
            vals = [int(x) for x in pre[k]]
            if vs:
                cells = cells + [(i, n - 1 - j) for (i, j) in cells]
                vals = vals + [n - 1 - x for x in vals]
            assert cnt[k] == brute.count_matching(sq, cells, vals)


def test_invalid_prefix_counts_zero():
    n = 6
    order = orders.md_ad_rows(n)
    bad = orders.identity(n) + [0]            # (1,1) == (0,0) on the diagonal
    assert oracle.count(n, D, order, bad)[0] == 0
    bad = orders.identity(n) + [7]            # value out of range
    assert oracle.count(n, D, order, bad)[0] == 0


def test_split_sums_equal_unsplit():
    n = 7
    order = orders.md_ad_rows(n)
    base = np.array([orders.identity(n)], np.uint8)
    total = _full_count(n, D)
    for depth in (n + 3, n + 10):
        pre, par = oracle.extend(n, D, order, base, depth)
        assert (par == 0).all()
        cnt, _ = oracle.count_many(n, D, order, pre, threads=4)
        assert int(cnt.sum()) == total


def test_extend_is_lexicographic_and_matches_partial_count():
    n = 6
    order = orders.md_ad_rows(n)
    base = np.array([orders.identity(n)], np.uint8)
    for depth in (n + 2, n + 5, n + 9):
        pre, _ = oracle.extend(n, D, order, base, depth)
        assert len(pre) == oracle.count(n, D, order[:depth], orders.identity(n))[0]
        keys = [tuple(r) for r in pre]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_sample_prefix_is_valid_and_deterministic():
    rng = np.random.Generator(np.random.PCG64(5))
    for n, flags in ((6, D), (8, D), (8, D | V), (9, D)):
        vs = bool(flags & V)
        order = orders.md_ad_rows(n, vsym=vs, first_rows=n - 3)
        depth = (n - 3) * len(orders.identity(n, vs))
        draws = rng.integers(0, 2**32, size=4096, dtype=np.uint32)
        p1, u1 = oracle.sample_prefix(n, flags, order, depth, draws)
        p2, u2 = oracle.sample_prefix(n, flags, order, depth, draws)
        assert p1 is not None and u1 == u2 and (p1 == p2).all()
        # valid: the partial count of exactly these cells is 1
        assert oracle.count(n, flags, order[:depth], p1)[0] == 1


def test_nodes_count_accepted_placements():
    # the last position of the order accepts exactly one value per square,
    # so nodes >= squares, and a full prefix has no nodes and one square
    n = 5
    order = orders.md_ad_rows(n)
    c, nd = oracle.count(n, D, order, orders.identity(n))
    assert nd >= c
    sq = brute.squares(n, True, row0=list(range(n)))
    full = [int(sq[0][i][j]) for (i, j) in order]
    assert oracle.count(n, D, order, full) == (1, 0)


# ------------------------------------------------------------ trim_tail --
# A final run of one line's off-diagonal cells can be dropped from a full
# order without changing any count (each of them is the last open cell of
# its column, and the values these force are those the line lacks).  Pinned
# on known totals and on brute force; and the two conditions of the rule
# (one line, no diagonal) each matter.

LATIN_ROW0_FIXED = {4: 24, 5: 1344, 6: 1128960}   # Latin squares 576, 161280,
# 812851200 of orders 4-6 (OEIS A002860), divided by the n! first rows


def _orders_to_trim(n, seed, shuffled=8):
    rng = np.random.default_rng(seed)
    out = [orders.md_ad_rows(n), orders.row_major(n), orders.hourglass(n),
           orders.heuristic_complete(n, orders.row0(n)),
           orders.heuristic_complete(n, orders.row0(n), squares=True)]
    rest = [(i, j) for i in range(1, n) for j in range(n)]
    for _ in range(shuffled):
        out.append(orders.row0(n) + [rest[k] for k in rng.permutation(len(rest))])
    return out


@pytest.mark.parametrize("n", [4, 5, 6])
def test_trimmed_orders_keep_the_known_totals(golden, n):
    dropped = 0
    # (ordinary squares of order 6 take the oracle minutes: orders 4 and 5)
    for flags in ((D, 0) if n < 6 else (D,)):
        for order in _orders_to_trim(n, n, 8 if n < 6 else 3):
            for window in (0, 3, 6, 100):
                t = orders.trim_tail(n, order, n, window, diagonal=bool(flags))
                assert t[:n] == order[:n] and set(t) <= set(order) and len(t) > n
                dropped += len(order) - len(t)
                got = oracle.count(n, flags, t, orders.identity(n))[0]
                if flags:
                    assert got * oracle.multiplier(n, D) == golden["dls_total_%d" % n]
                else:
                    assert got == LATIN_ROW0_FIXED[n]
    assert dropped > 0


@pytest.mark.parametrize("n", [4, 5])
def test_trimmed_orders_per_prefix_by_brute_force(n):
    # brute force lists whole squares; each prefix of the trimmed order
    # must have as many completions as squares agree with it on those cells
    sq = np.array(brute.squares(n, diagonal=True, row0=list(range(n))))
    for order in _orders_to_trim(n, 10 + n):
        t = orders.trim_tail(n, order, n, 100)
        depth = n + 3
        pre, _ = oracle.extend(n, D, t, np.array([orders.identity(n)], np.uint8), depth)
        c, _ = oracle.count_many(n, D, t, pre)
        cells = t[:depth]
        for p, k in zip(pre, c):
            match = np.all([sq[:, i, j] == p[q] for q, (i, j) in enumerate(cells)], axis=0)
            assert int(match.sum()) == int(k)


def test_trim_needs_one_line_and_no_diagonal():
    n = 6
    ref = _full_count(n, D)
    # row-major ends with row 5, whose end cell (5, 5) lies on the main
    # diagonal: the rule drops nothing, and dropping the row anyway (its
    # diagonal cells unchecked) changes the count
    rm = orders.row_major(n)
    assert orders.trim_tail(n, rm, n, 0) == rm
    assert oracle.count(n, D, rm[:-6], orders.identity(n))[0] != ref
    # without the diagonal rule the four inner cells of row 5 may go ...
    inner = [c for c in rm if c not in [(5, 1), (5, 2), (5, 3), (5, 4)]] + \
        [(5, 1), (5, 2), (5, 3), (5, 4)]
    t = orders.trim_tail(n, inner, n, 0)
    assert t == inner[:-4] and oracle.count(n, D, t, orders.identity(n))[0] == ref
    # ... but a final run on two lines may not: (5, 4) is forced by its
    # column and (4, 3) by its column only once (5, 3) is placed
    two = [c for c in rm if c not in [(4, 3), (5, 3), (5, 4)]] + [(5, 3), (4, 3), (5, 4)]
    assert oracle.count(n, D, two, orders.identity(n))[0] == ref
    assert oracle.count(n, D, two[:-2], orders.identity(n))[0] != ref


def test_trim_leaves_partial_orders():
    n = 6
    part = orders.md_ad_rows(n)[:30]
    assert orders.trim_tail(n, part, n) == part
    vs = orders.md_ad_rows(n, vsym=True)
    assert orders.trim_tail(n, vs[:14], 3, vsym=True) == vs[:14]
    odd = orders.row_major(5, vsym=True)
    assert orders.trim_tail(5, odd, 2, vsym=True) == odd


def _vsym_orders_to_trim(n, seed, shuffled):
    rng = np.random.default_rng(seed)
    w = n // 2
    out = [orders.md_ad_rows(n, vsym=True), orders.row_major(n, vsym=True),
           orders.heuristic_complete(n, orders.row0(n, True), vsym=True),
           orders.heuristic_complete(n, orders.row0(n, True), vsym=True, squares=True)]
    rest = [(i, j) for i in range(1, n) for j in range(w)]
    for _ in range(shuffled):
        out.append(orders.row0(n, True) + [rest[k] for k in rng.permutation(len(rest))])
    return out


@pytest.mark.parametrize("n", [4, 6])
def test_trimmed_symmetric_orders_by_brute_force(n):
    # vertically symmetric squares with row 0 the identity, with and without
    # the diagonal rule, listed by brute force; only row runs may drop
    dropped = 0
    for flags in (D | V, V):
        sq = brute.squares(n, diagonal=bool(flags & D), vsym=True, row0=list(range(n)))
        for order in _vsym_orders_to_trim(n, n, 6):
            for window in (0, 3, 100):
                t = orders.trim_tail(n, order, n // 2, window, diagonal=bool(flags & D),
                                     vsym=True)
                assert t[:n // 2] == order[:n // 2] and len(t) > n // 2
                dropped += len(order) - len(t)
                assert oracle.count(n, flags, t, orders.identity(n, True))[0] == len(sq)
    assert dropped > 0


def test_trimmed_symmetric_order8_and_a_column_run():
    n, flags = 8, D | V
    ref = _full_count(n, flags)
    for order in _vsym_orders_to_trim(n, 8, 0)[::2] + _vsym_orders_to_trim(n, 8, 0)[3:]:
        t = orders.trim_tail(n, order, 4, 6, vsym=True)
        assert oracle.count(n, flags, t, orders.identity(n, True))[0] == ref
    # a final run down a left column is not forced by its rows: dropping it
    # changes the count; the rule drops only its last cell (a run of one
    # cell is also a row's run)
    n, flags = 6, V
    ref = _full_count(n, flags)
    col = [c for c in orders.row_major(n, vsym=True) if c not in [(3, 1), (4, 1)]]
    col += [(3, 1), (4, 1)]
    assert orders.trim_tail(n, col, 3, 0, diagonal=False, vsym=True) == col[:-1]
    assert oracle.count(n, flags, col[:-1], orders.identity(n, True))[0] == ref
    assert oracle.count(n, flags, col[:-2], orders.identity(n, True))[0] != ref
