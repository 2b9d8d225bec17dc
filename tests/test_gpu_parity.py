"""GPU parity: the CUDA path against the oracle, bit-exact per prefix, on every
workload, both kernels and a range of launch shapes; the paper's printed
counts where the GPU reaches them; edge cases."""
import os

import numpy as np
import pytest

import oracle
from oracle import orders
import gpu_cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D, V = 1, 2
THREADS = max(1, min(16, os.cpu_count() or 1))


def _gpu_counts(dls, n, flags, order, pre, launch=None, plain=False):
    t = torch.from_numpy(np.ascontiguousarray(pre)).cuda()
    total = torch.zeros(1, dtype=torch.uint64, device="cuda")
    if plain:
        c = dls.count_plain(n, flags, order, t, total=total)
    else:
        c = dls.count(n, flags, order, t, total=total, launch=launch)
    torch.cuda.synchronize()
    c = c.cpu().numpy()
    tot = int(total.cpu().numpy()[0])
    assert tot == int(c.sum(dtype=np.uint64))
    return c


SHAPES = [
    dict(),
    dict(block_threads=32),
    dict(block_threads=512),
    dict(lanes_per_prefix=4),
    dict(lanes_per_prefix=32),
    dict(donate=-1),
    dict(check_every=1),
    dict(blocks_per_sm=1, block_threads=64),
    dict(words=1),
    dict(words=1, lanes_per_prefix=2, block_threads=64),
    dict(stack=1),
    dict(stack=1, block_threads=64, check_every=1),
]


def test_config1_order6_single_subproblem(dls, golden):
    wl = gpu_cases.split(dls, 6, D, 0)
    assert wl.prefixes.shape == (1, 6)
    ref, _ = oracle.count_many(6, D, wl.oracle_order, wl.oracle_prefixes)
    for sh in SHAPES:
        c = _gpu_counts(dls, 6, D, wl.order, wl.prefixes, dls.Launch(**sh))
        assert (c == ref).all(), sh
        assert int(c[0]) * dls.multiplier(6, D) == golden["dls_total_6"]
    c = _gpu_counts(dls, 6, D, wl.order, wl.prefixes, plain=True)
    assert (c == ref).all()


@pytest.mark.parametrize("n,flags,after", [(4, D, 0), (5, D, 3), (5, 0, 4), (6, D, 5),
                                           (6, D, 9), (6, D | V, 2), (6, 0, 8), (7, D, 4),
                                           (8, D | V, 6), (7, D, 14), (6, D, 12)])
def test_small_workloads_all_shapes(dls, n, flags, after):
    # (7, D, 14) and (6, D, 12) hold both diagonals in the prefix: the
    # snapshot search runs without diagonal words there
    wl = gpu_cases.split(dls, n, flags, after)
    ref, _ = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes, threads=THREADS)
    for sh in SHAPES:
        c = _gpu_counts(dls, n, flags, wl.order, wl.prefixes, dls.Launch(**sh))
        assert (c == ref).all(), sh
        c = _gpu_counts(dls, n, flags, wl.order, wl.prefixes,
                        dls.Launch(kernel=dls.KERNEL_PLAIN, **sh))
        assert (c == ref).all(), ("plain", sh)



def test_config2_order7_split10(dls):
    wl = gpu_cases.split(dls, 7, D, 10)
    assert len(wl.prefixes) > 1000
    ref, _ = oracle.count_many(7, D, wl.oracle_order, wl.oracle_prefixes, threads=THREADS)
    for sh in (dict(), dict(lanes_per_prefix=8), dict(block_threads=256)):
        c = _gpu_counts(dls, 7, D, wl.order, wl.prefixes, dls.Launch(**sh))
        assert (c == ref).all(), sh
    c = _gpu_counts(dls, 7, D, wl.order, wl.prefixes, plain=True)
    assert (c == ref).all()
    assert int(ref.sum()) == oracle.count(7, D, orders.md_ad_rows(7), orders.identity(7))[0]


@pytest.mark.parametrize("n,flags,rows", [(9, D, 4), (10, D, 5), (11, D, 6), (12, D, 7),
                                          (12, D | V, 6), (10, D | V, 4), (9, 0, 6),
                                          (10, D, 7)])
def test_larger_orders_from_sampled_partial_squares(dls, n, flags, rows):
    """Orders above 8 (row and column words in shared memory, or register
    fields for symmetric order 10): a few random partial squares with
    `rows` rows filled, decoded from the same seeded draws by both sides."""
    import dls_inputs
    vs = bool(flags & V)
    order = dls.fill_order(n, flags, first_rows=rows)
    o_order = orders.md_ad_rows(n, vsym=vs, first_rows=rows)
    assert [tuple(c) for c in order] == o_order
    depth = rows * len(orders.identity(n, vs))
    pre, o_pre = [], []
    for k in range(6):
        draws = dls_inputs.draws(1 << 14, seed=n * 100 + rows, stream=k)
        a, ua = dls.sample_prefix(n, flags, order, depth, draws)
        b, ub = oracle.sample_prefix(n, flags, o_order, depth, draws)
        assert ua == ub
        if b is None:
            continue
        assert (a == b).all()
        pre.append(a)
        o_pre.append(b)
    assert pre
    pre, o_pre = np.array(pre), np.array(o_pre)
    ref, _ = oracle.count_many(n, flags, o_order, o_pre, threads=THREADS)
    if rows < n - 3:
        assert (ref > 0).any()
    for sh in (dict(), dict(words=1), dict(lanes_per_prefix=8), dict(kernel=dls.KERNEL_PLAIN)):
        c = _gpu_counts(dls, n, flags, order, pre, dls.Launch(**sh))
        assert (c == ref).all(), sh


def test_snapshot_stack_refused_where_it_does_not_apply(dls):
    """The snapshot search needs register words and one lane per prefix."""
    # order 9 with every row after the prefix (no row 0): no wide words
    t9 = torch.from_numpy(np.zeros((1, 0), dtype=np.uint8)).cuda()
    t8 = torch.from_numpy(np.arange(8, dtype=np.uint8)[None]).cuda()
    for n, t, sh in ((9, t9, dict(stack=2)), (8, t8, dict(stack=2, words=1)),
                     (8, t8, dict(stack=2, lanes_per_prefix=2)),
                     (8, t8, dict(stack=2, kernel=dls.KERNEL_PLAIN, lanes_per_prefix=4)),
                     (8, t8, dict(stack=3))):
        with pytest.raises(dls.DlsError) as e:
            dls.count(n, D, dls.fill_order(n, D), t, launch=dls.Launch(**sh))
        assert e.value.code == 3, (n, sh)


def test_describe_launch_names_the_kernel(dls):
    o8, o9 = dls.fill_order(8, D), dls.fill_order(9, D)
    d = dls.describe_launch(8, D, o8, 15, 1000)
    assert d["kernel"] == "k_snapshot" and d["words"] == "registers"
    assert d["stack_entries"] > 0 and d["grid_blocks"] > 0
    assert dls.describe_launch(8, D, o8, 15, 1000, dls.Launch(stack=1))["kernel"] == "k_persistent"
    assert dls.describe_launch(8, D, o8, 15, 1000,
                               dls.Launch(kernel=dls.KERNEL_PLAIN))["kernel"] == "k_plain_snap"
    assert dls.describe_launch(8, D, o8, 15, 1000,
                               dls.Launch(kernel=dls.KERNEL_PLAIN, stack=1))["kernel"] == "k_plain"
    d9 = dls.describe_launch(9, D, o9, 17, 1000)
    assert d9["kernel"] == "k_snapshot" and d9["step"] == "snapshot, wide words"
    d9 = dls.describe_launch(9, D, o9, 5, 1000)  # rows 0-8 all searched
    assert d9["kernel"] == "k_persistent" and d9["words"] == "shared"
    assert dls.describe_launch(8, D, o8, 15, 0)["grid_blocks"] == 0
    with pytest.raises(dls.DlsError):
        dls.describe_launch(9, D, o9, 5, 10, dls.Launch(stack=2))


def test_lookahead_where_it_applies(dls):
    """Lookahead (Section 2.4.2): same counts, fewer nodes, where no cell
    after the prefix lies on a diagonal and without vertical symmetry;
    refused elsewhere."""
    for n, flags, after, kind in ((7, D, 14, dls.ORDER_HEURISTIC), (6, D, 10, dls.ORDER_HEURISTIC),
                                  (6, 0, 3, None), (5, 0, 4, None)):
        wl = gpu_cases.split(dls, n, flags, after, kind=kind)
        ref_c, ref_n = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes,
                                         threads=THREADS)
        t = torch.from_numpy(wl.prefixes).cuda()
        for sh in (dict(lookahead=1), dict(lookahead=1, block_threads=32, check_every=1)):
            nodes = torch.zeros(1, dtype=torch.uint64, device="cuda")
            c = dls.count(n, flags, wl.order, t, nodes=nodes, launch=dls.Launch(**sh))
            torch.cuda.synchronize()
            assert (c.cpu().numpy() == ref_c).all(), (n, flags, sh)
            assert int(nodes.cpu().numpy()[0]) <= int(ref_n.sum())
    for n, flags, after in ((6, D, 5), (6, D | V, 2)):
        wl = gpu_cases.split(dls, n, flags, after)
        with pytest.raises(dls.DlsError) as e:
            dls.count(n, flags, wl.order, torch.from_numpy(wl.prefixes).cuda(),
                      launch=dls.Launch(lookahead=1))
        assert e.value.code == 3


def test_fused_step_where_it_applies(dls):
    """The fused step (a following cell with one candidate is placed in the
    same iteration) makes the next iteration's move early: counts and node
    counts equal the oracle's, with the step on and off, in the persistent
    and plain kernels, with and without vertical symmetry; refused where
    diagonal words are in play, and with the lookahead."""
    for n, flags, after, kind in ((7, D, 14, dls.ORDER_HEURISTIC), (6, D, 10, dls.ORDER_HEURISTIC),
                                  (6, 0, 3, None), (5, 0, 4, None), (6, 0, 8, None),
                                  (8, D | V, 8, None), (6, V, 0, None)):
        wl = gpu_cases.split(dls, n, flags, after, kind=kind)
        ref_c, ref_n = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes,
                                         threads=THREADS)
        t = torch.from_numpy(wl.prefixes).cuda()
        depth = wl.prefixes.shape[1]
        for sh in (dict(fuse=1), dict(fuse=-1), dict(fuse=1, kernel=dls.KERNEL_PLAIN),
                   dict(fuse=1, block_threads=32, check_every=1), dict()):
            launch = dls.Launch(**sh)
            on = sh.get("fuse", 0) == 1 or (sh.get("fuse", 0) == 0 and not flags & V)
            assert dls.describe_launch(n, flags, wl.order, depth, len(t),
                                       launch)["fused"] == on
            nodes = torch.zeros(1, dtype=torch.uint64, device="cuda")
            c = dls.count(n, flags, wl.order, t, nodes=nodes, launch=launch)
            torch.cuda.synchronize()
            assert (c.cpu().numpy() == ref_c).all(), (n, flags, sh)
            assert int(nodes.cpu().numpy()[0]) == int(ref_n.sum()), (n, flags, sh)
    for n, flags, after, sh in ((6, D, 5, dict(fuse=1)), (6, D | V, 2, dict(fuse=1)),
                                (6, 0, 3, dict(fuse=1, lookahead=1)),
                                (6, 0, 3, dict(fuse=1, stack=1))):
        wl = gpu_cases.split(dls, n, flags, after)
        with pytest.raises(dls.DlsError) as e:
            dls.count(n, flags, wl.order, torch.from_numpy(wl.prefixes).cuda(),
                      launch=dls.Launch(**sh))
        assert e.value.code == 3, (n, flags, sh)
    # where it does not apply, the default runs the unfused step
    wl = gpu_cases.split(dls, 6, D, 5)
    assert not dls.describe_launch(6, D, wl.order, wl.prefixes.shape[1], 10)["fused"]


def test_snapshot_stack_deep_orders(dls):
    """Orders whose cells after the prefix are mostly free (row-major order
    from an empty square, so nothing is forced early): the snapshot stack
    runs at its bound; the host-buffer entry reports any overflow."""
    for n, flags, kind, after in ((6, D, dls.ORDER_ROW_MAJOR, 0), (6, 0, dls.ORDER_ROW_MAJOR, 3),
                                  (7, D, dls.ORDER_ROW_MAJOR, 9), (8, D | V, dls.ORDER_ROW_MAJOR, 2),
                                  (6, D | V, dls.ORDER_HEURISTIC, 0)):
        wl = gpu_cases.split(dls, n, flags, after, kind=kind)
        ref, _ = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes,
                                   threads=THREADS)
        for sh in (dict(stack=2), dict(stack=2, block_threads=32, check_every=1),
                   dict(stack=2, kernel=dls.KERNEL_PLAIN)):
            c = _gpu_counts(dls, n, flags, wl.order, wl.prefixes, dls.Launch(**sh))
            assert (c == ref).all(), (n, flags, kind, sh)
            hc, tot = dls.count_host(n, flags, wl.order, wl.prefixes, launch=dls.Launch(**sh))
            assert (hc == ref).all() and tot == int(ref.sum())


def test_register_words_refused_when_they_do_not_fit(dls):
    # order 9: register words only as the snapshot search's wide words, which
    # need at most 8 rows after the prefix; refused with the per-position
    # stack and with every row after the prefix
    order = dls.fill_order(9, D)
    t = torch.from_numpy(np.arange(9, dtype=np.uint8)[None]).cuda()
    t0 = torch.from_numpy(np.zeros((1, 0), np.uint8)).cuda()
    for tt, sh in ((t, dict(words=2, stack=1)), (t0, dict(words=2))):
        with pytest.raises(dls.DlsError) as e:
            dls.count(9, D, order, tt, launch=dls.Launch(**sh))
        assert e.value.code == 3


def test_node_counts_match_oracle(dls):
    for n, flags, after in ((6, D, 0), (7, D, 10), (6, D | V, 3), (5, 0, 5)):
        wl = gpu_cases.split(dls, n, flags, after)
        ref_c, ref_n = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes,
                                         threads=THREADS)
        t = torch.from_numpy(wl.prefixes).cuda()
        for sh in (dict(), dict(lanes_per_prefix=4), dict(kernel=dls.KERNEL_PLAIN),
                   dict(words=1), dict(stack=1)):
            nodes = torch.zeros(1, dtype=torch.uint64, device="cuda")
            c = dls.count(n, flags, wl.order, t, nodes=nodes, launch=dls.Launch(**sh))
            torch.cuda.synchronize()
            assert (c.cpu().numpy() == ref_c).all()
            assert int(nodes.cpu().numpy()[0]) == int(ref_n.sum()), (n, flags, sh)


@pytest.mark.slow
def test_config3_order8_diag64_sampled_against_oracle(dls):
    wl = gpu_cases.dls8_diag64(dls)
    c = _gpu_counts(dls, 8, D, wl.order, wl.prefixes)
    # the diagonals the oracle recounts: 4 of the 64, seed-chosen
    import dls_inputs
    check = dls_inputs.choose(64, 4, seed=1)
    sel = np.isin(wl.parents, check)
    # counts do not depend on the order of the cells after the prefix: the
    # oracle takes its own Section 2.3 order there (about 3x fewer nodes)
    o_fast = orders.heuristic_complete(8, wl.oracle_order[:wl.depth])
    ref, _ = oracle.count_many(8, D, o_fast, wl.oracle_prefixes[sel], threads=THREADS)
    assert (c[sel] == ref).all()
    # plain launch agrees everywhere
    c2 = _gpu_counts(dls, 8, D, wl.order, wl.prefixes, plain=True)
    assert (c2 == c).all()
    # and a lane-split launch
    c3 = _gpu_counts(dls, 8, D, wl.order, wl.prefixes, dls.Launch(lanes_per_prefix=4))
    assert (c3 == c).all()


@pytest.mark.parametrize("depth", [22, 25, 28, 31])
@pytest.mark.parametrize("suffix", ["heuristic", "heuristic_sq"])
def test_bench_configuration_against_oracle(dls, suffix, depth):
    """The order-8 workload exactly as the benchmark times it, at every split
    depth its autotuner can pick (14, 17, 20 or 23 cells past row 0: both
    diagonals and part of row 1 at 28), the Section 2.3 order (or its
    squared-count variant) after the split, counted through a CUDA-graph plan
    with the default launch and the 64-thread blocks the autotuner picks; the
    prefixes of 4 seed-chosen diagonals of the 64 against the oracle (its own
    order and prefixes)."""
    import dls_inputs
    from paper_1709_02599_gb300 import autotune
    n = 8
    order0 = dls.fill_order(n, D)
    ident = np.arange(n, dtype=np.uint8)[None]
    diags, _ = dls.extend_prefixes(n, D, order0, ident, n + (n - 1))
    picks = dls_inputs.choose(len(diags), 64, 0)         # the benchmark's seed-0 draw
    order, pre, par = autotune.build_problem(n, D, order0, diags[picks], depth, suffix)
    o_order = orders.heuristic_complete(n, orders.md_ad_rows(n)[:depth],
                                        squares=suffix == "heuristic_sq")
    # the tail run is dropped from the GPU's order; the oracle counts the
    # whole square
    assert [tuple(map(int, x)) for x in order] == orders.trim_tail(n, o_order, depth)
    o_diags, _ = oracle.extend(n, D, orders.md_ad_rows(n), np.array([orders.identity(n)],
                                                                        np.uint8), n + (n - 1))
    o_pre, o_par = oracle.extend(n, D, o_order, o_diags[picks], depth)
    assert (o_pre == pre).all() and (o_par == par).all()
    sel = np.isin(par, dls_inputs.choose(64, 4, seed=2))
    ref, _ = oracle.count_many(n, D, o_order, o_pre[sel], threads=THREADS)
    assert int(ref.sum()) > 0
    d_pre = torch.from_numpy(pre).cuda()
    for launch in (dict(), dict(fuse=-1), dict(block_threads=64), dict(lookahead=1)):
        counts = torch.empty(len(pre), dtype=torch.uint64, device="cuda")
        total = torch.empty(1, dtype=torch.uint64, device="cuda")
        plan = dls.Plan(n, D, order, d_pre, counts, total, dls.Launch(**launch))
        plan.launch()
        torch.cuda.synchronize()
        c = counts.cpu().numpy()
        plan.close()
        assert dls.describe_launch(n, D, order, depth, len(pre),
                                   dls.Launch(**launch))["kernel"] == "k_snapshot"
        assert int(total.cpu().numpy()[0]) == int(c.sum(dtype=np.uint64))
        assert (c[sel] == ref).all(), launch


@pytest.mark.slow
def test_config4_vsym10_smallest_against_oracle(dls):
    wl = gpu_cases.vsym10_rows2(dls)
    assert len(wl.prefixes) == 2000
    c = _gpu_counts(dls, 10, D | V, wl.order, wl.prefixes)
    c2 = _gpu_counts(dls, 10, D | V, wl.order, wl.prefixes, plain=True)
    assert (c2 == c).all()
    idx = np.argsort(c, kind="stable")[:20]
    # the oracle splits each checked prefix a few cells deeper so that all
    # host threads stay busy, and sums the parts per prefix
    o_fast = orders.heuristic_complete(10, wl.oracle_order[:wl.depth], True, True)
    sub, par = oracle.extend(10, D | V, o_fast, wl.oracle_prefixes[idx], wl.depth + 4)
    part, _ = oracle.count_many(10, D | V, o_fast, sub, threads=THREADS)
    ref = np.zeros(len(idx), np.uint64)
    np.add.at(ref, par, part)
    assert (c[idx] == ref).all()


@pytest.mark.slow
def test_paper_order8_total(dls, golden):
    # Section 5.1: 7 447 587 840 diagonal Latin squares of order 8 with row 0
    # fixed; split after both diagonals (14 cells past row 0)
    wl = gpu_cases.split(dls, 8, D, 14)
    c = _gpu_counts(dls, 8, D, wl.order, wl.prefixes)
    assert int(c.sum(dtype=np.uint64)) == golden["dls8_row0_fixed"]
    # dls_count_weighted: the same count times the row-0 multiplier 8!, and
    # with every weight 2^32 - 1 a weighted total past 2^64, both in 128 bits
    d_pre = torch.from_numpy(wl.prefixes).cuda()
    total = dls.count_weighted(8, D, wl.order, d_pre, multiply=True)
    assert total == golden["dls8_row0_fixed"] * 40320
    # (int32 -1 is the 32-bit pattern 2^32 - 1; the library reads uint32)
    w = torch.full((len(wl.prefixes),), -1, dtype=torch.int32, device="cuda")
    big = dls.count_weighted(8, D, wl.order, d_pre, weights=w)
    assert big == golden["dls8_row0_fixed"] * 0xFFFFFFFF and big >= 1 << 64


@pytest.mark.slow
def test_paper_partial_count_n10_k30(dls, golden):
    # Section 5.3: 284 086 571 712 partial diagonal Latin squares of order 10
    # with the first 30 cells in row-major order filled and row 0 fixed
    n = 10
    order = dls.fill_order(n, D, dls.ORDER_ROW_MAJOR)[:30]
    base = np.arange(n, dtype=np.uint8)[None]
    pre, _ = dls.extend_prefixes(n, D, order, base, 16)
    # the split itself against the oracle's enumerator
    o_pre, _ = oracle.extend(n, D, orders.row_major(n)[:30], base, 16)
    assert (pre == o_pre).all()
    c = _gpu_counts(dls, n, D, order, pre)
    assert int(c.sum(dtype=np.uint64)) == golden["n10_k30"]
    # a sample of prefixes against the oracle
    idx = np.arange(0, len(pre), len(pre) // 6)
    ref, _ = oracle.count_many(n, D, orders.row_major(n)[:30], o_pre[idx], threads=THREADS)
    assert (c[idx] == ref).all()


@pytest.mark.slow
def test_paper_partial_count_n10_k32(dls, golden):
    # Section 5.3: 12 611 543 636 160 partial diagonal Latin squares of order
    # 10 with the first 32 cells in row-major order filled and row 0 fixed;
    # split after 18 cells (~1e6 prefixes)
    n = 10
    order = dls.fill_order(n, D, dls.ORDER_ROW_MAJOR)[:32]
    base = np.arange(n, dtype=np.uint8)[None]
    pre, _ = dls.extend_prefixes(n, D, order, base, 18)
    o_pre, _ = oracle.extend(n, D, orders.row_major(n)[:32], base, 18)
    assert (pre == o_pre).all()
    c = _gpu_counts(dls, n, D, order, pre)
    assert int(c.sum(dtype=np.uint64)) == golden["n10_k32"]
    # a few prefixes against the oracle
    idx = np.arange(0, len(pre), len(pre) // 8)[:8]
    ref, _ = oracle.count_many(n, D, orders.row_major(n)[:32], o_pre[idx], threads=THREADS)
    assert (c[idx] == ref).all() and (ref > 0).any()


def test_paper_hourglass8_on_gpu(dls, golden):
    # Section 4.2: 22 192 248 hourglass designs of order 8
    n = 8
    order = dls.fill_order(n, D, dls.ORDER_HOURGLASS)[:8 + 7 + 7 + 6]
    base = np.arange(n, dtype=np.uint8)[None]
    pre, _ = dls.extend_prefixes(n, D, order, base, 8 + 7)
    c = _gpu_counts(dls, n, D, order, pre)
    assert int(c.sum(dtype=np.uint64)) == golden["hourglass8"]


def test_edge_cases(dls):
    order = dls.fill_order(6, D)
    # empty batch
    t = torch.zeros((0, 6), dtype=torch.uint8, device="cuda")
    c = dls.count(6, D, order, t)
    torch.cuda.synchronize()
    assert c.numel() == 0
    # complete squares as prefixes: 1 if valid, 0 if not
    o_order = orders.md_ad_rows(6)
    full, _ = oracle.extend(6, D, o_order, np.array([orders.identity(6)], np.uint8), 36)
    assert len(full) == 128
    bad = full[:5].copy()
    bad[:, 20] = (bad[:, 20] + 1) % 6
    pre = np.concatenate([full, bad])
    c = _gpu_counts(dls, 6, D, order, pre)
    ref, _ = oracle.count_many(6, D, o_order, pre)
    assert (c == ref).all() and c[:128].sum() == 128
    # one cell left
    c = _gpu_counts(dls, 6, D, order, full[:, :35])
    assert (c == 1).all()
    # invalid prefixes: repeated value, value out of range
    ok, _ = oracle.extend(6, D, o_order, np.array([orders.identity(6)], np.uint8), 10)
    bad = ok[:40].copy()
    bad[::2, 7] = 9
    bad[1::2, 9] = bad[1::2, 8]
    c = _gpu_counts(dls, 6, D, order, np.concatenate([ok[:40], bad]))
    ref, _ = oracle.count_many(6, D, o_order, np.concatenate([ok[:40], bad]))
    assert (c == ref).all() and (c[40:] == 0).all()
    # orders 1..3
    assert _gpu_counts(dls, 1, D, [(0, 0)], np.zeros((1, 0), np.uint8))[0] == 1
    for n in (2, 3):
        o = dls.fill_order(n, D)
        assert _gpu_counts(dls, n, D, o, np.arange(n, dtype=np.uint8)[None])[0] == 0
    # vertically symmetric odd orders are empty
    for n in (5, 7):
        o = dls.fill_order(n, D | V)
        c = _gpu_counts(dls, n, D | V, o, np.arange(n // 2, dtype=np.uint8)[None])
        assert c[0] == 0
    # the largest order: partial order of 16 + 6 cells, every mask bit in use
    o16 = [(0, j) for j in range(16)] + [(1, 1), (1, 14), (2, 2), (15, 0), (15, 15), (3, 5)]
    pre16 = np.arange(16, dtype=np.uint8)[None]
    c = _gpu_counts(dls, 16, D, o16, pre16)
    assert c[0] == oracle.count(16, D, o16, list(range(16)))[0]


def test_host_buffers_and_plan_and_streams(dls):
    wl = gpu_cases.split(dls, 7, D, 8)
    ref, _ = oracle.count_many(7, D, wl.oracle_order, wl.oracle_prefixes, threads=THREADS)
    # host-buffer entry point (pinned and pageable)
    pinned = torch.from_numpy(wl.prefixes).pin_memory()
    cnt, tot = dls.count_host(7, D, wl.order, pinned)
    assert (cnt == ref).all() and tot == int(ref.sum())
    cnt, tot = dls.count_host(7, D, wl.order, wl.prefixes,
                              launch=dls.Launch(kernel=dls.KERNEL_PLAIN))
    assert (cnt == ref).all()
    # graph plan, launched repeatedly
    t = torch.from_numpy(wl.prefixes).cuda()
    counts = torch.empty(len(t), dtype=torch.uint64, device="cuda")
    total = torch.empty(1, dtype=torch.uint64, device="cuda")
    plan = dls.Plan(7, D, wl.order, t, counts, total)
    for _ in range(3):
        counts.fill_(7)
        plan.launch()
        torch.cuda.synchronize()
        assert (counts.cpu().numpy() == ref).all()
        assert int(total.cpu().numpy()[0]) == int(ref.sum())
    plan.close()
    # two streams at once
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    c1 = torch.empty(len(t), dtype=torch.uint64, device="cuda")
    c2 = torch.empty(len(t), dtype=torch.uint64, device="cuda")
    torch.cuda.synchronize()
    dls.count(7, D, wl.order, t, counts=c1, stream=s1)
    dls.count(7, D, wl.order, t, counts=c2, stream=s2, launch=dls.Launch(lanes_per_prefix=2))
    torch.cuda.synchronize()
    assert (c1.cpu().numpy() == ref).all() and (c2.cpu().numpy() == ref).all()


def test_status_queries_after_counts_and_plans(dls):
    """dls_stream_status after dls_count_ex and dls_plan_status after a plan
    launch: a finished count reports DLS_OK and every prefix started, for
    the batched and the plain kernels, on a stream of our own."""
    wl = gpu_cases.split(dls, 7, D, 14)
    ref, _ = oracle.count_many(7, D, wl.oracle_order, wl.oracle_prefixes, threads=THREADS)
    P = len(wl.prefixes)
    d_pre = torch.from_numpy(wl.prefixes).cuda()
    st = torch.cuda.Stream()
    for launch in (dls.Launch(), dls.Launch(kernel=dls.KERNEL_PLAIN),
                   dls.Launch(stack=1), dls.Launch(lanes_per_prefix=4)):
        with torch.cuda.stream(st):
            c = dls.count(7, D, wl.order, d_pre, launch=launch, stream=st)
        assert dls.stream_status(st) == (0, P), launch
        assert (c.cpu().numpy() == ref).all()
        counts = torch.empty(P, dtype=torch.uint64, device="cuda")
        plan = dls.Plan(7, D, wl.order, d_pre, counts, None, launch)
        plan.launch(st)
        assert plan.status(st) == (0, P)
        assert (counts.cpu().numpy() == ref).all()
        plan.close()


def test_budget_and_abort_flag_on_the_gpu(dls):
    """A small iteration budget stops the count (DLS_ERR_TIMEOUT): every count
    not marked DLS_UNFINISHED below prefixes_started is exact, and counting the
    rest again completes the job.  An abort flag in device memory that is set
    stops it (DLS_ERR_ABORTED); one that stays clear changes nothing."""
    wl = gpu_cases.split(dls, 7, D, 14)
    ref, _ = oracle.count_many(7, D, wl.oracle_order, wl.oracle_prefixes, threads=THREADS)
    P = len(wl.prefixes)
    d_pre = torch.from_numpy(wl.prefixes).cuda()
    st = torch.cuda.Stream()
    for sh in (dict(), dict(kernel=dls.KERNEL_PLAIN), dict(stack=1), dict(lanes_per_prefix=4)):
        launch = dls.Launch(budget=32, check_every=8, **sh)
        with torch.cuda.stream(st):
            c = dls.count(7, D, wl.order, d_pre, launch=launch, stream=st)
        status, started = dls.stream_status(st)
        assert status == dls.ERR_TIMEOUT and 0 < started <= P, sh
        c = c.cpu().numpy()
        unfinished = (c & np.uint64(dls.UNFINISHED)) != 0
        assert unfinished.any()
        done = ~unfinished & (np.arange(P) < started)
        assert (c[done] == ref[done]).all(), sh
        redo = np.nonzero(~done)[0]
        with torch.cuda.stream(st):
            c2 = dls.count(7, D, wl.order, d_pre[torch.from_numpy(redo).cuda()],
                           launch=dls.Launch(**sh), stream=st)
        assert dls.stream_status(st) == (0, len(redo))
        c[redo] = c2.cpu().numpy()
        assert (c == ref).all(), sh
    for value, expect in ((1, dls.ERR_ABORTED), (0, 0)):
        flag = torch.full((1,), value, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(st):
            c = dls.count(7, D, wl.order, d_pre, launch=dls.Launch(abort_flag=flag.data_ptr()),
                          stream=st)
        status, started = dls.stream_status(st)
        assert status == expect
        if expect == 0:
            assert started == P and (c.cpu().numpy() == ref).all()


@pytest.mark.parametrize("depth", [25, 28])
def test_stack_cap_on_the_benchmark_workload(dls, depth):
    """The order-8 workload with the snapshot stack capped below its bound
    (entries 16 and 12, against 25 and 23): the lanes that would outgrow the
    cap defer their prefix, the recount pass counts those again, and the
    counts of 4 seed-chosen diagonals are the oracle's; every count and the
    total equal those of the uncapped launch, through plans too."""
    import dls_inputs
    from paper_1709_02599_gb300 import autotune
    n = 8
    order0 = dls.fill_order(n, D)
    ident = np.arange(n, dtype=np.uint8)[None]
    diags, _ = dls.extend_prefixes(n, D, order0, ident, n + (n - 1))
    picks = dls_inputs.choose(len(diags), 64, 0)
    order, pre, par = autotune.build_problem(n, D, order0, diags[picks], depth, "heuristic_sq")
    o_order = orders.heuristic_complete(n, orders.md_ad_rows(n)[:depth], squares=True)
    o_diags, _ = oracle.extend(n, D, orders.md_ad_rows(n), np.array([orders.identity(n)],
                                                                        np.uint8), n + (n - 1))
    o_pre, o_par = oracle.extend(n, D, o_order, o_diags[picks], depth)
    assert (o_pre == pre).all()
    sel = np.isin(par, dls_inputs.choose(64, 4, seed=3))
    ref, _ = oracle.count_many(n, D, o_order, o_pre[sel], threads=THREADS)
    d_pre = torch.from_numpy(pre).cuda()
    full = _gpu_counts(dls, n, D, order, pre)
    for cap in (16, 12):
        for launch in (dls.Launch(stack_cap=cap), dls.Launch(stack_cap=cap, block_threads=64),
                       dls.Launch(kernel=dls.KERNEL_PLAIN, stack_cap=cap)):
            assert dls.describe_launch(n, D, order, depth, len(pre), launch)["stack_entries"] == cap
            c = _gpu_counts(dls, n, D, order, pre, launch)
            assert (c == full).all(), launch
            assert (c[sel] == ref).all()
            counts = torch.empty(len(pre), dtype=torch.uint64, device="cuda")
            total = torch.empty(1, dtype=torch.uint64, device="cuda")
            plan = dls.Plan(n, D, order, d_pre, counts, total, launch)
            plan.launch()
            plan.launch()
            assert plan.status() == (0, len(pre))
            assert (counts.cpu().numpy() == full).all()
            assert int(total.cpu().numpy()[0]) == int(full.sum())
            plan.close()


@pytest.mark.parametrize("flags", [D, 0])
def test_order9_wide_words(dls, flags):
    """Order 9 on the wide-word snapshot search: random partial squares with
    4 rows filled (5 for ordinary squares), extended through the rest of both
    diagonals with the diagonal flag, so that every step runs (diagonal
    words, the fused step, the lookahead), plus a capped stack (deferred
    prefixes recounted) and the plain launch, against the oracle."""
    import dls_inputs
    rows = 4 if flags & D else 5
    order = dls.fill_order(9, flags, first_rows=rows)
    o_order = orders.md_ad_rows(9, first_rows=rows)
    depth = rows * 9
    pre, o_pre = [], []
    for k in range(8):
        draws = dls_inputs.draws(1 << 14, seed=9 * 100 + rows + 50, stream=k)
        a, _ = dls.sample_prefix(9, flags, order, depth, draws)
        b, _ = oracle.sample_prefix(9, flags, o_order, depth, draws)
        if b is None:
            continue
        pre.append(a)
        o_pre.append(b)
    pre, o_pre = np.array(pre), np.array(o_pre)
    assert (pre == o_pre).all()
    cases = [(pre, o_pre, depth)]
    if flags & D:
        diag = sum(1 for i, j in o_order[depth:] if i == j or i + j == 8)
        p2, _ = dls.extend_prefixes(9, flags, order, pre, depth + diag)
        o2, _ = oracle.extend(9, flags, o_order, o_pre, depth + diag)
        assert (p2 == o2).all() and len(p2) > 0
        cases.append((p2, o2, depth + diag))
    for p, op, d in cases:
        ref, _ = oracle.count_many(9, flags, o_order, op, threads=THREADS)
        shapes = [dict(), dict(kernel=dls.KERNEL_PLAIN), dict(stack_cap=4),
                  dict(block_threads=32, check_every=1)]
        if d > depth:
            shapes += [dict(fuse=-1), dict(lookahead=1), dict(stack_cap=3, block_threads=64)]
        for sh in shapes:
            info = dls.describe_launch(9, flags, order, d, len(p), dls.Launch(**sh))
            assert info["step"] == "snapshot, wide words", (sh, info)
            c = _gpu_counts(dls, 9, flags, order, p, dls.Launch(**sh))
            assert (c == ref).all(), (d, sh)
