"""CPU tests of the library's kernels and launch code.

The library is built with the host compiler against a stand-in CUDA
runtime (host_emulation.py, tests/host_kernels). In it, every CUDA thread is
a cooperative fiber, warp votes and shuffles complete once all lanes of the
warp reach them, and all blocks of a grid interleave at those points. The
kernels then run through the library's own C entry points: dls_count_ex,
dls_count_host, dls_count_host_noalloc, the CUDA-graph plans and
dls_describe_launch.

What this checks, against the oracle (which shares no code with it):
- the per-prefix counts, the total and the node count for every launch
  shape of the persistent and plain kernels: snapshot and per-position
  stacks, register and shared-memory words, lane splits, donation on and off
  and at every iteration, lookahead and fused step, several blocks sharing
  the queue;
- the host-buffer entries (the allocation-free one too) and plans replayed
  twice;
- the launch descriptions and the argument errors, which otherwise need a
  GPU.

The GPU tests remain the parity tests proper; this catches mistakes in the
kernels' warp-level logic on any machine."""
import numpy as np
import pytest

import gpu_cases
import oracle

D, V = 1, 2
ERR_BAD_ARG = 3
ERR_TIMEOUT = 6
ERR_ABORTED = 7
ERR_INTERNAL = 10
UNFINISHED = np.uint64(1 << 63)


# launch shapes: both kernel families, both stacks, both word placements,
# lane splits, donation off and at every iteration, small blocks and several
# blocks per multiprocessor (the stand-in device has two)
SHAPES = [
    dict(),
    dict(block_threads=32),
    dict(block_threads=32, check_every=1),
    dict(block_threads=64, blocks_per_sm=3),
    dict(donate=-1),
    dict(lanes_per_prefix=4),
    dict(lanes_per_prefix=32, block_threads=32),
    dict(words=1),
    dict(words=1, lanes_per_prefix=2, block_threads=64),
    dict(stack=1),
    dict(stack=1, block_threads=32, check_every=1),
    dict(fuse=-1),
]


def every(wl, step):
    """Every step-th prefix of a workload (both sides take the same ones):
    the emulated kernels run about 10^6 nodes per second, so the workloads
    here stay near 10^5 nodes."""
    return gpu_cases.Workload(wl.n, wl.flags, wl.order, wl.prefixes[::step], wl.oracle_order,
                              wl.oracle_prefixes[::step])


def check_counts(emu, wl, n, flags, shapes, nodes_exact=True):
    ref_c, ref_n = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes, threads=4)
    for sh in shapes:
        rc, res = emu.count("count", n, flags, wl.order, wl.prefixes, **sh)
        if rc == ERR_BAD_ARG and sh.get("fuse") == -1:
            continue
        assert rc == 0, (sh, rc)
        c, total, nodes = res
        assert (c == ref_c).all(), sh
        assert total == int(ref_c.sum()), sh
        if nodes_exact:
            assert nodes == int(ref_n.sum()), sh
        else:
            assert nodes <= int(ref_n.sum()), sh


@pytest.mark.parametrize("n,flags,after,kind,step", [
    (4, D, 0, None, 1), (5, D, 3, None, 1), (5, 0, 4, None, 1), (6, D, 5, None, 1),
    (6, D | V, 2, None, 1), (7, D, 14, None, 200), (6, D, 12, None, 1), (6, V, 4, None, 4),
    (6, D, 10, "heuristic", 1), (7, D, 11, "heuristic", 40)])
def test_kernels_against_oracle(dls, emulated, n, flags, after, kind, step):
    k = {None: None, "heuristic": dls.ORDER_HEURISTIC}[kind]
    wl = every(gpu_cases.split(dls, n, flags, after, kind=k), step)
    shapes = SHAPES + [dict(sh, kernel=1) for sh in SHAPES if "check_every" not in sh
                       and "donate" not in sh and "blocks_per_sm" not in sh]
    check_counts(emulated, wl, n, flags, shapes)


@pytest.mark.parametrize("n,flags,after,kind,step", [
    (6, D | V, 2, None, 1), (7, D, 14, None, 50), (6, D, 10, "heuristic", 1),
    (6, V, 4, None, 4)])
def test_kernels_on_trimmed_orders(dls, emulated, n, flags, after, kind, step):
    """Every kernel on orders shortened by dls_order_trim, against the oracle
    on its own trimmed order (counts and nodes) and on the whole order
    (counts)."""
    k = {None: None, "heuristic": dls.ORDER_HEURISTIC}[kind]
    wl = every(gpu_cases.split(dls, n, flags, after, kind=k, trim=True), step)
    full = every(gpu_cases.split(dls, n, flags, after, kind=k), step)
    assert len(wl.order) < len(full.order)
    shapes = [dict(), dict(kernel=1), dict(stack=1), dict(stack_cap=1)]
    check_counts(emulated, wl, n, flags, shapes)
    c_full, _ = oracle.count_many(n, flags, full.oracle_order, full.oracle_prefixes, threads=4)
    rc, res = emulated.count("count", n, flags, wl.order, wl.prefixes)
    assert rc == 0 and (res[0] == c_full).all()


def test_strided_queue_order(dls, emulated):
    """Where the grid's lanes get 16 prefixes or fewer each (and there are
    4 096 or more), the batched byte-word search takes its queue in a
    strided order (place k is prefix k * stride mod P): every prefix is
    still counted once, into its own slot, also through the recount pass of
    a capped stack and with the node count."""
    for n, flags, after, kind, shapes in (
            (7, D, 12, dls.ORDER_HEURISTIC, [dict(), dict(stack_cap=2)]),):
        wl = gpu_cases.split(dls, n, flags, after, kind=kind)
        P = len(wl.prefixes)
        for sh in shapes:
            rc, info = emulated.count("describe", n, flags, wl.order, wl.prefixes, **sh)
            assert rc == 0 and info["run"] == 2
            assert 4096 <= P <= 16 * info["grid_blocks"] * info["block_threads"], (P, info)
        check_counts(emulated, wl, n, flags, shapes)


def test_lookahead_and_fused_step(dls, emulated):
    """Where no cell after the prefix lies on a diagonal: the lookahead
    (without vertical symmetry) prunes (fewer nodes, same counts); the fused
    step (also with it) keeps the counts and the nodes."""
    for n, flags, after, kind, step in ((7, D, 14, dls.ORDER_HEURISTIC, 30),
                                        (6, 0, 8, None, 1000), (5, 0, 4, None, 1),
                                        (8, D | V, 8, None, 4), (6, V, 0, None, 1)):
        wl = every(gpu_cases.split(dls, n, flags, after, kind=kind), step)
        check_counts(emulated, wl, n, flags,
                     [dict(fuse=1), dict(fuse=1, kernel=1), dict(fuse=1, block_threads=32,
                                                                 check_every=1)])
        if flags & V:
            rc, _ = emulated.count("count", n, flags, wl.order, wl.prefixes, lookahead=1)
            assert rc == ERR_BAD_ARG
            continue
        check_counts(emulated, wl, n, flags,
                     [dict(lookahead=1), dict(lookahead=1, block_threads=32, check_every=1)],
                     nodes_exact=False)


def test_larger_orders_from_sampled_partial_squares(dls, emulated):
    """Orders 9, 10 (symmetric) and 12 (symmetric): shared-memory words, and
    register fields for symmetric order 10, through the per-position
    kernels."""
    for n, flags, rows in ((9, D, 4), (10, D | V, 5), (12, D | V, 7), (9, 0, 6)):
        wl = gpu_cases.sampled_rows(dls, n, flags, rows)
        check_counts(emulated, wl, n, flags,
                     [dict(), dict(words=1), dict(lanes_per_prefix=8), dict(kernel=1),
                      dict(block_threads=32, check_every=1)])


def test_queue_shared_by_many_blocks(dls, emulated):
    """Many prefixes, small blocks, several blocks per multiprocessor: the
    blocks take items from one queue in turns."""
    wl = every(gpu_cases.split(dls, 7, D, 11, kind=dls.ORDER_HEURISTIC), 8)
    assert len(wl.prefixes) > 7 * 32
    rc, info = emulated.count("describe", 7, D, wl.order, wl.prefixes, block_threads=32,
                   blocks_per_sm=4)
    assert rc == 0 and info["grid_blocks"] == 8
    check_counts(emulated, wl, 7, D, [dict(block_threads=32, blocks_per_sm=4),
                                          dict(block_threads=32, blocks_per_sm=4, stack=1)])


def test_host_buffer_entry_and_plans(dls, emulated):
    # order 6 (diagonal words in the search) and order 7 with both diagonals
    # in the prefix (the fused step by default)
    for n, after, step in ((6, 5, 1), (7, 14, 200)):
        wl = every(gpu_cases.split(dls, n, D, after), step)
        ref_c, _ = oracle.count_many(n, D, wl.oracle_order, wl.oracle_prefixes)
        for sh in (dict(), dict(stack=1), dict(kernel=1), dict(lanes_per_prefix=4)):
            for entry in ("host", "noalloc"):
                rc, (c, total, _) = emulated.count(entry, n, D, wl.order, wl.prefixes, **sh)
                assert rc == 0 and (c == ref_c).all(), (entry, sh)
                assert total == int(ref_c.sum()), (entry, sh)  # the plain 128-bit sum
            rc, (c, total, _) = emulated.count("plan", n, D, wl.order, wl.prefixes, **sh)
            assert rc == 0 and (c == ref_c).all() and total == int(ref_c.sum()), sh


def test_status_after_every_entry(dls, emulated):
    """A finished count reports DLS_OK and every prefix started, through
    dls_stream_status after dls_count_ex and dls_plan_status after a plan,
    for both kernel families.  With the snapshot stack bound forced below
    what the search needs (a hook of this CPU build only), the kernel sets
    its overflow flag and every entry reports DLS_ERR_INTERNAL: the status
    queries, dls_count_host and dls_count_host_noalloc."""
    wl = every(gpu_cases.split(dls, 7, D, 14), 100)
    P = len(wl.prefixes)
    for sh in (dict(), dict(kernel=1), dict(stack=1), dict(kernel=1, stack=1)):
        for entry in ("count", "plan"):
            rc, _ = emulated.count(entry, 7, D, wl.order, wl.prefixes, **sh)
            assert rc == 0 and emulated.last_status == (0, P), (entry, sh)
    for sh in (dict(), dict(kernel=1)):
        info = emulated.count("describe", 7, D, wl.order, wl.prefixes, **sh)[1]
        assert info["stack_entries"] > 1
        low = {"DLS_STANDIN_SNAP_CAP": 1}
        for entry in ("count", "plan"):
            rc, _ = emulated.count(entry, 7, D, wl.order, wl.prefixes, env=low, **sh)
            assert rc == 0 and emulated.last_status[0] == ERR_INTERNAL, (entry, sh)
        for entry in ("host", "noalloc"):
            rc, _ = emulated.count(entry, 7, D, wl.order, wl.prefixes, env=low, **sh)
            assert rc == ERR_INTERNAL, (entry, sh)
        # the per-position stack has no bound to exceed
        rc, _ = emulated.count("host", 7, D, wl.order, wl.prefixes, env=low, stack=1, **sh)
        assert rc == 0


@pytest.mark.parametrize("sh", [dict(), dict(kernel=1), dict(stack=1), dict(kernel=1, stack=1),
                                dict(lanes_per_prefix=4), dict(kernel=1, lanes_per_prefix=4)])
def test_budget_stops_and_the_rest_resumes(dls, emulated, sh):
    """A tiny iteration budget stops the count: DLS_ERR_TIMEOUT, the prefixes a
    lane was still searching marked DLS_UNFINISHED, those never handed out
    beyond prefixes_started.  Every other count is already exact, and
    counting the rest again without a budget completes the job."""
    wl = every(gpu_cases.split(dls, 7, D, 14), 7)
    ref, _ = oracle.count_many(7, D, wl.oracle_order, wl.oracle_prefixes)
    P = len(wl.prefixes)
    rc, res = emulated.count("count", 7, D, wl.order, wl.prefixes, budget=8, check_every=4,
                             block_threads=64, **sh)
    assert rc == 0
    status, started = emulated.last_status
    assert status == ERR_TIMEOUT and 0 < started <= P
    counts = res[0]
    unfinished = (counts & UNFINISHED) != 0
    assert unfinished.any()
    done = ~unfinished & (np.arange(P) < started)
    assert (counts[done] == ref[done]).all()
    redo = ~done
    rc, res2 = emulated.count("count", 7, D, wl.order, wl.prefixes[redo], **sh)
    assert rc == 0 and emulated.last_status == (0, int(redo.sum()))
    merged = counts.copy()
    merged[redo] = res2[0]
    assert (merged == ref).all()
    # the host-buffer entries return the status
    for entry in ("host", "noalloc"):
        rc, _ = emulated.count(entry, 7, D, wl.order, wl.prefixes, budget=8, check_every=4, **sh)
        assert rc == ERR_TIMEOUT, entry


def test_weighted_total(dls, emulated):
    """dls_count_weighted: the counts, and the sum of weight x count in 128
    bits times the row-0 multiplier (weights (k % 5) + 1 in the driver), for
    both kernel families.  (A total past 2^64 is tested on the GPU.)"""
    for n, after, step in ((7, 14, 7),):
        wl = every(gpu_cases.split(dls, n, D, after), step)
        ref, _ = oracle.count_many(n, D, wl.oracle_order, wl.oracle_prefixes)
        w = np.arange(len(ref)) % 5 + 1
        expect = sum(int(c) * int(x) for c, x in zip(ref, w)) * oracle.multiplier(n, D)
        for sh in (dict(), dict(kernel=1)):
            rc, res = emulated.count("weighted", n, D, wl.order, wl.prefixes, **sh)
            assert rc == 0 and (res[0] == ref).all(), (n, sh)
            assert emulated.last_total128 == expect, (n, sh)


@pytest.mark.parametrize("n,after,step", [(7, 14, 7), (6, 5, 1)])
def test_stack_cap_defers_and_recounts(dls, emulated, n, after, step):
    """A stack cap far below the bound: lanes that would outgrow it defer
    their prefix, the recount pass counts those again with the full bound,
    and every count and the total are the oracle's (plans, both host-buffer
    entries, the weighted total; the batched and the plain snapshot
    kernels).  describe reports the cap."""
    wl = every(gpu_cases.split(dls, n, D, after), step)
    ref, _ = oracle.count_many(n, D, wl.oracle_order, wl.oracle_prefixes)
    P = len(ref)
    for sh in (dict(stack_cap=2), dict(stack_cap=1, block_threads=32),
               dict(kernel=1, stack_cap=2)):
        rc, info = emulated.count("describe", n, D, wl.order, wl.prefixes, **sh)
        assert rc == 0 and info["stack_entries"] == sh["stack_cap"], sh
        rc, res = emulated.count("plan", n, D, wl.order, wl.prefixes, **sh)
        assert rc == 0 and emulated.last_status == (0, P), sh
        assert (res[0] == ref).all() and res[1] == int(ref.sum()), sh
        for entry in ("host", "noalloc"):
            rc, res = emulated.count(entry, n, D, wl.order, wl.prefixes, **sh)
            assert rc == 0 and (res[0] == ref).all(), (entry, sh)
        rc, res = emulated.count("weighted", n, D, wl.order, wl.prefixes, **sh)
        w = np.arange(P) % 5 + 1
        assert rc == 0 and (res[0] == ref).all()
        assert emulated.last_total128 == sum(int(c) * int(x) for c, x in zip(ref, w)) * \
            oracle.multiplier(n, D)


def test_abort_flag(dls, emulated):
    """A set abort flag stops the count before any prefix is finished
    (DLS_ERR_ABORTED); a flag that stays clear changes nothing."""
    wl = every(gpu_cases.split(dls, 7, D, 14), 7)
    ref, _ = oracle.count_many(7, D, wl.oracle_order, wl.oracle_prefixes)
    P = len(wl.prefixes)
    for sh in (dict(), dict(kernel=1), dict(stack=1)):
        rc, res = emulated.count("count", 7, D, wl.order, wl.prefixes, abort=1, **sh)
        assert rc == 0 and emulated.last_status[0] == ERR_ABORTED, sh
        c = res[0]
        assert ((c == 0) | ((c & UNFINISHED) != 0)).all()
        rc, res = emulated.count("count", 7, D, wl.order, wl.prefixes, abort=2, **sh)
        assert rc == 0 and emulated.last_status == (0, P) and (res[0] == ref).all(), sh
        rc, _ = emulated.count("plan", 7, D, wl.order, wl.prefixes, abort=1, **sh)
        assert rc == 0 and emulated.last_status[0] == ERR_ABORTED
        rc, _ = emulated.count("host", 7, D, wl.order, wl.prefixes, abort=1, **sh)
        assert rc == ERR_ABORTED


def test_describe_launch_and_argument_errors(dls, emulated):
    o8 = dls.fill_order(8, D)
    p8 = np.zeros((10, 15), np.uint8)
    rc, d = emulated.count("describe", 8, D, o8, p8)
    assert rc == 0 and d["run"] == 2 and d["words"] == 2 and d["stack_entries"] > 0
    assert d["fused"] == 0  # diagonal cells remain after depth 15
    rc, d = emulated.count("describe", 8, D, o8, np.zeros((10, 28), np.uint8))
    assert rc == 0 and d["fused"] == 1  # both diagonals inside the prefix
    rc, d = emulated.count("describe", 8, D, o8, p8, kernel=1)
    assert rc == 0 and d["run"] == 3
    rc, d = emulated.count("describe", 8, D, o8, p8, stack=1)
    assert rc == 0 and d["run"] == 0 and d["stack_entries"] == 0
    # order 9: the wide words where at most 8 rows have cells after the
    # prefix (row 0 inside it), else the per-position search
    o9 = dls.fill_order(9, D)
    rc, d = emulated.count("describe", 9, D, o9, np.zeros((10, 17), np.uint8))
    assert rc == 0 and d["run"] == 2 and d["words"] == 2 and d["step"] == 3
    rc, d = emulated.count("describe", 9, D, o9, np.zeros((10, 5), np.uint8))
    assert rc == 0 and d["run"] == 0 and d["words"] == 1
    rc, d = emulated.count("describe", 9, D, o9, np.zeros((10, 17), np.uint8), words=1)
    assert rc == 0 and d["run"] == 0 and d["words"] == 1
    for n, order, depth, sh in (
            (9, o9, 5, dict(stack=2)), (8, o8, 15, dict(stack=2, words=1)),
            (8, o8, 15, dict(stack=2, lanes_per_prefix=2)), (8, o8, 15, dict(stack=3)),
            (8, o8, 15, dict(fuse=1)), (8, o8, 15, dict(lookahead=1)),
            (8, o8, 28, dict(fuse=1, lookahead=1)), (8, o8, 28, dict(fuse=2)),
            (8, o8, 15, dict(block_threads=48)), (8, o8, 15, dict(lanes_per_prefix=3)),
            (9, o9, 17, dict(words=2, stack=1)), (8, o8, 15, dict(check_every=3))):
        rc, _ = emulated.count("count", n, D, order, np.zeros((4, depth), np.uint8), **sh)
        assert rc == ERR_BAD_ARG, (n, depth, sh)


def test_edge_cases(dls, emulated):
    """The GPU edge-case test's inputs, with several launch shapes: an empty
    batch, whole squares as prefixes, one cell left, invalid prefixes,
    orders 1 to 3, odd vertically symmetric orders and order 16 with every
    mask bit in use."""
    from oracle import orders
    shapes = (dict(), dict(stack=1), dict(kernel=1), dict(block_threads=32, check_every=1))

    def counts(n, flags, order, pre, sh):
        rc, res = emulated.count("count", n, flags, order, pre, **sh)
        assert rc == 0, (n, sh)
        return res[0]

    order = dls.fill_order(6, D)
    o_order = orders.md_ad_rows(6)
    ident = np.array([orders.identity(6)], np.uint8)
    full, _ = oracle.extend(6, D, o_order, ident, 36)
    bad = full[:5].copy()
    bad[:, 20] = (bad[:, 20] + 1) % 6
    ok, _ = oracle.extend(6, D, o_order, ident, 10)
    inval = ok[:40].copy()
    inval[::2, 7] = 9
    inval[1::2, 9] = inval[1::2, 8]
    o16 = [(0, j) for j in range(16)] + [(1, 1), (1, 14), (2, 2), (15, 0), (15, 15), (3, 5)]
    ref16 = oracle.count(16, D, o16, list(range(16)))[0]
    for sh in shapes:
        assert len(counts(6, D, order, np.zeros((0, 6), np.uint8), sh)) == 0
        pre = np.concatenate([full, bad])
        c = counts(6, D, order, pre, sh)
        assert (c == oracle.count_many(6, D, o_order, pre)[0]).all() and c[:128].sum() == 128
        assert (counts(6, D, order, full[:, :35], sh) == 1).all()
        pre = np.concatenate([ok[:40], inval])
        c = counts(6, D, order, pre, sh)
        assert (c == oracle.count_many(6, D, o_order, pre)[0]).all() and (c[40:] == 0).all()
        assert counts(1, D, [(0, 0)], np.zeros((1, 0), np.uint8), sh)[0] == 1
        for n in (2, 3):
            o = dls.fill_order(n, D)
            assert counts(n, D, o, np.arange(n, dtype=np.uint8)[None], sh)[0] == 0
        for n in (5, 7):
            o = dls.fill_order(n, D | V)
            assert counts(n, D | V, o, np.arange(n // 2, dtype=np.uint8)[None], sh)[0] == 0
        c = counts(16, D, o16, np.arange(16, dtype=np.uint8)[None], sh)
        assert c[0] == ref16, sh


def test_bench_configuration_sample(dls, emulated):
    """The benchmark's launch as the autotuner chose it on the GB300 (split
    depth 25, squared-count order after the split, fused step, blocks of
    64) on every 100th prefix of one of its 64 diagonal fillings."""
    import dls_inputs
    from oracle import orders
    from paper_1709_02599_gb300 import autotune
    n, depth = 8, 25
    order0 = dls.fill_order(n, D)
    ident = np.arange(n, dtype=np.uint8)[None]
    diags, _ = dls.extend_prefixes(n, D, order0, ident, n + (n - 1))
    pick = dls_inputs.choose(len(diags), 64, 0)[dls_inputs.choose(64, 1, 3)]
    order, pre, _ = autotune.build_problem(n, D, order0, diags[pick], depth, "heuristic_sq")
    o_order = orders.heuristic_complete(n, orders.md_ad_rows(n)[:depth], squares=True)
    o_diags, _ = oracle.extend(n, D, orders.md_ad_rows(n),
                               np.array([orders.identity(n)], np.uint8), n + (n - 1))
    o_pre, _ = oracle.extend(n, D, o_order, o_diags[pick], depth)
    # the benchmark's order drops the tail run: the oracle runs the same
    # (shortened) order, so node counts compare too
    o_order = orders.trim_tail(n, o_order, depth)
    assert [tuple(map(int, c)) for c in order] == o_order
    wl = every(gpu_cases.Workload(n, D, order, pre, o_order, o_pre), 100)
    rc, info = emulated.count("describe", n, D, wl.order, wl.prefixes, block_threads=64)
    assert rc == 0 and info["run"] == 2 and info["fused"] == 1
    check_counts(emulated, wl, n, D, [dict(block_threads=64), dict(block_threads=64, fuse=-1),
                                      dict(kernel=1, block_threads=64)])
