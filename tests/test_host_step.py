"""CPU tests of the kernels' snapshot search step.

snap_step (dls_snapshot.cuh), the step that k_snapshot and k_plain_snap run
on every lane, is compiled for the host with a shim of the few CUDA builtins
it uses (tests/host_step). It then runs on one lane per prefix, with no
warp and no donation. For each workload and each variant of the step
(plain, diagonal words, vertical symmetry, lookahead, fused), these are
checked against the oracle, which shares no code with it:
- per-prefix completion counts, bit for bit;
- node counts: equal to the oracle's, except the lookahead, which prunes;
- every step leaves the lane at a valid position, with the stack within the
  kernel's bound. Each stack slot starts as 0xff bytes, so a read of a stale
  slot shows.

The bound is restated here from its rule: a position after the prefix whose
cell lies on a line with all other cells earlier in the order has at most
one candidate and never makes an entry."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import gpu_cases
import oracle
from oracle import orders

D, V = 1, 2
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1709_02599_gb300", "csrc")


@pytest.fixture(scope="module")
def step_check(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    exe = str(tmp_path_factory.mktemp("host_step") / "step_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(HERE, "host_step"), "-I", CSRC,
                    "-o", exe, os.path.join(HERE, "host_step", "step_check.cpp")],
                   check=True, capture_output=True, text=True)
    return exe


def entry_bound(order, n, flags, depth):
    """Positions from depth to the one before the last whose cell is not the
    last open cell of a row, a column or (with the diagonal flag) a
    diagonal; with vertical symmetry (left-half cells) only columns and the
    diagonal line -- the n left cells on either diagonal -- force a cell."""
    diag, vsym = bool(flags & D), bool(flags & V)
    rowc, colc = [0] * n, [0] * n
    mdc = adc = dline = 0
    bound = 0
    for t in range(len(order) - 1):
        i, j = int(order[t][0]), int(order[t][1])
        md, ad = diag and i == j, diag and i + j == n - 1
        if vsym:
            forced = colc[j] == n - 1 or ((md or ad) and dline == n - 1)
        else:
            forced = (rowc[i] == n - 1 or colc[j] == n - 1 or (md and mdc == n - 1)
                      or (ad and adc == n - 1))
        if t >= depth and not forced:
            bound += 1
        rowc[i] += 1
        colc[j] += 1
        mdc += md
        adc += ad
        dline += md or ad
    return max(1, bound)


def run_step(exe, tmp_path, n, flags, mode, order, prefixes, depth, cap, split=None):
    ob = tmp_path / "order.bin"
    pb = tmp_path / "prefixes.bin"
    np.ascontiguousarray(order, dtype=np.uint8).tofile(ob)
    np.ascontiguousarray(prefixes, dtype=np.uint8).tofile(pb)
    extra = [str(x) for x in split] if split else []
    r = subprocess.run([exe, str(n), str(flags), str(mode), str(ob), str(pb), str(depth),
                        str(cap)] + extra, capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    out = np.array([[int(x) for x in line.split()] for line in r.stdout.splitlines()],
                   dtype=np.uint64).reshape(-1, 2)
    stats = r.stderr.split()
    info = {stats[k]: int(stats[k + 1]) for k in range(0, len(stats), 2)}
    return out[:, 0], out[:, 1], info


def check_workload(exe, tmp_path, wl, n, flags):
    depth = wl.prefixes.shape[1]
    ref_c, ref_n = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes, threads=4)
    cap = entry_bound(wl.order, n, flags, depth)
    diag_after = bool(flags & D) and any(int(i) == int(j) or int(i) + int(j) == n - 1
                                         for i, j in wl.order[depth:])
    modes = [0] if diag_after else ([0, 2] if flags & V else [0, 1, 2])
    iters = {}
    for mode in modes:
        c, nd, info = run_step(exe, tmp_path, n, flags, mode, wl.order, wl.prefixes, depth, cap)
        assert (c == ref_c).all(), (n, flags, mode)
        if mode == 1:
            assert (nd <= ref_n).all()
        else:
            assert (nd == ref_n).all(), (n, flags, mode)
        assert info["badpos"] == 0 and info["overflow"] == 0, info
        assert info["maxsp"] <= cap, (info, cap)
        iters[mode] = info["iters"]
    if 2 in iters:
        assert iters[2] <= iters[0]
    return iters


@pytest.mark.parametrize("n,flags,after,kind", [
    (4, D, 0, None), (5, D, 3, None), (5, 0, 4, None), (6, D, 5, None), (6, D, 9, None),
    (6, D | V, 2, None), (7, D, 4, None), (7, D, 14, None), (6, D, 12, None),
    (6, V, 0, None),
    (7, D, 14, "heuristic"), (6, D, 10, "heuristic"), (7, D, 11, "heuristic"),
    (8, D | V, 8, "heuristic"), (6, D, 0, "row_major"), (6, 0, 3, "row_major")])
def test_step_against_oracle(dls, step_check, tmp_path, n, flags, after, kind):
    k = {None: None, "heuristic": dls.ORDER_HEURISTIC, "row_major": dls.ORDER_ROW_MAJOR}[kind]
    wl = gpu_cases.split(dls, n, flags, after, kind=k)
    check_workload(step_check, tmp_path, wl, n, flags)


@pytest.mark.parametrize("n,flags,after,kind", [
    (6, D | V, 2, None), (6, V, 0, None), (8, D | V, 8, "heuristic"), (7, D, 14, "heuristic"),
    (6, D, 10, "heuristic"), (6, 0, 3, "row_major"), (7, D, 4, None)])
def test_step_on_trimmed_orders(dls, step_check, tmp_path, n, flags, after, kind):
    """Orders shortened by dls_order_trim (the oracle runs its own trim_tail
    of its order, so node counts compare too); the counts must also be those
    of the whole order."""
    k = {None: None, "heuristic": dls.ORDER_HEURISTIC, "row_major": dls.ORDER_ROW_MAJOR}[kind]
    wl = gpu_cases.split(dls, n, flags, after, kind=k, trim=True)
    full = gpu_cases.split(dls, n, flags, after, kind=k)
    assert len(wl.order) < len(full.order) and (wl.prefixes == full.prefixes).all()
    check_workload(step_check, tmp_path, wl, n, flags)
    c_trim, _ = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes, threads=4)
    c_full, _ = oracle.count_many(n, flags, full.oracle_order, full.oracle_prefixes, threads=4)
    assert (c_trim == c_full).all()


@pytest.mark.parametrize("n,k,depth", [(6, 15, 8), (6, 20, 9), (7, 18, 9), (5, 12, 5)])
def test_step_on_partial_orders(dls, step_check, tmp_path, n, k, depth):
    """Partial orders (the first k row-major cells, as for Section 5.3's
    partial counts): the last cell can have several candidates."""
    order = dls.fill_order(n, 0, dls.ORDER_ROW_MAJOR)[:k]
    o_order = [tuple(map(int, c)) for c in order]
    base = np.arange(n, dtype=np.uint8)[None]
    pre, _ = dls.extend_prefixes(n, 0, order, base, depth)
    o_pre, _ = oracle.extend(n, 0, o_order, base, depth)
    wl = gpu_cases.Workload(n, 0, order, pre, o_order, o_pre)
    check_workload(step_check, tmp_path, wl, n, 0)


@pytest.mark.parametrize("flags", [D, 0])
def test_wide_step_on_order9(dls, step_check, tmp_path, flags):
    """Order 9 (the wide words: values 0-7 in byte slots, value 8 a bit of
    its own) on random partial squares: 4 and 5 rows filled (5 and 6 for
    ordinary squares; with the diagonal flag the diagonals are searched),
    and 4 rows plus the rest of both diagonals (every step mode: plain,
    lookahead, fused)."""
    for rows in ((4, 5) if flags & D else (5, 6)):
        wl = gpu_cases.sampled_rows(dls, 9, flags, rows, count=4)
        check_workload(step_check, tmp_path, wl, 9, flags)
    if flags & D:
        wl = gpu_cases.sampled_rows(dls, 9, D, 4, count=4)
        # the diagonal cells of rows 4-8 follow the filled rows in the order
        diag = sum(1 for i, j in wl.oracle_order[wl.depth:] if i == j or i + j == 8)
        depth = wl.depth + diag
        pre, _ = dls.extend_prefixes(9, D, wl.order, wl.prefixes, depth)
        o_pre, _ = oracle.extend(9, D, wl.oracle_order, wl.oracle_prefixes, depth)
        wl2 = gpu_cases.Workload(9, D, wl.order, pre, wl.oracle_order, o_pre, depth=depth)
        iters = check_workload(step_check, tmp_path, wl2, 9, D)
        assert set(iters) == {0, 1, 2}
        # the same on orders shortened by dls_order_trim (the oracle runs its
        # own trim_tail of its order; counts also equal the whole order's)
        t = dls.order_trim(9, D, wl.order, depth)
        o_t = orders.trim_tail(9, wl.oracle_order, depth)
        assert [tuple(map(int, c)) for c in t] == o_t and len(t) < len(wl.order)
        wl3 = gpu_cases.Workload(9, D, t, pre, o_t, o_pre, depth=depth)
        check_workload(step_check, tmp_path, wl3, 9, D)
        c_t, _ = oracle.count_many(9, D, o_t, o_pre, threads=4)
        c_f, _ = oracle.count_many(9, D, wl.oracle_order, o_pre, threads=4)
        assert (c_t == c_f).all()


def test_step_on_one_diagonal_of_the_order8_workload(dls, step_check, tmp_path):
    """One of the 64 diagonal fillings of the order-8 benchmark workload,
    split at depth 25 with the squared-count order after the split (the
    benchmark's configuration): the fused step needs far fewer iterations."""
    import dls_inputs
    from oracle import orders
    from paper_1709_02599_gb300 import autotune
    n, depth = 8, 25
    order0 = dls.fill_order(n, D)
    ident = np.arange(n, dtype=np.uint8)[None]
    diags, _ = dls.extend_prefixes(n, D, order0, ident, n + (n - 1))
    pick = dls_inputs.choose(len(diags), 1, 5)
    order, pre, _ = autotune.build_problem(n, D, order0, diags[pick], depth, "heuristic_sq")
    o_order = orders.heuristic_complete(n, orders.md_ad_rows(n)[:depth], squares=True)
    o_diags, _ = oracle.extend(n, D, orders.md_ad_rows(n), np.array([orders.identity(n)],
                                                                    np.uint8), n + (n - 1))
    o_pre, _ = oracle.extend(n, D, o_order, o_diags[pick], depth)
    # the benchmark's order drops the tail run: the oracle runs the same
    # (shortened) order, so node counts compare too
    o_order = orders.trim_tail(n, o_order, depth)
    assert [tuple(map(int, c)) for c in order] == o_order
    wl = gpu_cases.Workload(n, D, order, pre, o_order, o_pre)
    iters = check_workload(step_check, tmp_path, wl, n, D)
    assert set(iters) == {0, 1, 2}
    assert iters[2] < 0.75 * iters[0], iters


# ------------------------------------------------ the per-position step --
# dfs_step (dls_search.cuh): k_persistent and k_plain (orders above 8, lane
# splits, shared-memory words) and, with the symmetry flag taken at run
# time, the serving kernel.


def check_position_step(exe, tmp_path, wl, n, flags):
    depth = wl.prefixes.shape[1]
    ref_c, ref_n = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes, threads=4)
    fits = n * (n // 2) <= 64 if flags & V else n <= 8
    splits = [None]
    if depth + 2 <= len(wl.order) - 2:
        splits += [(2, depth + 2), (3, min(depth + 5, len(wl.order) - 2))]
    ran = 0
    for mode in ([10] if fits else []) + [11, 12]:
        for split in splits:
            c, nd, info = run_step(exe, tmp_path, n, flags, mode, wl.order, wl.prefixes, depth,
                                   1, split)
            assert (c == ref_c).all(), (n, flags, mode, split)
            assert (nd == ref_n).all(), (n, flags, mode, split)
            assert info["badpos"] == 0, info
            assert info["maxsp"] <= len(wl.order) - 2 - depth, info
            ran += 1
    return ran


@pytest.mark.parametrize("n,flags,after", [(6, D, 5), (6, D | V, 2), (5, 0, 4), (6, D, 12),
                                           (6, V, 0)])
def test_position_step_against_oracle(dls, step_check, tmp_path, n, flags, after):
    wl = gpu_cases.split(dls, n, flags, after)
    assert check_position_step(step_check, tmp_path, wl, n, flags) >= 6


@pytest.mark.parametrize("n,flags,rows", [(9, D, 4), (10, D | V, 5), (12, D | V, 7), (9, 0, 6),
                                          (10, D, 5), (11, D, 6)])
def test_position_step_on_larger_orders(dls, step_check, tmp_path, n, flags, rows):
    """Orders above 8 from sampled partial squares: shared-memory words (and
    register fields for symmetric order 10).  Rows chosen so that some
    sampled squares have completions."""
    wl = gpu_cases.sampled_rows(dls, n, flags, rows)
    assert len(wl.prefixes) > 0
    ref, _ = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes, threads=4)
    assert int(ref.sum()) > 0
    check_position_step(step_check, tmp_path, wl, n, flags)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_steps_on_every_order_length_and_depth(dls, step_check, tmp_path, n):
    """Degenerate shapes: every prefix of the row-major order as a partial
    order (one cell up to the whole square), split at every depth from 0 to
    its length, with the plain and fused snapshot steps and the per-position
    step (orders 2 to 4 in full; order 5 at a few lengths)."""
    full = dls.fill_order(n, 0, dls.ORDER_ROW_MAJOR)
    lengths = range(1, len(full) + 1) if n < 5 else (1, 2, 6, 12, 19, 24, 25)
    for length in lengths:
        order = full[:length]
        o_order = [tuple(map(int, c)) for c in order]
        for depth in range(length + 1):
            pre, _ = dls.extend_prefixes(n, 0, order, np.zeros((1, 0), np.uint8), depth)
            if len(pre) == 0:
                continue
            pre = pre[::max(1, len(pre) // 200)]
            ref_c, ref_n = oracle.count_many(n, 0, o_order, pre)
            cap = entry_bound(order, n, 0, depth)
            for mode in (0, 2, 11):
                c, nd, info = run_step(step_check, tmp_path, n, 0, mode, order, pre, depth, cap)
                assert (c == ref_c).all() and (nd == ref_n).all(), (length, depth, mode)
                assert info["badpos"] == 0 and info["overflow"] == 0, (length, depth, mode)
