"""CPU tests of the library's kernels and launch code.

dls_kernels.cu is built with the host compiler against a stand-in CUDA
runtime (tests/host_kernels). In it, every CUDA thread is a cooperative
fiber, warp votes and shuffles complete once all lanes of the warp reach
them, and all blocks of a grid interleave at those points. The kernels then
run through the library's own C entry points: dls_count_ex, dls_count_host,
the CUDA-graph plans and dls_describe_launch. Two source-level substitutions
are made in a temporary copy, because the host compiler has no
__shared__:
- the dynamic shared array becomes a per-block buffer;
- each static shared array becomes a per-block buffer too.

What this checks, against the oracle (which shares no code with it):
- the per-prefix counts, the total and the node count for every launch
  shape of the persistent and plain kernels: snapshot and per-position
  stacks, register and shared-memory words, lane splits, donation on and off
  and at every iteration, lookahead and fused step, several blocks sharing
  the queue;
- the host-buffer entry and plans replayed twice;
- the launch descriptions and the argument errors, which otherwise need a
  GPU.

The GPU tests remain the parity tests proper; this catches mistakes in the
kernels' warp-level logic on any machine."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import gpu_cases
import oracle

D, V = 1, 2
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1709_02599_gb300", "csrc")
HK = os.path.join(HERE, "host_kernels")
FIELDS = ["kernel", "block_threads", "blocks_per_sm", "lanes_per_prefix", "split_pos",
          "donate", "check_every", "words", "stack", "lookahead", "fuse"]
ERR_BAD_ARG = 3


def host_kernel_source(text):
    """The kernel source with its shared arrays turned into per-block
    buffers of the stand-in runtime, and the stand-in launch appended."""
    text = text.replace("extern __shared__ uint32_t smem[];",
                        "uint32_t *smem = static_cast<uint32_t *>(::shim::dynamic_smem());")
    pat = re.compile(r"__shared__\s+([A-Za-z_][\w ]*?)\s+(\w+)\[(\d+)\];")
    lines = text.split("\n")
    for k, line in enumerate(lines):
        m = pat.search(line)
        if m:
            t, name, count = m.groups()
            lines[k] = (line[:m.start()] + "%s *%s = static_cast<%s *>(::shim::block_shared("
                        "sizeof(%s) * %s, %d));" % (t, name, t, t, count, k) + line[m.end():])
    text = "\n".join(lines) + '\n#include "launch_kparams.inc"\n'
    assert "__shared__" not in text
    return text


@pytest.fixture(scope="module")
def kernel_check(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("host_kernels")
    src = d / "dls_kernels_host.cpp"
    with open(os.path.join(CSRC, "dls_kernels.cu")) as f:
        src.write_text(host_kernel_source(f.read()))
    exe = str(d / "kernel_check")
    r = subprocess.run([gxx, "-O1", "-std=c++17", "-w", "-I", HK,
                        "-I", os.path.join(HERE, "host_step"), "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src),
                        os.path.join(CSRC, "dls_host.cpp"), os.path.join(HK, "simt.cpp"),
                        os.path.join(HK, "kernel_check.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe, d


def run(kc, entry, n, flags, order, prefixes, **launch):
    exe, d = kc
    prefixes = np.ascontiguousarray(prefixes, dtype=np.uint8)
    np.ascontiguousarray(order, dtype=np.uint8).tofile(d / "order.bin")
    prefixes.tofile(d / "prefixes.bin")
    depth = prefixes.shape[1] if prefixes.ndim == 2 else 0
    r = subprocess.run([exe, entry, str(n), str(flags), str(d / "order.bin"),
                        str(d / "prefixes.bin"), str(depth)]
                       + [str(launch.get(k, 0)) for k in FIELDS],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    lines = r.stdout.split("\n")
    rc = int(lines[0].split()[1])
    if rc != 0:
        return rc, None
    if entry == "describe":
        keys = ["run", "words", "block_threads", "grid_blocks", "smem_bytes", "stack_entries",
                "fused"]
        return 0, dict(zip(keys, map(int, lines[1].split())))
    head = lines[1].split()
    total, nodes = int(head[1]), int(head[3])
    counts = np.array([int(x) for x in lines[2:] if x.strip()], dtype=np.uint64)
    return 0, (counts, total, nodes)


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


def check_counts(kc, wl, n, flags, shapes, nodes_exact=True):
    ref_c, ref_n = oracle.count_many(n, flags, wl.oracle_order, wl.oracle_prefixes, threads=4)
    for sh in shapes:
        rc, res = run(kc, "count", n, flags, wl.order, wl.prefixes, **sh)
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
def test_kernels_against_oracle(dls, kernel_check, n, flags, after, kind, step):
    k = {None: None, "heuristic": dls.ORDER_HEURISTIC}[kind]
    wl = every(gpu_cases.split(dls, n, flags, after, kind=k), step)
    shapes = SHAPES + [dict(sh, kernel=1) for sh in SHAPES if "check_every" not in sh
                       and "donate" not in sh and "blocks_per_sm" not in sh]
    check_counts(kernel_check, wl, n, flags, shapes)


def test_lookahead_and_fused_step(dls, kernel_check):
    """Where no cell after the prefix lies on a diagonal and without vertical
    symmetry: the lookahead prunes (fewer nodes, same counts); the fused step
    keeps the counts and the nodes."""
    for n, flags, after, kind, step in ((7, D, 14, dls.ORDER_HEURISTIC, 30),
                                        (6, 0, 8, None, 1000), (5, 0, 4, None, 1)):
        wl = every(gpu_cases.split(dls, n, flags, after, kind=kind), step)
        check_counts(kernel_check, wl, n, flags,
                     [dict(fuse=1), dict(fuse=1, kernel=1), dict(fuse=1, block_threads=32,
                                                                 check_every=1)])
        check_counts(kernel_check, wl, n, flags,
                     [dict(lookahead=1), dict(lookahead=1, block_threads=32, check_every=1)],
                     nodes_exact=False)


def test_larger_orders_from_sampled_partial_squares(dls, kernel_check):
    """Orders 9, 10 (symmetric) and 12 (symmetric): shared-memory words, and
    register fields for symmetric order 10, through the per-position
    kernels."""
    for n, flags, rows in ((9, D, 4), (10, D | V, 5), (12, D | V, 7), (9, 0, 6)):
        wl = gpu_cases.sampled_rows(dls, n, flags, rows)
        check_counts(kernel_check, wl, n, flags,
                     [dict(), dict(words=1), dict(lanes_per_prefix=8), dict(kernel=1),
                      dict(block_threads=32, check_every=1)])


def test_queue_shared_by_many_blocks(dls, kernel_check):
    """Many prefixes, small blocks, several blocks per multiprocessor: the
    blocks take items from one queue in turns."""
    wl = every(gpu_cases.split(dls, 7, D, 11, kind=dls.ORDER_HEURISTIC), 8)
    assert len(wl.prefixes) > 7 * 32
    rc, info = run(kernel_check, "describe", 7, D, wl.order, wl.prefixes, block_threads=32,
                   blocks_per_sm=4)
    assert rc == 0 and info["grid_blocks"] == 8
    check_counts(kernel_check, wl, 7, D, [dict(block_threads=32, blocks_per_sm=4),
                                          dict(block_threads=32, blocks_per_sm=4, stack=1)])


def test_host_buffer_entry_and_plans(dls, kernel_check):
    wl = gpu_cases.split(dls, 6, D, 5)
    ref_c, _ = oracle.count_many(6, D, wl.oracle_order, wl.oracle_prefixes)
    for sh in (dict(), dict(stack=1), dict(kernel=1), dict(lanes_per_prefix=4)):
        rc, (c, total, _) = run(kernel_check, "host", 6, D, wl.order, wl.prefixes, **sh)
        assert rc == 0 and (c == ref_c).all(), sh
        assert total == int(ref_c.sum()), sh  # the plain 128-bit sum
        rc, (c, total, _) = run(kernel_check, "plan", 6, D, wl.order, wl.prefixes, **sh)
        assert rc == 0 and (c == ref_c).all() and total == int(ref_c.sum()), sh


def test_describe_launch_and_argument_errors(dls, kernel_check):
    o8 = dls.fill_order(8, D)
    p8 = np.zeros((10, 15), np.uint8)
    rc, d = run(kernel_check, "describe", 8, D, o8, p8)
    assert rc == 0 and d["run"] == 2 and d["words"] == 2 and d["stack_entries"] > 0
    assert d["fused"] == 0  # diagonal cells remain after depth 15
    rc, d = run(kernel_check, "describe", 8, D, o8, np.zeros((10, 28), np.uint8))
    assert rc == 0 and d["fused"] == 1  # both diagonals inside the prefix
    rc, d = run(kernel_check, "describe", 8, D, o8, p8, kernel=1)
    assert rc == 0 and d["run"] == 3
    rc, d = run(kernel_check, "describe", 8, D, o8, p8, stack=1)
    assert rc == 0 and d["run"] == 0 and d["stack_entries"] == 0
    o9 = dls.fill_order(9, D)
    rc, d = run(kernel_check, "describe", 9, D, o9, np.zeros((10, 17), np.uint8))
    assert rc == 0 and d["run"] == 0 and d["words"] == 1
    for n, order, depth, sh in (
            (9, o9, 17, dict(stack=2)), (8, o8, 15, dict(stack=2, words=1)),
            (8, o8, 15, dict(stack=2, lanes_per_prefix=2)), (8, o8, 15, dict(stack=3)),
            (8, o8, 15, dict(fuse=1)), (8, o8, 15, dict(lookahead=1)),
            (8, o8, 28, dict(fuse=1, lookahead=1)), (8, o8, 28, dict(fuse=2)),
            (8, o8, 15, dict(block_threads=48)), (8, o8, 15, dict(lanes_per_prefix=3)),
            (9, o9, 17, dict(words=2)), (8, o8, 15, dict(check_every=3))):
        rc, _ = run(kernel_check, "count", n, D, order, np.zeros((4, depth), np.uint8), **sh)
        assert rc == ERR_BAD_ARG, (n, depth, sh)
