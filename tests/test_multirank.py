"""The multi-rank path on CPU: world size 2 over gloo.  Each rank counts its
slice of the prefixes (here with the oracle, standing in for its GPU) and the
exact total is reduced across ranks; a rank that fails is seen by the other
through the process group, not by a hang."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import orders

D = 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path, fail_rank):
    import datetime
    import torch.distributed as dist
    from paper_1709_02599_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    n = 7
    o = orders.md_ad_rows(n)
    pre, _ = oracle.extend(n, D, o, np.array([orders.identity(n)], np.uint8), n + 8)
    if rank == fail_rank:
        # leaves between steps, before its collective: the peer must not hang
        os._exit(3)
    try:
        idx, local, total = shard.count_sharded(
            lambda p: oracle.count_many(n, D, o, p, threads=2)[0], pre, rank, world)
        big = shard.allreduce_total((1 << 63) + rank)   # beyond int64
        np.save(out_path % rank, np.array([total, len(idx), int(local.sum()),
                                           big >> 32, big & 0xFFFFFFFF], dtype=object),
                allow_pickle=True)
    except Exception as e:  # the surviving rank reports the failure
        np.save(out_path % rank, np.array(["error", repr(e)], dtype=object), allow_pickle=True)
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_shards_partition_the_batch():
    from paper_1709_02599_gb300 import shard
    for n_items in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            for mode in ("interleave", "block"):
                parts = [shard.shard_indices(n_items, r, world, mode) for r in range(world)]
                allidx = np.concatenate(parts) if parts else np.zeros(0)
                assert sorted(allidx.tolist()) == list(range(n_items))


def test_two_ranks_gloo_total(tmp_path):
    world = 2
    port = _free_port()
    out = str(tmp_path / "r%d.npy")
    mp.start_processes(_worker, args=(world, port, out, -1), nprocs=world, join=True,
                       start_method="spawn")
    n = 7
    o = orders.md_ad_rows(n)
    ref = oracle.count(n, D, o, orders.identity(n))[0]
    res = [np.load(out % r, allow_pickle=True) for r in range(world)]
    assert all(int(r[0]) == ref for r in res)
    pre, _ = oracle.extend(n, D, o, np.array([orders.identity(n)], np.uint8), n + 8)
    assert sum(int(r[1]) for r in res) == len(pre)
    assert sum(int(r[2]) for r in res) == ref
    big = (int(res[0][3]) << 32) | int(res[0][4])
    assert big == (1 << 64) + 1


def test_failed_rank_is_detected_not_hung(tmp_path):
    world = 2
    port = _free_port()
    out = str(tmp_path / "r%d.npy")
    ctx = mp.start_processes(_worker, args=(world, port, out, 1), nprocs=world, join=False,
                             start_method="spawn")
    ok = False
    for _ in range(120):
        try:
            if ctx.join(timeout=1):
                break
        except mp.ProcessExitedException:
            ok = True
            break
    for p in ctx.processes:
        if p.is_alive():
            p.join(timeout=60)
    assert ok or any(p.exitcode == 3 for p in ctx.processes)
    # the survivor recorded the error instead of a result (or exited)
    r0 = out % 0
    if os.path.exists(r0):
        rec = np.load(r0, allow_pickle=True)
        assert rec[0] == "error"


def _bench_worker(rank, world, port, out_path):
    """bench.py's rank logic for --scaling strong, the oracle standing in for
    each rank's GPU: rank 0's choice is broadcast, each rank counts its
    interleaved share of the one problem, the total is reduced exactly, and
    rank 0 checks its rows of the chosen diagonals against the oracle."""
    import datetime
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        spec = bench.SPECS["dls8_diag64"]
        units = 4
        mine = (28, "heuristic_sq", {}) if rank == 0 else (31, "given", {"block_threads": 32})
        depth, suffix, cfg = bench.agree_on_choice(mine, world, "strong")
        o_order, pre, par = spec.oracle_sample(0, units, np.arange(units), depth, suffix)
        share = bench.rank_share(len(pre), rank, world, "strong")
        local, _ = oracle.count_many(spec.n, spec.flags, o_order, pre[share], threads=2)
        total = bench.reduce_squares(int(local.sum()), world)
        checked = None
        if rank == 0:
            chk, _, _ = bench.oracle_check(spec, 0, units, depth, suffix, pre[share],
                                           par[share], local, 2, share, par)
            checked = chk["agree"]
        np.save(out_path % rank, np.array([depth, suffix, len(share), total, checked],
                                          dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_bench_strong_scaling_rank_logic(tmp_path):
    world = 2
    port = _free_port()
    out = str(tmp_path / "b%d.npy")
    mp.start_processes(_bench_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    import bench
    spec = bench.SPECS["dls8_diag64"]
    o_order, pre, _ = spec.oracle_sample(0, 4, np.arange(4), 28, "heuristic_sq")
    ref, _ = oracle.count_many(spec.n, spec.flags, o_order, pre, threads=4)
    res = [np.load(out % r, allow_pickle=True) for r in range(world)]
    assert all(int(r[0]) == 28 and r[1] == "heuristic_sq" for r in res)   # rank 0's choice
    assert sum(int(r[2]) for r in res) == len(pre)
    assert all(int(r[3]) == int(ref.sum()) for r in res)
    assert res[0][4] is True
