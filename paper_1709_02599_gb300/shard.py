"""Splitting a prefix batch over ranks (one process per GPU).

The prefixes of Section 5.2 are independent work units, so ranks take
disjoint slices and the only exchange is the sum of the per-rank totals --
one scalar, reduced exactly (two 32-bit halves of each 64-bit count, so any
total below 2^64 * world survives).  Nothing else crosses ranks.
"""
import numpy as np


def shard_indices(n_items, rank, world, mode="interleave"):
    """Indices of the units rank `rank` of `world` takes.  'interleave'
    deals units round-robin (neighbouring prefixes have similar cost, so this
    spreads cost evenly); 'block' gives contiguous ranges."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    if mode == "interleave":
        return np.arange(rank, n_items, world, dtype=np.int64)
    if mode == "block":
        lo = (n_items * rank) // world
        hi = (n_items * (rank + 1)) // world
        return np.arange(lo, hi, dtype=np.int64)
    raise ValueError("mode must be 'interleave' or 'block'")


def allreduce_total(local_total, group=None):
    """Exact sum over ranks of a non-negative integer below 2^64 (torch
    process group, any backend).  Returns a Python int."""
    import torch
    import torch.distributed as dist
    v = int(local_total)
    if v < 0 or v >= 1 << 64:
        raise ValueError("total out of range")
    parts = torch.tensor([v & 0xFFFFFFFF, v >> 32], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        parts = parts.cuda()
    dist.all_reduce(parts, group=group)
    lo, hi = (int(x) for x in parts.cpu().tolist())
    return lo + (hi << 32)


def count_sharded(count_fn, prefixes, rank, world, group=None, mode="interleave"):
    """Counts this rank's share of `prefixes` with count_fn (uint8 [P, d] ->
    uint64 [P]) and returns (indices, local counts, global total)."""
    idx = shard_indices(len(prefixes), rank, world, mode)
    local = np.asarray(count_fn(prefixes[idx]), dtype=np.uint64)
    total = allreduce_total(int(local.sum(dtype=np.uint64)), group)
    return idx, local, total
