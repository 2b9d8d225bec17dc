"""Workunits with a quorum and a checkpoint (Section 5.2).

Section 5.2 splits the order-9 search into independent workunits, one per
assignment of the first cells (the prefix split).  The paper ran them twice
over.  On the volunteer grid (Section 5.2.1) each workunit went to two hosts,
and a result counted only when the two copies agreed; otherwise two new
copies were issued.  On the cluster (Section 5.2.2) a control process kept
the pool of workunits and accumulated their results.

Here a workunit is a batch of consecutive prefixes, counted in one launch.

    res = run_workunits(n, flags, order, prefixes, "run.jsonl", batch=1 << 20,
                        quorum=(Launch(), Launch(kernel=KERNEL_PLAIN)))
    res["counts"], res["total"]

quorum: the launch shapes that each count every workunit.  With two or more
(the quorum of 2: for instance the batched kernel and the plain one, two
different code paths), the per-prefix counts of all of them must agree.  If
they do not, the whole quorum is counted again, up to max_rounds times.

The checkpoint is a JSON-lines file plus a sidecar file of counts
(`path` + ".counts", one uint64 per prefix).
- The first line names the problem: a digest of n, flags, the order, the
  prefixes and the batch size.  A run on another problem is refused.
- Each accepted workunit appends one line: its prefix range, the sum of its
  counts and a digest of its counts.  This happens after its counts are in
  the sidecar file.
- A restarted run skips the workunits whose lines and counts agree, and
  counts again any other one.  That covers a run killed at any point, a line
  cut short, and counts that do not match their line.  A line cut short at
  the end of the file is removed before new lines are appended.

Counting goes through `counter(prefixes, launch)`, which returns uint64
counts.  The default counts on the GPU through the library (dls_count_ex);
it needs CUDA.  Tests pass their own counter."""
import hashlib
import json
import os

import numpy as np

VERSION = 1


def _digest(*parts):
    h = hashlib.sha256()
    for p in parts:
        h.update(p if isinstance(p, bytes) else repr(p).encode())
    return h.hexdigest()


def gpu_counter(n, flags, order):
    """counter(prefixes, launch) on the GPU (the library's dls_count_ex)."""
    import torch

    from . import count

    def counter(prefixes, launch):
        t = torch.from_numpy(np.ascontiguousarray(prefixes, dtype=np.uint8)).cuda()
        c = count(n, flags, order, t, launch=launch)
        torch.cuda.synchronize()
        return c.cpu().numpy().astype(np.uint64)

    return counter


def _read_checkpoint(path, config):
    """Accepted workunit records {unit: record} of a checkpoint, or {} when
    there is none.  Raises ValueError if it belongs to another problem."""
    if not os.path.exists(path):
        return {}
    done = {}
    with open(path) as f:
        lines = f.read().split("\n")
    try:
        head = json.loads(lines[0])
    except (ValueError, IndexError):
        head = None
    if not head or head.get("kind") != "dls-workunits":
        raise ValueError("%s is not a workunit checkpoint" % path)
    if head.get("config") != config or head.get("version") != VERSION:
        raise ValueError("%s belongs to another problem" % path)
    for line in lines[1:]:
        try:
            rec = json.loads(line)
        except ValueError:
            continue  # a line cut short by an interrupted run
        if isinstance(rec, dict) and "unit" in rec:
            done[int(rec["unit"])] = rec
    return done


def _drop_torn_tail(path):
    """Cuts a line that an interrupted run left unfinished (no final newline)
    off the end of the checkpoint, so that the next record starts on a line
    of its own instead of being joined to the fragment and lost."""
    with open(path, "rb+") as f:
        data = f.read()
        if data and not data.endswith(b"\n"):
            f.truncate(data.rfind(b"\n") + 1)


def run_workunits(n, flags, order, prefixes, path, batch=1 << 20, quorum=None, counter=None,
                  max_rounds=3):
    """Counts every prefix (uint8 [P, depth]) through workunits of `batch`
    prefixes, checkpointed at `path`.  Returns a dict: 'counts' (uint64
    [P]), 'total' (exact int), 'units', 'units_counted' (this run),
    'units_resumed', 'disagreements' (quorum rounds that did not agree)."""
    from . import Launch

    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(-1, 2)
    prefixes = np.ascontiguousarray(prefixes, dtype=np.uint8)
    if prefixes.ndim != 2:
        raise ValueError("prefixes must be a [P, depth] array")
    if batch < 1 or max_rounds < 1:
        raise ValueError("batch and max_rounds must be positive")
    quorum = tuple(quorum) if quorum else (Launch(),)
    if counter is None:
        counter = gpu_counter(n, flags, order)
    P = len(prefixes)
    config = _digest(VERSION, int(n), int(flags), order.tobytes(), prefixes.shape,
                     prefixes.tobytes(), int(batch))
    done = _read_checkpoint(path, config)
    if not os.path.exists(path):
        with open(path, "w") as f:
            f.write(json.dumps({"kind": "dls-workunits", "version": VERSION, "config": config,
                                "n_prefixes": P, "batch": int(batch)}) + "\n")
    else:
        _drop_torn_tail(path)
    side = path + ".counts"
    if not os.path.exists(side) or os.path.getsize(side) != 8 * P:
        np.zeros(P, np.uint64).tofile(side)
    counts = np.memmap(side, dtype=np.uint64, mode="r+", shape=(P,)) if P else \
        np.zeros(0, np.uint64)
    units = (P + batch - 1) // batch
    counted = resumed = disagreements = 0
    for u in range(units):
        s, e = u * batch, min(P, (u + 1) * batch)
        rec = done.get(u)
        if (rec is not None and rec.get("start") == s and rec.get("stop") == e
                and rec.get("sha256") == _digest(np.asarray(counts[s:e]).tobytes())):
            resumed += 1
            continue
        for rounds in range(1, max_rounds + 1):
            got = [np.asarray(counter(prefixes[s:e], launch), dtype=np.uint64)
                   for launch in quorum]
            if all(g.shape == (e - s,) and (g == got[0]).all() for g in got):
                break
            disagreements += 1
        else:
            raise RuntimeError("workunit %d: the quorum did not agree in %d rounds"
                               % (u, max_rounds))
        counts[s:e] = got[0]
        if P:
            counts.flush()
        line = {"unit": u, "start": s, "stop": e, "sum": int(got[0].sum(dtype=object)),
                "sha256": _digest(got[0].tobytes()), "rounds": rounds}
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")
            f.flush()
            os.fsync(f.fileno())
        counted += 1
    out = np.array(counts, dtype=np.uint64)
    return {"counts": out, "total": int(sum(int(x) for x in out)), "units": units,
            "units_counted": counted, "units_resumed": resumed,
            "disagreements": disagreements}


def count_split(n, flags, depth, path, batch=1 << 20, quorum=1, counter=None,
                first_rows=1):
    """Section 5.2's run: row 0 fixed to 0..n-1, the cells after it in the
    Section 2.3 order (Fig. 1 for order 9), every valid assignment of the
    first `depth` cells one prefix, counted through run_workunits (quorum 2:
    the batched kernel and the plain per-position one).  Returns
    run_workunits' dict plus 'prefixes', 'row0_fixed' (the exact count with
    row 0 fixed) and 'squares' (x the row-0 multiplier)."""
    from . import (KERNEL_PLAIN, ORDER_HEURISTIC, Launch, extend_prefixes, fill_order,
                   multiplier)
    order = fill_order(n, flags, ORDER_HEURISTIC, first_rows)
    w = n // 2 if flags & 2 else n
    base = np.arange(w, dtype=np.uint8)[None]
    prefixes, _ = extend_prefixes(n, flags, order, base, depth)
    launches = (Launch(), Launch(kernel=KERNEL_PLAIN, stack=1))[:max(1, quorum)]
    res = run_workunits(n, flags, order, prefixes, path, batch=batch, quorum=launches,
                        counter=counter)
    res["prefixes"] = len(prefixes)
    res["row0_fixed"] = res["total"]
    res["squares"] = res["total"] * multiplier(n, flags)
    return res


def main(argv=None):
    """python -m paper_1709_02599_gb300.workunits --n 9 --depth 19
    --checkpoint dls9.jsonl [--quorum 2] prints one JSON line: the exact
    count with row 0 fixed and the number of squares.  Interrupted, the same
    command resumes from the checkpoint."""
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--vsym", action="store_true")
    ap.add_argument("--depth", type=int, required=True,
                    help="prefix length, row 0 included (order 9, Section 5.2: 19)")
    ap.add_argument("--checkpoint", required=True)
    ap.add_argument("--batch", type=int, default=1 << 20)
    ap.add_argument("--quorum", type=int, default=1, choices=(1, 2))
    a = ap.parse_args(argv)
    flags = 1 | (2 if a.vsym else 0)
    res = count_split(a.n, flags, a.depth, a.checkpoint, batch=a.batch, quorum=a.quorum)
    print(json.dumps({k: v for k, v in res.items() if k != "counts"}))
    return 0


__all__ = ["run_workunits", "gpu_counter", "count_split"]


if __name__ == "__main__":
    main()
