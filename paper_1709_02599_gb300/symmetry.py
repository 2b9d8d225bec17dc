"""Counting with symmetry breaking (Section 4, Algorithm 6).

    res = count_symmetry_broken(8, DIAGONAL)
    res["total"]    # squares with row 0 fixed, e.g. 7 447 587 840 for n = 8

Every hourglass (row 0, both diagonals, last row) is enumerated by the prefix
split, dls_hourglass_classes keeps the canonical ones with their class sizes
(GPU), and dls_count_weighted counts the completions of the canonical ones
and sums class size x completions in 128 bits (GPU; Corollary 1).

For orders whose hourglasses do not fit in memory at once (order 9 has
1.49e9), count_symmetry_broken_resumable does the same in workunits.  A
workunit is a batch of short prefixes of the hourglass order (row 0 and the
main diagonal).  Each is extended to its hourglasses, the canonical ones are
kept, and their weighted completions are counted.  The batches go through
workunits.run_workunits, with its checkpoint and optional quorum.
"""
import ctypes

import numpy as np

from . import (_lib, lib, count as dls_count, count_weighted, extend_prefixes, fill_order,
               order_complete, order_trim, DIAGONAL, VSYM, ORDER_HOURGLASS, ORDER_HEURISTIC,
               Launch)


def hourglass_len(n, vsym=False):
    """Number of hourglass cells (left half with vsym)."""
    o = fill_order(n, DIAGONAL | (VSYM if vsym else 0), ORDER_HOURGLASS)
    w = n // 2 if vsym else n
    cells = set()
    for j in range(n):
        cells |= {(0, j), (n - 1, j)}
    for i in range(n):
        cells |= {(i, i), (i, n - 1 - i)}
    k = sum(1 for (i, j) in cells if j < w)
    assert {tuple(map(int, c)) for c in o[:k]} == {c for c in cells if c[1] < w}
    return k


def hourglass_classes(n, flags, order, d_hourglasses, stream=None):
    """Class sizes (uint32 CUDA tensor) of the hourglasses in d_hourglasses
    (uint8 CUDA tensor [count, len]); 0 for non-canonical ones."""
    import torch
    hg = d_hourglasses.contiguous()
    count, ln = hg.shape
    out = torch.empty(count, dtype=torch.int32, device=hg.device)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.uint8).reshape(-1, 2))
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _lib.check(lib().dls_hourglass_classes(n, flags, o.ctypes.data_as(_lib.u8p), ln,
                                           ctypes.c_void_p(hg.data_ptr()) if count else None,
                                           count, ctypes.c_void_p(out.data_ptr()) if count else None,
                                           ctypes.c_void_p(st)), "dls_hourglass_classes")
    return out


def count_symmetry_broken(n, flags=DIAGONAL, launch=None, min_items=1 << 20):
    """Squares with row 0 fixed to 0..n-1, counted through canonical
    hourglasses.  Returns a dict with the total and the class statistics."""
    import torch
    vsym = bool(flags & VSYM)
    order, k = hourglass_order(n, flags)
    ident = np.arange(n // 2 if vsym else n, dtype=np.uint8)[None]
    hg, _ = extend_prefixes(n, flags, order, ident, k)
    d_hg = torch.from_numpy(hg).cuda()
    sizes = hourglass_classes(n, flags, order[:k], d_hg)
    canon = torch.nonzero(sizes > 0).flatten()
    sz = sizes[canon].cpu().numpy().astype(np.int64)
    reps = hg[canon.cpu().numpy()]
    # split the representatives further (Section 5.2) until there are enough
    # independent items to keep every lane busy; each item keeps the class
    # size of its representative
    depth, items, parent = k, reps, np.arange(len(reps), dtype=np.int64)
    while len(items) < min_items and depth < len(order) - 2:
        items, par = extend_prefixes(n, flags, order, items, depth + 1)
        parent = parent[par]
        depth += 1
    # Algorithm 6's Total += Cnt * multiple in the library: each item weighs
    # the class size of its representative, the weighted sum is taken in 128
    # bits on the device (dls_count_weighted)
    d_items = torch.from_numpy(items).cuda()
    weights = torch.from_numpy(sz[parent].astype(np.int32)).cuda()
    counts = torch.empty(len(items), dtype=torch.uint64, device="cuda")
    total = count_weighted(n, flags, order, d_items, weights=weights, counts=counts,
                           launch=launch)
    ct = counts.cpu().numpy()
    return {"total": total, "hourglasses": int(len(hg)), "classes": int(len(canon)),
            "class_size_sum": int(sizes.sum().item()), "max_class": int(sz.max()) if len(sz) else 0,
            "squares_counted": int(ct.sum()), "items": int(len(items)), "split_depth": depth,
            "order": order, "hourglass_values": hg, "class_sizes": sizes.cpu().numpy()}


def hourglass_order(n, flags):
    """The hourglass cells (row 0, main diagonal, anti-diagonal, last row;
    left half with vertical symmetry) followed by the other cells in the
    Section 2.3 order, shortened by dls_order_trim (the counts stay the
    same).  Returns (order, number of hourglass cells)."""
    vsym = bool(flags & VSYM)
    k = hourglass_len(n, vsym)
    order = fill_order(n, flags, ORDER_HOURGLASS)
    order = order_complete(n, flags, order, k, ORDER_HEURISTIC)
    return order_trim(n, flags, order, k), k


def weighted_counter(n, flags, order, k, classes_fn=None, count_fn=None, min_items=1 << 20,
                     tally=None):
    """counter(bases, launch) for workunits.run_workunits.  bases are prefixes
    of the first cells of `order` (k hourglass cells first).  For each base
    it returns the sum, over the canonical hourglasses that extend it, of
    class size x completions (Corollary 1).

    classes_fn(hourglasses) -> class sizes, and count_fn(prefixes, launch) ->
    completion counts; both default to the library on the GPU.  tally (a
    dict, optional) receives, per batch of bases (keyed by their bytes), the
    number of hourglasses extending them and the sum of the class sizes of
    the canonical ones among them."""
    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(-1, 2)
    if classes_fn is None:
        def classes_fn(hg):
            import torch
            return hourglass_classes(n, flags, order[:k],
                                     torch.from_numpy(hg).cuda()).cpu().numpy()
    if count_fn is None:
        def count_fn(prefixes, launch):
            import torch
            c = dls_count(n, flags, order, torch.from_numpy(prefixes).cuda(), launch=launch)
            torch.cuda.synchronize()
            return c.cpu().numpy()

    def counter(bases, launch):
        bases = np.ascontiguousarray(bases, dtype=np.uint8)
        out = np.zeros(len(bases), np.uint64)
        hg, hpar = extend_prefixes(n, flags, order, bases, k)
        if len(hg) == 0:
            if tally is not None:
                tally[bases.tobytes()] = (0, 0)
            return out
        sizes = np.asarray(classes_fn(hg)).astype(np.int64)
        if tally is not None:
            tally[bases.tobytes()] = (int(len(hg)), int(sizes.sum()))
        canon = np.nonzero(sizes > 0)[0]
        if len(canon) == 0:
            return out
        reps, rbase, rsize = hg[canon], hpar[canon], sizes[canon].astype(np.uint64)
        # split the representatives further while there are few of them
        # (Section 5.2), so that every lane has work
        depth, items, parent = k, reps, np.arange(len(reps), dtype=np.int64)
        while len(items) < min_items and depth < len(order) - 2:
            nxt, par = extend_prefixes(n, flags, order, items, depth + 1)
            if len(nxt) == 0:
                break
            items, parent, depth = nxt, parent[par], depth + 1
        per_rep = np.zeros(len(reps), np.uint64)
        if len(items) and len(items[0]) == depth:
            np.add.at(per_rep, parent, np.asarray(count_fn(items, launch), dtype=np.uint64))
        np.add.at(out, rbase, rsize * per_rep)
        return out

    return counter


def count_symmetry_broken_resumable(n, flags, path, batch=64, quorum=1, base_depth=None,
                                    classes_fn=None, count_fn=None, min_items=1 << 20):
    """count_symmetry_broken in workunits of `batch` base prefixes (row 0
    and the main diagonal by default), checkpointed at `path`.  Returns
    workunits.run_workunits' dict with 'total' = squares with row 0 fixed,
    plus 'bases' and 'base_depth'.

    A quorum (2: the batched and the plain kernel) covers the completion
    counts only: the class sizes come from the one canonisation kernel.
    They are checked instead by an invariant of the whole run -- every
    hourglass lies in exactly one class, so the class sizes of the canonical
    hourglasses add up to the number of hourglasses.  That needs every
    workunit, so it is checked when this call counted all of them
    ('class_check' True; None when some were resumed from the checkpoint)
    and a failure raises RuntimeError."""
    from . import KERNEL_PLAIN
    from .workunits import run_workunits
    order, k = hourglass_order(n, flags)
    w = n // 2 if flags & VSYM else n
    if base_depth is None:
        base_depth = w
        while base_depth < k and int(order[base_depth][0]) == int(order[base_depth][1]):
            base_depth += 1  # the main-diagonal cells after row 0
    if not w <= base_depth <= k:
        raise ValueError("base_depth must lie between row 0 and the hourglass")
    ident = np.arange(w, dtype=np.uint8)[None]
    bases, _ = extend_prefixes(n, flags, order, ident, base_depth)
    launches = (Launch(), Launch(kernel=KERNEL_PLAIN, stack=1))[:max(1, quorum)]
    tally = {}
    res = run_workunits(n, flags, order, bases, path, batch=batch, quorum=launches,
                        counter=weighted_counter(n, flags, order, k, classes_fn, count_fn,
                                                 min_items, tally=tally))
    res["bases"] = int(len(bases))
    res["base_depth"] = int(base_depth)
    res["class_check"] = None
    if res["units_resumed"] == 0 and len(bases):
        hourglasses = sum(h for h, _ in tally.values())
        size_sum = sum(c for _, c in tally.values())
        if hourglasses != size_sum:
            raise RuntimeError("class sizes add up to %d, not to the %d hourglasses"
                               % (size_sum, hourglasses))
        res["class_check"] = True
        res["hourglasses"] = hourglasses
    return res


def main(argv=None):
    """python -m paper_1709_02599_gb300.symmetry --n 9 --checkpoint sym9.jsonl
    prints one JSON line: the squares with row 0 fixed, counted through
    canonical hourglasses in resumable workunits."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--vsym", action="store_true")
    ap.add_argument("--checkpoint", required=True)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--quorum", type=int, default=1, choices=(1, 2))
    a = ap.parse_args(argv)
    flags = DIAGONAL | (VSYM if a.vsym else 0)
    res = count_symmetry_broken_resumable(a.n, flags, a.checkpoint, batch=a.batch,
                                          quorum=a.quorum)
    print(json.dumps({k: v for k, v in res.items() if k != "counts"}))
    return 0


if __name__ == "__main__":
    main()
