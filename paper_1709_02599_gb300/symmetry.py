"""Counting with symmetry breaking (Section 4, Algorithm 6).

    res = count_symmetry_broken(8, DIAGONAL)
    res["total"]    # squares with row 0 fixed, e.g. 7 447 587 840 for n = 8

Every hourglass (row 0, both diagonals, last row) is enumerated by the prefix
split, dls_hourglass_classes keeps the canonical ones with their class sizes
(GPU), dls_count counts the completions of the canonical ones (GPU), and the
total is the sum of class size x completions (Corollary 1).
"""
import ctypes

import numpy as np

from . import (_lib, lib, count as dls_count, extend_prefixes, fill_order, order_complete,
               DIAGONAL, VSYM, ORDER_HOURGLASS, ORDER_HEURISTIC, Launch)


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
    k = hourglass_len(n, vsym)
    order = fill_order(n, flags, ORDER_HOURGLASS)
    order = order_complete(n, flags, order, k, ORDER_HEURISTIC)
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
    counts = dls_count(n, flags, order, torch.from_numpy(items).cuda(), launch=launch)
    torch.cuda.synchronize()
    ct = counts.cpu().numpy()
    per_rep = np.zeros(len(reps), dtype=object)
    for r, c in zip(parent, ct):
        per_rep[r] += int(c)
    total = sum(int(s) * int(c) for s, c in zip(sz, per_rep))
    return {"total": total, "hourglasses": int(len(hg)), "classes": int(len(canon)),
            "class_size_sum": int(sizes.sum().item()), "max_class": int(sz.max()) if len(sz) else 0,
            "squares_counted": int(ct.sum()), "items": int(len(items)), "split_depth": depth,
            "order": order, "hourglass_values": hg, "class_sizes": sizes.cpu().numpy()}
