"""Monte Carlo estimate of the number of squares (Section 5.3).

The estimate works in four steps:
1. Count N^k, the partial squares whose first k cells of the fill order are
   filled (row-major order in Section 5.3, row 0 fixed).
2. Draw a sample of those partial squares.
3. Count the completions of each to a whole square.
4. Take N^k x (mean completions) as the estimate of the number of squares
   with row 0 fixed. Its standard error is N^k x (sample standard
   deviation) / sqrt(sample size).

    res = estimate(10, DIAGONAL, 30, ranks)     # ranks: integers in [0, N^k)

Sampling is by rank. A draw r selects the r-th k-cell partial square in
lexicographic order of its values along the fill order. It is found by
counting descent:
- count the k-cell completions of every extension one cell deeper;
- step into the extension whose range of ranks holds r;
- repeat until k cells are filled.

Uniform ranks therefore give a uniform sample, and the ranks are the only
random numbers (the caller draws them, e.g. dls_inputs.ranks). Every count
runs in the library's CUDA kernels (dls_count). This module only splits the
work and picks extensions.
"""
import numpy as np

from . import (DIAGONAL, ORDER_HEURISTIC, ORDER_ROW_MAJOR, count, extend_prefixes,
               fill_order, order_complete, order_trim)


def _first_cells(n, flags):
    """Values of the cells before the search: row 0 = 0..n-1 (left half
    with vertical symmetry)."""
    w = n // 2 if flags & 2 else n
    return np.arange(w, dtype=np.uint8)[None]


def counts_split(n, flags, order, prefixes, min_items=1 << 18, launch=None):
    """Count(prefix) for every prefix (uint8 [P, d]) under `order`, on the
    GPU.  While there are fewer than min_items work items and more than two
    cells remain, the prefixes are split one cell deeper (Section 5.2) and
    the parts summed back per prefix.  Returns uint64 [P]."""
    import torch
    prefixes = np.ascontiguousarray(prefixes, dtype=np.uint8)
    P, d = prefixes.shape
    if P == 0:
        return np.zeros(0, np.uint64)
    items, parent = prefixes, np.arange(P, dtype=np.int64)
    while len(items) < min_items and d < len(order) - 2:
        items, par = extend_prefixes(n, flags, order, items, d + 1)
        parent = parent[par]
        d += 1
        if len(items) == 0:
            break
    out = np.zeros(P, np.uint64)
    if len(items):
        c = count(n, flags, order, torch.from_numpy(items).cuda(), launch=launch)
        torch.cuda.synchronize()
        np.add.at(out, parent, c.cpu().numpy())
    return out


def select_by_rank(n, flags, order_k, ranks, start_depth=None, launch=None):
    """The ranks[i]-th k-cell partial square (k = len(order_k)) in
    lexicographic order of the values along order_k, for every rank.

    Returns (prefixes uint8 [m, k], total), total = N^k.  Ranks must lie in
    [0, total)."""
    order_k = np.ascontiguousarray(order_k, dtype=np.uint8).reshape(-1, 2)
    k = len(order_k)
    first = _first_cells(n, flags)
    d0 = first.shape[1] if start_depth is None else start_depth
    base, _ = extend_prefixes(n, flags, order_k, first, d0)
    c = counts_split(n, flags, order_k, base, launch=launch)
    cum = np.cumsum(c.astype(object))
    total = int(cum[-1]) if len(cum) else 0
    ranks = [int(r) for r in np.asarray(ranks).ravel()]
    if any(r < 0 or r >= total for r in ranks):
        raise ValueError("ranks must lie in [0, N^k)")
    m = len(ranks)
    cum_i = np.array([int(x) for x in cum], dtype=object)
    pick = np.searchsorted(cum_i.astype(float), np.array(ranks, dtype=float), side="right")
    cur = np.zeros((m, d0), np.uint8)
    rem = []
    for s, r in enumerate(ranks):
        i = int(pick[s])
        # floating-point searchsorted is a first guess; settle it exactly
        while i > 0 and cum_i[i - 1] > r:
            i -= 1
        while cum_i[i] <= r:
            i += 1
        cur[s] = base[i]
        rem.append(r - (int(cum_i[i - 1]) if i > 0 else 0))
    for d in range(d0, k):
        kids, par = extend_prefixes(n, flags, order_k, cur, d + 1)
        kc = (np.ones(len(kids), np.uint64) if d + 1 == k
              else counts_split(n, flags, order_k, kids, launch=launch))
        nxt = np.zeros((m, d + 1), np.uint8)
        starts = np.searchsorted(par, np.arange(m), side="left")
        ends = np.searchsorted(par, np.arange(m), side="right")
        for s in range(m):
            acc = 0
            for j in range(starts[s], ends[s]):
                cj = int(kc[j])
                if rem[s] < acc + cj:
                    nxt[s] = kids[j]
                    rem[s] -= acc
                    break
                acc += cj
            else:  # pragma: no cover - the counts above guarantee a child
                raise RuntimeError("rank selection lost its path")
        cur = nxt
    return cur, total


def estimate(n, flags, k, ranks, order_k=None, start_depth=None, min_items=1 << 18,
             launch=None):
    """Section 5.3's estimate from the partial squares selected by `ranks`.

    order_k: the first k cells (default: row-major, as in Section 5.3); the
    completion counts use the Section 2.3 order for the remaining cells,
    shortened by dls_order_trim.
    Returns a dict: 'n_k' (exact N^k), 'samples' (the k-cell prefixes),
    'completions' (uint64 per sample), 'mean', 'estimate', 'stderr'."""
    flags = int(flags)
    if order_k is None:
        order_k = fill_order(n, flags, ORDER_ROW_MAJOR)[:k]
    order_k = np.ascontiguousarray(order_k, dtype=np.uint8).reshape(-1, 2)
    samples, n_k = select_by_rank(n, flags, order_k, ranks, start_depth, launch=launch)
    full = order_trim(n, flags, order_complete(n, flags, order_k, len(order_k), ORDER_HEURISTIC),
                      len(order_k))
    comp = counts_split(n, flags, full, samples, min_items=min_items, launch=launch)
    vals = [int(v) for v in comp]
    m = len(vals)
    mean = sum(vals) / m if m else 0.0
    var = sum((v - mean) ** 2 for v in vals) / (m - 1) if m > 1 else 0.0
    return {"n_k": n_k, "samples": samples, "completions": comp, "mean": mean,
            "estimate": n_k * mean, "stderr": n_k * (var / m) ** 0.5 if m else 0.0}


__all__ = ["counts_split", "select_by_rank", "estimate", "DIAGONAL"]


def main(argv=None):
    """python -m paper_1709_02599_gb300.montecarlo --n 10 --k 30 --samples 8
    prints one JSON line: N^k, the estimate and its standard error (ranks
    from dls_inputs.ranks with the given seed)."""
    import argparse
    import json
    import os
    import sys
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=10)
    ap.add_argument("--k", type=int, default=30)
    ap.add_argument("--samples", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--start-depth", type=int, default=0)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import dls_inputs
    order_k = fill_order(a.n, DIAGONAL, ORDER_ROW_MAJOR)[:a.k]
    sd = a.start_depth or None
    t0 = time.perf_counter()
    _, n_k = select_by_rank(a.n, DIAGONAL, order_k, [0], sd)
    t1 = time.perf_counter()
    res = estimate(a.n, DIAGONAL, a.k, dls_inputs.ranks(n_k, a.samples, a.seed), order_k, sd)
    t2 = time.perf_counter()
    print(json.dumps({"n": a.n, "k": a.k, "n_k": n_k, "samples": a.samples, "seed": a.seed,
                      "mean_completions": res["mean"], "estimate": res["estimate"],
                      "stderr": res["stderr"], "squares_counted": int(res["completions"].sum()),
                      "completions": [int(v) for v in res["completions"]],
                      "seconds_n_k": t1 - t0, "seconds_sample": t2 - t1}))


if __name__ == "__main__":
    main()
