"""Autotuner for the batched count: split depth, fill order after the prefix,
lanes per prefix, placement of the row/column words, block size and the
snapshot stack's cap.

Every trial counts the same squares: the base prefixes are extended to the
candidate split depth with the same leading cells, and only the cells after
the split are reordered (counts do not depend on their order; Section 2.3
shows the search size does), and every order is shortened by dls_order_trim
(a final run of cells forced by their columns or rows is dropped).  A trial
is timed as a CUDA-graph launch (dls_plan_*) with CUDA events; all trials
must report the same total.

    best = tune(n, flags, order, base, depths=[...])
    best["order"], best["depth"], best["launch"]    # Launch fields dict

Results are cached per device and problem in _build/autotune.json.
"""
import hashlib
import json
import os
import time

import numpy as np

from . import (Launch, Plan, ORDER_HEURISTIC, ORDER_HEURISTIC_SQ, ORDER_MD_AD_ROWS,
               KERNEL_PERSISTENT, TAIL_WINDOW,
               extend_prefixes, order_complete, order_trim)

SUFFIXES = {"given": None, "heuristic": ORDER_HEURISTIC, "heuristic_sq": ORDER_HEURISTIC_SQ}
SHAPES = [
    {},
    {"block_threads": 64},
    {"block_threads": 256},
    {"stack_cap": 17, "block_threads": 64},
    {"stack_cap": 15, "block_threads": 64},
    {"stack_cap": 17},
    {"stack_cap": 20},
    {"fuse": -1},
    {"fuse": -1, "block_threads": 64},
    {"lookahead": 1},
    {"lookahead": 1, "block_threads": 64},
    {"check_every": 16},
    {"stack": 1},
    {"words": 1},
    {"words": 1, "block_threads": 256},
    {"lanes_per_prefix": 2},
    {"words": 1, "lanes_per_prefix": 2},
]
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(n, flags, order, base, depths, suffixes, shapes, dev):
    h = hashlib.sha1()
    h.update(repr((n, flags, list(depths), list(suffixes), shapes, dev, TAIL_WINDOW)).encode())
    h.update(np.ascontiguousarray(order, dtype=np.uint8).tobytes())
    b = np.ascontiguousarray(base, dtype=np.uint8)
    h.update(repr(b.shape).encode())
    h.update(b.tobytes())
    return h.hexdigest()


def _load_cache():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1)
    os.replace(tmp, _CACHE)


def build_problem(n, flags, order, base, depth, suffix, window=TAIL_WINDOW):
    """(order, prefixes, parents) for one split depth and suffix rule.  The
    order is then shortened by dls_order_trim (window None: not), which
    leaves every count and the prefixes as they are."""
    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(-1, 2)
    if SUFFIXES[suffix] is not None:
        order = order_complete(n, flags, order, depth, SUFFIXES[suffix])
    if window is not None:
        order = order_trim(n, flags, order, depth, window)
    pre, par = extend_prefixes(n, flags, order, base, depth)
    return order, pre, par


def time_plan(n, flags, order, d_pre, launch, reps=2):
    """Seconds per pass (min over reps) and the total."""
    import torch
    P = d_pre.shape[0]
    counts = torch.empty(max(P, 1), dtype=torch.uint64, device=d_pre.device)
    total = torch.empty(1, dtype=torch.uint64, device=d_pre.device)
    plan = Plan(n, flags, order, d_pre, counts, total, launch)
    stream = torch.cuda.current_stream()
    plan.launch(stream)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.launch(stream)
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / 1e3)
    tot = int(total.cpu().numpy()[0])
    plan.close()
    return best, tot


def tune(n, flags, order, base, depths, suffixes=("given", "heuristic", "heuristic_sq"), shapes=None,
         reps=2, use_cache=True, log=None):
    """Two stages: (split depth, suffix) with the default launch shape, then
    the launch shape for the best of those.  Returns a dict with the chosen
    'depth', 'suffix', 'launch' (Launch fields), 'order' (uint8 [L, 2]),
    'seconds' and the list of 'trials'."""
    import torch
    shapes = SHAPES if shapes is None else shapes
    dev = torch.cuda.get_device_name()
    key = _key(n, flags, order, base, depths, suffixes, shapes, dev)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        hit = dict(cache[key])
        hit["order"] = np.array(hit["order"], np.uint8)
        hit["cached"] = True
        return hit
    trials = []
    total_ref = None
    best = None
    built = {}
    for depth in depths:
        for suffix in suffixes:
            o, pre, _ = build_problem(n, flags, order, base, depth, suffix)
            d_pre = torch.from_numpy(pre).cuda()
            built[(depth, suffix)] = (o, d_pre)
            sec, tot = time_plan(n, flags, o, d_pre, Launch(kernel=KERNEL_PERSISTENT), reps)
            if total_ref is None:
                total_ref = tot
            if tot != total_ref:
                raise RuntimeError("autotune: totals differ between trials")
            trials.append({"depth": depth, "suffix": suffix, "launch": {}, "seconds": sec,
                           "prefixes": int(pre.shape[0])})
            if log:
                log(trials[-1])
            if best is None or sec < best["seconds"]:
                best = trials[-1]
    o, d_pre = built[(best["depth"], best["suffix"])]
    for k in list(built):
        if k != (best["depth"], best["suffix"]):
            del built[k]
    from . import DlsError
    for sh in shapes:
        if not sh:
            continue
        try:
            sec, tot = time_plan(n, flags, o, d_pre, Launch(**sh), reps)
        except DlsError as e:
            if e.code != 3:      # a shape that does not apply to this problem
                raise
            continue
        if tot != total_ref:
            raise RuntimeError("autotune: totals differ between trials")
        trials.append({"depth": best["depth"], "suffix": best["suffix"], "launch": sh,
                       "seconds": sec, "prefixes": int(d_pre.shape[0])})
        if log:
            log(trials[-1])
        if sec < best["seconds"]:
            best = trials[-1]
    result = {"depth": best["depth"], "suffix": best["suffix"], "launch": best["launch"],
              "seconds": best["seconds"], "total": total_ref, "trials": trials,
              "order": [list(map(int, c)) for c in o], "device": dev, "when": time.time()}
    if use_cache:
        cache[key] = result
        _save_cache(cache)
    out = dict(result)
    out["order"] = np.array(result["order"], np.uint8)
    out["cached"] = False
    return out
