#!/usr/bin/env python
"""Throughput of the GPU enumerator of diagonal Latin squares.

One step = one pass of the whole search over one batch: order 8, row 0 fixed
to the identity, 64 seed-drawn main-diagonal fillings, each split 20 cells
past row 0 (~1.17 M independent prefixes, ~2.5e8 squares), counted by the
persistent kernel launched from a CUDA graph.  Reported:

* value     -- squares enumerated per second (exact counts), device-timed
               with CUDA events on the launching stream, L2 flushed between
               steps;
* plain     -- the same for the one-thread-per-prefix launch with the same
               search step (what batching gains), and with the per-position
               step (plain_per_position_step);
* e2e       -- through dls_count_host (host buffers, copies inside the timed
               region);
* roofline  -- integer-issue roofline of the search kernel;
* oracle_check -- the oracle recounts 4 of the 64 diagonal fillings from its
               own order and split: prefixes and counts must agree exactly
               (the bench fails otherwise);
* cpu_baseline -- the oracle's rate on that sample, on the host cores;
* workloads.vsym10_rows2 -- the same for the largest single-GPU
               configuration: vertically symmetric order 10, 2000 seed-drawn
               fillings of rows 1-2, the 20 smallest checked by the oracle;
* serving   -- a replay of the serving mix with latency percentiles.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With torchrun (N > 1) each rank counts its own 64 diagonals (seed = rank) and
rank 0 prints the line (weak scaling, no collective on the data path); with
--scaling strong the ranks split one 64-diagonal problem (interleaved
prefixes, rank 0's tuned split) and the exact total is reduced.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import dls_inputs  # noqa: E402

METRIC = "diagonal Latin squares enumerated/sec on 1 GB300 (exact count) vs plain launch; p99 latency"
UNIT = "squares/s"
DIAGS, AFTER_ROW0 = 64, 20
# the fewest integer operations a search node takes in the bitmask form:
# isolate + clear the lowest candidate bit (4), mark and unmark the row and
# column words (4), next cell's forbidden mask and complement (2), the depth
# step (1), the loop test (1)
OPS_PER_NODE = 12
ISSUE_LANES_PER_SM = 4 * 32      # 4 schedulers x 32 lanes, one instruction/clk
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) per prefix of the batched kernel, per (workload,
# kernel, step, fused, split depth), from an ncu capture of that build (the
# summaries under profiles/ give the commands); a kernel or depth without a
# capture of its current build reports traffic null.  Order 8: 16 of the 64
# diagonals at depth 25 (stack cap 17, blocks of 64, strided queue), 149 590
# prefixes, 4 972 544 B read.  Symmetric order 10 (the field-shift search,
# which keeps the queue in order): 100 of the 2 000 rows-1-2 prefixes at
# depth 23, 125 320 prefixes, 3 914 240 B read.
_BW = ("dls8_diag64", "k_snapshot", "snapshot, byte words", True)
TRAFFIC_PER_PREFIX = {
    _BW + (25,): 4972544 / 149590,
    ("vsym10_rows2", "k_snapshot", "snapshot, field shifts", False, 23): 3914240 / 125320,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="under torchrun: weak = each rank counts its own 64 diagonals "
                         "(seed = rank); strong = the ranks split one 64-diagonal problem")
    ap.add_argument("--no-config4", action="store_true",
                    help="skip the second leg (vertically symmetric order 10, 2000 rows-1-2 "
                         "prefixes)")
    ap.add_argument("--workload", default="dls8_diag64", choices=["dls8_diag64", "vsym10_rows2"])
    ap.add_argument("--diagonals", type=int, default=0,
                    help="base prefixes per rank (0 = the workload's own: 64 diagonal "
                         "fillings / 2000 row prefixes; fewer only for profiling captures)")
    ap.add_argument("--launch", default="", help="json dict of Launch fields (skips the "
                    "launch-shape stage of the autotuner)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="split 20 cells past row 0, cells after the split row by row")
    ap.add_argument("--suffix", default="", choices=["", "given", "heuristic", "heuristic_sq"],
                    help="fix the order of the cells after the split")
    ap.add_argument("--depth", type=int, default=0,
                    help="fix the split depth (cells from the start of the order)")
    ap.add_argument("--serve-jobs", type=int, default=100,
                    help="also replay this many jobs of the serving mix (Poisson arrivals "
                         "at 200/s) and report latency percentiles")
    ap.add_argument("--serve-limit", type=float, default=150.0,
                    help="seconds after which the serving replay stops")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------ workloads --

class Dls8Diag64:
    """Order 8, row 0 identity, `units` seed-drawn main-diagonal fillings
    (row 0 + main diagonal), split 20 cells past row 0 by default.  The
    oracle checks the counts of 4 seed-chosen fillings of the 64."""
    name, n, flags, units, unit_name = "dls8_diag64", 8, 1, DIAGS, "diagonal fillings"
    default_depth = 8 + AFTER_ROW0
    depths = [8 + 14, 8 + 17, 8 + 20, 8 + 23]
    first_rows = 1
    check_units = 4
    check_rule = "4 seed-chosen diagonal fillings of the 64"
    oracle_extra = 0          # cells the oracle splits deeper for its threads

    def base_depth(self):
        return self.n + (self.n - 1)

    def product_base(self, dls, seed, k):
        order = dls.fill_order(self.n, self.flags, first_rows=self.first_rows)
        # row 0 = 0..n-1; with vertical symmetry the order lists its left half
        w = self.n // 2 if self.flags & 2 else self.n
        ident = np.arange(w, dtype=np.uint8)[None]
        allb, _ = dls.extend_prefixes(self.n, self.flags, order, ident, self.base_depth())
        picks = dls_inputs.choose(len(allb), k, seed)
        return order, allb[picks]

    def check_bases(self, seed, gpu_base_sums):
        """Indices (into the run's base prefixes) of the bases the oracle
        checks."""
        return dls_inputs.choose(len(gpu_base_sums), self.check_units, seed + 1000)

    def oracle_sample(self, seed, units, base_idx, depth, suffix):
        """The oracle's own order and prefixes for the run's base prefixes
        `base_idx` (of the `units` drawn with `seed`), split at `depth` (cells
        after the split in `suffix` order).  Returns (order, prefixes,
        parents): parents[k] = position in base_idx of prefix k's base."""
        import oracle
        from oracle import orders
        vs = bool(self.flags & 2)
        o_order = orders.md_ad_rows(self.n, vsym=vs, first_rows=self.first_rows)
        if suffix in ("heuristic", "heuristic_sq"):
            o_order = orders.heuristic_complete(self.n, o_order[:depth], True, vs,
                                                squares=suffix == "heuristic_sq")
        ident = np.array([orders.identity(self.n, vs)], np.uint8)
        allb, _ = oracle.extend(self.n, self.flags, o_order, ident, self.base_depth())
        picks = dls_inputs.choose(len(allb), units, seed)
        pre, par = oracle.extend(self.n, self.flags, o_order, allb[picks][np.asarray(base_idx)],
                                 depth)
        return o_order, pre, par


class Vsym10Rows2(Dls8Diag64):
    """Order 10, vertically symmetric, row 0 identity; `units` seed-drawn
    fillings of rows 1 and 2 out of the 2 153 120 valid ones.  The oracle
    checks the 20 with the smallest GPU counts."""
    name, n, flags, units, unit_name = "vsym10_rows2", 10, 3, 2000, "rows-1-2 prefixes"
    default_depth = 19
    depths = [17, 19, 21, 23]
    first_rows = 3
    check_units = 20
    check_rule = "the 20 rows-1-2 prefixes of the 2000 with the smallest GPU counts"
    oracle_extra = 4

    def base_depth(self):
        return 15

    def check_bases(self, seed, gpu_base_sums):
        return np.argsort(np.asarray(gpu_base_sums, dtype=np.uint64), kind="stable")[
            :self.check_units]


SPECS = {"dls8_diag64": Dls8Diag64(), "vsym10_rows2": Vsym10Rows2()}


def run_oracle(spec, o_order, pre, threads, extra=0):
    """Oracle counts of `pre` (summed back from `extra` cells deeper, where
    the split is finer for the threads).  Returns (counts per prefix, nodes,
    seconds)."""
    import oracle
    t0 = time.perf_counter()
    if extra:
        depth = min(pre.shape[1] + extra, len(o_order) - 1)
        sub, par = oracle.extend(spec.n, spec.flags, o_order, pre, depth)
        c, nd = oracle.count_many(spec.n, spec.flags, o_order, sub, threads=threads)
        counts = np.zeros(len(pre), np.uint64)
        np.add.at(counts, par, c)
        nodes = int(nd.sum())
    else:
        counts, nd = oracle.count_many(spec.n, spec.flags, o_order, pre, threads=threads)
        nodes = int(nd.sum())
    return counts, nodes, time.perf_counter() - t0


def oracle_check(spec, seed, units, depth, suffix, pre, par, counts, threads, share=None,
                 par_all=None):
    """The oracle counts the prefixes of the bases spec.check_bases() picks,
    from its own order and split; they must equal the GPU's prefixes byte for
    byte and its counts exactly (RuntimeError otherwise).  pre / par / counts
    are this rank's rows; under strong scaling `share` holds their indices in
    the whole problem and par_all its parents, and only this rank's rows of
    the checked bases are compared.  Returns the line's 'oracle_check'
    object, the oracle's rate on that sample (squares/s) and the number of
    prefixes it counted."""
    if share is None:
        share, par_all = np.arange(len(pre), dtype=np.int64), par
    sums = np.zeros(units, np.uint64)
    np.add.at(sums, par, counts)
    idx = np.asarray(spec.check_bases(seed, sums))
    o_order, o_pre, o_par = spec.oracle_sample(seed, units, idx, depth, suffix)
    c, _, dt = run_oracle(spec, o_order, o_pre, threads, spec.oracle_extra)
    agree = True
    for k, b in enumerate(idx):
        o_rows = np.nonzero(o_par == k)[0]       # the oracle's prefixes of base b
        g_all = np.nonzero(par_all == b)[0]      # their places in the whole problem
        mine = np.nonzero(par == b)[0]           # this rank's rows of base b
        if len(g_all) != len(o_rows):
            agree = False
            continue
        at = o_rows[np.searchsorted(g_all, share[mine])]
        if not ((pre[mine] == o_pre[at]).all() and (counts[mine] == c[at]).all()):
            agree = False
    squares = int(c.sum())
    out = {"bases": int(len(idx)), "which": spec.check_rule, "prefixes": int(len(o_pre)),
           "squares": squares, "agree": agree, "oracle_seconds": round(dt, 2)}
    if not agree:
        raise RuntimeError("oracle check failed: %s" % json.dumps(out))
    return out, (squares / dt if dt > 0 else None), len(o_pre)


# --------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.rows = []
        self.proc = None
        self.bus_id = bus_id

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.bus_id:
            cmd[1:1] = ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm = []
        mx = []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[4 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_bus_id(dev):
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        dom = getattr(p, "pci_domain_id", 0)
        bus = getattr(p, "pci_bus_id", None)
        devid = getattr(p, "pci_device_id", 0)
        if bus is None:
            return None
        return "%08X:%02X:%02X.0" % (dom, bus, devid)
    except Exception:
        return None


# ---------------------------------------------------------- measurement --

def timed_steps(launch_fn, stream, steps, flush):
    """Per-step CUDA events around launch_fn on `stream`, L2 flushed between
    steps (outside the events).  Returns the list of step times (s)."""
    import torch
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            launch_fn()
            b.record(stream)
            evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) / 1e3 for a, b in evs]


def serving_leg(n_jobs, limit_s, seed=0, **cfg):
    """Replays the seeded serving mix in real time against the
    continuous-batching server (dls_server_cfg fields in cfg); returns the
    'serving' object of the line."""
    from paper_1709_02599_gb300 import serving
    specs = dls_inputs.serving_jobs(n_jobs, seed=seed)
    jobs = []
    for sp in specs:
        b = serving.build_job(sp["n"], sp["vsym"], sp["rows"], sp["draws"])
        if b is None:
            continue
        flags, order, prefix = b
        jobs.append(dict(n=sp["n"], flags=flags, order=order, prefix=prefix,
                         arrival=sp["arrival"], rows=sp["rows"]))
    srv = serving.Server(**cfg)
    # one untimed warm-up job so that the first epoch pays no start-up cost
    srv.submit(jobs[0]["n"], jobs[0]["flags"], jobs[0]["order"], jobs[0]["prefix"])
    srv.drain()
    done, makespan = serving.run_stream(srv, jobs, time_limit_s=limit_s)
    st = srv.stats()
    srv.close()
    lat = np.array([done[k][0] for k in sorted(done)]) * 1e3
    squares = sum(done[k][1] for k in done)
    span = jobs[-1]["arrival"] if jobs else 0.0
    out = {"jobs": len(jobs), "completed": len(done), "unfinished": len(jobs) - len(done),
           "offered_rate_hz": len(jobs) / span if span > 0 else None,
           "served_rate_hz": len(done) / makespan if makespan > 0 else None,
           "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
           "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
           "max_ms": float(lat.max()) if len(lat) else None,
           "squares": int(squares), "squares_per_s": squares / makespan if makespan else None,
           "makespan_s": makespan, "epochs": st["epochs"], "lanes": st["lanes"],
           "device_bytes": st["device_bytes"],
           "mix": "order uniform {6,7,8,9}, diagonal or vertically symmetric, 2..N-3 rows "
                  "fixed, Poisson 200/s, seed %d" % seed}
    if out["unfinished"]:
        out["note"] = "stopped after %.0f s with jobs unfinished" % limit_s
    # the served counts of the jobs of order <= 8, recounted by the batch
    # kernels (each job split 2^14 ways), after the replay
    from paper_1709_02599_gb300.montecarlo import counts_split
    small = [k for k in sorted(done) if jobs[k]["n"] <= 8]
    try:
        bad = 0
        for k in small:
            j = jobs[k]
            ref = counts_split(j["n"], j["flags"], j["order"],
                               np.asarray(j["prefix"], np.uint8)[None], min_items=1 << 14)
            bad += int(int(ref[0]) != int(done[k][1]))
        out["batch_check"] = {"jobs": len(small), "agree": bad == 0, "mismatches": bad,
                              "rule": "every completed job of order <= 8 recounted by the "
                                      "batch kernels"}
    except Exception as e:  # the check must not lose the serving numbers
        out["batch_check"] = {"jobs": len(small), "error": repr(e)[:200]}
    return out


def rank_share(n_prefixes, rank, ws, scaling):
    """Indices of the prefixes this rank counts: all of its own problem under
    weak scaling (each rank draws its own base prefixes), an interleaved
    share of the one common problem under strong scaling."""
    if scaling == "strong" and ws > 1:
        from paper_1709_02599_gb300 import shard
        return shard.shard_indices(n_prefixes, rank, ws)
    return np.arange(n_prefixes, dtype=np.int64)


def agree_on_choice(choice, ws, scaling):
    """Under strong scaling every rank must count the same problem: rank 0's
    tuned (depth, suffix, launch) is broadcast to the others."""
    if scaling != "strong" or ws < 2:
        return choice
    import torch.distributed as dist
    box = [choice]
    dist.broadcast_object_list(box, src=0)
    return box[0]


def reduce_squares(local, ws):
    """Exact sum of the ranks' square counts (one scalar collective)."""
    if ws < 2:
        return int(local)
    from paper_1709_02599_gb300 import shard
    return shard.allreduce_total(int(local))


def reference_arm(args):
    """The oracle, as it stands, on the host cores: each step a bounded sample
    (one diagonal's prefixes) of the same workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    spec = SPECS[args.workload]
    base_idx = dls_inputs.choose(spec.units, 1, 1000)
    o_order, pre, _ = spec.oracle_sample(0, spec.units, base_idx, spec.default_depth,
                                         "heuristic_sq")
    for _ in range(args.warmup):
        run_oracle(spec, o_order, pre, threads)
    sq = 0
    t = 0.0
    for _ in range(args.steps):
        c, _, dt = run_oracle(spec, o_order, pre, threads)
        sq += int(c.sum())
        t += dt
    value = sq / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": spec.name, "n": spec.n,
                   "sample": "1 of the %d %s per step" % (spec.units, spec.unit_name),
                   "prefixes_per_step": int(len(pre))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "all %d prefixes of 1 seed-chosen base prefix of the %d, "
                                   "cells after the split in the squared-count Section 2.3 "
                                   "order"
                                   % (len(pre), spec.units)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_leg(dls, spec, args, steps, stream, flush, seed, rank, ws, units=None,
            plain_per_position=True):
    # under strong scaling every rank draws the same base prefixes
    seed = 0 if args.scaling == "strong" else seed
    """One workload: autotune (cached), then the graph-launched batched count
    timed over `steps` steps, the plain launches, the host-buffer entry, the
    roofline and the oracle check.  Returns (leg dict, step seconds, squares
    per step, the plan's count of our kernel launches per step)."""
    import torch
    from paper_1709_02599_gb300 import autotune
    N, FLAGS = spec.n, spec.flags
    units = units or spec.units
    order0, base = spec.product_base(dls, seed, units)
    fixed = json.loads(args.launch) if args.launch else None
    tuned = None
    if args.no_autotune:
        depth_sel = args.depth or spec.default_depth
        suffix_sel, cfg = args.suffix or "given", fixed or {}
    else:
        t0 = time.perf_counter()
        suffixes = (args.suffix,) if args.suffix else ("given", "heuristic", "heuristic_sq")
        shapes = [{}] if fixed is not None else None
        best = autotune.tune(N, FLAGS, order0, base, [args.depth] if args.depth else spec.depths,
                             suffixes=suffixes, shapes=shapes)
        depth_sel, suffix_sel = best["depth"], best["suffix"]
        cfg = fixed if fixed is not None else best["launch"]
        tuned = {"trials": len(best["trials"]), "cached": best["cached"],
                 "seconds": round(time.perf_counter() - t0, 2),
                 "candidates": "split depth %s x order after the split {given, heuristic, "
                               "heuristic_sq}, "
                               "then %d launch shapes" % (spec.depths,
                                                          len(shapes or autotune.SHAPES) - 1)}
    depth_sel, suffix_sel, cfg = agree_on_choice((depth_sel, suffix_sel, cfg), ws, args.scaling)
    order, pre, par = autotune.build_problem(N, FLAGS, order0, base, depth_sel, suffix_sel)
    P_all = len(pre)
    share = rank_share(P_all, rank, ws, args.scaling)
    par_all = par
    pre, par = np.ascontiguousarray(pre[share]), par[share]
    P, depth = pre.shape
    d_pre = torch.from_numpy(pre).to("cuda")
    counts = torch.empty(P, dtype=torch.uint64, device="cuda")
    total = torch.empty(1, dtype=torch.uint64, device="cuda")
    launch = dls.Launch(**cfg)
    plan = dls.Plan(N, FLAGS, order, d_pre, counts, total, launch)
    run = dls.describe_launch(N, FLAGS, order, depth, P, launch)

    # node count of the workload (separately compiled counting variant,
    # untimed) and the exact square count
    nodes_t = torch.zeros(1, dtype=torch.uint64, device="cuda")
    with torch.cuda.stream(stream):
        dls.count(N, FLAGS, order, d_pre, counts=counts, total=total, nodes=nodes_t,
                  launch=launch, stream=stream)
    torch.cuda.synchronize()
    squares = int(total.cpu().numpy()[0])
    nodes = int(nodes_t.cpu().numpy()[0])

    for _ in range(max(args.warmup, 0)):
        plan.launch(stream)
    torch.cuda.synchronize()

    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(gpu_bus_id(torch.cuda.current_device())) if rank == 0 else None
    if sampler:
        sampler.start()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    times = timed_steps(lambda: plan.launch(stream), stream, steps, flush)
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop() if sampler else None
    if int(total.cpu().numpy()[0]) != squares:
        raise RuntimeError("count changed between runs")
    counts_np = counts.cpu().numpy()
    step_s = sum(times) / len(times)
    if ws > 1:
        t = torch.tensor([step_s], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_s = float(t.item())

    # plain one-thread-per-prefix launches on the same workload: with the same
    # search step (the batching comparison) and with the per-position step
    def plain_leg(stack):
        pl = dls.Launch(kernel=dls.KERNEL_PLAIN, words=cfg.get("words", 0), stack=stack)
        pplan = dls.Plan(N, FLAGS, order, d_pre, counts, total, pl)
        for _ in range(max(args.warmup, 1)):
            pplan.launch(stream)
        torch.cuda.synchronize()
        pt = timed_steps(lambda: pplan.launch(stream), stream, steps, flush)
        if int(total.cpu().numpy()[0]) != squares:
            raise RuntimeError("plain launch count differs")
        pplan.close()
        p_step = sum(pt) / len(pt)
        return {"value": squares / p_step, "unit": UNIT, "ms_per_step": 1e3 * p_step,
                "kernel": dls.describe_launch(N, FLAGS, order, depth, P, pl)["kernel"],
                "speedup_of_batched": p_step / step_s}
    plain = plain_pp = None
    if not args.no_plain:
        plain = plain_leg(0)
        if plain["kernel"] != "k_plain" and plain_per_position:
            plain_pp = plain_leg(1)

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        pinned_in = torch.from_numpy(pre).pin_memory()
        pinned_out = torch.empty(P, dtype=torch.int64).pin_memory()
        for _ in range(2):
            dls.count_host(N, FLAGS, order, pinned_in, pinned_out, launch, stream)
        e2e_t = []
        for _ in range(steps):
            t0 = time.perf_counter()
            _, tot = dls.count_host(N, FLAGS, order, pinned_in, pinned_out, launch, stream)
            e2e_t.append(time.perf_counter() - t0)
            if tot != squares:
                raise RuntimeError("host-buffer count differs")
        e2e_step = sum(e2e_t) / len(e2e_t)
        e2e = {"value": squares / e2e_step, "unit": UNIT, "h2d_bytes_per_step": int(P * depth),
               "d2h_bytes_per_step": int(P * 8), "entry": "dls_count_host"}

    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    sm_max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak_tops = sms * ISSUE_LANES_PER_SM * sm_max_mhz * 1e6 / 1e12
    achieved_tops = nodes * OPS_PER_NODE / step_s / 1e12
    # the traffic figures belong to the kernel variant they were captured on
    tkey = (spec.name, run["kernel"], run["step"], bool(run.get("fused")), depth)
    leg = {
        "value": squares / step_s, "unit": UNIT, "steps": steps,
        "ms_per_step": 1e3 * step_s,
        "config": {"workload": spec.name if units == spec.units else
                   "%s (profiling case: %d %s)" % (spec.name, units, spec.unit_name),
                   "n": N, "flags": "diagonal" + (", vertically symmetric" if FLAGS & 2 else ""),
                   "row0": "identity", spec.unit_name.replace(" ", "_"): units, "seed": "rank",
                   "split_depth": int(depth_sel), "suffix_order": suffix_sel,
                   "order_cells": int(len(order)),
                   "tail_dropped": int(N * (N // 2 if FLAGS & 2 else N) - len(order)),
                   "tail_rule": "dls_order_trim: the order's final cells, each the last "
                                "open cell of its column, complete every filling in exactly "
                                "one way, so the search stops before them; counts are of "
                                "whole squares (checked against the oracle's whole order)",
                   "prefixes": int(P), "squares_per_step": squares, "nodes_per_step": nodes,
                   "kernel": run["kernel"] + " (CUDA graph)", "launch": cfg, "resolved": run,
                   "autotune": tuned,
                   "l2": "flushed: 256 MiB write between timed steps"},
        "plain": plain,
        "plain_per_position_step": plain_pp,
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops,
                     "unit": "Tops/s", "frac": achieved_tops / peak_tops,
                     "traffic": (TRAFFIC_PER_PREFIX[tkey] * P if tkey in TRAFFIC_PER_PREFIX
                                 else None),
                     "algorithmic_bytes": int(P * (depth + 8)),
                     "ops_per_node": OPS_PER_NODE,
                     "peak_from": "%d SMs x 4 schedulers x 32 lanes x %.0f MHz" % (sms, sm_max_mhz)},
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        chk, rate, n_pre = oracle_check(spec, seed, units, depth_sel, suffix_sel, pre, par,
                                        counts_np, threads, share, par_all)
        leg["oracle_check"] = chk
        leg["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "all %d prefixes of %s, same split and fill order as "
                                         "the GPU run (%d squares, %.1f s)"
                                         % (n_pre, spec.check_rule, chk["squares"],
                                            chk["oracle_seconds"])}
    plan.close()
    return leg, step_s, squares


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import paper_1709_02599_gb300 as dls

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    seed = rank
    spec = SPECS[args.workload]
    leg, step_s, squares = run_leg(dls, spec, args, args.steps, stream, flush, seed, rank, ws,
                                   units=args.diagonals or spec.units)
    squares_all = reduce_squares(squares, ws)
    value = squares_all / step_s
    e2e = leg["e2e"]
    if e2e is not None and ws > 1:
        e2e = dict(e2e, note="per-rank rate (host timers are not reduced)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
        "scaling": args.scaling, "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": leg["config"],
        "plain": leg["plain"],
        "plain_per_position_step": leg["plain_per_position_step"],
        "e2e": e2e,
        "roofline": leg["roofline"],
        "gpu_launches": args.steps,
        "clocks": leg["clocks"],
        "wall_s_timed_region": leg["wall_s_timed_region"],
    }
    for k in ("oracle_check", "cpu_baseline"):
        if k in leg:
            line[k] = leg[k]
    # the largest single-GPU configuration as a second leg: the vertically
    # symmetric order-10 workload, fewer steps (one pass is ~1 s)
    if not args.no_config4 and spec.name != "vsym10_rows2" and not args.diagonals:
        leg4, step4, squares4 = run_leg(dls, SPECS["vsym10_rows2"], args, min(args.steps, 5),
                                        stream, flush, seed, rank, ws, plain_per_position=False)
        leg4["value"] = reduce_squares(squares4, ws) / step4
        leg4["gpu_launches"] = leg4["steps"]
        line["workloads"] = {"vsym10_rows2": leg4}
    if rank == 0 and args.serve_jobs > 0:
        line["serving"] = serving_leg(args.serve_jobs, args.serve_limit)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
