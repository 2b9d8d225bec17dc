"""CPU tests of bench.py's host side: the reference arm's JSON line, the
oracle sample of its CPU legs (the same prefixes and fill order as the GPU
leg counts), and the clock sampler's summary."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
import dls_inputs
import oracle
from oracle import orders

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["config"]["workload"] == "dls8_diag64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_sample_is_the_gpu_workload(dls):
    """The CPU legs time the oracle on prefixes that the GPU leg also counts:
    the same seed-chosen diagonal fillings, split at the same depth, with the
    same order of the cells after the split."""
    from paper_1709_02599_gb300 import autotune
    spec = bench.SPECS["dls8_diag64"]
    order0, base = spec.product_base(dls, 0, spec.units)
    for depth, suffix in ((25, "heuristic_sq"), (28, "heuristic")):
        sub = dls_inputs.choose(spec.units, 2, 1000)
        o_order, o_pre, o_par = spec.oracle_sample(0, spec.units, sub, depth, suffix)
        order, pre, par = autotune.build_problem(spec.n, spec.flags, order0, base[sub], depth,
                                                 suffix)
        # the GPU's order is the oracle's with the tail run dropped
        assert [tuple(map(int, c)) for c in order] == orders.trim_tail(spec.n, o_order, depth)
        assert len(order) < len(o_order)
        assert pre.shape == o_pre.shape and (pre == o_pre).all() and (par == o_par).all()
    # and the oracle counts them: a few prefixes, against their own split
    c, _ = oracle.count_many(spec.n, spec.flags, o_order, o_pre[:50], threads=4)
    assert c.dtype == np.uint64 and len(c) == 50
    # the symmetric order-10 workload: 2000 of the 2 153 120 fillings of rows
    # 1-2 below the (left-half) identity row, split at every depth the
    # autotuner tries
    spec = bench.SPECS["vsym10_rows2"]
    order0, base = spec.product_base(dls, 0, spec.units)
    assert base.shape == (2000, 15) and (base[:, :5] == np.arange(5)).all()
    idx = np.arange(0, 2000, 250)
    for depth in spec.depths:
        for suffix in ("given", "heuristic_sq"):
            order, pre, par = autotune.build_problem(spec.n, spec.flags, order0, base[idx],
                                                     depth, suffix)
            o_order, o_pre, o_par = spec.oracle_sample(0, spec.units, idx, depth, suffix)
            assert [tuple(map(int, c)) for c in order] == orders.trim_tail(
                spec.n, o_order, depth, vsym=True)
            assert (pre == o_pre).all() and (par == o_par).all()


def test_oracle_check_agrees_and_catches_a_wrong_count(dls):
    """bench.oracle_check on an 8-diagonal profiling case: counts the oracle
    itself produced for the checked diagonals pass; one count off by one, a
    missing prefix's count, or a prefix of another base, raise."""
    from paper_1709_02599_gb300 import autotune
    spec = bench.SPECS["dls8_diag64"]
    units, depth, suffix = 8, 28, "heuristic_sq"
    order0, base = spec.product_base(dls, 0, units)
    order, pre, par = autotune.build_problem(spec.n, spec.flags, order0, base, depth, suffix)
    idx = spec.check_bases(0, np.zeros(units, np.uint64))
    o_order, o_pre, o_par = spec.oracle_sample(0, units, idx, depth, suffix)
    ref, _ = oracle.count_many(spec.n, spec.flags, o_order, o_pre, threads=os.cpu_count())
    counts = np.zeros(len(pre), np.uint64)
    for k, b in enumerate(idx):
        counts[par == b] = ref[o_par == k]
    out, rate, n_pre = bench.oracle_check(spec, 0, units, depth, suffix, pre, par, counts,
                                          os.cpu_count())
    assert out["agree"] and out["bases"] == 4 and n_pre == len(o_pre) and rate > 0
    assert out["squares"] == int(ref.sum())
    bad = counts.copy()
    k = int(np.nonzero(np.isin(par, idx) & (counts > 0))[0][0])
    bad[k] += 1
    try:
        bench.oracle_check(spec, 0, units, depth, suffix, pre, par, bad, 2)
    except RuntimeError as e:
        assert "oracle check failed" in str(e)
    else:
        raise AssertionError("a wrong count passed the check")


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def join(self, timeout=None):
        pass


def test_clock_sampler_summary():
    s = bench.ClockSampler()
    s.proc, s.thread = _Done(), _Done()
    s.rows = [["2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"],
              ["2025", "2070", "1380", "0x4", "Not Active", "Not Active", "Not Active",
               "Active"],
              ["[N/A]", "2070", "x", "x", "x", "x", "x", "x"],
              ["1995", "2070", "1400", "0x4", "Not Active", "Active", "Not Active", "Active"]]
    out = s.stop()
    assert out == {"sm_mhz": 2025.0, "sm_max_mhz": 2070.0, "samples": 3,
                   "reasons": ["hw_thermal_slowdown", "sw_power_cap"]}
    empty = bench.ClockSampler()
    assert empty.stop() is None
