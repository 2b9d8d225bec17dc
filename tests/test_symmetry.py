"""Symmetry breaking (Section 4): GPU canonisation against the oracle's
Algorithm 5, and the paper's printed class and square counts."""
import os

import numpy as np
import pytest

import oracle
from oracle import orders

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
D, V = 1, 2
THREADS = max(1, min(16, os.cpu_count() or 1))


def _oracle_order(n, vs):
    hc = orders.hourglass_cells(n, vs)
    return hc, hc + [c for c in orders.md_ad_rows(n, vsym=vs) if c not in hc]


@pytest.mark.parametrize("n,flags", [(5, D), (6, D), (7, D), (6, D | V), (8, D | V)])
def test_classes_match_oracle_everywhere(dls, n, flags):
    from paper_1709_02599_gb300 import symmetry
    vs = bool(flags & V)
    res = symmetry.count_symmetry_broken(n, flags)
    hc, full = _oracle_order(n, vs)
    assert [tuple(map(int, c)) for c in res["order"][:len(hc)]] == hc
    o_hg, _ = oracle.extend(n, flags, full, np.array([orders.identity(n, vs)], np.uint8),
                            len(hc))
    assert (o_hg == res["hourglass_values"]).all()
    ref = oracle.hourglass_classes(n, flags, full, o_hg, threads=THREADS)
    assert (res["class_sizes"].astype(np.int64) == ref).all()
    assert res["class_size_sum"] == len(o_hg)
    direct = oracle.count(n, flags, orders.md_ad_rows(n, vsym=vs), orders.identity(n, vs))[0]
    assert res["total"] == direct


def test_order8_classes_and_total(dls, golden):
    # Section 4.2: 22 192 248 hourglasses in 116 857 classes (at most 192
    # each); Section 5.1: 7 447 587 840 squares with row 0 fixed
    from paper_1709_02599_gb300 import symmetry
    res = symmetry.count_symmetry_broken(8, D)
    assert res["hourglasses"] == golden["hourglass8"]
    assert res["class_size_sum"] == golden["hourglass8"]
    assert res["classes"] == golden["hourglass8_classes"]
    assert res["max_class"] == 192
    assert res["total"] == golden["dls8_row0_fixed"]
    # the GPU's class sizes against the oracle on a sample of hourglasses
    hc, full = _oracle_order(8, False)
    idx = np.arange(0, res["hourglasses"], 997)
    ref = oracle.hourglass_classes(8, D, full, res["hourglass_values"][idx], threads=THREADS)
    assert (res["class_sizes"][idx].astype(np.int64) == ref).all()
    # include canonical ones in the sample
    canon = np.nonzero(res["class_sizes"])[0][::50]
    ref = oracle.hourglass_classes(8, D, full, res["hourglass_values"][canon], threads=THREADS)
    assert (res["class_sizes"][canon].astype(np.int64) == ref).all()


@pytest.mark.slow
def test_vsym10_total(dls, golden):
    # Section 5.4: 82 731 715 264 512 vertically symmetric diagonal Latin
    # squares of order 10 (row 0 fixed), classes of at most 2^5 * 4! = 768
    from paper_1709_02599_gb300 import symmetry
    res = symmetry.count_symmetry_broken(10, D | V)
    assert res["max_class"] <= 768
    assert res["class_size_sum"] == res["hourglasses"]
    hc, full = _oracle_order(10, True)
    idx = np.arange(0, res["hourglasses"], 4999)
    ref = oracle.hourglass_classes(10, D | V, full, res["hourglass_values"][idx], threads=THREADS)
    assert (res["class_sizes"][idx].astype(np.int64) == ref).all()
    assert res["total"] == golden["vsym10_row0_fixed"]


def test_order8_total_resumable(dls, golden, tmp_path):
    """The same total through workunits of base prefixes (row 0 and the main
    diagonal: 1 854 bases), the class sizes and completions on the GPU."""
    from paper_1709_02599_gb300 import symmetry
    res = symmetry.count_symmetry_broken_resumable(8, D, str(tmp_path / "sym8.jsonl"), batch=256)
    assert res["bases"] == 1854 and res["base_depth"] == 15 and res["units"] == 8
    assert res["total"] == golden["dls8_row0_fixed"]
