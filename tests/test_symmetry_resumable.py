"""CPU tests of the resumable symmetry-broken count (Section 4 through the
workunits of Section 5.2): the library's kernels, built for the CPU on the
stand-in runtime, give the class sizes and the completion counts; the totals
must be the oracle's, also after an interrupted run resumes."""
import dataclasses

import numpy as np
import pytest

import oracle
from oracle import orders

D, V = 1, 2


def primitives(emulated, n, flags, calls=None):
    from paper_1709_02599_gb300 import symmetry
    order, k = symmetry.hourglass_order(n, flags)

    def classes_fn(hg):
        rc, sizes = emulated.classes(n, flags, order[:k], hg)
        assert rc == 0
        return sizes

    def count_fn(prefixes, launch):
        if calls is not None:
            calls.append(len(prefixes))
            if len(calls) == 3:
                raise RuntimeError("lost the device")
        rc, res = emulated.count("count", n, flags, order, prefixes, **dataclasses.asdict(launch))
        assert rc == 0
        return res[0]

    return classes_fn, count_fn


@pytest.mark.parametrize("n,flags", [(6, D), (7, D), (6, D | V), (8, D | V)])
def test_totals_equal_the_oracle(dls, emulated, tmp_path, n, flags):
    from paper_1709_02599_gb300 import symmetry
    vs = bool(flags & V)
    direct = oracle.count(n, flags, orders.md_ad_rows(n, vsym=vs), orders.identity(n, vs))[0]
    cf, nf = primitives(emulated, n, flags)
    res = symmetry.count_symmetry_broken_resumable(n, flags, str(tmp_path / "s.jsonl"), batch=8,
                                                   classes_fn=cf, count_fn=nf, min_items=1)
    assert res["total"] == direct
    assert res["units"] == (res["bases"] + 7) // 8 and res["units_counted"] == res["units"]
    assert res["class_check"] is True


def test_a_wrong_class_size_is_caught(dls, emulated, tmp_path):
    # the quorum covers the completion counts; a wrong class size from the
    # canonisation (one size one too large, from a fake of the call) breaks
    # the whole-run invariant and the run raises
    from paper_1709_02599_gb300 import symmetry
    cf, nf = primitives(emulated, 6, D)

    def off_by_one(hg):
        sizes = np.array(cf(hg), copy=True)
        nz = np.nonzero(sizes)[0]
        if len(nz):
            sizes[nz[0]] += 1
        return sizes

    with pytest.raises(RuntimeError, match="class sizes"):
        symmetry.count_symmetry_broken_resumable(6, D, str(tmp_path / "w.jsonl"), batch=8,
                                                 quorum=2, classes_fn=off_by_one, count_fn=nf,
                                                 min_items=1)


def test_interrupted_run_resumes_and_quorum_agrees(dls, emulated, tmp_path):
    from paper_1709_02599_gb300 import symmetry
    path = str(tmp_path / "r.jsonl")
    calls = []
    cf, nf = primitives(emulated, 7, D, calls)
    with pytest.raises(RuntimeError):
        symmetry.count_symmetry_broken_resumable(7, D, path, batch=16, classes_fn=cf,
                                                 count_fn=nf, min_items=1)
    cf, nf = primitives(emulated, 7, D)
    res = symmetry.count_symmetry_broken_resumable(7, D, path, batch=16, classes_fn=cf,
                                                   count_fn=nf, min_items=1)
    assert res["units_resumed"] == 2 and res["total"] == 171200
    assert res["class_check"] is None  # some units came from the checkpoint
    res = symmetry.count_symmetry_broken_resumable(7, D, str(tmp_path / "q.jsonl"), batch=64,
                                                   quorum=2, classes_fn=cf, count_fn=nf,
                                                   min_items=256)
    assert res["total"] == 171200 and res["disagreements"] == 0


def test_per_base_weights_sum_to_the_class_sizes(dls, emulated):
    """With every completion count 1, a base's weight is the sum of the
    class sizes of its canonical hourglasses; over all bases that is the
    number of hourglasses (every hourglass is in exactly one class)."""
    from paper_1709_02599_gb300 import symmetry
    n, flags = 7, D
    order, k = symmetry.hourglass_order(n, flags)
    cf, _ = primitives(emulated, n, flags)
    ones = lambda prefixes, launch: np.ones(len(prefixes), np.uint64)
    counter = symmetry.weighted_counter(n, flags, order, k, cf, ones, min_items=1)
    bases, _ = dls.extend_prefixes(n, flags, order, np.arange(n, dtype=np.uint8)[None], 13)
    hg, _ = dls.extend_prefixes(n, flags, order, bases, k)
    w = counter(bases, None)
    assert int(w.sum()) == len(hg) == 19008
