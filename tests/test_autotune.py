"""The autotuner: every trial counts the same squares, the chosen setting
reproduces the oracle's counts, and the result is cached."""
import numpy as np
import pytest

import oracle
from oracle import orders

pytestmark = pytest.mark.gpu
D = 1


def test_autotune_small_problem(dls, tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_1709_02599_gb300 import autotune
    monkeypatch.setattr(autotune, "_CACHE", str(tmp_path / "cache.json"))
    n = 7
    order = dls.fill_order(n, D)
    ident = np.arange(n, dtype=np.uint8)[None]
    base, _ = dls.extend_prefixes(n, D, order, ident, n + 6)       # row 0 + main diagonal
    base = base[::5]
    best = autotune.tune(n, D, order, base, [n + 8, n + 10], shapes=autotune.SHAPES[:3])
    assert not best["cached"]
    assert best["depth"] in (n + 8, n + 10) and best["suffix"] in autotune.SUFFIXES
    assert len(best["trials"]) == 2 * len(autotune.SUFFIXES) + 2
    # the chosen setting gives the oracle's per-prefix counts
    o, pre, _ = autotune.build_problem(n, D, order, base, best["depth"], best["suffix"])
    c = dls.count(n, D, o, torch.from_numpy(pre).cuda(), launch=dls.Launch(**best["launch"]))
    torch.cuda.synchronize()
    o_order = orders.md_ad_rows(n)
    o_base, _ = oracle.extend(n, D, o_order, np.array([orders.identity(n)], np.uint8), n + 6)
    o_pre, _ = oracle.extend(n, D, o_order, o_base[::5], best["depth"])
    assert (o_pre == pre).all()
    ref, _ = oracle.count_many(n, D, o_order, o_pre, threads=8)
    assert (c.cpu().numpy() == ref).all()
    assert best["total"] == int(ref.sum())
    again = autotune.tune(n, D, order, base, [n + 8, n + 10], shapes=autotune.SHAPES[:3])
    assert again["cached"] and again["depth"] == best["depth"]
