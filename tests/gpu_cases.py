"""Workload construction for the GPU tests.

Each workload is built twice from the same seeded indices (dls_inputs): once
by the library (fill order, prefix split -- what the GPU counts) and once by
the oracle (its own order and enumerator -- what the oracle counts).  The two
must agree byte for byte; the oracle only ever sees its own arrays."""
import numpy as np

import dls_inputs
import oracle
from oracle import orders

D, V = 1, 2


class Workload:
    def __init__(self, n, flags, order, prefixes, oracle_order, oracle_prefixes, **extra):
        self.n, self.flags = n, flags
        self.order, self.prefixes = order, prefixes
        self.oracle_order, self.oracle_prefixes = oracle_order, oracle_prefixes
        self.__dict__.update(extra)
        assert [tuple(c) for c in order] == list(oracle_order)
        assert prefixes.shape == oracle_prefixes.shape
        assert (prefixes == oracle_prefixes).all()


def split(dls, n, flags, after_row0, first_rows=1, kind=None, trim=False):
    """Row 0 identity, every valid prefix `after_row0` cells past row 0.
    kind: None = main diagonal, anti-diagonal, rows; dls.ORDER_ROW_MAJOR;
    dls.ORDER_HEURISTIC (the Section 2.3 order after row 0).  trim: both
    orders shortened after the prefix (dls_order_trim on the library's side,
    the oracle's trim_tail on the oracle's)."""
    vs = bool(flags & V)
    if kind is None:
        order = dls.fill_order(n, flags, first_rows=first_rows)
        o_order = orders.md_ad_rows(n, vsym=vs, first_rows=first_rows)
    elif kind == dls.ORDER_ROW_MAJOR:
        order = dls.fill_order(n, flags, kind=kind)
        o_order = orders.row_major(n, vsym=vs)
    else:
        w0 = len(orders.identity(n, vs))
        order = dls.order_complete(n, flags, dls.fill_order(n, flags)[:w0], w0, kind)
        o_order = orders.heuristic_complete(n, orders.row0(n, vs), bool(flags & D), vs)
    w = len(orders.identity(n, vs))
    depth = min(len(o_order), w + after_row0)
    if trim:
        order = dls.order_trim(n, flags, order, depth)
        o_order = orders.trim_tail(n, o_order, depth, diagonal=bool(flags & D), vsym=vs)
        assert [tuple(map(int, c)) for c in order] == o_order
    base = np.array([orders.identity(n, vs)], np.uint8)
    pre, _ = dls.extend_prefixes(n, flags, order, base, depth)
    o_pre, _ = oracle.extend(n, flags, o_order, base, depth)
    return Workload(n, flags, order, pre, o_order, o_pre, depth=depth)


def dls8_diag64(dls, seed=0, k=64, after_row0=20):
    """Order 8, row 0 identity, k seed-drawn main-diagonal fillings, each split
    `after_row0` cells past row 0."""
    n = 8
    order = dls.fill_order(n, D)
    o_order = orders.md_ad_rows(n)
    ident = np.array([orders.identity(n)], np.uint8)
    diags, _ = dls.extend_prefixes(n, D, order, ident, n + (n - 1))
    o_diags, _ = oracle.extend(n, D, o_order, ident, n + (n - 1))
    assert (diags == o_diags).all()
    picks = dls_inputs.choose(len(diags), k, seed)
    pre, par = dls.extend_prefixes(n, D, order, diags[picks], n + after_row0)
    o_pre, o_par = oracle.extend(n, D, o_order, o_diags[picks], n + after_row0)
    assert (par == o_par).all()
    return Workload(n, D, order, pre, o_order, o_pre, parents=par, picks=picks,
                    n_diags=len(diags), depth=n + after_row0)


def vsym10_rows2(dls, seed=0, k=2000):
    """Order 10 vertically symmetric, rows 1-2 fixed after the identity row;
    k seed-drawn prefixes out of all valid ones."""
    n = 10
    order = dls.fill_order(n, D | V, first_rows=3)
    o_order = orders.md_ad_rows(n, vsym=True, first_rows=3)
    ident = np.array([orders.identity(n, True)], np.uint8)
    allp, _ = dls.extend_prefixes(n, D | V, order, ident, 3 * (n // 2))
    o_allp, _ = oracle.extend(n, D | V, o_order, ident, 3 * (n // 2))
    assert (allp == o_allp).all()
    picks = dls_inputs.choose(len(allp), k, seed)
    return Workload(n, D | V, order, allp[picks], o_order, o_allp[picks],
                    population=len(allp), depth=3 * (n // 2))


def sampled_rows(dls, n, flags, rows, count=6):
    """Up to `count` random partial squares with `rows` rows filled (row 0
    included), each decoded from the same seeded draws by the library's and
    the oracle's samplers (draws that run out are skipped by both)."""
    vs = bool(flags & V)
    order = dls.fill_order(n, flags, first_rows=rows)
    o_order = orders.md_ad_rows(n, vsym=vs, first_rows=rows)
    depth = rows * len(orders.identity(n, vs))
    pre, o_pre = [], []
    for k in range(count):
        draws = dls_inputs.draws(1 << 14, seed=n * 100 + rows, stream=k)
        a, ua = dls.sample_prefix(n, flags, order, depth, draws)
        b, ub = oracle.sample_prefix(n, flags, o_order, depth, draws)
        assert ua == ub
        if b is None:
            continue
        pre.append(a)
        o_pre.append(b)
    return Workload(n, flags, order, np.array(pre, np.uint8).reshape(-1, depth), o_order,
                    np.array(o_pre, np.uint8).reshape(-1, depth), depth=depth)


def _cheap(n, vsym, k):
    # the oracle must finish these quickly: order 9 with 2-3 rows fixed has
    # 1e6..1e10 completions per job, order 8 with 2 rows ~1e6
    return not (n == 9 and k <= 3) and not (n == 8 and k == 2 and not vsym)


def make_jobs(dls, count, seed=11):
    """`count` serving jobs of the synthetic mix (dls_inputs.serving_jobs),
    built by the library (serving.build_job) and by the oracle from the same
    draws, cheap enough for the oracle."""
    from paper_1709_02599_gb300 import serving
    jobs = []
    for spec in dls_inputs.serving_jobs(10 * count, seed=seed):
        n, vs, k = spec["n"], spec["vsym"], spec["rows"]
        if not _cheap(n, vs, k):
            continue
        built = serving.build_job(n, vs, k, spec["draws"])
        flags = D | (V if vs else 0)
        w = n // 2 if vs else n
        o_order = orders.md_ad_rows(n, vsym=vs, first_rows=k)
        o_pre, _ = oracle.sample_prefix(n, flags, o_order, k * w, spec["draws"])
        if built is None:
            assert o_pre is None
            continue
        bflags, order, prefix = built
        o_order = orders.heuristic_complete(n, o_order[:k * w], True, vs)
        assert [tuple(c) for c in order] == o_order and (prefix == o_pre).all()
        jobs.append(dict(n=n, flags=flags, order=order, prefix=prefix, o_order=o_order,
                         o_prefix=o_pre, arrival=spec["arrival"]))
        if len(jobs) == count:
            break
    return jobs


def oracle_counts(jobs):
    """The oracle's count of each job."""
    return [oracle.count(j["n"], j["flags"], j["o_order"], j["o_prefix"])[0] for j in jobs]
