"""Pins of the oracle's hourglass canonisation (Section 4.1-4.2, Algorithm 5)
that do not go through the GPU.

* Orbits by an independent enumeration: every hourglass of a small order is
  mapped by each generator of the group of M-transformations that keep
  hourglasses -- the vertical mirror (not for vertically symmetric squares,
  Section 5.4), the swap of the symmetric row and column pair k, N-1-k, and
  adjacent transpositions of the indices 1..N/2-1 paired with their mirrors,
  which generate the paired permutations -- followed by renaming the symbols
  so that row 0 reads 0..N-1.  The connected components of the resulting
  graph are the classes.  Algorithm 5, as the oracle implements it, must give
  each class's lexicographically least member (cells compared in row-major
  order) the number of members, and every other member 0.  This code shares
  nothing with the oracle: no transformation loop, no image list, no
  pairwise ComputeDistinct; the orbit of a design is reached by closure.
* Corollary 1 on the CPU: the completions of the canonical hourglasses,
  weighted by class size, add up to the whole count with row 0 fixed.
* The paper's figures for order 8 (Section 4.2): 22 192 248 hourglass
  designs, 116 857 of them canonical, no class larger than 192.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import orders

D, V = oracle.DIAGONAL, oracle.VSYM


def _hourglasses(n, flags):
    """Hourglass cells, the oracle's full order and every hourglass (values
    of those cells, row 0 the identity)."""
    vs = bool(flags & V)
    hc = orders.hourglass_cells(n, vs)
    full = hc + [c for c in orders.md_ad_rows(n, vsym=vs) if c not in hc]
    hg, _ = oracle.extend(n, flags, full, np.array([orders.identity(n, vs)], np.uint8), len(hc))
    return hc, full, hg


def _grids(n, flags, cells, values):
    """[M, n, n] int arrays, -1 where empty; with vertical symmetry the mirror
    cell (i, n-1-j) holds n-1-v."""
    g = np.full((len(values), n, n), -1, np.int16)
    for t, (i, j) in enumerate(cells):
        g[:, i, j] = values[:, t]
        if flags & V:
            g[:, i, n - 1 - j] = n - 1 - values[:, t].astype(np.int16)
    return g


def _generators(n, vsym, with_mirror=True):
    """(row map, column map) pairs: cell (i, j) moves to (r[i], c[j])."""
    ident = list(range(n))
    h = n // 2
    gens = []
    if with_mirror and not vsym:
        gens.append((ident, [n - 1 - j for j in range(n)]))
    for k in range(h):
        s = ident[:]
        s[k], s[n - 1 - k] = n - 1 - k, k
        gens.append((s, s))
    for a in range(1, h - 1):
        s = ident[:]
        s[a], s[a + 1] = a + 1, a
        s[n - 1 - a], s[n - 2 - a] = n - 2 - a, n - 1 - a
        gens.append((s, s))
    return gens


def _move(grids, rmap, cmap):
    n = grids.shape[1]
    rinv = np.argsort(rmap)
    cinv = np.argsort(cmap)
    out = grids[:, rinv][:, :, cinv]
    # rename the symbols so that row 0 reads 0..n-1
    ren = np.argsort(out[:, 0, :], axis=1)  # ren[v] = column of v in row 0
    filled = out >= 0
    renamed = np.take_along_axis(ren, np.where(filled, out, 0).reshape(len(out), -1),
                                 axis=1).reshape(out.shape)
    return np.where(filled, renamed, -1).astype(np.int16)


def _keys(grids):
    # row-major bytes, -1 (empty) as 0: byte order is the lexicographic order
    return [bytes(r) for r in (grids + 1).astype(np.uint8).reshape(len(grids), -1)]


def _orbit_classes(n, flags, cells, values, with_mirror=True):
    """Class size at each class's least member, 0 elsewhere, by closure under
    the generators (union-find over the images)."""
    grids = _grids(n, flags, cells, values)
    keys = _keys(grids)
    index = {k: t for t, k in enumerate(keys)}
    assert len(index) == len(keys)
    parent = list(range(len(keys)))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for rmap, cmap in _generators(n, bool(flags & V), with_mirror):
        img = _keys(_move(grids, rmap, cmap))
        for t, k in enumerate(img):
            u = index[k]  # the image of an hourglass is an hourglass
            a, b = find(t), find(u)
            if a != b:
                parent[a] = b
    members = {}
    for t in range(len(keys)):
        members.setdefault(find(t), []).append(t)
    out = np.zeros(len(keys), np.int64)
    for ms in members.values():
        least = min(ms, key=lambda t: keys[t])
        out[least] = len(ms)
    return out


CASES = [(5, D), (6, D), (7, D), (6, D | V), (8, D | V)]


@pytest.mark.parametrize("n,flags", CASES)
def test_classes_are_the_orbits(n, flags):
    hc, full, hg = _hourglasses(n, flags)
    expect = _orbit_classes(n, flags, hc, hg)
    got = oracle.hourglass_classes(n, flags, full, hg, threads=os.cpu_count() or 1)
    assert (got == expect).all(), (n, flags)
    assert int(got.sum()) == len(hg)
    # class sizes divide the order of the group (orbit-stabiliser)
    h = n // 2
    group = (1 if flags & V else 2) * 2 ** h * int(np.prod(range(1, h)))
    assert all(group % int(s) == 0 for s in got[got > 0])


def test_a_missing_generator_changes_the_classes():
    # the check above is sensitive to the group: without the vertical mirror
    # the orbits of order 6 split, and the oracle's classes no longer match
    hc, full, hg = _hourglasses(6, D)
    partial = _orbit_classes(6, D, hc, hg, with_mirror=False)
    got = oracle.hourglass_classes(6, D, full, hg)
    assert (got != partial).any()
    assert (got > 0).sum() < (partial > 0).sum()


@pytest.mark.parametrize("n,flags,total", [(6, D, 128), (7, D, 171200), (6, D | V, 64),
                                           (8, D | V, 3612672)])
def test_corollary1_total_on_the_cpu(n, flags, total):
    # Corollary 1: sum over canonical hourglasses of class size x completions
    # = squares with row 0 fixed, also counted directly
    hc, full, hg = _hourglasses(n, flags)
    sizes = oracle.hourglass_classes(n, flags, full, hg, threads=os.cpu_count() or 1)
    canon = np.nonzero(sizes)[0]
    counts, _ = oracle.count_many(n, flags, full, hg[canon], threads=os.cpu_count() or 1)
    weighted = sum(int(s) * int(c) for s, c in zip(sizes[canon], counts))
    vs = bool(flags & V)
    direct = oracle.count(n, flags, orders.md_ad_rows(n, vsym=vs), orders.identity(n, vs))[0]
    assert weighted == direct == total


@pytest.mark.slow
def test_order8_class_statistics(golden):
    # Section 4.2: 22 192 248 hourglass designs of order 8, 116 857 classes,
    # at most 192 designs in one; batches of main-diagonal fillings keep the
    # memory small (~21 s on 8 threads)
    n = 8
    hc = orders.hourglass_cells(n)
    full = hc + [c for c in orders.md_ad_rows(n) if c not in hc]
    ndiag = n + sum(1 for (i, j) in hc[n:] if i == j)
    bases, _ = oracle.extend(n, D, full, np.array([orders.identity(n)], np.uint8), ndiag)
    assert len(bases) == 1854
    total = canonical = largest = size_sum = 0
    for s in range(0, len(bases), 64):
        hg, _ = oracle.extend(n, D, full, bases[s:s + 64], len(hc))
        cls = oracle.hourglass_classes(n, D, full, hg, threads=os.cpu_count() or 1)
        total += len(hg)
        canonical += int((cls > 0).sum())
        largest = max(largest, int(cls.max()))
        size_sum += int(cls.sum())
    assert total == size_sum == golden["hourglass8"]
    assert canonical == golden["hourglass8_classes"]
    # the paper's bound, attained: a design whose stabiliser is trivial has
    # one image per element of the group (2 * 2^4 * 3! = 192)
    assert largest == golden["hourglass8_max_class"]
