"""Brute-force square lister for tiny orders.

Test infrastructure only.  It pins the oracle with a method that shares
nothing with a cell-by-cell search: squares are built a whole row at a time
from the list of all N! permutations (the row-by-row approach the paper
describes and rejects for speed in Section 2.1), keeping a partial square only
while its columns hold distinct values and, for diagonal squares, its
diagonal cells hold distinct values.  Vertically symmetric squares (Section
5.4) use only the permutations p with p[j] + p[N-1-j] == N-1.

Use it for N <= 6; the row lists grow like N!.
"""
import itertools

import numpy as np


def permutations(n, vsym=False):
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.int8).reshape(-1, n)
    if vsym:
        perms = perms[(perms.astype(np.int16) + perms[:, ::-1] == n - 1).all(axis=1)]
    return perms


def squares(n, diagonal=True, vsym=False, row0=None, chunk=20000):
    """All N x N squares (int8 [S, N, N]) whose rows are permutations, whose
    columns hold distinct values, whose two diagonals hold distinct values if
    ``diagonal``, whose rows are vertically symmetric if ``vsym`` and whose
    row 0 equals ``row0`` (any row 0 if None)."""
    perms = permutations(n, vsym)
    if row0 is None:
        first = perms
    else:
        r0 = np.asarray(row0, dtype=np.int8).reshape(1, n)
        ok = (perms == r0).all(axis=1).any()
        first = r0 if ok else perms[:0]
    cols = np.arange(n)
    # partial squares: [T, r, n]
    part = first.reshape(-1, 1, n).copy()
    for r in range(1, n):
        kept = []
        for s in range(0, len(part), chunk):
            blk = part[s:s + chunk]                       # [T, r, n]
            T = len(blk)
            # column clash: candidate value equals a value above it
            clash = np.zeros((T, len(perms)), dtype=bool)
            for q in range(r):
                clash |= (blk[:, q, None, :] == perms[None, :, :]).any(axis=2)
            if diagonal:
                md_above = blk[:, np.arange(r), np.arange(r)]          # [T, r]
                ad_above = blk[:, np.arange(r), n - 1 - np.arange(r)]  # [T, r]
                md_new = perms[:, r]                                   # [C]
                ad_new = perms[:, n - 1 - r]
                clash |= (md_above[:, :, None] == md_new[None, None, :]).any(axis=1)
                clash |= (ad_above[:, :, None] == ad_new[None, None, :]).any(axis=1)
            t_idx, c_idx = np.nonzero(~clash)
            if len(t_idx):
                kept.append(np.concatenate([blk[t_idx], perms[c_idx][:, None, :]], axis=1))
        part = np.concatenate(kept, axis=0) if kept else np.zeros((0, r + 1, n), np.int8)
    del cols
    return part


def count_matching(sq, cells, values):
    """How many squares of ``sq`` carry ``values`` in ``cells``."""
    if len(sq) == 0:
        return 0
    ok = np.ones(len(sq), dtype=bool)
    for (i, j), v in zip(cells, values):
        ok &= sq[:, i, j] == v
    return int(ok.sum())
