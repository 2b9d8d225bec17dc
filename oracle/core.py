"""ctypes front end of ``dls_oracle.c``.

Test infrastructure only (see the package docstring).  The C file is compiled
with plain ``gcc -O2`` into ``oracle/_build/liboracle.so`` the first time it is
needed, or by ``build()``.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

DIAGONAL = 1
VSYM = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dls_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the C oracle (gcc, no GPU needed).  Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L",
                               "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_count.argtypes = [ctypes.c_int, ctypes.c_uint, u8p, ctypes.c_int,
                                 u8p, ctypes.c_int, u64p, u64p]
    lib.oracle_count.restype = ctypes.c_int
    lib.oracle_count_many.argtypes = [ctypes.c_int, ctypes.c_uint, u8p, ctypes.c_int,
                                      u8p, ctypes.c_int, ctypes.c_int64, u64p, u64p,
                                      ctypes.c_int]
    lib.oracle_count_many.restype = ctypes.c_int
    lib.oracle_extend.argtypes = [ctypes.c_int, ctypes.c_uint, u8p, ctypes.c_int,
                                  u8p, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                  u8p, ctypes.c_int64, i64p]
    lib.oracle_extend.restype = ctypes.c_int64
    lib.oracle_sample_prefix.argtypes = [ctypes.c_int, ctypes.c_uint, u8p, ctypes.c_int,
                                         ctypes.c_int, u32p, ctypes.c_int64, u8p]
    lib.oracle_sample_prefix.restype = ctypes.c_int64
    lib.oracle_hourglass_classes.argtypes = [ctypes.c_int, ctypes.c_uint, u8p, ctypes.c_int,
                                             u8p, ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_long), ctypes.c_int]
    lib.oracle_hourglass_classes.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _order_array(order):
    arr = np.ascontiguousarray(np.asarray(order, dtype=np.uint8).reshape(-1, 2))
    if arr.size == 0:
        arr = np.zeros((1, 2), np.uint8)[:0]
    return arr


def count(n, flags, order, prefix=()):
    """Count completions of one prefix.  Returns (count, nodes)."""
    lib = _load()
    o = _order_array(order)
    p = np.ascontiguousarray(np.asarray(prefix, dtype=np.uint8).reshape(-1))
    buf = p if p.size else np.zeros(1, np.uint8)
    c = ctypes.c_uint64(0)
    nd = ctypes.c_uint64(0)
    rc = lib.oracle_count(n, flags, _ptr(o if o.size else np.zeros(2, np.uint8), ctypes.c_uint8),
                          len(o), _ptr(buf, ctypes.c_uint8), p.size,
                          ctypes.byref(c), ctypes.byref(nd))
    if rc != 0:
        raise ValueError("oracle_count: bad arguments")
    return int(c.value), int(nd.value)


def count_many(n, flags, order, prefixes, threads=1):
    """Count completions of each row of ``prefixes`` (uint8 [P, depth]).

    Returns (counts uint64 [P], nodes uint64 [P])."""
    lib = _load()
    o = _order_array(order)
    pre = np.ascontiguousarray(np.asarray(prefixes, dtype=np.uint8))
    if pre.ndim != 2:
        raise ValueError("prefixes must be 2-D")
    P, depth = pre.shape
    counts = np.zeros(P, np.uint64)
    nodes = np.zeros(P, np.uint64)
    if P == 0:
        return counts, nodes
    buf = pre if pre.size else np.zeros(1, np.uint8)
    rc = lib.oracle_count_many(n, flags, _ptr(o if o.size else np.zeros(2, np.uint8), ctypes.c_uint8),
                               len(o), _ptr(buf, ctypes.c_uint8), depth, P,
                               _ptr(counts, ctypes.c_uint64), _ptr(nodes, ctypes.c_uint64),
                               int(threads))
    if rc != 0:
        raise ValueError("oracle_count_many: bad arguments")
    return counts, nodes


def extend(n, flags, order, base, depth):
    """All valid assignments of the first ``depth`` order cells extending the
    rows of ``base`` (uint8 [B, base_depth]).  Returns (prefixes [M, depth],
    parents int64 [M])."""
    lib = _load()
    o = _order_array(order)
    b = np.ascontiguousarray(np.asarray(base, dtype=np.uint8))
    if b.ndim == 1:
        b = b.reshape(1, -1)
    B, bd = b.shape
    bbuf = b if b.size else np.zeros(1, np.uint8)
    obuf = o if o.size else np.zeros(2, np.uint8)
    cap = 1 << 16
    while True:
        out = np.zeros((cap, max(depth, 1)), np.uint8)
        parents = np.zeros(cap, np.int64)
        total = lib.oracle_extend(n, flags, _ptr(obuf, ctypes.c_uint8), len(o),
                                  _ptr(bbuf, ctypes.c_uint8), bd, B, depth,
                                  _ptr(out, ctypes.c_uint8), cap,
                                  _ptr(parents, ctypes.c_int64))
        if total < 0:
            raise ValueError("oracle_extend: bad arguments")
        if total <= cap:
            return out[:total, :depth].copy(), parents[:total].copy()
        cap = int(total)


def sample_prefix(n, flags, order, depth, draws):
    """Draw-driven random prefix; returns (prefix uint8 [depth], draws used)
    or (None, -1) if the draws ran out."""
    lib = _load()
    o = _order_array(order)
    d = np.ascontiguousarray(np.asarray(draws, dtype=np.uint32))
    out = np.zeros(max(depth, 1), np.uint8)
    used = lib.oracle_sample_prefix(n, flags, _ptr(o if o.size else np.zeros(2, np.uint8), ctypes.c_uint8),
                                    len(o), depth,
                                    _ptr(d if d.size else np.zeros(1, np.uint32), ctypes.c_uint32),
                                    d.size, _ptr(out, ctypes.c_uint8))
    if used < 0:
        return None, -1
    return out[:depth].copy(), int(used)


def hourglass_classes(n, flags, order, hourglasses, threads=1):
    """Class size of each hourglass (rows of ``hourglasses``: values of the
    first cells of ``order``) if it is canonic, else 0 (Algorithm 5)."""
    lib = _load()
    o = _order_array(order)
    hg = np.ascontiguousarray(np.asarray(hourglasses, dtype=np.uint8))
    if hg.ndim != 2 or hg.shape[1] > len(o):
        raise ValueError("hourglasses must be 2-D and no longer than the order")
    out = np.zeros(len(hg), dtype=np.int_)
    if len(hg):
        lib.oracle_hourglass_classes(n, flags, _ptr(o, ctypes.c_uint8), hg.shape[1],
                                     _ptr(hg, ctypes.c_uint8), len(hg),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                     int(threads))
    if (out < 0).any():
        raise ValueError("oracle_hourglass_classes: bad arguments")
    return out


def multiplier(n, flags):
    """Number of squares per square with row 0 fixed to 0..N-1.

    Diagonal (and ordinary) Latin squares: every relabelling of the symbols
    keeps the square valid and maps row 0 to the identity in exactly one way,
    so the total is N! times the fixed-row count (Section 2.2; Section 5.2.1
    multiplies the order-9 count by 9!).  Vertically symmetric squares: only
    relabellings that commute with v -> N-1-v keep the symmetry; for even N
    there are 2^(N/2) (N/2)! of them (choose the image pair of each of the N/2
    symbol pairs and an orientation), so that is the factor."""
    if flags & VSYM:
        if n % 2 == 1:
            return 1
        h = n // 2
        return (2 ** h) * math.factorial(h)
    return math.factorial(n)
