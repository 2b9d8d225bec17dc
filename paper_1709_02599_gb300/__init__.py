"""GB300 enumerator of diagonal Latin squares (Kochemazov, Vatutin, Zaikin).

Python binding of the C ABI in include/dls.h: every function here only
marshals arguments and calls libdls.so; every step of the count runs in the
library's CUDA kernels (or, for prefix generation, in its host C++ code).
PyTorch provides device memory and streams.

    import paper_1709_02599_gb300 as dls
    order = dls.fill_order(8, dls.DIAGONAL)             # md, ad, rows
    base = np.arange(8, dtype=np.uint8)[None]          # row 0 = identity
    pre, _ = dls.extend_prefixes(8, dls.DIAGONAL, order, base, 8 + 20)
    counts = dls.count(8, dls.DIAGONAL, order, torch.from_numpy(pre).cuda())
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (DIAGONAL, VSYM, DLS_MAX_N, ORDER_MD_AD_ROWS, ORDER_ROW_MAJOR,  # noqa: F401
                   ORDER_HOURGLASS, ORDER_HEURISTIC, ORDER_HEURISTIC_SQ, KERNEL_PERSISTENT,
                   KERNEL_PLAIN, ERR_TIMEOUT, ERR_ABORTED, UNFINISHED,
                   DlsError)


@dataclass
class Launch:
    """Launch shape (dls_launch_t); zero fields take the library defaults."""
    kernel: int = KERNEL_PERSISTENT
    block_threads: int = 0
    blocks_per_sm: int = 0
    lanes_per_prefix: int = 0
    split_pos: int = 0
    donate: int = 0
    check_every: int = 0
    words: int = 0
    stack: int = 0
    lookahead: int = 0
    fuse: int = 0
    budget: int = 0        # search iterations per lane before stopping (0 = none)
    abort_flag: int = 0    # address of an int the kernel polls (0 = none)
    stack_cap: int = 0     # snapshot entries per lane (0 = the bound)

    def c(self):
        return _lib.LaunchT(self.kernel, self.block_threads, self.blocks_per_sm,
                            self.lanes_per_prefix, self.split_pos, self.donate,
                            self.check_every, self.words, self.stack, self.lookahead,
                            self.fuse, self.budget, self.stack_cap, self.abort_flag or None)


def lib():
    return _lib.load()


def _u8(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _order(order):
    o = _u8(order).reshape(-1, 2)
    return o, o.ctypes.data_as(_lib.u8p), len(o)


def fill_order(n, flags=DIAGONAL, kind=ORDER_MD_AD_ROWS, first_rows=1):
    """Fill order as uint8 [L, 2] (i, j) pairs."""
    L = lib()
    buf = np.zeros((DLS_MAX_N * DLS_MAX_N, 2), np.uint8)
    ln = ctypes.c_int(0)
    _lib.check(L.dls_fill_order(n, flags, kind, first_rows, buf.ctypes.data_as(_lib.u8p),
                                DLS_MAX_N * DLS_MAX_N, ctypes.byref(ln)), "dls_fill_order")
    return buf[:ln.value].copy()


def order_complete(n, flags, order, keep, kind=ORDER_HEURISTIC):
    """Keep the first ``keep`` cells of ``order`` and append the rest of the
    square by the rule of ``kind`` (dls_order_complete)."""
    L = lib()
    o, op, ol = _order(order)
    if keep > ol:
        raise ValueError("keep exceeds the order length")
    buf = np.zeros((DLS_MAX_N * DLS_MAX_N, 2), np.uint8)
    ln = ctypes.c_int(0)
    _lib.check(L.dls_order_complete(n, flags, op, keep, kind, buf.ctypes.data_as(_lib.u8p),
                                    DLS_MAX_N * DLS_MAX_N, ctypes.byref(ln)),
               "dls_order_complete")
    return buf[:ln.value].copy()


TAIL_WINDOW = 6


def order_trim(n, flags, order, keep, window=TAIL_WINDOW):
    """``order`` shortened without changing any count (dls_order_trim): the
    cells of the last cell's row or column among the last ``window`` cells
    move to the end, then the run of that line's off-diagonal cells at the
    end is dropped -- each of them is the last open cell of its column (row)
    and the values these force are exactly those the line lacks.  The first
    ``keep`` cells stay in place.  With vertical symmetry only a row's run
    drops; partial orders come back unchanged."""
    L = lib()
    o, op, ol = _order(order)
    buf = np.zeros((DLS_MAX_N * DLS_MAX_N, 2), np.uint8)
    ln = ctypes.c_int(0)
    _lib.check(L.dls_order_trim(n, flags, op, ol, keep, window, buf.ctypes.data_as(_lib.u8p),
                                DLS_MAX_N * DLS_MAX_N, ctypes.byref(ln)), "dls_order_trim")
    return buf[:ln.value].copy()


def extend_prefixes(n, flags, order, base, depth):
    """All valid assignments of the first ``depth`` order cells extending
    the rows of ``base`` (uint8 [B, base_depth]).  Returns (uint8 [M, depth],
    int64 parents [M])."""
    L = lib()
    o, op, ol = _order(order)
    b = _u8(base)
    if b.ndim == 1:
        b = b.reshape(1, -1)
    nb, bd = b.shape
    bptr = b.ctypes.data_as(_lib.u8p) if b.size else None
    need = ctypes.c_int64(0)
    cap = 1 << 16
    while True:
        out = np.zeros((cap, max(depth, 1)), np.uint8)
        par = np.zeros(cap, np.int64)
        rc = L.dls_extend_prefixes(n, flags, op, ol, bptr, bd, nb, depth,
                                   out.ctypes.data_as(_lib.u8p), cap,
                                   par.ctypes.data_as(_lib.i64p), ctypes.byref(need))
        if rc == _lib.ERR_CAPACITY:
            cap = int(need.value)
            continue
        _lib.check(rc, "dls_extend_prefixes")
        m = int(need.value)
        return out[:m, :depth].copy(), par[:m].copy()


def sample_prefix(n, flags, order, depth, draws):
    """Draw-driven random prefix -> (uint8 [depth], draws used); (None, -1)
    when the draws run out."""
    L = lib()
    o, op, ol = _order(order)
    d = np.ascontiguousarray(np.asarray(draws, dtype=np.uint32))
    out = np.zeros(max(depth, 1), np.uint8)
    used = ctypes.c_int64(0)
    rc = L.dls_sample_prefix(n, flags, op, ol, depth, d.ctypes.data_as(_lib.u32p), d.size,
                             out.ctypes.data_as(_lib.u8p), ctypes.byref(used))
    if rc == _lib.ERR_CAPACITY:
        return None, -1
    _lib.check(rc, "dls_sample_prefix")
    return out[:depth].copy(), int(used.value)


def estimate_nodes(n, flags, order, prefix, seed=0, probes=256):
    """Knuth's random-descent estimate of the search nodes below ``prefix``
    (uint8 values along ``order``): ``probes`` seeded descents, their mean
    (dls_estimate_nodes).  0.0 for an invalid prefix."""
    L = lib()
    o, op, ol = _order(order)
    p = _u8(prefix).ravel()
    out = ctypes.c_double(0.0)
    _lib.check(L.dls_estimate_nodes(n, flags, op, ol,
                                    p.ctypes.data_as(_lib.u8p) if p.size else None, p.size,
                                    int(seed) & ((1 << 64) - 1), probes, ctypes.byref(out)),
               "dls_estimate_nodes")
    return out.value


def multiplier(n, flags):
    return lib().dls_multiplier(n, flags).value()


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def describe_launch(n, flags, order, depth, n_prefixes, launch=None):
    """The kernel and launch shape dls_count_ex would use (dls_describe_launch):
    a dict with 'kernel' (k_snapshot / k_persistent / k_plain_snap / k_plain), 'words'
    ('registers' or 'shared'), 'block_threads', 'grid_blocks', 'smem_bytes',
    'stack_entries', 'fused' (the snapshot search's fused step), 'step' (which
    search step runs)."""
    o, op, ol = _order(order)
    cfg = (launch or Launch()).c()
    info = _lib.LaunchInfo()
    _lib.check(lib().dls_describe_launch(n, flags, op, ol, depth, n_prefixes,
                                         ctypes.byref(cfg), ctypes.byref(info)),
               "dls_describe_launch")
    return {"kernel": _lib.RUN_NAMES[info.run],
            "words": "registers" if info.words == 2 else "shared",
            "block_threads": info.block_threads, "grid_blocks": info.grid_blocks,
            "smem_bytes": info.smem_bytes, "stack_entries": info.stack_entries,
            "fused": bool(info.fused), "step": _lib.STEP_NAMES[info.step]}


def count(n, flags, order, prefixes, counts=None, total=None, nodes=None, launch=None,
          stream=None):
    """Count completions of every prefix on the GPU.

    prefixes: torch uint8 CUDA tensor [P, depth] (contiguous).
    counts / total / nodes: optional torch uint64 CUDA tensors ([P], [1], [1])
    to write into; counts is allocated when None.  Asynchronous on
    ``stream`` (default: torch's current stream).  Returns counts."""
    import torch
    if prefixes.dtype != torch.uint8 or not prefixes.is_cuda or prefixes.dim() != 2:
        raise ValueError("prefixes must be a 2-D uint8 CUDA tensor")
    prefixes = prefixes.contiguous()
    P, depth = prefixes.shape
    if counts is None:
        counts = torch.empty(P, dtype=torch.uint64, device=prefixes.device)
    o, op, ol = _order(order)
    cfg = (launch or Launch()).c()
    _lib.check(lib().dls_count_ex(n, flags, op, ol, _dev_ptr(prefixes) if P else None, depth,
                                  P, _dev_ptr(counts), _dev_ptr(total), _dev_ptr(nodes),
                                  ctypes.byref(cfg), _stream_handle(stream)), "dls_count_ex")
    return counts


def count_weighted(n, flags, order, prefixes, weights=None, counts=None, multiply=False,
                   launch=None, stream=None):
    """Sum of weight x Count over the prefixes, in 128 bits on the device
    (dls_count_weighted): Algorithm 6's total when the weights are class
    sizes; the plain total with weights=None; times the row-0 multiplier
    with multiply=True.  prefixes: uint8 CUDA tensor [P, depth]; weights:
    int32/uint32 CUDA tensor [P] or None; counts: uint64 CUDA tensor [P] to
    receive the counts, or None.  Synchronous; returns a Python int."""
    import torch
    if prefixes.dtype != torch.uint8 or not prefixes.is_cuda or prefixes.dim() != 2:
        raise ValueError("prefixes must be a 2-D uint8 CUDA tensor")
    prefixes = prefixes.contiguous()
    P, depth = prefixes.shape
    if weights is not None:
        weights = weights.contiguous()
        if weights.dtype not in (torch.int32, torch.uint32) or weights.shape != (P,):
            raise ValueError("weights must be a [P] 32-bit CUDA tensor")
    o, op, ol = _order(order)
    cfg = (launch or Launch()).c()
    tot = _lib.U128()
    _lib.check(lib().dls_count_weighted(n, flags, op, ol, _dev_ptr(prefixes) if P else None,
                                        depth, P, _dev_ptr(weights), _dev_ptr(counts),
                                        1 if multiply else 0, ctypes.byref(tot),
                                        ctypes.byref(cfg), _stream_handle(stream)),
               "dls_count_weighted")
    return tot.value()


def count_plain(n, flags, order, prefixes, counts=None, total=None, stream=None):
    """The plain one-thread-per-prefix launch (dls_count_plain)."""
    import torch
    prefixes = prefixes.contiguous()
    P, depth = prefixes.shape
    if counts is None:
        counts = torch.empty(P, dtype=torch.uint64, device=prefixes.device)
    o, op, ol = _order(order)
    _lib.check(lib().dls_count_plain(n, flags, op, ol, _dev_ptr(prefixes) if P else None,
                                     depth, P, _dev_ptr(counts), _dev_ptr(total),
                                     _stream_handle(stream)), "dls_count_plain")
    return counts


def count_host(n, flags, order, prefixes, counts_out=None, launch=None, stream=None):
    """Host-buffer entry point (dls_count_host): prefixes and counts in host
    memory (numpy or CPU torch tensors; pinned memory makes the copies
    asynchronous).  Synchronous.  Returns (counts uint64 [P], total int)."""
    pre = prefixes
    if hasattr(pre, "numpy"):
        pre_np = pre.numpy()
    else:
        pre_np = np.ascontiguousarray(np.asarray(pre, dtype=np.uint8))
    if pre_np.ndim != 2:
        raise ValueError("prefixes must be 2-D")
    P, depth = pre_np.shape
    if counts_out is None:
        counts_out = np.zeros(P, np.uint64)
    cnt_np = counts_out.numpy() if hasattr(counts_out, "numpy") else counts_out
    o, op, ol = _order(order)
    tot = _lib.U128()
    cfg = (launch or Launch()).c()
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _lib.check(lib().dls_count_host(n, flags, op, ol,
                                    ctypes.c_void_p(pre_np.ctypes.data) if P else None,
                                    depth, P, ctypes.c_void_p(cnt_np.ctypes.data),
                                    ctypes.byref(tot), ctypes.byref(cfg), sh),
               "dls_count_host")
    return counts_out, tot.value()


def release():
    lib().dls_release()


def stream_status(stream=None):
    """Status of the last count enqueued on ``stream`` (dls_stream_status):
    waits for the stream; returns (status code, prefixes started).  Status
    DLS_ERR_INTERNAL (10) means the counts are not to be trusted."""
    out = _lib.CountStatus()
    _lib.check(lib().dls_stream_status(_stream_handle(stream), ctypes.byref(out)),
               "dls_stream_status")
    return int(out.status), int(out.prefixes_started)


class Plan:
    """One dls_count_ex call frozen into a CUDA graph (dls_plan_*)."""

    def __init__(self, n, flags, order, prefixes, counts, total=None, launch=None):
        self._keep = (prefixes, counts, total)
        o, op, ol = _order(order)
        P, depth = prefixes.shape
        cfg = (launch or Launch()).c()
        h = ctypes.c_void_p(0)
        _lib.check(lib().dls_plan_create(ctypes.byref(h), n, flags, op, ol,
                                         _dev_ptr(prefixes) if P else None, depth, P,
                                         _dev_ptr(counts), _dev_ptr(total),
                                         ctypes.byref(cfg)), "dls_plan_create")
        self._h = h

    def launch(self, stream=None):
        _lib.check(lib().dls_plan_launch(self._h, _stream_handle(stream)), "dls_plan_launch")

    def status(self, stream=None):
        """(status code, prefixes started) of the last launch on ``stream``
        (dls_plan_status); waits for the stream."""
        out = _lib.CountStatus()
        _lib.check(lib().dls_plan_status(self._h, _stream_handle(stream), ctypes.byref(out)),
                   "dls_plan_status")
        return int(out.status), int(out.prefixes_started)

    def close(self):
        if self._h:
            lib().dls_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
