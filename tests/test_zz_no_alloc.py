"""The allocation-free host-buffer entry point, dls_count_host_noalloc.

It is meant for callers that cannot let the library call cudaMalloc (their
own pool owns the device memory, or their path must not pay the implicit
synchronisation of cudaMalloc/cudaFree).  Its device staging and queue head
live in a fixed array inside the library, shared by every call.  This test
calls it through the C ABI twice in a row, on different workloads, and checks
each result against the regular host-buffer entry point dls_count_host and
against the oracle's counts of the same prefixes -- integer counts, so they
must agree exactly -- and checks that an oversized call is refused.  It sits
in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import gpu_cases
import oracle

pytestmark = pytest.mark.gpu

D, V = 1, 2


def _noalloc(dls, lib, n, flags, order, pre):
    from paper_1709_02599_gb300 import _lib
    o = np.ascontiguousarray(np.asarray(order, dtype=np.uint8).reshape(-1, 2))
    pre = np.ascontiguousarray(pre, dtype=np.uint8)
    P, depth = pre.shape
    counts = np.full(P, 0xDEADBEEF, np.uint64)
    tot = _lib.U128()
    cfg = dls.Launch().c()
    rc = lib.dls_count_host_noalloc(n, flags, o.ctypes.data_as(_lib.u8p), len(o),
                                    ctypes.c_void_p(pre.ctypes.data) if P else None, depth, P,
                                    ctypes.c_void_p(counts.ctypes.data), ctypes.byref(tot),
                                    ctypes.byref(cfg), None)
    return rc, counts, tot.value()


def test_noalloc_matches_host_entry_on_two_calls(dls):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    lib = dls.lib()
    first = gpu_cases.split(dls, 7, D, 8)          # order 7, many prefixes
    second = gpu_cases.split(dls, 8, D | V, 6)     # vertically symmetric, fewer
    assert len(second.prefixes) < len(first.prefixes)
    for wl in (first, second):
        rc, got, got_total = _noalloc(dls, lib, wl.n, wl.flags, wl.order, wl.prefixes)
        assert rc == 0, dls.lib().dls_strerror(rc)
        ref, ref_total = dls.count_host(wl.n, wl.flags, wl.order, wl.prefixes)
        assert (got == ref).all()
        assert got_total == ref_total == int(ref.sum())
        exact, _ = oracle.count_many(wl.n, wl.flags, wl.oracle_order, wl.oracle_prefixes,
                                     threads=4)
        assert (got == exact).all()
    # the plain kernel through the same entry point (no queue head needed)
    from paper_1709_02599_gb300 import _lib
    o = np.ascontiguousarray(first.order)
    counts = np.zeros(len(first.prefixes), np.uint64)
    cfg = dls.Launch(kernel=dls.KERNEL_PLAIN).c()
    rc = lib.dls_count_host_noalloc(7, D, o.ctypes.data_as(_lib.u8p), len(o),
                                    ctypes.c_void_p(first.prefixes.ctypes.data),
                                    first.prefixes.shape[1], len(first.prefixes),
                                    ctypes.c_void_p(counts.ctypes.data), None,
                                    ctypes.byref(cfg), None)
    assert rc == 0
    ref, _ = dls.count_host(7, D, first.order, first.prefixes)
    assert (counts == ref).all()


def test_noalloc_rejects_oversized_calls(dls):
    lib = dls.lib()
    from paper_1709_02599_gb300 import _lib
    cap = 4 << 20
    n, depth = 8, 28
    P = cap // (depth + 8) + 1
    pre = np.zeros((P, depth), np.uint8)
    counts = np.zeros(P, np.uint64)
    o = np.ascontiguousarray(dls.fill_order(n, D))
    rc = lib.dls_count_host_noalloc(n, D, o.ctypes.data_as(_lib.u8p), len(o),
                                    ctypes.c_void_p(pre.ctypes.data), depth, P,
                                    ctypes.c_void_p(counts.ctypes.data), None, None, None)
    assert rc == _lib.ERR_CAPACITY
    assert (counts == 0).all()
