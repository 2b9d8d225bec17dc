"""Continuous-batching serving of counting jobs (dls_server_* in dls.h).

    srv = Server(budget=4096)
    jid = srv.submit(n, flags, order, prefix)
    srv.step()                      # one epoch
    for jid, count in srv.poll(): ...

``run_stream`` replays a list of jobs with arrival times in real time against
a server and returns per-job latencies and counts.
"""
import ctypes
import time

import numpy as np

from . import _lib, lib, DIAGONAL, VSYM, ORDER_HEURISTIC, fill_order, order_complete, \
    sample_prefix


class Server:
    def __init__(self, **cfg):
        L = lib()
        c = _lib.ServerCfg()
        L.dls_server_default_cfg(ctypes.byref(c))
        for k, v in cfg.items():
            setattr(c, k, v)
        h = ctypes.c_void_p(0)
        _lib.check(L.dls_server_create(ctypes.byref(c), ctypes.byref(h)), "dls_server_create")
        self._h = h
        self.cfg = c

    def submit(self, n, flags, order, prefix):
        o = np.ascontiguousarray(np.asarray(order, dtype=np.uint8).reshape(-1, 2))
        p = np.ascontiguousarray(np.asarray(prefix, dtype=np.uint8).reshape(-1))
        jid = ctypes.c_int64(0)
        _lib.check(lib().dls_server_submit(self._h, n, flags, o.ctypes.data_as(_lib.u8p), len(o),
                                           p.ctypes.data_as(_lib.u8p) if p.size else None,
                                           p.size, ctypes.byref(jid)), "dls_server_submit")
        return int(jid.value)

    def step(self):
        _lib.check(lib().dls_server_step(self._h), "dls_server_step")

    def poll(self, cap=4096):
        ids = np.zeros(cap, np.int64)
        cnt = np.zeros(cap, np.uint64)
        k = ctypes.c_int(0)
        _lib.check(lib().dls_server_poll(self._h, ids.ctypes.data_as(_lib.i64p),
                                         cnt.ctypes.data_as(_lib.u64p), cap, ctypes.byref(k)),
                   "dls_server_poll")
        return [(int(ids[t]), int(cnt[t])) for t in range(k.value)]

    def stats(self):
        st = _lib.ServerStats()
        _lib.check(lib().dls_server_get_stats(self._h, ctypes.byref(st)), "dls_server_get_stats")
        return {f: int(getattr(st, f)) for f, _ in st._fields_}

    def drain(self, timeout_s=600.0):
        """Step until no job is pending or active; returns [(id, count)]."""
        out = []
        t0 = time.perf_counter()
        while True:
            self.step()
            out += self.poll()
            st = self.stats()
            if st["pending"] == 0 and st["active"] == 0:
                self.step()
                out += self.poll()
                return out
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain in %.0f s" % timeout_s)

    def abort(self):
        """Stop the server (dls_server_abort; any thread): the next step
        raises DlsError with code ABORTED instead of launching an epoch."""
        _lib.check(lib().dls_server_abort(self._h), "dls_server_abort")

    def close(self):
        if self._h:
            lib().dls_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_job(n, vsym, rows, draws, suffix=ORDER_HEURISTIC):
    """(flags, order, prefix) of a serving job: rows 0..rows-1 fixed to a
    random valid partial square decoded from `draws`; the cells after them in
    the order of ``suffix``.  None if the draws ran out."""
    flags = DIAGONAL | (VSYM if vsym else 0)
    order = fill_order(n, flags, first_rows=rows)
    w = n // 2 if vsym else n
    depth = rows * w
    prefix, _ = sample_prefix(n, flags, order, depth, draws)
    if prefix is None:
        return None
    if suffix is not None:
        order = order_complete(n, flags, order, depth, suffix)
    return flags, order, prefix


def run_stream(server, jobs, time_limit_s=None):
    """Replays jobs (dicts with 'arrival' seconds, 'n', 'flags', 'order',
    'prefix') in real time.  Returns {job index: (latency_s, count)} and the
    makespan; jobs unfinished at time_limit_s are left out."""
    order_idx = sorted(range(len(jobs)), key=lambda k: jobs[k]["arrival"])
    t0 = time.perf_counter()
    nxt = 0
    id2k = {}
    arrive = {}
    done = {}
    while len(done) < len(jobs):
        now = time.perf_counter() - t0
        while nxt < len(order_idx) and jobs[order_idx[nxt]]["arrival"] <= now:
            k = order_idx[nxt]
            j = jobs[k]
            jid = server.submit(j["n"], j["flags"], j["order"], j["prefix"])
            id2k[jid] = k
            arrive[k] = t0 + j["arrival"]
            nxt += 1
        server.step()
        tnow = time.perf_counter()
        for jid, cnt in server.poll():
            k = id2k[jid]
            done[k] = (tnow - arrive[k], cnt)
        if nxt == len(order_idx):
            st = server.stats()
            if st["pending"] == 0 and st["active"] == 0 and len(done) == len(jobs):
                break
        elif server.stats()["active"] == 0 and server.stats()["pending"] == 0:
            # idle until the next arrival
            wait = jobs[order_idx[nxt]]["arrival"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.01))
        if time_limit_s is not None and time.perf_counter() - t0 > time_limit_s:
            break
    return done, time.perf_counter() - t0
