"""Python front end of the continuous-batching request server (mt_server_* in
include/motifs.h): submission, the round loop, Poisson arrivals and latency
percentiles.  All counting runs in the library's kernels."""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import MT_OK, _check, _ptr, load_library

_vp = ctypes.c_void_p


class Server:
    """Continuous-batching server over resident per-k tables."""

    def __init__(self, tables: dict, memory_budget: int = 8 << 30, max_slots: int = 64,
                 round_cost: float = 1.6e9, method: int = 0):
        self.lib = load_library()
        self.tables = dict(tables)
        ts = [self.tables[k].handle if k in self.tables else None for k in (3, 4, 5, 6)]
        h = _vp()
        _check(self.lib.mt_server_create(*ts, int(memory_budget), int(max_slots),
                                         float(round_cost), ctypes.byref(h)), "mt_server_create")
        self.handle = h.value
        if method:
            _check(self.lib.mt_server_set_method(self.handle, int(method)),
                   "mt_server_set_method")

    def submit(self, k: int, g) -> int:
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(g.col, dtype=np.int32)
        if col.size == 0:
            col = np.zeros(1, np.int32)
        rid = ctypes.c_uint64()
        _check(self.lib.mt_server_submit(self.handle, int(k), int(g.n), int(rp[-1]), _ptr(rp),
                                         _ptr(col), ctypes.byref(rid)), "mt_server_submit")
        return int(rid.value)

    def step(self):
        c, a, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.mt_server_step(self.handle, ctypes.byref(c), ctypes.byref(a),
                                       ctypes.byref(p)), "mt_server_step")
        return c.value, a.value, p.value

    def result(self, rid: int, k: int):
        """(state, histogram or None, latency ms, status)."""
        st = ctypes.c_int32()
        lat = ctypes.c_double()
        C = self.tables[k].num_classes
        out = np.empty(C, np.uint64)
        status = self.lib.mt_server_result(self.handle, rid, ctypes.byref(st), _ptr(out),
                                           ctypes.byref(lat))
        if status != MT_OK:
            return 3, None, lat.value, status
        return st.value, (out if st.value == 2 else None), lat.value, status

    def used_bytes(self) -> int:
        u = ctypes.c_size_t()
        _check(self.lib.mt_server_used_bytes(self.handle, ctypes.byref(u)), "mt_server_used_bytes")
        return int(u.value)

    def free(self):
        if getattr(self, "handle", None):
            self.lib.mt_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def run_stream(server: Server, requests, arrivals_s=None, timeout_s: float = 600.0):
    """Drive the server until every request is done.

    `requests` is a list of (k, graph); `arrivals_s` their arrival offsets in
    seconds (None: all at once).  Returns per-request results, latencies (ms,
    submission to completion on the host clock) and the wall time."""
    n = len(requests)
    arrivals = np.zeros(n) if arrivals_s is None else np.asarray(arrivals_s, dtype=np.float64)
    order = np.argsort(arrivals, kind="stable")
    ids = [None] * n
    done = {}
    lat = np.zeros(n)
    t0 = time.perf_counter()
    nxt = 0
    outstanding = {}
    while len(done) < n:
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError("serving stream did not finish")
        while nxt < n and arrivals[order[nxt]] <= now:
            i = int(order[nxt])
            k, g = requests[i]
            ids[i] = server.submit(k, g)
            outstanding[ids[i]] = i
            nxt += 1
        completed, active, pending = server.step()
        if outstanding:
            for rid, i in list(outstanding.items()):
                st, hist, ms, status = server.result(rid, requests[i][0])
                if st >= 2:
                    done[i] = (st, hist, status)
                    lat[i] = ms
                    del outstanding[rid]
        if active == 0 and pending == 0 and not outstanding and nxt < n:
            time.sleep(max(0.0, min(0.001, arrivals[order[nxt]] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    return [done[i] for i in range(n)], lat, wall


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
