"""Python side of the continuous-batching server (lider_server_* in the C ABI).

The scheduler, the admission against a memory budget, the per-slot CUDA
streams and staging, and the latency record all live in the native library;
this module marshals arguments, keeps each request's host buffers alive until
it completes, and drives a Poisson load for measurement.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import lider
from .lider import LiderError, ServerCounters, ServerParams, _check, _lib


class Ticket:
    """One submitted request; result() waits for it (the GIL is released
    while waiting) and returns (ids, scores) as host arrays, or raises the
    error of its batch."""

    __slots__ = ("server", "ticket", "queries", "ids", "scores", "_rc", "_msg")

    def __init__(self, server, ticket, queries, ids, scores):
        self.server, self.ticket, self.queries, self.ids, self.scores = server, ticket, queries, ids, scores
        self._rc = None
        self._msg = ""

    def _wait(self, timeout: float | None):
        if self._rc is None:
            rc = _lib.lider_server_wait(self.server._h, self.ticket, -1.0 if timeout is None else float(timeout))
            if rc == lider.ETIMEDOUT:
                raise TimeoutError(lider.last_error())
            self._rc, self._msg = rc, (lider.last_error() if rc else "")
            self.queries = None
            self.server._open.pop(self.ticket, None)

    def result(self, timeout: float | None = None):
        self._wait(timeout)
        if self._rc:
            raise LiderError(self._rc, self._msg)
        return self.ids, self.scores


class Server:
    """Continuous batching over a lider.Index (which must outlive the server).

    c: clusters probed per query; slots: batches in flight; max_batch: queries
    per batch (and per request); max_k: largest k; mem_budget: bytes of search
    scratch the batches in flight may hold together; max_wait_us: batching
    window while the device is busy."""

    def __init__(self, index, c: int, *, slots: int = 3, max_batch: int = 8192, max_k: int = 100,
                 mem_budget: int = 16 << 30, max_wait_us: float = 200.0):
        p = ServerParams(c, slots, max_batch, max_k, mem_budget, max_wait_us)
        h = ctypes.c_void_p()
        _check(_lib.lider_server_create(ctypes.c_void_p(index.handle), ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        self._open = {}          # ticket -> Ticket not yet waited for
        self.index, self.d, self.max_batch, self.max_k = index, index.d, max_batch, max_k

    def submit(self, queries: np.ndarray, k: int) -> Ticket:
        q = np.ascontiguousarray(queries, dtype=np.float32)
        if q.ndim != 2 or q.shape[1] != self.d:
            raise ValueError(f"queries must be (nq, {self.d})")
        nq = q.shape[0]
        ids = np.empty((nq, k), dtype=np.int64)
        sc = np.empty((nq, k), dtype=np.float32)
        t = ctypes.c_int64()
        _check(_lib.lider_server_submit(self._h, q.ctypes.data, nq, k, ids.ctypes.data, sc.ctypes.data,
                                        ctypes.byref(t)))
        tk = Ticket(self, t.value, q, ids, sc)
        self._open[t.value] = tk
        return tk

    def stats(self) -> dict:
        st = ServerCounters()
        _check(_lib.lider_server_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def latencies_ms(self, clear: bool = False) -> np.ndarray:
        total = ctypes.c_int64()
        _check(_lib.lider_server_latencies(self._h, None, 0, 0, ctypes.byref(total)))
        out = np.empty(total.value + 1024, dtype=np.float64)   # room for completions in between
        _check(_lib.lider_server_latencies(self._h, out.ctypes.data, out.shape[0], int(clear), ctypes.byref(total)))
        return out[:min(total.value, out.shape[0])].copy()

    def close(self):
        """Finish every submitted request (their results stay readable), then
        stop the server."""
        if getattr(self, "_h", None) is not None and self._h.value:
            for tk in list(self._open.values()):
                tk._wait(None)
            _lib.lider_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_schedule(rate_qps: float, duration_s: float, ks=(10, 100), max_req: int = 256, n_queries: int = 10000,
                     seed: int = 0):
    """Arrival times (s), sizes, k and query offsets of a Poisson request
    stream: sizes log-uniform in [1, max_req] queries, k drawn from ks, the
    offered load rate_qps queries/s on average."""
    rng = np.random.default_rng(seed)
    mean_size = (max_req - 1) / np.log(max_req) if max_req > 1 else 1.0
    req_rate = rate_qps / mean_size
    n = int(req_rate * duration_s * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / req_rate, size=n))
    size = np.clip(np.exp(rng.uniform(0, np.log(max_req), size=n)), 1, max_req).astype(np.int64)
    k = rng.choice(np.asarray(ks), size=n)
    off = rng.integers(0, n_queries - size + 1)
    keep = t < duration_s
    return t[keep], size[keep], k[keep], off[keep]


def run_load(server: Server, queries: np.ndarray, schedule):
    """Submit each request of `schedule` at its arrival time and return
    [(offset, size, k, ticket)]."""
    t_arr, size, k, off = schedule
    sent = []
    t0 = time.perf_counter()
    for i in range(t_arr.shape[0]):
        target = t0 + t_arr[i]
        while True:
            dt = target - time.perf_counter()
            if dt <= 0:
                break
            if dt > 2e-4:
                time.sleep(dt - 1e-4)
        o, s = int(off[i]), int(size[i])
        sent.append((o, s, int(k[i]), server.submit(queries[o:o + s], int(k[i]))))
    return sent


__all__ = ["Server", "Ticket", "LiderError", "poisson_schedule", "run_load"]
