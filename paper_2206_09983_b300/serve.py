"""Streaming request loop over resident graphs (continuous batching).

A request is a batch of edges for one tenant (one mn_graph: its edge ring,
adjacency, DEBI words and window stay resident on the device).  Each tenant
has one CUDA stream (owned by its graph) and one worker thread; the C calls
release the GIL, so batches of different tenants run on the device at the
same time.  Requests are admitted continuously -- as soon as their tenant's
slot is free and the device-memory budget has room for them -- not in waves.
With ``merge=True`` a tenant's queued requests are admitted together as one
batch (up to max_batch); the batch's results then belong to all of them.
Within a tenant, requests run in arrival order, so each request's result is
the one the paper's snapshot loop (Alg. 1) gives for that batch sequence.

Admission by memory: a request reserves its staging bytes (24 B per edge) plus
an estimate of its result lists (a running average of record bytes per edge
for that tenant, times a safety factor) from a shared budget, and releases
them when it completes.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import mnemonic as M


@dataclass
class Request:
    tenant: str
    edges: np.ndarray
    t_arrival: float
    rid: int
    t_admit: float = 0.0
    t_done: float = 0.0
    batch_id: int = 0
    count_pos: list = field(default_factory=list)
    count_neg: list = field(default_factory=list)
    rows_pos: list = field(default_factory=list)
    rows_neg: list = field(default_factory=list)
    merged_with: int = 1
    error: str = ""

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class _Tenant:
    def __init__(self, name: str, graph, keep_rows: bool, count_only: bool):
        self.name = name
        self.graph = graph
        self.queue: collections.deque = collections.deque()
        self.keep_rows = keep_rows
        self.count_only = count_only
        self.bytes_per_edge = 64.0      # running estimate of result bytes per inserted edge
        self.thread = None
        self.batches = []               # per device batch: (edges, requests, seconds in the insert call)


class Server:
    """Continuous-batching front end for a set of tenant graphs."""

    def __init__(self, mem_budget_bytes: int = 1 << 30, merge: bool = False,
                 max_batch: int = 1 << 16, safety: float = 2.0):
        self.budget = int(mem_budget_bytes)
        self.in_use = 0
        self.peak_in_use = 0
        self.inflight = 0               # device batches admitted and not yet completed
        self.merge = merge
        self.max_batch = max_batch
        self.safety = safety
        self.tenants: dict[str, _Tenant] = {}
        self.cv = threading.Condition()
        self.closed = False
        self.done: list[Request] = []
        self._rid = 0

    # ------------------------------------------------------------ setup
    def add_tenant(self, name: str, graph, keep_rows: bool = False, count_only: bool = False):
        t = _Tenant(name, graph, keep_rows, count_only)
        self.tenants[name] = t
        t.thread = threading.Thread(target=self._worker, args=(t,), daemon=True)
        t.thread.start()
        return t

    # ------------------------------------------------------------ requests
    def submit(self, tenant: str, edges: np.ndarray, t_arrival: float | None = None) -> Request:
        with self.cv:
            self._rid += 1
            r = Request(tenant, edges, time.perf_counter() if t_arrival is None else t_arrival,
                        self._rid)
            self.tenants[tenant].queue.append(r)
            self.cv.notify_all()
            return r

    def _need(self, t: _Tenant, n: int) -> int:
        return int(24 * n + self.safety * t.bytes_per_edge * n)

    def _take(self, t: _Tenant):
        """Requests to admit now for tenant t (under the lock), or None."""
        if not t.queue:
            return None
        first = t.queue[0]
        need = self._need(t, len(first.edges))
        # a request larger than the whole budget is admitted alone when idle
        if self.in_use + need > self.budget and self.in_use > 0:
            return None
        reqs = [t.queue.popleft()]
        n = len(first.edges)
        while self.merge and t.queue:
            nxt = t.queue[0]
            extra = self._need(t, len(nxt.edges))
            if n + len(nxt.edges) > self.max_batch or self.in_use + need + extra > self.budget:
                break
            reqs.append(t.queue.popleft())
            n += len(nxt.edges)
            need += extra
        self.in_use += need
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        self.inflight += 1
        return reqs, need

    def _worker(self, t: _Tenant):
        while True:
            with self.cv:
                got = None
                while not self.closed:
                    got = self._take(t)
                    if got is not None:
                        break
                    self.cv.wait(0.05)
                if got is None:
                    return
            reqs, need = got
            now = time.perf_counter()
            for r in reqs:
                r.t_admit = now
            edges = reqs[0].edges if len(reqs) == 1 else np.concatenate([r.edges for r in reqs])
            err = ""
            res = None
            rows = ([], [])
            t_ins = time.perf_counter()
            # any failure is reported on the batch's requests, and the worker
            # goes on: its reservation is released below either way
            try:
                res = t.graph.insert(edges, count_only=t.count_only)
            except M.MnError as e:
                err = str(e)
            except Exception as e:                     # noqa: BLE001 -- reported per request
                err = f"{type(e).__name__}: {e}"
            t.batches.append((len(edges), len(reqs), time.perf_counter() - t_ins))
            if res is not None and t.keep_rows and not t.count_only:
                try:
                    for qi in range(len(res.count_pos)):
                        rows[0].append(t.graph.fetch_rows(qi, +1))
                        rows[1].append(t.graph.fetch_rows(qi, -1))
                except Exception as e:                 # noqa: BLE001 -- reported per request
                    err = f"{type(e).__name__}: {e}"
            done = time.perf_counter()
            with self.cv:
                for r in reqs:
                    r.t_done = done
                    r.merged_with = len(reqs)
                    r.error = err
                    if res is not None:
                        r.batch_id = res.batch_id
                        r.count_pos = list(res.count_pos)
                        r.count_neg = list(res.count_neg)
                        r.rows_pos, r.rows_neg = rows
                    self.done.append(r)
                if res is not None and len(edges):
                    rec = t.graph.layouts
                    out = sum((res.count_pos[i] + res.count_neg[i]) * rec[i][2]
                              for i in range(len(res.count_pos)))
                    t.bytes_per_edge = 0.8 * t.bytes_per_edge + 0.2 * out / len(edges)
                self.in_use -= need
                self.inflight -= 1
                self.cv.notify_all()

    def drain(self, timeout: float = 600.0):
        """Wait until every submitted request has completed."""
        deadline = time.perf_counter() + timeout
        with self.cv:
            # an admitted batch counts until it completes, also one that
            # reserved no bytes (a request without edges)
            while any(t.queue for t in self.tenants.values()) or self.inflight > 0:
                left = deadline - time.perf_counter()
                if left <= 0:
                    raise TimeoutError("requests still pending")
                self.cv.wait(min(left, 0.05))

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.tenants.values():
            if t.thread is not None:
                t.thread.join(timeout=60)

    # ------------------------------------------------------------ reports
    def latency_ms(self, tenant: str | None = None):
        lat = [1e3 * r.latency for r in self.done if tenant is None or r.tenant == tenant]
        if not lat:
            return {"p50": None, "p99": None, "n": 0}
        return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "n": len(lat)}


def poisson_batches(rng: np.random.Generator, total_edges: int, lo: int, hi: int,
                    rate_edges_per_s: float):
    """Arrival schedule: (t_offset_s, size) with log-uniform sizes in [lo, hi]
    and exponential gaps so that the offered load is rate_edges_per_s."""
    out, t, n = [], 0.0, 0
    mean = (hi - lo) / np.log(hi / lo)        # mean of a log-uniform on [lo, hi]
    while n < total_edges:
        size = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        size = min(size, total_edges - n)
        t += rng.exponential(mean / rate_edges_per_s)
        out.append((t, size))
        n += size
    return out
