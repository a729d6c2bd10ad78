"""Host logic of the serving loop (no GPU): admission by memory budget,
per-tenant order, merging of queued requests, overlap across tenants."""
import threading
import time
from types import SimpleNamespace

import numpy as np

from paper_2206_09983_b300 import mnemonic as M
from paper_2206_09983_b300.serve import Server, poisson_batches


class FakeGraph:
    """Stands in for mn_graph: sleeps per edge and records its calls."""

    def __init__(self, log, name, per_edge=2e-6):
        self.log, self.name, self.per_edge = log, name, per_edge
        self.layouts = [(3, 3, 40)]
        self.batch = 0
        self.lock = threading.Lock()

    def insert(self, edges, count_only=False):
        t0 = time.perf_counter()
        time.sleep(self.per_edge * len(edges) + 0.002)
        with self.lock:
            self.batch += 1
            b = self.batch
        self.log.append((self.name, b, t0, time.perf_counter(), len(edges)))
        return SimpleNamespace(batch_id=b, count_pos=[len(edges)], count_neg=[0])


def edges(n):
    return np.zeros(n, dtype=M.EDGE_DTYPE)


def test_budget_order_and_overlap():
    log = []
    s = Server(mem_budget_bytes=400_000, merge=False)
    for name in ("a", "b", "c"):
        s.add_tenant(name, FakeGraph(log, name))
    reqs = []
    for i in range(30):
        reqs.append(s.submit("abc"[i % 3], edges(1000 + 37 * i)))
    s.drain()
    s.close()
    assert all(r.t_done > 0 and not r.error for r in reqs)
    assert s.peak_in_use <= 400_000
    for name in "abc":
        mine = [r for r in reqs if r.tenant == name]
        assert [r.batch_id for r in mine] == sorted(r.batch_id for r in mine)
        assert [r.count_pos[0] for r in mine] == [len(r.edges) for r in mine]
    # batches of different tenants overlapped in time
    spans = sorted((t0, t1, n) for n, _, t0, t1, _ in log)
    assert any(spans[i + 1][0] < spans[i][1] and spans[i + 1][2] != spans[i][2]
               for i in range(len(spans) - 1))


def test_merge_queued_requests():
    log = []
    s = Server(mem_budget_bytes=1 << 30, merge=True, max_batch=10_000)
    g = FakeGraph(log, "a", per_edge=2e-5)
    s.add_tenant("a", g)
    reqs = [s.submit("a", edges(500)) for _ in range(12)]
    s.drain()
    s.close()
    assert max(r.merged_with for r in reqs) > 1          # queued requests were batched
    assert sum(n for *_, n in log) == 12 * 500           # every edge inserted once
    assert all(sum(len(r.edges) for r in reqs if r.batch_id == b) <= 10_000
               for b in {r.batch_id for r in reqs})


def test_oversized_request_admitted_alone():
    log = []
    s = Server(mem_budget_bytes=10_000, merge=False)
    s.add_tenant("a", FakeGraph(log, "a"))
    r = s.submit("a", edges(5000))
    s.drain()
    s.close()
    assert r.t_done > 0


def test_poisson_schedule_covers_stream():
    rng = np.random.default_rng(5)
    sch = poisson_batches(rng, 1_000_000, 1024, 262144, 5e6)
    assert sum(n for _, n in sch) == 1_000_000
    assert all(1 <= n <= 262144 for _, n in sch)
    ts = [t for t, _ in sch]
    assert ts == sorted(ts)


def test_drain_waits_for_empty_requests():
    """A request with no edges reserves no result bytes, yet drain() must
    still wait until it has completed (its insert call takes time too)."""
    log = []
    s = Server(mem_budget_bytes=1 << 20, merge=False)
    s.add_tenant("a", FakeGraph(log, "a", per_edge=0.0))
    reqs = [s.submit("a", edges(0)) for _ in range(5)]
    s.drain()
    done = [r.t_done > 0 for r in reqs]
    s.close()
    assert all(done) and len(log) == 5


class FailingGraph(FakeGraph):
    """Raises on its second insert call."""

    def insert(self, edges, count_only=False):
        if self.batch == 1:
            self.batch += 1
            raise ValueError("device gone")
        return super().insert(edges, count_only)


def test_failed_insert_is_reported_and_the_worker_goes_on():
    log = []
    s = Server(mem_budget_bytes=1 << 20, merge=False)
    s.add_tenant("a", FailingGraph(log, "a"))
    reqs = [s.submit("a", edges(100)) for _ in range(4)]
    s.drain(timeout=30)
    s.close()
    assert [bool(r.error) for r in reqs] == [False, True, False, False]
    assert "ValueError" in reqs[1].error
    assert s.in_use == 0 and s.inflight == 0
