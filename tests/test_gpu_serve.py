"""Serving loop on the device: tenants' batches run concurrently on their own
streams; each request's result is the same alone and in the mix, and equals
the oracle's dS for that batch."""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M
from paper_2206_09983_b300.serve import Server

pytestmark = pytest.mark.gpu


def tenant_a():
    s = gen.uniform_stream(300, 8000, 2, 3, seed=301, attr_range=3)
    qs = [gen.q_cycle(3, labels=[0, -1, 1], iso=True),
          gen.q_path(2, labels=[1, 2], iso=False, temporal="chain")]
    return s, qs, 3000


def tenant_b():
    s = gen.rmat_stream(10, 16000, 0.57, 0.19, 0.19, 4, 1.2, 2, 100, seed=302)
    qs = [gen.q_path(3, labels=[0, 1, 0], iso=True, temporal="chain"),
          gen.q_out_star(3, labels=[0, 1, 2], iso=True, temporal="chain")]
    return s, qs, 6000


def tenant_c():
    s = gen.uniform_stream(100, 6000, 2, 2, seed=303)
    qs = [gen.q_cycle(3, iso=False)]
    return s, qs, 2000


def sizes(n, seed):
    rng = np.random.default_rng(seed)
    out, lo = [], 0
    while lo < n:
        k = int(min(n - lo, rng.integers(200, 1500)))
        out.append((lo, lo + k))
        lo += k
    return out


def make(s, qs, window):
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=window,
                max_batch=1500, max_queries=len(qs))
    for q in qs:
        g.register_query(q)
    return g


def run(tenants):
    srv = Server(mem_budget_bytes=64 << 20, merge=False, max_batch=1500)
    graphs = {}
    for name, (s, qs, w) in tenants.items():
        graphs[name] = make(s, qs, w)
        srv.add_tenant(name, graphs[name], keep_rows=True)
    reqs = {name: [] for name in tenants}
    plans = {name: sizes(len(tenants[name][0]["src"]), hash(name) % 1000) for name in tenants}
    k = 0
    while any(k < len(p) for p in plans.values()):
        for name, p in plans.items():
            if k < len(p):
                lo, hi = p[k]
                reqs[name].append((lo, hi, srv.submit(name, M.edges_from_stream(tenants[name][0], lo, hi))))
        k += 1
    srv.drain()
    srv.close()
    for g in graphs.values():
        g.close()
    return reqs, srv


def test_results_same_alone_and_in_the_mix():
    A = tenant_a()
    alone, _ = run({"a": A})
    mixed, srv = run({"a": A, "b": tenant_b(), "c": tenant_c()})
    ra, rm = alone["a"], mixed["a"]
    assert len(ra) == len(rm)
    for (lo, hi, x), (_, _, y) in zip(ra, rm):
        assert not x.error and not y.error
        assert x.count_pos == y.count_pos and x.count_neg == y.count_neg
        for qi in range(len(A[1])):
            assert (x.rows_pos[qi] == y.rows_pos[qi]).all() and (x.rows_neg[qi] == y.rows_neg[qi]).all()
    # and they are the oracle's per-batch dS (count window of 3000 edges)
    s, qs, W = A
    lo_w = 0
    for lo, hi, r in ra:
        xexp = max(0, hi - lo_w - W)
        for qi, q in enumerate(qs):
            pos = oracle.delta(s, lo_w, hi, lo, hi, q)
            assert (r.rows_pos[qi] == pos).all() and len(r.rows_pos[qi]) == len(pos)
            neg = oracle.delta(s, lo_w, hi, lo_w, lo_w + xexp, q)
            assert len(r.rows_neg[qi]) == len(neg) and (r.rows_neg[qi] == neg).all()
        lo_w += xexp
    # the other tenants' requests all completed too
    assert all(not r.error for name in ("b", "c") for _, _, r in mixed[name])
    assert srv.latency_ms()["n"] == sum(len(v) for v in mixed.values())


def test_merged_requests_equal_the_oracle_for_the_concatenated_batch():
    """merge=True (the mode the serving benchmark runs): requests that queue
    while the tenant's previous batch is on the GPU are admitted together as
    one device batch; every request of a merged group reports that batch's
    result, which must equal the oracle's dS+ / dS- for the concatenated
    edges under the count window."""
    s, qs, W = tenant_a()
    g = make(s, qs, W)
    srv = Server(mem_budget_bytes=64 << 20, merge=True, max_batch=1500)
    srv.add_tenant("a", g, keep_rows=True)
    plan = [(lo, min(len(s["src"]), lo + 150)) for lo in range(0, len(s["src"]), 150)]
    reqs = [srv.submit("a", M.edges_from_stream(s, lo, hi)) for lo, hi in plan]
    srv.drain()
    srv.close()
    g.close()
    assert all(not r.error for r in reqs)
    assert max(r.merged_with for r in reqs) > 1, "no requests were merged"
    # device batches: consecutive requests sharing a batch id, in arrival order
    groups = []
    for (lo, hi), r in zip(plan, reqs):
        if groups and groups[-1][2].batch_id == r.batch_id:
            groups[-1][1] = hi
            groups[-1][3] += 1
        else:
            groups.append([lo, hi, r, 1])
    assert sum(gr[3] for gr in groups) == len(reqs)
    lo_w = 0
    for lo, hi, r, n_req in groups:
        assert r.merged_with == n_req
        x = max(0, hi - lo_w - W)
        for qi, q in enumerate(qs):
            pos = oracle.delta(s, lo_w, hi, lo, hi, q)
            neg = oracle.delta(s, lo_w, hi, lo_w, lo_w + x, q)
            assert r.count_pos[qi] == len(pos) and r.count_neg[qi] == len(neg)
            assert len(r.rows_pos[qi]) == len(pos) and (r.rows_pos[qi] == pos).all()
            assert len(r.rows_neg[qi]) == len(neg) and (r.rows_neg[qi] == neg).all()
        lo_w += x
