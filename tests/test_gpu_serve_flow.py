"""Serving on a NetFlow-shaped stream (the generator of the serving
workload at reduced scale: 200K hosts, client -> server flows with Zipf
activity and popularity, ~8 parallel edges per pair, 6 protocol labels):
requests of log-uniform size arrive faster than the GPU serves them, queued
requests are merged into device batches under a memory budget, and every
checked device batch's lists equal the CPU oracle's dS+ / dS- for the
concatenated edges under the count window (batches 0, 1, 2, 3 and every
4th)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M
from paper_2206_09983_b300.serve import Server, poisson_batches

pytestmark = pytest.mark.gpu


def test_flow_stream_serving_sampled_parity():
    from paper_2206_09983_b300 import build
    build.build()
    s = gen.flow_stream(200_000, 1_600_000, 6, seed=0x4D4E0055, zipf_s=1.1)
    W, MB = 1 << 20, 1 << 16
    qs = [gen.q_path(2, labels=[0, 1], iso=True, temporal="chain"),
          gen.q_path(3, labels=[0, -1, 0], iso=True, temporal="chain")]
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=W, max_batch=MB,
                max_queries=len(qs), out_capacity=1 << 16)
    for lo in range(0, W, MB):
        g.insert(M.edges_from_stream(s, lo, lo + MB), count_only=True)
    for q in qs:
        g.register_query(q)
    rng = np.random.default_rng(0x5E50)
    sched = poisson_batches(rng, 400_000, 1 << 10, MB, 1e12)     # a backlog: requests queue and merge
    srv = Server(mem_budget_bytes=256 << 20, merge=True, max_batch=MB)
    srv.add_tenant("flow", g, keep_rows=True)
    pos, plan, reqs = W, [], []
    for _, size in sched:
        plan.append((pos, pos + size))
        reqs.append(srv.submit("flow", M.edges_from_stream(s, pos, pos + size)))
        pos += size
    srv.drain()
    srv.close()
    g.close()
    assert all(not r.error for r in reqs)
    assert max(r.merged_with for r in reqs) > 1, "no requests were merged"
    groups = []
    for (lo, hi), r in zip(plan, reqs):
        if groups and groups[-1][2].batch_id == r.batch_id:
            groups[-1][1] = hi
        else:
            groups.append([lo, hi, r])
    lo_w, checked = 0, 0
    for k, (lo, hi, r) in enumerate(groups):
        x = max(0, hi - lo_w - W)
        if k in (0, 1, 2, 3) or k % 4 == 0:
            for qi, q in enumerate(qs):
                pos_rows = oracle.delta(s, lo_w, hi, lo, hi, q)
                neg_rows = oracle.delta(s, lo_w, hi, lo_w, lo_w + x, q)
                assert r.count_pos[qi] == len(pos_rows) and r.count_neg[qi] == len(neg_rows), (k, qi)
                assert (r.rows_pos[qi] == pos_rows).all() and (r.rows_neg[qi] == neg_rows).all(), (k, qi)
            checked += 1
        lo_w += x
    assert checked >= 4
