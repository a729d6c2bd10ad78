"""mn_count_static_noalloc: the static count for callers that must not
allocate device memory during the call (memory fully reserved by another
framework, latency-critical serving loops).  Its seed scratch is a fixed
device array inside the library; the result must equal mn_count_static.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test; it also passes alone in a fresh
process.
"""
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

pytestmark = pytest.mark.gpu


def test_noalloc_count_matches_allocating_count_twice_in_a_row():
    from paper_2206_09983_b300 import build
    build.build()
    s = gen.uniform_stream(300, 12000, 2, 3, seed=99, attr_range=4)
    qs = [gen.q_cycle(3, labels=[0, -1, 1], iso=True),
          gen.q_path(2, labels=[1, 2], iso=False, temporal="chain")]
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=6000,
                max_batch=2000, max_queries=len(qs))
    try:
        qids = [g.register_query(q) for q in qs]
        for lo in range(0, 8000, 2000):
            g.insert(M.edges_from_stream(s, lo, lo + 2000))
        for qi in qids:
            a1 = g.count_static_noalloc(qi)          # first call: also sets up the scratch
            a2 = g.count_static_noalloc(qi)          # second call reuses the shared scratch
            ref = g.count_static(qi)
            assert a1 == ref and a2 == ref
            wlo, whi, _ = g.info()
            assert ref == oracle.count_static(s, wlo, whi, qs[qi])
        # the window moves: the scratch must not carry the previous call's counts
        g.insert(M.edges_from_stream(s, 8000, 10000))
        for qi in qids:
            b1 = g.count_static_noalloc(qi)
            b2 = g.count_static_noalloc(qi)
            assert b1 == b2 == g.count_static(qi)
    finally:
        g.close()
