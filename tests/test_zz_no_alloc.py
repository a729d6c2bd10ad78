"""mn_count_static_noalloc: the static count for callers that must not
allocate device memory during the call (memory fully reserved by another
framework, latency-critical serving loops).  Its seed scratch is a fixed
device array inside the library; the result must equal mn_count_static.

The test checks that the call allocates nothing (the graph's device-memory
accounting is unchanged across it, with the live window grown past the seed
buffer the allocating count last sized) and that it returns the same counts
as mn_count_static and the oracle.

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
        g.insert(M.edges_from_stream(s, 0, 1000))
        g.count_static(qids[0])                      # sizes its seed buffer for 1,000 live edges
        for lo in range(1000, 8000, 2000):           # the window grows to 6,000 live edges
            g.insert(M.edges_from_stream(s, lo, min(8000, lo + 2000)))
        # the no-allocation calls first, before anything that may allocate
        m0 = g.memory_info()
        got = {}
        for qi in qids:
            a1 = g.count_static_noalloc(qi)          # the first call also sets up the scratch
            a2 = g.count_static_noalloc(qi)          # the second reuses the shared scratch
            got[qi] = (a1, a2)
        m1 = g.memory_info()
        assert (m1["used"], m1["peak"]) == (m0["used"], m0["peak"]), "the no-allocation path allocated"
        for qi in qids:
            ref = g.count_static(qi)                 # grows its seed buffer past 1,000 edges
            assert got[qi] == (ref, ref)
            wlo, whi, _ = g.info()
            assert ref == oracle.count_static(s, wlo, whi, qs[qi])
        assert g.memory_info()["used"] > m1["used"], "the window did not outgrow the seed buffer"
        # the window moves: the scratch must not carry the previous call's counts
        g.insert(M.edges_from_stream(s, 8000, 10000))
        m2 = g.memory_info()
        for qi in qids:
            b1 = g.count_static_noalloc(qi)
            b2 = g.count_static_noalloc(qi)
            assert g.memory_info() == m2
            assert b1 == b2 == g.count_static(qi)
    finally:
        g.close()
