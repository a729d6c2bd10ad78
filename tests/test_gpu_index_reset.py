"""Periodic reset of the candidate index and memory accounting through the C
ABI: after mn_reset_index every query's DEBI words over the live window are
those the stream built (explicitly deleted edges included), and the next
batches' results equal the oracle's; mn_memory_info reports the bytes held,
their peak and the budget."""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import assert_rows_equal, vm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def test_reset_rebuilds_the_same_index_and_results_stay_exact():
    s = gen.rmat_stream(9, 8000, 0.57, 0.19, 0.19, 4, 1.2, 3, 1000, seed=0x1D)
    qs = [gen.q_path(2, labels=[0, 1], vmask=vm(None, 0, None), iso=True, temporal="chain"),
          gen.q_cycle(3, labels=[-1, 0, -1], vmask=vm(None, None, None), iso=False, temporal="none")]
    n, W, B = len(s["src"]), 3000, 1000
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=W, max_batch=W,
                max_queries=len(qs), mem_budget=1 << 30)
    try:
        g.insert(M.edges_from_stream(s, 0, W), count_only=True)
        for q in qs:
            g.register_query(q)
        batches = list(oracle.window_batches(n, B, W, W))
        for lo, hi, hi_new, x in batches[:2]:
            g.insert(M.edges_from_stream(s, hi, hi_new))
        lo, hi, _ = g.info()
        g.delete(np.arange(lo + 10, lo + 400, 7, dtype=np.uint64))
        before = [g.read_debi(qi, lo, hi) for qi in range(len(qs))]
        assert any(b.any() for b in before)
        g.reset_index()
        for qi in range(len(qs)):
            assert np.array_equal(g.read_debi(qi, lo, hi), before[qi]), f"query {qi}"
        # the next batches against the oracle (the deleted edges stay deleted)
        dead = set(range(lo + 10, lo + 400, 7))
        for lo_b, hi_b, hi_new, x in batches[2:4]:
            r = g.insert(M.edges_from_stream(s, hi_b, hi_new))
            alive = np.array([i not in dead for i in range(lo_b, hi_new)], dtype=np.uint8)
            for qi, q in enumerate(qs):
                pos = oracle.delta(s, lo_b, hi_new, hi_b, hi_new, q, alive=alive)
                assert r.count_pos[qi] == len(pos)
                assert_rows_equal(g.fetch_rows(qi, +1), pos, f"query {qi} dS+ after reset")
        mem = g.memory_info()
        assert 0 < mem["used"] <= mem["peak"] <= mem["budget"] == 1 << 30
    finally:
        g.close()
