"""Queued batches (MN_ASYNC + mn_batch_wait) through the C ABI: the same
results as synchronous inserts and as the oracle, the graph refusing other
calls while a batch is queued, and a queued batch that fails validation
applying nothing."""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import assert_rows_equal, make_graph, vm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def _stream_and_queries():
    s = gen.rmat_stream(10, 24000, 0.57, 0.19, 0.19, 6, 1.2, 3, 1000, seed=0xA5)
    rng = np.random.default_rng(5)
    lab = lambda k: [int(x) for x in rng.integers(0, 6, size=k)]  # noqa: E731
    qs = [gen.q_path(3, labels=lab(3), vmask=vm(0, None, None, 1), iso=True, temporal="chain"),
          gen.q_cycle(3, labels=lab(3), vmask=vm(None, None, None), iso=False, temporal="none"),
          gen.q_out_star(3, labels=lab(3), vmask=vm(None, 2, None, None), iso=True, temporal="chain")]
    return s, qs


def test_async_matches_sync_and_oracle():
    """Window 6,000, batches of 2,500 (a ragged last one): every batch queued
    with MN_ASYNC (host and device input alternating), host work done while it
    runs, then completed; counts and sorted lists equal the synchronous
    path's, and the counts equal the oracle's."""
    s, qs = _stream_and_queries()
    n = len(s["src"])
    W, B = 6000, 2500
    ga = make_graph(s, window=W, max_batch=W, max_queries=len(qs))
    gs = make_graph(s, window=W, max_batch=W, max_queries=len(qs))
    import torch
    dev_edges = torch.from_numpy(M.edges_from_stream(s, 0, n).view(np.uint8)).cuda()
    try:
        for g in (ga, gs):
            g.insert(M.edges_from_stream(s, 0, W), count_only=True)
            for q in qs:
                g.register_query(q)
        for k, (lo, hi, hi_new, x) in enumerate(oracle.window_batches(n, B, W, W)):
            if k % 2:
                bid = ga.insert_async(None, device_ptr=dev_edges.data_ptr() + 24 * hi, n=hi_new - hi)
            else:
                bid = ga.insert_async(M.edges_from_stream(s, hi, hi_new))
            nxt = M.edges_from_stream(s, hi_new, min(n, hi_new + B))    # host work meanwhile
            ra = ga.wait(bid)
            assert ra.batch_id == bid
            rs = gs.insert(M.edges_from_stream(s, hi, hi_new))
            assert (ra.seq_lo, ra.seq_hi, ra.expired_lo, ra.expired_hi) == \
                (rs.seq_lo, rs.seq_hi, rs.expired_lo, rs.expired_hi) == (hi, hi_new, lo, lo + x)
            assert ra.count_pos == rs.count_pos and ra.count_neg == rs.count_neg, f"batch {k}"
            for qi, q in enumerate(qs):
                for sign in (+1, -1):
                    assert_rows_equal(ga.fetch_rows(qi, sign), gs.fetch_rows(qi, sign),
                                      f"batch {k} query {qi} sign {sign}")
                if k in (0, 3):
                    assert ra.count_pos[qi] == len(oracle.delta(s, lo, hi_new, hi, hi_new, q))
                    if x:
                        assert ra.count_neg[qi] == len(oracle.delta(s, lo, hi_new, lo, lo + x, q))
            del nxt
    finally:
        ga.close()
        gs.close()


def test_async_state_rules():
    """While a batch is queued: insert, static counts and deletes give
    MN_ERR_STATE; waiting completes it; waiting again on the completed id is
    fine; an unknown id is an invalid argument."""
    s, qs = _stream_and_queries()
    g = make_graph(s, window=4000, max_batch=4000, max_queries=len(qs))
    try:
        g.insert(M.edges_from_stream(s, 0, 4000), count_only=True)
        qid = g.register_query(qs[0])
        bid = g.insert_async(M.edges_from_stream(s, 4000, 6000))
        for call in (lambda: g.insert(M.edges_from_stream(s, 6000, 7000)),
                     lambda: g.count_static(qid),
                     lambda: g.delete([4100])):
            with pytest.raises(M.MnError) as e:
                call()
            assert e.value.status == -9                            # MN_ERR_STATE
        r = g.wait(bid)
        assert (r.seq_lo, r.seq_hi) == (4000, 6000)
        g.wait(bid)                                                # completed already: fine
        with pytest.raises(M.MnError) as e:
            g.wait(bid + 5)
        assert e.value.status == -1                                # MN_ERR_INVALID_ARG
        r2 = g.insert(M.edges_from_stream(s, 6000, 7000))          # the graph is usable again
        assert (r2.seq_lo, r2.seq_hi) == (6000, 7000)
    finally:
        g.close()


def test_async_validation_error_applies_nothing():
    """A queued batch whose timestamps go backwards is reported by
    mn_batch_wait as MN_ERR_TS_ORDER; the live window is unchanged and the
    next valid batch gives the oracle's dS+."""
    s, qs = _stream_and_queries()
    g = make_graph(s, window=5000, max_batch=5000, max_queries=1)
    try:
        g.insert(M.edges_from_stream(s, 0, 5000), count_only=True)
        qid = g.register_query(qs[1])
        before = g.info()
        bad = M.edges_from_stream(s, 5000, 5100).copy()
        bad["ts"][50] = bad["ts"][10]                              # not strictly increasing
        bid = g.insert_async(bad)
        with pytest.raises(M.MnError) as e:
            g.wait(bid)
        assert e.value.status == -3                                # MN_ERR_TS_ORDER
        assert g.info() == before
        r = g.insert(M.edges_from_stream(s, 5000, 6000))
        assert r.count_pos[qid] == len(oracle.delta(s, 0, 6000, 5000, 6000, qs[1]))
    finally:
        g.close()
