"""The enumerator's one device-side wait (an idle warp polling its slot of
the work-splitting queue, Sec. VI pull-based distribution) has a bound that
the host sets (mn_set_wait_limit).

* With a tiny bound, idle warps give their slots up almost at once; giving
  up is the normal exit and never loses work, so every list still equals the
  oracle's and subtrees are still handed over.
* With MN_WAIT_HOLD (a flag that nothing on the device ever clears), every
  idle wait runs to its bound: the batch reports MN_ERR_TIMEOUT through a
  status word -- no trap, no hang -- and the next batch under the default
  bound is exact again.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import assert_rows_equal, make_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def hub_stream():
    """R-MAT with hubs (4,096 vertices, 4 edge labels): label slices of
    ~100-200 entries, so busy warps split work for the idle ones."""
    return gen.rmat_stream(12, 24000, 0.57, 0.19, 0.19, 4, 1.2, 2, 100, seed=0x4D4E0077)


def hub_queries():
    return [gen.q_path(3, labels=[0, 1, 0], iso=True, temporal="chain"),
            gen.q_out_star(3, labels=[0, 0, 1], iso=True, temporal="chain")]


def check_batch(g, s, qs, lo, hi, hi_new, x, r):
    for qi, q in enumerate(qs):
        pos = oracle.delta(s, lo, hi_new, hi, hi_new, q)
        assert r.count_pos[qi] == len(pos)
        assert_rows_equal(g.fetch_rows(qi, +1), pos, f"q{qi} dS+")
        if x:
            neg = oracle.delta(s, lo, hi_new, lo, lo + x, q)
            assert r.count_neg[qi] == len(neg)
            assert_rows_equal(g.fetch_rows(qi, -1), neg, f"q{qi} dS-")


def test_tiny_wait_bound_is_still_exact():
    s, qs = hub_stream(), hub_queries()
    W, B = 12000, 4000
    split = 0
    for bound in (1, 64):
        with make_graph(s, window=W, max_batch=W) as g:
            g.insert(M.edges_from_stream(s, 0, W), count_only=True)
            for q in qs:
                g.register_query(q)
            g.set_wait_limit(bound)
            g.reset_stats()
            for lo_b in range(W, 24000, B):        # G1 = [lo_b - W, lo_b + B); the oldest B expire
                r = g.insert(M.edges_from_stream(s, lo_b, lo_b + B))
                check_batch(g, s, qs, lo_b - W, lo_b, lo_b + B, B, r)
            split += g.stats()["tasks_split"]
    assert split > 0, "no subtree was handed over: the wait was never exercised"


def test_wait_that_runs_out_reports_timeout_and_recovers():
    s, qs = hub_stream(), hub_queries()
    W, B = 12000, 4000
    with make_graph(s, window=W, max_batch=W) as g:
        g.insert(M.edges_from_stream(s, 0, W), count_only=True)
        for q in qs:
            g.register_query(q)
        g.set_wait_limit(64, hold=True)
        with pytest.raises(M.MnError) as ei:
            g.insert(M.edges_from_stream(s, W, W + B))
        assert ei.value.status == -7                       # MN_ERR_TIMEOUT
        # the batch was applied (its counts may be partial); the next one is exact
        assert g.info()[:2] == (B, W + B)
        g.set_wait_limit(0)
        r = g.insert(M.edges_from_stream(s, W + B, W + 2 * B))
        check_batch(g, s, qs, B, W + B, W + 2 * B, B, r)
        wlo, whi, _ = g.info()
        for qi, q in enumerate(qs):
            assert g.count_static(qi) == oracle.count_static(s, wlo, whi, q)


def test_wait_limit_arguments():
    s = hub_stream()
    with make_graph(s, window=1000, max_batch=500) as g:
        with pytest.raises(M.MnError):
            g._check(g._lib.mn_set_wait_limit(g._h, 1 << 31, 0))
        with pytest.raises(M.MnError):
            g._check(g._lib.mn_set_wait_limit(g._h, 10, 0x80))
