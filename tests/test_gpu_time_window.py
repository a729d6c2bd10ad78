"""Time-window snapshots (mn_set_time_window) through the C ABI against the
oracle: after each batch with newest timestamp T the edges with ts <= T - w
expire, their dS- computed on G1 before removal.  Timestamps have random gaps,
so a time window and a count window differ; a window shorter than a batch's
time span also expires edges of the batch itself."""
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


def _stream():
    s = gen.rmat_stream(9, 9000, 0.57, 0.19, 0.19, 4, 1.2, 3, 1000, seed=0x7E)
    rng = np.random.default_rng(0x7E)
    s["ts"] = np.cumsum(rng.integers(1, 6, size=len(s["src"]))).astype(np.int64)
    qs = [gen.q_path(2, labels=[0, 1], vmask=vm(None, 0, None), iso=True, temporal="chain"),
          gen.q_cycle(3, labels=[-1, 0, -1], vmask=vm(None, None, None), iso=False, temporal="none"),
          gen.q_out_star(3, labels=[0, 1, 2], vmask=vm(1, None, None, None), iso=True, temporal="chain")]
    return s, qs


@pytest.mark.parametrize("window", [6000, 1000])
def test_time_window_matches_oracle(window):
    s, qs = _stream()
    n, B = len(s["src"]), 700
    ts = s["ts"]
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=0, max_batch=B,
                edge_capacity=8192, max_queries=len(qs))
    try:
        for q in qs:
            g.register_query(q)
        g.set_time_window(window)
        lo, hi, k, expired = 0, 0, 0, 0
        while hi < n:
            hi_new = min(n, hi + B)
            cut = ts[hi_new - 1] - window
            lo_new = lo + int(np.searchsorted(ts[lo:hi_new], cut, side="right"))
            x = lo_new - lo
            r = g.insert(M.edges_from_stream(s, hi, hi_new))
            assert (r.seq_lo, r.seq_hi, r.expired_lo, r.expired_hi) == (hi, hi_new, lo, lo + x), f"batch {k}"
            if k % 3 == 1 or hi_new == n:
                for qi, q in enumerate(qs):
                    pos = oracle.delta(s, lo, hi_new, hi, hi_new, q)
                    neg = oracle.delta(s, lo, hi_new, lo, lo + x, q)
                    assert r.count_pos[qi] == len(pos) and r.count_neg[qi] == len(neg), f"batch {k} q {qi}"
                    assert_rows_equal(g.fetch_rows(qi, +1), pos, f"batch {k} query {qi} dS+")
                    assert_rows_equal(g.fetch_rows(qi, -1), neg, f"batch {k} query {qi} dS-")
            expired += x
            lo, hi, k = lo_new, hi_new, k + 1
            assert g.info()[:2] == (lo, hi)
        assert expired > 0
        if window < 3 * B:                 # the window is shorter than a batch's time span
            assert lo > n - B
    finally:
        g.close()


def test_time_window_arguments():
    s, _ = _stream()
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=2000, max_batch=500,
                max_queries=1)
    try:
        with pytest.raises(M.MnError) as e:
            g.set_time_window(100)                     # a count window is set already
        assert e.value.status == -1
        with pytest.raises(M.MnError) as e:
            g.set_time_window(-5)
        assert e.value.status == -1
        g.set_time_window(0)
    finally:
        g.close()
