"""DEBI neighbourhood filtering on the device (mn_set_filtering) against the
plain reference oracle/debi_filter.py:

* the query tree, the bitmaps TD(u) / BU(u) and the filtered DEBI words equal
  the oracle's after every batch -- the frontier maintenance (insertions,
  count-window expiry, explicit deletions, a query registered while the
  filtering is on) reaches exactly the sets of one top-down and one
  bottom-up pass over the live graph;
* enumeration with the filtering on gives the oracle's lists (the filter only
  removes vertices no embedding uses), and it does prune seeds.
"""
import numpy as np
import pytest

from oracle import debi_filter as F
from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import assert_rows_equal, make_graph, vm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def check_sets(g, s, qs, lo, hi, alive=None):
    for qi, q in enumerate(qs):
        TD, BU, (root, parent, tedge, order) = F.filter_sets(s, lo, hi, q, alive)
        groot, gpar, gted, gtd, gbu = g.read_filter(qi)
        assert (groot, gpar, gted) == (root, parent, tedge), f"query {qi}: tree"
        assert (gtd == TD).all(), f"query {qi}: TD differs at {np.argwhere(gtd != TD)[:5].tolist()}"
        assert (gbu == BU).all(), f"query {qi}: BU differs at {np.argwhere(gbu != BU)[:5].tolist()}"
        words = g.read_debi(qi, lo, hi)
        want = F.filtered_words(s, lo, hi, q, alive)
        assert (words == want).all(), f"query {qi}: filtered words"


def filter_queries(iso=True):
    return [gen.q_path(3, labels=[0, 1, 0], vmask=vm(0, None, 1, None), iso=iso, temporal="chain"),
            gen.q_cycle(4, labels=[0, -1, 1, 0], vmask=vm(None, 1, None, 0), iso=iso),
            gen.q_out_star(3, labels=[1, 0, 2], vmask=vm(0, None, None, 1), iso=iso),
            gen.q_tree6(labels=[0, 1, 2, 0, 1], vmask=vm(1, None, 0, None, None, 0), iso=iso,
                        temporal="chain")]


@pytest.mark.parametrize("iso", [True, False])
def test_filter_sets_follow_a_sliding_window(iso):
    """R-MAT window (1,024 vertices, 3 edge labels, window 4,000, batches of
    2,000): sets and words equal the
    oracle after the preload and after every batch, lists equal the oracle."""
    s = gen.rmat_stream(10, 12000, 0.57, 0.19, 0.19, 3, 1.2, 2, 100, seed=0x4D4E0090 + iso)
    qs = filter_queries(iso)
    W, B = 4000, 2000
    with make_graph(s, window=W, max_batch=W) as g:
        g.insert(M.edges_from_stream(s, 0, W), count_only=True)
        for q in qs:
            g.register_query(q)
        g.set_filtering(True)
        check_sets(g, s, qs, 0, W)
        g.reset_stats()
        for lo_b in range(W, 12000, B):
            r = g.insert(M.edges_from_stream(s, lo_b, lo_b + B))
            lo = lo_b - W                         # G1 = [lo, lo_b + B); [lo, lo + B) expires
            for qi, q in enumerate(qs):
                pos = oracle.delta(s, lo, lo_b + B, lo_b, lo_b + B, q)
                neg = oracle.delta(s, lo, lo_b + B, lo, lo + B, q)
                assert r.count_pos[qi] == len(pos) and r.count_neg[qi] == len(neg)
                assert_rows_equal(g.fetch_rows(qi, +1), pos, f"filtered dS+ q{qi}")
                assert_rows_equal(g.fetch_rows(qi, -1), neg, f"filtered dS- q{qi}")
            check_sets(g, s, qs, lo + B, lo_b + B)
        st = g.stats()
        assert st["seeds_filtered"] > 0 and st["filter_changes"] > 0


def test_filter_with_deletes_and_late_registration():
    """Explicit deletions (the reverse pass), then a query registered while
    the filtering is on, on a dense uniform multigraph."""
    s = gen.uniform_stream(150, 6000, 2, 3, seed=0x4D4E0092, attr_range=3)
    qs = filter_queries(True)[:2]
    rng = np.random.default_rng(0x92)
    with make_graph(s, max_batch=3000, capacity=6000) as g:
        for q in qs:
            g.register_query(q)
        g.set_filtering(True)
        g.insert(M.edges_from_stream(s, 0, 3000))
        check_sets(g, s, qs, 0, 3000)
        dele = np.sort(rng.choice(3000, size=700, replace=False)).astype(np.uint64)
        r = g.delete(dele)
        alive = np.ones(3000, dtype=np.uint8)
        mask = np.zeros(3000, dtype=np.uint8)
        mask[dele.astype(np.int64)] = 1
        for qi, q in enumerate(qs):
            neg = oracle.delta(s, 0, 3000, 0, 0, q, batch_mask=mask)
            assert r.count_neg[qi] == len(neg)
            assert_rows_equal(g.fetch_rows(qi, -1), neg, f"delete dS- q{qi}")
        alive[dele.astype(np.int64)] = 0
        check_sets(g, s, qs, 0, 3000, alive)
        r = g.insert(M.edges_from_stream(s, 3000, 6000))
        alive6 = np.concatenate([alive, np.ones(3000, dtype=np.uint8)])
        for qi, q in enumerate(qs):
            bm = np.zeros(6000, dtype=np.uint8)
            bm[3000:] = 1
            pos = oracle.delta(s, 0, 6000, 0, 0, q, alive=alive6, batch_mask=bm)
            assert_rows_equal(g.fetch_rows(qi, +1), pos, f"insert after delete q{qi}")
        q3 = filter_queries(True)[3]
        qs.append(q3)
        qi3 = g.register_query(q3)
        check_sets(g, s, qs, 0, 6000, alive6)
        assert g.count_static(qi3) == oracle.count_static(s, 0, 6000, q3, alive=alive6)
        g.set_filtering(False)
        assert g.count_static(qi3) == oracle.count_static(s, 0, 6000, q3, alive=alive6)
