"""Insert batches launched as one CUDA graph each (mn_set_graph_capture):
the recorded chain -- ingest, adjacency update, filtering, work units, order
choice, enumeration of dS- and dS+ -- gives the oracle's lists; the graph is
updated in place from batch to batch and instantiated again only when the
chain's shape changes (a ragged last batch sorts in fewer merge passes)."""
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


def device_edges(s):
    import torch
    packed = M.edges_from_stream(s, 0, len(s["src"]))
    return torch.from_numpy(packed.view(np.uint8).copy()).cuda()


def check(g, s, qs, lo, hi, hi_new, x, r, what):
    for qi, q in enumerate(qs):
        pos = oracle.delta(s, lo, hi_new, hi, hi_new, q)
        neg = oracle.delta(s, lo, hi_new, lo, lo + x, q) if x else np.zeros((0, q["nv"] + len(q["edges"])),
                                                                           dtype=np.uint64)
        assert r.count_pos[qi] == len(pos) and r.count_neg[qi] == len(neg), what
        assert_rows_equal(g.fetch_rows(qi, +1), pos, f"{what} q{qi} dS+")
        assert_rows_equal(g.fetch_rows(qi, -1), neg, f"{what} q{qi} dS-")


def test_graph_batches_are_exact_and_updated_in_place():
    s = gen.rmat_stream(10, 20000, 0.57, 0.19, 0.19, 4, 1.2, 2, 100, seed=0x4D4E00A0)
    qs = [gen.q_path(3, labels=[0, 1, 0], iso=True, temporal="chain"),
          gen.q_cycle(3, labels=[0, -1, 1], vmask=vm(0, None, 1), iso=True)]
    d = device_edges(s)
    W, B = 6000, 3000
    with make_graph(s, window=W, max_batch=W) as g:
        g.insert(None, device_ptr=d.data_ptr(), n=W, count_only=True)
        for q in qs:
            g.register_query(q)
        g.set_graph_capture(True)
        g.reset_stats()
        nb = 0
        for lo_b in range(W, 20000, B):
            hi_new = min(20000, lo_b + B)
            r = g.insert(None, device_ptr=d.data_ptr() + 24 * lo_b, n=hi_new - lo_b)
            lo = r.expired_lo
            check(g, s, qs, lo, lo_b, hi_new, r.expired_hi - r.expired_lo, r, f"graph batch {nb}")
            nb += 1
        st = g.stats()
        assert st["graph_launches"] == nb
        assert 1 <= st["graph_instantiations"] <= 3, st["graph_instantiations"]


def test_graph_with_filtering_and_learned_orders():
    s = gen.rmat_stream(10, 18000, 0.57, 0.19, 0.19, 3, 1.2, 2, 100, seed=0x4D4E00A1)
    qs = [gen.q_path(3, labels=[0, 1, 0], vmask=vm(0, None, 1, None), iso=True, temporal="chain"),
          gen.q_out_star(3, labels=[1, 0, 2], vmask=vm(0, None, None, 1), iso=True)]
    d = device_edges(s)
    W, B = 6000, 2000
    with make_graph(s, window=W, max_batch=W) as g:
        g.insert(None, device_ptr=d.data_ptr(), n=W, count_only=True)
        for q in qs:
            g.register_query(q)
        g.set_filtering(True)
        g.set_graph_capture(True)
        g.set_order_policy("explore")
        g.reset_stats()
        k = 0
        for lo_b in range(W, 18000, B):
            if k == 3:
                g.train_order_model(epochs=50, lr=2e-3)
                g.set_order_policy("learned")
            r = g.insert(None, device_ptr=d.data_ptr() + 24 * lo_b, n=B)
            check(g, s, qs, lo_b - W, lo_b, lo_b + B, B, r, f"graph+filter batch {k}")
            k += 1
        st = g.stats()
        assert st["graph_launches"] == k and st["seeds_filtered"] > 0
