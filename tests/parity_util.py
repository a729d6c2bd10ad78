"""Shared drivers for the GPU-vs-oracle parity tests."""
import numpy as np

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M


def vm(*labels):
    """Query vertex masks from single vertex labels (None = any)."""
    return [0 if l is None else (1 << l) for l in labels]


def c1_queries():
    """The tiny exact config: a labelled directed triangle, two label sets,
    under isomorphism and homomorphism."""
    qs = []
    for iso in (True, False):
        qs.append(gen.q_cycle(3, labels=[-1, -1, -1], vmask=vm(0, 0, 0), iso=iso))
        qs.append(gen.q_cycle(3, labels=[0, -1, -1], vmask=vm(0, 1, 2), iso=iso))
    return qs


def make_graph(stream, window=0, max_batch=4096, out_capacity=0, max_queries=16, capacity=None):
    n = len(stream["src"])
    return M.Graph(stream["num_vertices"], stream["num_edge_labels"], vmask=stream["vmask"],
                   window=window, max_batch=max_batch,
                   edge_capacity=0 if window else (capacity or n), out_capacity=out_capacity,
                   max_queries=max_queries)


def assert_rows_equal(gpu_rows, orc_rows, what=""):
    assert gpu_rows.shape == orc_rows.shape, f"{what}: gpu {gpu_rows.shape} vs oracle {orc_rows.shape}"
    if len(gpu_rows):
        bad = np.nonzero((gpu_rows != orc_rows).any(axis=1))[0]
        assert len(bad) == 0, f"{what}: first mismatch row {bad[0]}: {gpu_rows[bad[0]]} vs {orc_rows[bad[0]]}"


def run_stream_parity(stream, queries, batch, window=0, preload=0, only=None, max_batch=None,
                      out_capacity=0, check_static_every=0):
    """Insert the stream batch by batch; compare every (or the listed)
    batch's dS+ and dS- lists with the oracle for every query."""
    n = len(stream["src"])
    g = make_graph(stream, window=window, max_batch=max_batch or max(batch, preload, 1),
                   out_capacity=out_capacity, max_queries=max(len(queries), 1))
    checked = 0
    try:
        if preload:
            g.insert(M.edges_from_stream(stream, 0, preload), count_only=True)
        qids = [g.register_query(q) for q in queries]
        for k, (lo, hi, hi_new, x) in enumerate(oracle.window_batches(n, batch, window, preload)):
            r = g.insert(M.edges_from_stream(stream, hi, hi_new))
            assert (r.seq_lo, r.seq_hi, r.expired_lo, r.expired_hi) == (hi, hi_new, lo, lo + x)
            if only is not None and k not in only:
                continue
            for qi, q in zip(qids, queries):
                pos = oracle.delta(stream, lo, hi_new, hi, hi_new, q)
                assert r.count_pos[qi] == len(pos), f"batch {k} query {qi}: count+"
                assert_rows_equal(g.fetch_rows(qi, +1), pos, f"batch {k} query {qi} dS+")
                if x:
                    neg = oracle.delta(stream, lo, hi_new, lo, lo + x, q)
                    assert r.count_neg[qi] == len(neg), f"batch {k} query {qi}: count-"
                    assert_rows_equal(g.fetch_rows(qi, -1), neg, f"batch {k} query {qi} dS-")
                else:
                    assert r.count_neg[qi] == 0
                if check_static_every and k % check_static_every == 0:
                    assert g.count_static(qi) == oracle.count_static(stream, lo + x, hi_new, q)
            checked += 1
    finally:
        g.close()
    return checked
