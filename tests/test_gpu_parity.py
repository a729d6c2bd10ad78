"""CUDA path vs the CPU oracle, element by element (sorted embedding lists and
exact counts), through the C ABI.  Integer results: bit-exact."""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import (assert_rows_equal, c1_queries, make_graph, run_stream_parity, vm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def rmat_small(seed, scale=10, m=30000, labels=8, vlabels=4):
    return gen.rmat_stream(scale, m, 0.57, 0.19, 0.19, labels, 1.2, vlabels, 1000, seed=seed)


def test_c1_tiny_triangle_every_batch():
    """2,000 vertices, 20,000 uniform edges, batches of 256 (78 full + a
    ragged 32), triangle queries under isomorphism and homomorphism."""
    s = gen.uniform_stream(2000, 20000, 3, 4, seed=0x4D4E0001, attr_range=1)
    n = run_stream_parity(s, c1_queries(), batch=256, check_static_every=13)
    assert n == 79


def test_c1_many_parallel_edges_small_vertex_set():
    """Dense multigraph (60 vertices): long adjacency runs, many parallel
    edges, self-loops; several 32-wide chunks per segment."""
    s = gen.uniform_stream(60, 6000, 2, 2, seed=11, attr_range=3)
    qs = [gen.q_cycle(3, iso=True), gen.q_cycle(3, iso=False),
          gen.q_path(2, labels=[0, 1], iso=True, temporal="chain"),
          gen.q_cycle(2, iso=False)]
    run_stream_parity(s, qs, batch=700, only={0, 1, 4, 8})


def shape_queries(rng, temporal="chain", iso=True, elabels=8, vlabels=4):
    """The config-2 shapes with random labels: 4-vertex path, 4-cycle, 5-star,
    6-vertex tree."""
    def lab(k):
        return [int(x) for x in rng.integers(0, elabels, size=k)]

    def vl(k):
        return [int(x) if rng.random() < 0.5 else None for x in rng.integers(0, vlabels, size=k)]

    return [
        gen.q_path(3, labels=lab(3), vmask=vm(*vl(4)), iso=iso, temporal=temporal),
        gen.q_cycle(4, labels=lab(4), vmask=vm(*vl(4)), iso=iso, temporal=temporal),
        gen.q_out_star(4, labels=lab(4), vmask=vm(*vl(5)), iso=iso, temporal=temporal),
        gen.q_tree6(labels=lab(5), vmask=vm(*vl(6)), iso=iso, temporal=temporal),
    ]


@pytest.mark.parametrize("seed", [1, 2])
def test_rmat_sliding_window_temporal(seed):
    """R-MAT power-law multigraph, count window with preload, batches that
    span two sort tiles with a ragged tail; dS+ and dS- every batch."""
    s = rmat_small(100 + seed)
    rng = np.random.default_rng(seed)
    qs = shape_queries(rng)
    run_stream_parity(s, qs, batch=3000, window=9000, preload=9000)


def test_rmat_window_no_temporal_homo():
    s = rmat_small(7, scale=9, m=12000, labels=4, vlabels=2)
    rng = np.random.default_rng(7)
    qs = shape_queries(rng, temporal="none", iso=False, elabels=4, vlabels=2)
    qs[3] = dict(qs[3], iso=True)
    run_stream_parity(s, qs, batch=2500, window=5000, preload=2000)


def test_large_batches_many_tiles():
    """Batches of 9,000 edges: five sort tiles and a ragged tail."""
    s = rmat_small(9, scale=11, m=40000)
    rng = np.random.default_rng(9)
    qs = shape_queries(rng)[:2]
    run_stream_parity(s, qs, batch=9000, window=20000, only={0, 1, 3})


def test_random_queries_multi_query_launch():
    """Twelve random trees and chorded cycles (3..8 vertices) in one graph, on
    a dense multigraph (120 vertices, average degree 50): every query goes
    through one seed list and one enumerator launch per phase."""
    s = gen.uniform_stream(120, 6000, 2, 3, seed=21)
    rng = np.random.default_rng(21)
    qs = []
    for i in range(12):
        nv = int(rng.integers(3, 9))
        kind = "tree" if i % 2 == 0 else "cycle"
        q = gen.random_query(rng, nv, kind, 3, 2, chords=int(rng.integers(1, 3)) if nv >= 4 else 0)
        q["vmask"] = [m if rng.random() < 0.5 else 0 for m in q["vmask"]]
        q["iso"] = bool(i % 3 != 0)
        q["temporal"] = ["chain", "none", "pairs"][i % 3]
        if q["temporal"] == "pairs":
            k = len(q["edges"])
            q["prec"] = [(0, k - 1), (1, 0)] if k >= 2 else []
        qs.append(q)
    run_stream_parity(s, qs, batch=750, window=2000, preload=2000, only={0, 1})


def test_thirty_two_uneven_queries_one_launch():
    """32 concurrent queries of 3..8 vertices (random labelled trees and
    cycles with 1-2 chords, isomorphism, temporal chain) on an R-MAT
    multigraph (scale 10, 12,000 edges, 8 Zipf edge labels): every query's
    seeds of both phases go through one enumerator launch per batch."""
    s = gen.rmat_stream(10, 12000, 0.57, 0.19, 0.19, 8, 1.2, 4, 1000, seed=0x4D4E0003)
    rng = np.random.default_rng(0x4D4E0003)
    qs = []
    for i in range(32):
        nv = int(rng.integers(3, 9))
        kind = "tree" if i % 2 == 0 else "cycle"
        q = gen.random_query(rng, nv, kind, 8, 4, chords=int(rng.integers(1, 3)) if nv >= 4 else 0,
                             iso=True, temporal="chain")
        q["vmask"] = [m if rng.random() < 0.5 else 0 for m in q["vmask"]]
        qs.append(q)
    run_stream_parity(s, qs, batch=3000, window=6000, preload=6000, only={0, 1})


def test_output_lists_regrow_exactly():
    """A tiny initial list capacity: lists are regrown and re-enumerated."""
    s = gen.uniform_stream(300, 5000, 2, 2, seed=5)
    qs = [gen.q_path(2, iso=False), gen.q_cycle(3, iso=False)]
    run_stream_parity(s, qs, batch=1000, out_capacity=4)


def test_debi_words_match_edgematcher():
    s = rmat_small(31, scale=9, m=8000)
    rng = np.random.default_rng(31)
    qs = shape_queries(rng)
    qs[0]["edges"][0] = qs[0]["edges"][0][:3] + (100, 700) + qs[0]["edges"][0][5:]
    t = int(s["ts"][4000])
    qs[1]["edges"][1] = qs[1]["edges"][1][:5] + (t, gen.INT64_MAX)
    with make_graph(s, window=5000, max_batch=2000) as g:
        g.insert(M.edges_from_stream(s, 0, 2000))
        qids = [g.register_query(q) for q in qs]          # bulk edgeMatcher
        for lo in range(2000, 8000, 2000):
            g.insert(M.edges_from_stream(s, lo, lo + 2000))  # ingest-time edgeMatcher
        lo, hi, _ = g.info()
        for qi, q in zip(qids, qs):
            assert (g.read_debi(qi, lo, hi) == oracle.debi_words(s, lo, hi, q)).all()


def test_adjacency_is_sorted_live_window():
    """Label-partitioned adjacency = lexicographic sort of the live edges by
    (vertex * L + label, neighbour, seq), both directions."""
    s = rmat_small(41, scale=10, m=20000)
    L = s["num_edge_labels"]
    with make_graph(s, window=7000, max_batch=3000) as g:
        for lo in range(0, 20000, 3000):
            g.insert(M.edges_from_stream(s, lo, min(20000, lo + 3000)))
            wlo, whi, _ = g.info()
            seq = np.arange(wlo, whi, dtype=np.uint64)
            src = s["src"][wlo:whi].astype(np.uint64)
            dst = s["dst"][wlo:whi].astype(np.uint64)
            lab = s["label"][wlo:whi].astype(np.uint64)
            for d, (v, w) in enumerate([(src, dst), (dst, src)]):
                key = v * L + lab
                order = np.lexsort((seq, w, key))
                k, b, sq = g.read_adjacency(d)
                assert (k == key[order]).all() and (b == w[order]).all() and (sq == seq[order]).all()


def test_static_count_and_invariant():
    """|S(G2)| = |S(G)| + |dS+| - |dS-| on the device path, batch by batch."""
    s = rmat_small(51, scale=9, m=10000, labels=3, vlabels=2)
    q = gen.q_path(2, labels=[0, 1], iso=True, temporal="none")
    with make_graph(s, window=4000, max_batch=1500) as g:
        qi = g.register_query(q)
        prev = 0
        for lo in range(0, 10000, 1500):
            r = g.insert(M.edges_from_stream(s, lo, min(10000, lo + 1500)))
            now = g.count_static(qi)
            assert now == prev + r.count_pos[qi] - r.count_neg[qi]
            wlo, whi, _ = g.info()
            assert now == oracle.count_static(s, wlo, whi, q)
            prev = now


def test_explicit_deletes():
    """mn_delete_batch: dS- on the graph before removal, then the deleted
    edges stay invisible to later batches and to new queries."""
    s = gen.uniform_stream(80, 3000, 2, 2, seed=61, attr_range=2)
    qs = [gen.q_cycle(3, iso=True), gen.q_path(2, labels=[0, -1], iso=False, temporal="chain")]
    rng = np.random.default_rng(61)
    n = 3000
    with make_graph(s, max_batch=2000) as g:
        qids = [g.register_query(q) for q in qs]
        g.insert(M.edges_from_stream(s, 0, 2000))
        dele = np.sort(rng.choice(2000, size=300, replace=False)).astype(np.uint64)
        r = g.delete(dele)
        alive = np.ones(2000, dtype=np.uint8)
        mask = np.zeros(2000, dtype=np.uint8)
        mask[dele.astype(np.int64)] = 1
        for qi, q in zip(qids, qs):
            neg = oracle.delta(s, 0, 2000, 0, 0, q, alive=alive, batch_mask=mask)
            assert r.count_neg[qi] == len(neg)
            assert_rows_equal(g.fetch_rows(qi, -1), neg, "delete dS-")
        alive[dele.astype(np.int64)] = 0
        r = g.insert(M.edges_from_stream(s, 2000, n))
        alive_all = np.concatenate([alive, np.ones(n - 2000, dtype=np.uint8)])
        for qi, q in zip(qids, qs):
            bm = np.zeros(n, dtype=np.uint8)
            bm[2000:] = 1
            pos = oracle.delta(s, 0, n, 0, 0, q, alive=alive_all, batch_mask=bm)
            assert_rows_equal(g.fetch_rows(qi, +1), pos, "insert after delete")
        # a query registered after the deletion does not see deleted edges
        q2 = gen.q_cycle(3, iso=False)
        qi2 = g.register_query(q2)
        assert g.count_static(qi2) == oracle.count_static(s, 0, n, q2, alive=alive_all)
        # deleting a dead or repeated seq is rejected and changes nothing
        with pytest.raises(M.MnError) as ei:
            g.delete(np.array([dele[0]], dtype=np.uint64))
        assert ei.value.status == -1
        with pytest.raises(M.MnError):
            g.delete(np.array([2500, 2500], dtype=np.uint64))
        assert g.count_static(qi2) == oracle.count_static(s, 0, n, q2, alive=alive_all)


def test_invalid_batches_apply_nothing():
    s = gen.uniform_stream(100, 4000, 2, 2, seed=71)
    q = gen.q_cycle(3, iso=False)
    with make_graph(s, window=2000, max_batch=1000) as g:
        qi = g.register_query(q)
        g.insert(M.edges_from_stream(s, 0, 1000))
        bad = M.edges_from_stream(s, 1000, 2000)
        bad["src"][500] = 100                     # vertex out of range
        with pytest.raises(M.MnError) as ei:
            g.insert(bad)
        assert ei.value.status == -2
        bad = M.edges_from_stream(s, 1000, 2000)
        bad["ts"][700] = bad["ts"][699]           # not strictly increasing
        with pytest.raises(M.MnError) as ei:
            g.insert(bad)
        assert ei.value.status == -3
        old = M.edges_from_stream(s, 0, 10)       # older than the last timestamp
        with pytest.raises(M.MnError):
            g.insert(old)
        assert g.info()[:2] == (0, 1000)
        r = g.insert(M.edges_from_stream(s, 1000, 2000))
        pos = oracle.delta(s, 0, 2000, 1000, 2000, q)
        assert_rows_equal(g.fetch_rows(qi, +1), pos, "after rejected batches")
        assert r.count_pos[qi] == len(pos)


def test_work_budget_timeout_is_reported_and_recoverable():
    """A bounded device loop that runs out returns MN_ERR_TIMEOUT through a
    status word (no trap, no hang); the context and the graph stay usable."""
    s = gen.uniform_stream(50, 3000, 1, 1, seed=81)
    q = gen.q_path(3, iso=False)
    with make_graph(s, max_batch=1000) as g:
        qi = g.register_query(q)
        g.insert(M.edges_from_stream(s, 0, 1000))
        g.set_work_budget(2)
        with pytest.raises(M.MnError) as ei:
            g.insert(M.edges_from_stream(s, 1000, 2000))
        assert ei.value.status == -7
        g.set_work_budget(0)
        r = g.insert(M.edges_from_stream(s, 2000, 3000))
        pos = oracle.delta(s, 0, 3000, 2000, 3000, q)
        assert r.count_pos[qi] == len(pos)
        assert g.count_static(qi) == oracle.count_static(s, 0, 3000, q)


def test_empty_batch_and_single_edge_query():
    s = gen.uniform_stream(30, 500, 2, 3, seed=91, attr_range=5)
    q1 = gen.make_query(2, [(0, 1, 1, (1, 4))], vmask=vm(0, None), iso=True)
    with make_graph(s, window=300, max_batch=200) as g:
        qi = g.register_query(q1)
        r = g.insert(M.edges_from_stream(s, 0, 0))
        assert r.count_pos == [0] and r.count_neg == [0]
        for lo in range(0, 500, 200):
            hi = min(500, lo + 200)
            g.insert(M.edges_from_stream(s, lo, hi))
        wlo, whi, _ = g.info()
        assert g.count_static(qi) == oracle.count_static(s, wlo, whi, q1)


def test_sorted_fetch_is_the_oracle_order_without_host_sorting():
    """MN_FETCH_SORTED: the device sorts a list by (vertex tuple, edge-seq
    tuple) -- records of odd and even vertex counts (padded layouts), lists
    of 10^5 records (many merge passes), windows at offsets of the sorted
    list, and a later unsorted fetch of the same batch stays sorted."""
    s = gen.uniform_stream(300, 8000, 2, 2, seed=0x4D4E00B0)
    qs = [gen.q_path(2, iso=False), gen.q_path(3, labels=[0, 1, 0], iso=True, temporal="chain")]
    with make_graph(s, window=5000, max_batch=5000) as g:
        for q in qs:
            g.register_query(q)
        g.insert(M.edges_from_stream(s, 0, 5000), count_only=True)
        g.insert(M.edges_from_stream(s, 5000, 8000))
        for qi, q in enumerate(qs):
            nv = q["nv"]
            for sign, (blo, bhi) in ((+1, (5000, 8000)), (-1, (0, 3000))):
                want = oracle.delta(s, 0, 8000, blo, bhi, q)
                v, sq = g.fetch(qi, sign, sorted=True)
                got = np.concatenate([v.astype(np.uint64), sq], axis=1)
                assert got.shape == want.shape and (got == want).all(), (qi, sign)
                if len(want) > 1000:
                    v2, s2 = g.fetch(qi, sign, offset=777, max_records=500, sorted=True)
                    part = np.concatenate([v2.astype(np.uint64), s2], axis=1)
                    assert (part == want[777:1277]).all()
                v3, s3 = g.fetch(qi, sign)            # the list stays sorted for this batch
                assert (np.concatenate([v3.astype(np.uint64), s3], axis=1) == want).all()
        assert max(len(oracle.delta(s, 0, 8000, 5000, 8000, q)) for q in qs) > 100000


def test_maximum_query_size():
    """Queries at the maximum size -- a directed 16-cycle (16 vertices, 16
    edges) under isomorphism and a 15-edge path (16 vertices) under
    homomorphism, one vertex label per query vertex -- over a sliding window:
    every batch's dS+ and dS- equal the oracle's."""
    s = gen.uniform_stream(200, 20000, 16, 4, seed=0x4D4E00D0)
    labels = [i % 4 for i in range(16)]
    vm = [1 << i for i in range(16)]
    qs = [gen.q_cycle(16, labels=labels, vmask=vm, iso=True),
          gen.q_path(15, labels=labels[:15], vmask=vm, iso=False)]
    assert all(q["nv"] == M.MN_MAX_QV for q in qs) and len(qs[0]["edges"]) == M.MN_MAX_QE
    W, B = 14000, 3000
    found = 0
    with make_graph(s, window=W, max_batch=W) as g:
        g.insert(M.edges_from_stream(s, 0, W), count_only=True)
        for q in qs:
            g.register_query(q)
        for lo_b in (W, W + B):
            r = g.insert(M.edges_from_stream(s, lo_b, lo_b + B))
            lo = lo_b - W                        # G1 = [lo, lo_b + B); [lo, lo + B) expires
            for qi, q in enumerate(qs):
                pos = oracle.delta(s, lo, lo_b + B, lo_b, lo_b + B, q)
                neg = oracle.delta(s, lo, lo_b + B, lo, lo + B, q)
                assert r.count_pos[qi] == len(pos) and r.count_neg[qi] == len(neg), (lo_b, qi)
                assert_rows_equal(g.fetch_rows(qi, +1), pos, f"max-size q{qi} dS+ at {lo_b}")
                assert_rows_equal(g.fetch_rows(qi, -1), neg, f"max-size q{qi} dS- at {lo_b}")
                found += len(pos) + len(neg)
    assert found > 1000
