"""Launch configurations and result-list sizing against the CPU oracle.

* Every configuration the autotuner tries (resident blocks per SM x split
  threshold x split depth x pre-split threshold, and shared-memory staging
  of long last-depth ranges) gives the oracle's lists, on an R-MAT window where
  busy warps do hand subtrees to idle ones; both set explicitly and walked by
  the online autotuner on live batches.
* Multi-label data vertices with query label masks that are proper subsets
  of the data masks (the subset test of the label definition, Sec. II-B).
* Lists that overflow are grown and only their (query, phase) seeds run
  again; lists are then sized from the running records-per-edge estimate so
  later batches need no second launch.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import assert_rows_equal, make_graph, run_stream_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


W, B = 8000, 2000


def split_stream(batches=40):
    """R-MAT, 4,096 vertices, 4 edge labels: hub label slices of ~100-200
    entries (long enough to split) and 10^4-10^5 embeddings per batch."""
    return gen.rmat_stream(12, W + batches * B, 0.57, 0.19, 0.19, 4, 1.2, 2, 100, seed=0x4D4E0078)


def split_queries():
    return [gen.q_path(3, labels=[0, 1, 0], iso=True, temporal="chain"),
            gen.q_cycle(4, labels=[0, 0, 1, 0], iso=True, temporal="none"),
            gen.q_out_star(3, labels=[0, 0, 1], iso=True, temporal="chain")]


_ORACLE = {}


def expected(s, qs, k):
    """Oracle dS+ / dS- of batch k (G1 = [k B, W + (k + 1) B)); streams of
    different lengths are different streams."""
    key = (len(s["src"]), k)
    if key not in _ORACLE:
        lo, hi = k * B, W + k * B
        _ORACLE[key] = [(oracle.delta(s, lo, hi + B, hi, hi + B, q), oracle.delta(s, lo, hi + B, lo, lo + B, q))
                      for q in qs]
    return _ORACLE[key]


def check(g, s, qs, k, r, what):
    for qi, (pos, neg) in enumerate(expected(s, qs, k)):
        assert r.count_pos[qi] == len(pos) and r.count_neg[qi] == len(neg), f"{what} batch {k} q{qi}"
        assert_rows_equal(g.fetch_rows(qi, +1), pos, f"{what} batch {k} q{qi} dS+")
        assert_rows_equal(g.fetch_rows(qi, -1), neg, f"{what} batch {k} q{qi} dS-")


def fresh(s, qs):
    g = make_graph(s, window=W, max_batch=W)
    g.insert(M.edges_from_stream(s, 0, W), count_only=True)
    for q in qs:
        g.register_query(q)
    return g


def test_autotune_candidate_list():
    s, qs = split_stream(), split_queries()
    with fresh(s, qs) as g:
        cands = g.autotune_candidates()
        mx = g.get_tuning()["max_blocks_per_sm"]
    assert len(cands) == 20 and len(set(cands)) == 20
    assert {c[0] for c in cands} == {mx}
    assert {c[1] for c in cands} == {40, 64, 128}
    assert {c[3] for c in cands} == {0.0, 20.0, 22.0}
    assert sorted(c[4] for c in cands if c[4]) == [256, 1024]


def test_every_autotune_configuration_set_explicitly():
    """Paper order: the pre-split threshold has no effect there (nothing
    predicts work), the other axes do."""
    s, qs = split_stream(), split_queries()
    with fresh(s, qs) as g0:
        cands = g0.autotune_candidates()
    split = 0
    for bps, smin, sdep, th, sl in cands:
        with fresh(s, qs) as g:
            g.set_tuning(bps, smin, sdep)
            g.set_presplit(th)
            g.set_slice_staging(sl)
            t = g.get_tuning()
            assert (t["blocks_per_sm"], t["split_min"], t["presplit_log2"]) == (bps, smin, th)
            g.reset_stats()
            for k in (0, 1):
                r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
                check(g, s, qs, k, r, f"bps {bps} split_min {smin} depth {sdep} presplit {th} staging {sl}")
            split += g.stats()["tasks_split"]
    assert split > 0, "no configuration split any work"


def test_learned_presplit_is_exact_and_splits():
    """Learned order with pre-splitting at a threshold every seed passes
    (2^1 predicted cycles): each seed's first depth goes to the queue in
    pieces; lists stay the oracle's and subtrees are handed over."""
    s, qs = split_stream(), split_queries()
    with fresh(s, qs) as g:
        g.set_order_policy("explore")
        for k in range(3):
            r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
            check(g, s, qs, k, r, "explore")
        g.train_order_model(epochs=100, lr=2e-3)
        g.set_order_policy("learned")
        g.set_presplit(1.0)
        g.reset_stats()
        for k in range(3, 6):
            r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
            check(g, s, qs, k, r, "learned + presplit")
        assert g.stats()["tasks_split"] > 0


def test_online_autotuner_batches_are_exact():
    """Under learned orders the margin trial runs first (6 batches; each seed
    whose choice depends on the margin takes the paper's order or the model's
    pick at random), then each batch of the tuning walk runs under another
    launch candidate, then the filtering trial keeps the DEBI filtering up to
    date over 8 batches that alternate between enumerating without it and
    with it; every one of them (and the batches after the
    choices) equals the oracle, each query keeps the margin of its fewest
    estimated SM cycles, and the filtering is kept only when it is at least
    3% faster."""
    s, qs = split_stream(56), split_queries()
    with fresh(s, qs) as g:
        g.set_order_policy("explore")
        for k in range(3):
            r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
            check(g, s, qs, k, r, "explore")
        g.train_order_model(epochs=100, lr=2e-3)
        g.set_order_policy("learned")
        n = len(g.autotune_candidates())
        assert g.autotune_filter_result() is None and g.autotune_margin_result() is None
        g.autotune(1)
        active, left = g.autotune_state()
        # 6 margin-trial batches, the candidates, then 4 + 4 filtering-trial
        # batches (off and on alternating)
        assert active and left == 6 + n + 8
        g.reset_stats()
        k = 3
        while k < 3 + left + 2:
            r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
            check(g, s, qs, k, r, "autotune")
            assert g.autotune_state()[1] == max(0, left - (k - 2))
            k += 1
        assert not g.autotune_state()[0]
        assert g.stats()["tasks_split"] > 0
        ft = g.autotune_filter_result()
        assert ft is not None and ft["ms_per_kedge_off"] > 0 and ft["ms_per_kedge_on"] > 0
        assert ft["filtering_kept"] == (ft["ms_per_kedge_on"] < 0.97 * ft["ms_per_kedge_off"])
        mt = g.autotune_margin_result()
        assert mt is not None and mt["margins"] == [0.0, 0.5, 1.0, 2.0, 3.0, 6.0]
        assert all(v > 0 for v in mt["cycles_per_seed"])
        assert mt["kept"] == mt["margins"][int(np.argmin(mt["cycles_per_seed"]))] == g.get_order_margin()
        for qi in range(len(qs)):                      # each query: the fewest estimated SM cycles
            cyc = np.array(mt["query_cycles_per_seed"][qi])
            if cyc.sum() > 0:
                assert g.get_order_margin(qi) == mt["margins"][int(np.argmin(cyc))]
            else:                                      # no seed of it depended on the margin
                assert g.get_order_margin(qi) == mt["kept"]
        assert g.stats()["seeds_filtered"] > 0         # the trial's filtered batches pruned seeds


def test_order_margin_is_exact_and_checked():
    """The learned order at margins 0 (the model trusted outright) and 3, and
    with a different margin per query: lists equal the oracle's; the margin
    changes the picks, so the work differs; negative, infinite and NaN margins
    and unknown query ids are refused."""
    s, qs = split_stream(), split_queries()
    with fresh(s, qs) as g:
        assert g.get_order_margin() == 1.0 and [g.get_order_margin(q) for q in range(len(qs))] == [1.0] * len(qs)
        for bad in (-0.5, float("inf"), float("nan")):
            with pytest.raises(M.MnError):
                g.set_order_margin(bad)
            with pytest.raises(M.MnError):
                g.set_query_margin(0, bad)
        with pytest.raises(M.MnError):
            g.set_query_margin(len(qs), 1.0)
        with pytest.raises(M.MnError):
            g.get_order_margin(len(qs))
        g.set_order_policy("explore")
        for k in range(3):
            r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
            check(g, s, qs, k, r, "explore")
        g.train_order_model(epochs=100, lr=2e-3)
        g.set_order_policy("learned")
        work = []
        for k, m in ((3, 0.0), (4, 3.0)):
            g.set_order_margin(m)
            assert g.get_order_margin() == m
            g.reset_stats()
            r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
            check(g, s, qs, k, r, f"margin {m}")
            st = g.stats()
            work.append(st["entries_scanned"] + st["binds"])
        assert work[0] != work[1]
        for qi, m in enumerate((0.0, 3.0, 0.5)):
            g.set_query_margin(qi, m)
        assert [g.get_order_margin(q) for q in range(len(qs))] == [0.0, 3.0, 0.5]
        assert g.get_order_margin() == 3.0             # later queries: the last set_order_margin
        r = g.insert(M.edges_from_stream(s, W + 5 * B, W + 6 * B))
        check(g, s, qs, 5, r, "margins per query")


def test_multi_label_vertices_subset_masks():
    """Data vertices carry 1-4 labels; query masks are single labels, pairs of
    labels (proper subsets of many data masks) and "any"."""
    s = gen.rmat_stream(11, 24000, 0.57, 0.19, 0.19, 4, 1.2, 4, 100, seed=0x4D4E0079,
                        multi_label_p=0.35)
    pop = np.array([bin(int(m)).count("1") for m in s["vmask"]])
    assert (pop >= 2).mean() > 0.3
    qs = [gen.q_path(3, labels=[0, 1, 0], vmask=[0b0011, 0, 0b0100, 0b1001], iso=True, temporal="chain"),
          gen.q_cycle(3, labels=[0, -1, 1], vmask=[0b0110, 0b0001, 0], iso=True),
          gen.q_out_star(3, labels=[0, 1, 0], vmask=[0b1100, 0b0011, 0b0001, 0], iso=False, temporal="chain"),
          gen.q_tree6(labels=[0, 1, 0, 2, 0], vmask=[0b0101, 0, 0b0011, 0b1000, 0b0110, 0b0010], iso=True,
                      temporal="chain")]
    run_stream_parity(s, qs, batch=3000, window=9000, preload=9000)


def test_only_overflowing_lists_run_again_then_presized():
    """One query with many embeddings per batch, one with few: with a tiny
    initial capacity only the first query's lists overflow and run again;
    from then on its lists are sized ahead from the records-per-edge
    estimate and later batches take a single launch."""
    s = gen.uniform_stream(200, 14000, 2, 2, seed=0x4D4E007A, attr_range=100)
    qs = [gen.q_path(2, iso=False),                                    # ~10^5 per batch
          gen.make_query(2, [(0, 1, 0, (0, 1))], iso=True)]             # ~10 per batch
    with make_graph(s, window=6000, max_batch=2000, out_capacity=64) as g:
        for lo in range(0, 6000, 2000):
            g.insert(M.edges_from_stream(s, lo, lo + 2000), count_only=True)
        for q in qs:
            g.register_query(q)
        reruns = []
        for k, lo_b in enumerate(range(6000, 14000, 2000)):
            st0 = g.stats()
            r = g.insert(M.edges_from_stream(s, lo_b, lo_b + 2000))
            st1 = g.stats()
            reruns.append(st1["rerun_launches"] - st0["rerun_launches"])
            lo = lo_b - 6000                      # G1 = [lo, lo_b + 2000); [lo, lo + 2000) expires
            for qi, q in enumerate(qs):
                pos = oracle.delta(s, lo, lo_b + 2000, lo_b, lo_b + 2000, q)
                neg = oracle.delta(s, lo, lo_b + 2000, lo, lo + 2000, q)
                assert r.count_pos[qi] == len(pos) and r.count_neg[qi] == len(neg)
                assert_rows_equal(g.fetch_rows(qi, +1), pos, f"batch {k} q{qi} dS+")
                assert_rows_equal(g.fetch_rows(qi, -1), neg, f"batch {k} q{qi} dS-")
            assert r.count_pos[1] <= 64 and r.count_neg[1] <= 64, "the sparse query must fit"
            assert r.count_pos[0] > 64
        assert reruns[0] == 1, reruns
        assert sum(reruns[1:]) == 0, reruns


@pytest.mark.parametrize("min_entries", [32, 100])
def test_slice_staging_is_exact(min_entries):
    """Last-depth candidate ranges read through shared-memory windows filled
    by bulk asynchronous copies (mn_set_slice_staging): the oracle's lists,
    with ranges that span several 128-entry windows and ragged ends, with
    work handed between warps, and with the DEBI filtering on."""
    s, qs = split_stream(), split_queries()
    with fresh(s, qs) as g:
        with pytest.raises(M.MnError):
            g.set_slice_staging(5)
        g.set_slice_staging(min_entries)
        assert g.get_slice_staging() == min_entries
        g.reset_stats()
        for k in (0, 1):
            r = g.insert(M.edges_from_stream(s, W + k * B, W + (k + 1) * B))
            check(g, s, qs, k, r, f"staged >= {min_entries}")
        st = g.stats()
        assert st["entries_staged"] > 0 and st["tasks_split"] > 0
        g.set_filtering(True)
        g.reset_stats()
        r = g.insert(M.edges_from_stream(s, W + 2 * B, W + 3 * B))
        check(g, s, qs, 2, r, f"staged >= {min_entries}, filtered")
        assert g.stats()["entries_staged"] > 0
        g.set_slice_staging(0)
        g.reset_stats()
        r = g.insert(M.edges_from_stream(s, W + 3 * B, W + 4 * B))
        check(g, s, qs, 3, r, "staging off")
        assert g.stats()["entries_staged"] == 0
