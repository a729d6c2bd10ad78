"""Seed sharding through the C ABI: three graphs on one device, each with one
shard of the same stream's seeds, against the unsharded graph and the oracle.
Per batch and query: the shards' lists are disjoint, their union (sorted) is
the unsharded list, and their counts sum to it, for dS+ and dS-; static
counts add up the same way, and explicit deletes too."""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M
from paper_2206_09983_b300 import shard

from parity_util import assert_rows_equal, make_graph, vm

pytestmark = pytest.mark.gpu

SHARDS = 3


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2206_09983_b300 import build
    build.build()


def _setup():
    s = gen.rmat_stream(10, 20000, 0.57, 0.19, 0.19, 6, 1.2, 3, 1000, seed=0x5D)
    rng = np.random.default_rng(9)
    lab = lambda k: [int(x) for x in rng.integers(0, 6, size=k)]  # noqa: E731
    qs = [gen.q_path(3, labels=lab(3), vmask=vm(0, None, None, None), iso=True, temporal="chain"),
          gen.q_cycle(3, labels=lab(3), vmask=vm(None, None, None), iso=False, temporal="none"),
          gen.q_out_star(3, labels=lab(3), vmask=vm(None, 1, None, None), iso=True, temporal="chain")]
    return s, qs


def _disjoint(parts):
    rows = [r for r in parts if len(r)]
    if not rows:
        return True
    allr = np.concatenate(rows, axis=0)
    return len(np.unique(allr, axis=0)) == len(allr)


def test_shards_union_is_the_unsharded_result():
    s, qs = _setup()
    n = len(s["src"])
    W, B = 5000, 2000
    full = make_graph(s, window=W, max_batch=W, max_queries=len(qs))
    parts = [make_graph(s, window=W, max_batch=W, max_queries=len(qs)) for _ in range(SHARDS)]
    try:
        for i, g in enumerate(parts):
            g.set_shard(i, SHARDS)
        for g in [full] + parts:
            g.insert(M.edges_from_stream(s, 0, W), count_only=True)
            for q in qs:
                g.register_query(q)
        nonempty = 0
        for k, (lo, hi, hi_new, x) in enumerate(oracle.window_batches(n, B, W, W)):
            batch = M.edges_from_stream(s, hi, hi_new)
            rf = full.insert(batch)
            rp = [g.insert(batch) for g in parts]
            assert shard.merge_counts([r.count_pos for r in rp]) == rf.count_pos, f"batch {k} dS+"
            assert shard.merge_counts([r.count_neg for r in rp]) == rf.count_neg, f"batch {k} dS-"
            for qi, q in enumerate(qs):
                for sign in (+1, -1):
                    pr = [g.fetch_rows(qi, sign) for g in parts]
                    assert _disjoint(pr), f"batch {k} query {qi} sign {sign}: shards overlap"
                    ref = full.fetch_rows(qi, sign)
                    assert_rows_equal(shard.merge_rows(pr), ref, f"batch {k} query {qi} sign {sign}")
                    nonempty += int(len(ref) > 0 and sum(len(r) > 0 for r in pr) > 1)
                if k == 1:
                    assert rf.count_pos[qi] == len(oracle.delta(s, lo, hi_new, hi, hi_new, q))
        assert nonempty > 0, "no list was split over several shards"
        for qi in range(len(qs)):
            assert sum(g.count_static(qi) for g in parts) == full.count_static(qi)
        # explicit deletes: dS- of the deleted edges, split the same way
        lo, hi, nq = full.info()
        dels = np.arange(hi - 300, hi, 3, dtype=np.uint64)
        rf = full.delete(dels)
        rp = [g.delete(dels) for g in parts]
        assert shard.merge_counts([r.count_neg for r in rp]) == rf.count_neg
        for qi in range(len(qs)):
            assert_rows_equal(shard.merge_rows([g.fetch_rows(qi, -1) for g in parts]),
                              full.fetch_rows(qi, -1), f"delete query {qi}")
    finally:
        for g in [full] + parts:
            g.close()


def test_set_shard_rejects_bad_arguments():
    s, _ = _setup()
    g = make_graph(s, window=1000, max_batch=1000)
    try:
        for idx, cnt in ((0, 0), (2, 2), (5, 3)):
            with pytest.raises(M.MnError) as e:
                g.set_shard(idx, cnt)
            assert e.value.status == -1
        g.set_shard(1, 2)
        g.set_shard(0, 1)
    finally:
        g.close()
