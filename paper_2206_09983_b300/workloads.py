"""Named synthetic workloads (stream recipes and query sets).

The paper's datasets (NetFlow, LSBench, LANL; Sec. VII) are not available; these
seeded streams stand in for their shapes.  Only inputs are defined here.

rmat20_window: R-MAT power-law multigraph (a, b, c) = (0.57, 0.19, 0.19),
  2^20 vertices, 2^24 edges, 8 edge labels Zipf(1.2), 4 vertex labels
  uniform, int32 attribute uniform in [0, 1000), strictly increasing
  timestamps.  Count window 2^22 edges (the first 2^22 edges preloaded without
  reporting), then batches of 65,536 insertions each expiring 65,536 edges.
  Queries: 4-vertex path, 4-cycle, 5-star, 6-vertex tree, isomorphism, edge
  timestamps increasing in query-edge order.  Labels: path, cycle and tree
  from the seeded rejection search against the CPU oracle
  (tests/golden/calibrate_rmat20_queries.py); the star uses the four rarest
  edge labels, and its exact count on the first batch (98,341 new embeddings)
  was checked with that script's --check mode.  The search keeps a batch's
  lists listable: a 5-star at an R-MAT hub with frequent labels has ~10^7
  embeddings per batch.
"""
from __future__ import annotations

import numpy as np

from . import gen

RMAT20 = dict(
    name="rmat20_window",
    scale=20, num_edges=1 << 24, a=0.57, b=0.19, c=0.19,
    elabels=8, label_zipf=1.2, vlabels=4, attr_range=1000, seed=0x4D4E0002,
    window=1 << 22, batch=1 << 16,
)


def rmat20_stream() -> dict:
    """The whole 2^24-edge stream (always generated in full, so every user of
    a prefix sees the same edges)."""
    w = RMAT20
    return gen.rmat_stream(w["scale"], w["num_edges"], w["a"], w["b"], w["c"],
                           w["elabels"], w["label_zipf"], w["vlabels"], w["attr_range"], w["seed"])


def _vm(labels):
    return [0 if l is None else 1 << l for l in labels]


# (edge labels, vertex labels) per shape, from the seeded rejection search.
RMAT20_LABELS = {
    "path4": ([1, 2, 2], [3, None, None, 2]),
    "cycle4": ([0, 1, 0, 0], [3, None, 0, None]),
    "star5": ([5, 4, 6, 7], [0, 2, 3, 3, 2]),
    "tree6": ([7, 2, 5, 5, 7], [3, None, 0, 2, None, 3]),
}


def rmat20_queries(labels: dict | None = None) -> list:
    L = labels or RMAT20_LABELS
    kw = dict(iso=True, temporal="chain")
    el, vl = L["path4"]
    qp = gen.q_path(3, labels=el, vmask=_vm(vl), **kw)
    el, vl = L["cycle4"]
    qc = gen.q_cycle(4, labels=el, vmask=_vm(vl), **kw)
    el, vl = L["star5"]
    qs = gen.q_out_star(4, labels=el, vmask=_vm(vl), **kw)
    el, vl = L["tree6"]
    qt = gen.q_tree6(labels=el, vmask=_vm(vl), **kw)
    return [qp, qc, qs, qt]


QUERY_NAMES = ["path4", "cycle4", "star5", "tree6"]


def c3_query(nv, edges, elabels, vlabels):
    """One query of the batched-queries workload: the given shape and labels,
    isomorphism, timestamps increasing along the query edges."""
    return gen.make_query(nv, [(s, d, int(l)) for (s, d), l in zip(edges, elabels)], _vm(vlabels),
                          iso=True, temporal="chain")


# The 32 uneven queries of the batched-queries workload (index, n_q, edges,
# edge labels, vertex labels; the comment is the oracle's exact |dS+| of the
# first batch after the preloaded window), from the oracle-driven search in
# tests/golden/calibrate_rmat20_c3.py: random trees (even index) and cycles
# with 1-2 chords (odd index) of 3-8 vertices, labels drawn so that the first
# batch's |dS+| lies in [2^11, 2^17].  Every tree reached that range; under
# the temporal chain the chorded cycles either explode or have very few
# embeddings, and the search kept the largest count it could certify (0 to
# 5,997 new embeddings per batch): uneven queries by construction.
RMAT20_C3_QUERIES = [
    (0, 6, [(1, 0), (1, 2), (3, 0), (4, 0), (5, 0)], [6, 7, 7, 7, 7], [1, 0, 2, 2, 1, 3]),  # 39954
    (1, 7, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 0), (0, 4), (2, 5)], [6, 5, 6, 1, 3, 4, 6, 6, 1], [None, 1, 1, 2, 1, 2, 2]),  # 0
    (2, 4, [(0, 1), (0, 2), (2, 3)], [0, 7, 5], [1, 3, 1, 2]),  # 9118
    (3, 4, [(0, 1), (1, 2), (2, 3), (3, 0), (2, 0)], [2, 4, 0, 0, 0], [None, None, 3, 2]),  # 4637
    (4, 7, [(0, 1), (2, 1), (1, 3), (0, 4), (1, 5), (6, 3)], [7, 2, 7, 5, 7, 5], [1, 1, 2, 1, 1, 0, 3]),  # 68644
    (5, 4, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (3, 1)], [2, 1, 0, 4, 4, 3], [2, 0, 3, 0]),  # 3
    (6, 7, [(1, 0), (1, 2), (0, 3), (4, 3), (3, 5), (4, 6)], [3, 4, 7, 4, 4, 5], [2, 2, 2, 1, 1, 2, 1]),  # 43161
    (7, 4, [(0, 1), (1, 2), (2, 3), (3, 0), (3, 1)], [3, 5, 0, 0, 1], [2, None, 0, 2]),  # 77
    (8, 5, [(0, 1), (2, 0), (3, 1), (2, 4)], [4, 2, 2, 2], [3, 0, 3, 2, 2]),  # 108316
    (9, 8, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 7), (7, 0), (6, 3)], [2, 7, 4, 4, 6, 0, 5, 7, 2], [2, 2, 2, 1, 1, 0, 0, 0]),  # 0
    (10, 6, [(0, 1), (0, 2), (3, 2), (4, 1), (1, 5)], [6, 1, 7, 3, 4], [1, 1, 1, 3, 3, 2]),  # 49974
    (11, 7, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 0), (2, 0), (3, 6)], [6, 6, 7, 1, 4, 6, 0, 7, 7], [3, 1, 0, 3, 2, 1, 2]),  # 0
    (12, 8, [(1, 0), (2, 0), (3, 2), (3, 4), (5, 0), (6, 1), (7, 0)], [6, 4, 6, 6, 2, 3, 6], [0, 3, 3, 1, 1, 3, 3, 2]),  # 98395
    (13, 4, [(0, 1), (1, 2), (2, 3), (3, 0), (2, 0), (1, 3)], [4, 2, 2, 0, 3, 3], [None, 2, 2, 0]),  # 4
    (14, 4, [(0, 1), (2, 0), (3, 2)], [5, 6, 1], [2, 2, None, 0]),  # 40888
    (15, 5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 3), (4, 1)], [7, 2, 1, 5, 6, 0, 2], [3, 1, 2, 1, 2]),  # 4
    (16, 7, [(1, 0), (2, 0), (1, 3), (4, 3), (5, 4), (6, 0)], [7, 5, 7, 6, 1, 4], [1, 3, 0, 0, 3, 0, 3]),  # 41214
    (17, 5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (3, 0)], [3, 7, 5, 0, 4, 6], [3, 2, 3, 2, None]),  # 182
    (18, 4, [(0, 1), (1, 2), (3, 0)], [5, 1, 3], [1, 1, 3, 1]),  # 9266
    (19, 3, [(0, 1), (1, 2), (2, 0)], [-1, 0, 0], [None, 1, 2]),  # 5997
    (20, 4, [(0, 1), (2, 1), (3, 2)], [3, 7, 5], [1, None, None, 1]),  # 58778
    (21, 8, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 7), (7, 0), (6, 2)], [1, 7, 4, 5, 3, 1, 5, 6, 2], [1, 3, 1, 0, 2, 0, 1, 3]),  # 1
    (22, 6, [(1, 0), (0, 2), (1, 3), (0, 4), (5, 4)], [7, 5, 2, 4, 2], [1, 2, 1, 2, 2, 0]),  # 108162
    (23, 5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 3)], [4, 2, 3, 3, 1, 0], [2, None, 0, 0, None]),  # 314
    (24, 4, [(1, 0), (2, 1), (3, 0)], [3, 3, 4], [2, 3, 3, None]),  # 49379
    (25, 3, [(0, 1), (1, 2), (2, 0)], [1, 0, 0], [2, None, None]),  # 5227
    (26, 3, [(0, 1), (0, 2)], [1, 1], [3, 0, 3]),  # 21793
    (27, 7, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 0), (3, 6), (5, 1)], [7, 1, 5, 6, 5, 6, 3, 7, 5], [1, 1, 3, 0, 3, 1, None]),  # 0
    (28, 6, [(1, 0), (2, 0), (2, 3), (4, 0), (2, 5)], [5, 7, 5, 6, 7], [1, 0, 3, 3, 0, 3]),  # 105042
    (29, 3, [(0, 1), (1, 2), (2, 0)], [0, 0, 0], [3, 0, None]),  # 3993
    (30, 5, [(1, 0), (1, 2), (2, 3), (4, 3)], [3, 3, 3, 6], [1, 3, None, 0, 1]),  # 96870
    (31, 7, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 0), (2, 5), (3, 0)], [7, 4, 7, 7, 5, 1, 7, 6, 1], [None, 3, 2, 1, 2, 3, 0]),  # 0
]


def rmat20_c3_queries() -> list:
    return [c3_query(nv, edges, el, vl) for _, nv, edges, el, vl in RMAT20_C3_QUERIES]


def rmat20_c3_names() -> list:
    return [f"q{i}_{'tree' if i % 2 == 0 else 'cycle'}{nv}" for i, nv, *_ in RMAT20_C3_QUERIES]


# Benchmark workloads on the rmat20 stream: the four config-2 queries, and
# the batched uneven queries (the 32 above plus the four) in one graph.
WORKLOADS = {
    "rmat20_window": dict(name="rmat20_window", window=RMAT20["window"], batch=RMAT20["batch"],
                          queries=rmat20_queries, query_names=lambda: list(QUERY_NAMES),
                          out_capacity=1 << 21),
    "rmat20_uneven": dict(name="rmat20_uneven", window=RMAT20["window"], batch=RMAT20["batch"],
                          queries=lambda: rmat20_c3_queries() + rmat20_queries(),
                          query_names=lambda: rmat20_c3_names() + list(QUERY_NAMES),
                          out_capacity=1 << 18),
}


# ---------------------------------------------------------------- serving workload

# NetFlow-like serving stream (BASELINE config 5): 10M hosts (10% servers),
# client -> server flows by Zipf(1.1) client activity and server popularity,
# 10% uniform background flows, geometric repeats (mean 8) of each drawn host
# pair (8.1 timestamped parallel edges per distinct pair in the first 2^22),
# 6 protocol labels Zipf(1.1), one vertex label, 200M edges; count window
# 2^24 edges, Poisson arrivals of log-uniform batches in [2^10, 2^18].
FLOW = dict(name="flow10m_serve", hosts=10_000_000, num_edges=200_000_000, elabels=6, zipf=1.1,
            seed=0x4D4E0005, window=1 << 24, batch=1 << 16, max_batch=1 << 18)


def flow_chunks():
    w = FLOW
    return gen.flow_chunks(w["hosts"], w["num_edges"], w["elabels"], w["seed"], zipf_s=w["zipf"])


def flow_prefix(n: int) -> dict:
    """The first n edges of the serving stream (always the same edges: the
    stream is generated chunk by chunk in arrival order)."""
    parts, have = [], 0
    for c in flow_chunks():
        parts.append(c)
        have += len(c["src"])
        if have >= n:
            break
    out = {k: np.concatenate([p[k] for p in parts])[:n] for k in ("src", "dst", "label", "attr", "ts")}
    out["vmask"] = np.ones(FLOW["hosts"], dtype=np.uint32)
    out["num_vertices"] = FLOW["hosts"]
    out["num_edge_labels"] = FLOW["elabels"]
    return out


def flow_query(nv, edges, elabels):
    """A standing query of the serving workload: the given shape and
    protocol labels (-1 = any), isomorphism, timestamps increasing along the
    query edges; one vertex label, so no vertex constraint."""
    return gen.make_query(nv, [(s, d, int(l)) for (s, d), l in zip(edges, elabels)], None,
                          iso=True, temporal="chain")


# The 8 standing queries (index, n_q, edges, protocol labels; the comment is
# the oracle's exact |dS+| of the first batch of 65,536 edges after the
# preloaded window), from the oracle-driven search in
# tests/golden/calibrate_flow_queries.py: directed paths and forked paths, the
# shapes that stay listable on a stream whose hub clients and servers make
# stars explode.
FLOW_QUERIES = [
    (2, 4, [(0, 1), (1, 2), (2, 3)], [-1, -1, -1]),  # 2175
    (5, 5, [(0, 1), (1, 2), (2, 3), (1, 4)], [0, 5, 3, 0]),  # 13085
    (9, 5, [(0, 1), (1, 2), (2, 3), (2, 4)], [-1, 0, 0, 0]),  # 19248
    (11, 6, [(0, 1), (1, 2), (2, 3), (3, 4), (1, 5)], [2, 0, -1, 0, 1]),  # 4557
    (15, 5, [(0, 1), (1, 2), (2, 3), (2, 4)], [1, -1, -1, -1]),  # 14650
    (19, 5, [(0, 1), (1, 2), (2, 3), (2, 4)], [3, 0, -1, 0]),  # 3978
    (21, 5, [(0, 1), (1, 2), (2, 3), (1, 4)], [0, 1, 0, 3]),  # 34682
    (35, 5, [(0, 1), (1, 2), (2, 3), (1, 4)], [2, 3, 0, 2]),  # 7709
]


def flow_queries() -> list:
    return [flow_query(nv, edges, el) for _, nv, edges, el in FLOW_QUERIES]
