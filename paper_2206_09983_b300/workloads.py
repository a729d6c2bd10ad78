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
