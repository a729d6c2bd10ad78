"""Parity at the benchmark's full size (the rmat20 stream: 2^20 vertices,
window 2^22 edges, batches of 65,536), for both benchmark workloads -- the
four calibrated queries (rmat20_window) and the 36 batched uneven queries
(rmat20_uneven: 32 random trees and chorded cycles plus the four) -- in the
launch configurations bench.py times (device-resident batches, count-only
preload, queries registered on the full window): the plain path (paper
order, default launch), and the learned arm (orders picked by the work
model trained on three explore batches, then tuned online on live batches as
the benchmark does: the per-query margin trial of the learned order, the walk
over launch parameters, pre-splitting and slice staging, and the trial of the
DEBI filtering; the two checked batches run in whatever configuration the
autotuner kept).

The oracle cannot list a whole batch quickly, so per batch and query:
* sampled exactness: for a seeded sample of the batch's edges, the GPU records
  that contain a sampled edge equal the oracle's embeddings containing a
  sampled edge (the oracle's delta with the sample as its batch);
* properties of every record: it is a valid embedding of the live window
  (endpoints, labels, vertex labels, injectivity, temporal order), it contains
  a batch edge, and no record repeats.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2206_09983_b300 import workloads
from paper_2206_09983_b300 import mnemonic as M

pytestmark = pytest.mark.gpu


_STREAM = {}


# batches the learned arm may spend before its checked ones: 3 explore
# batches, then the autotuner (6 margin-trial batches, one per launch
# candidate, 6 for the filtering trial)
LEARNED_SPAN = 48


@pytest.fixture(scope="module", params=[("rmat20_window", "plain"), ("rmat20_uneven", "plain"),
                                        ("rmat20_window", "learned"), ("rmat20_uneven", "learned")],
                ids=lambda p: f"{p[0]}-{p[1]}")
def run(request):
    import torch
    from paper_2206_09983_b300 import build
    build.build()
    name, mode = request.param
    wl = workloads.WORKLOADS[name]
    W, B = wl["window"], wl["batch"]
    if "s" not in _STREAM:
        _STREAM["s"] = workloads.rmat20_stream()
    s = _STREAM["s"]
    span = LEARNED_SPAN if mode == "learned" else 0
    packed = M.edges_from_stream(s, 0, W + (span + 2) * B)
    d = torch.from_numpy(packed.view(np.uint8)).cuda()
    qs = wl["queries"]()
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=W, max_batch=B,
                max_queries=len(qs), stream=torch.cuda.current_stream().cuda_stream,
                out_capacity=wl["out_capacity"])
    for lo in range(0, W, B):
        g.insert(None, device_ptr=d.data_ptr() + 24 * lo, n=B, count_only=True)
    qids = [g.register_query(q) for q in qs]
    pos = W
    if mode == "learned":
        g.set_order_policy("explore")
        for _ in range(3):
            g.insert(None, device_ptr=d.data_ptr() + 24 * pos, n=B)
            pos += B
        g.train_order_model(epochs=300, lr=2e-3)
        g.set_order_policy("learned")
        g.autotune(1)
        while g.autotune_state()[0]:
            assert pos < W + span * B, "autotuner needs more batches than the fixture packed"
            g.insert(None, device_ptr=d.data_ptr() + 24 * pos, n=B)
            pos += B
        print(f"{name}: kept {g.get_tuning()}, filtering trial {g.autotune_filter_result()}")
    out = []
    for _ in range(2):
        hi = pos
        r = g.insert(None, device_ptr=d.data_ptr() + 24 * hi, n=B)
        rows = {(qi, sg): g.fetch_rows(qi, sg) for qi in qids for sg in (+1, -1)}
        out.append((hi - W, hi, hi + B, r, rows))
        pos += B
    g.close()
    return s, qs, out


def check_valid(s, q, rows, lo, hi_new, blo, bhi):
    nv, ne = q["nv"], len(q["edges"])
    f = rows[:, :nv].astype(np.int64)
    g = rows[:, nv:].astype(np.int64)
    assert ((g >= lo) & (g < hi_new)).all(), "edge outside the live window"
    for e, (a, b, lab, alo, ahi, tlo, thi) in enumerate(q["edges"]):
        sq = g[:, e]
        assert (s["src"][sq] == f[:, a]).all() and (s["dst"][sq] == f[:, b]).all()
        if lab >= 0:
            assert (s["label"][sq] == lab).all()
        assert ((s["attr"][sq] >= alo) & (s["attr"][sq] < ahi)).all()
    for u in range(nv):
        m = np.uint32(q["vmask"][u])
        assert ((s["vmask"][f[:, u]] & m) == m).all()
    if q["iso"]:
        fs = np.sort(f, axis=1)
        assert (np.diff(fs, axis=1) != 0).all(), "vertex map not injective"
    for a, b in oracle.precedence_pairs(q):
        assert (s["ts"][g[:, a]] < s["ts"][g[:, b]]).all()
    inb = (g >= blo) & (g < bhi)
    assert inb.any(axis=1).all(), "record without a batch edge"
    if len(rows) > 1:
        assert len(np.unique(rows, axis=0)) == len(rows), "repeated record"


@pytest.mark.parametrize("k", [0, 1])
def test_fullsize_records_are_valid_and_unique(run, k):
    s, qs, out = run
    lo, hi, hi_new, r, rows = out[k]
    B = hi_new - hi
    for qi, q in enumerate(qs):
        pos = rows[(qi, +1)]
        neg = rows[(qi, -1)]
        assert len(pos) == r.count_pos[qi] and len(neg) == r.count_neg[qi]
        check_valid(s, q, pos, lo, hi_new, hi, hi_new)
        check_valid(s, q, neg, lo, hi_new, lo, lo + B)


@pytest.mark.parametrize("k", [0, 1])
def test_fullsize_sampled_exact(run, k):
    s, qs, out = run
    lo, hi, hi_new, r, rows = out[k]
    B = hi_new - hi
    rng = np.random.default_rng(1234 + k)
    for sign, base in ((+1, hi), (-1, lo)):
        pick = rng.choice(B, size=48 if len(qs) <= 8 else 24, replace=False) + base
        # plus the 8 batch edges with the highest-degree endpoints (the hub
        # tail, where subtrees are split and donated)
        deg = np.bincount(s["src"][lo:hi_new], minlength=s["num_vertices"]) + \
            np.bincount(s["dst"][lo:hi_new], minlength=s["num_vertices"])
        bsl = np.arange(base, base + B)
        hub = bsl[np.argsort(-(deg[s["src"][bsl]] + deg[s["dst"][bsl]]), kind="stable")[:8]]
        pick = np.unique(np.concatenate([pick, hub]))
        mask = np.zeros(hi_new - lo, dtype=np.uint8)
        mask[pick - lo] = 1
        for qi, q in enumerate(qs):
            got = rows[(qi, sign)]
            nv = q["nv"]
            sel = np.isin(got[:, nv:], pick.astype(np.uint64)).any(axis=1)
            want = oracle.delta(s, lo, hi_new, 0, 0, q, batch_mask=mask)
            sub = got[sel]
            assert sub.shape == want.shape, f"query {qi} sign {sign}: {sub.shape} vs {want.shape}"
            assert (sub == want).all()
