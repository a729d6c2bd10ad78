"""The learned matching-order model on the device.

* Forward and gradient kernels (tcgen05 tensor cores, BF16 x BF16 -> FP32
  in TMEM) against the FP64 reference oracle/mlp_ref.py.  Forward tolerance,
  from the arithmetic: the only source of disagreement beyond FP32 rounding is
  a layer-1 activation that lands on the other side of a BF16 rounding
  boundary (one BF16 ulp, 2^-8 relative); the bound per output row is
  2^-7 * sum_k |w3_k| sum_h |W2_hk| |h1_h| plus 1e-4 relative FP32 slack.
  Gradient tolerance, 2e-2 of the largest entry of each parameter group: the
  device rounds dZ2 and dZ1 to BF16 as MMA operands (2^-9 relative per
  element, two roundings on the path to dW1), and a ReLU input or layer-1
  activation within the forward's error of a boundary flips one row's
  contribution; both stay far below 2e-2 of the group's scale on 200 rows.
* Exactness: every candidate order enumerates the same sets (explore policy
  picks orders at random; lists equal the oracle's).
* Gain: after training on logged work, the learned policy does less work
  (adjacency entries tested + candidates bound) than the paper order on the
  same held-out batches, with identical lists.
"""
import numpy as np
import pytest

from oracle import mlp_ref, oracle
from paper_2206_09983_b300 import gen
from paper_2206_09983_b300 import mnemonic as M

from parity_util import assert_rows_equal

pytestmark = pytest.mark.gpu


def bf16_bits(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def rand_params(rng, scale=0.15):
    p = rng.normal(0, scale, mlp_ref.COUNT).astype(np.float32)
    return p


def test_mlp_forward_matches_fp64_reference():
    rng = np.random.default_rng(11)
    p = rand_params(rng)
    xb = bf16_bits(rng.uniform(0, 8, (777, mlp_ref.NF)))
    x = mlp_ref.bf16_bits_to_f64(xb)
    y = M.mlp_forward(p, xb)
    yr, c = mlp_ref.forward(p.astype(np.float64), x)
    P = c["P"]
    bound = 2.0 ** -7 * (np.abs(c["h1"]) @ np.abs(c["W2"]) @ np.abs(P["w3"])) + 1e-4 * (1 + np.abs(yr))
    assert (np.abs(y - yr) <= bound).all(), float(np.max(np.abs(y - yr) - bound))


def test_mlp_gradient_matches_fp64_reference():
    rng = np.random.default_rng(12)
    p = rand_params(rng)
    xb = bf16_bits(rng.uniform(0, 8, (200, mlp_ref.NF)))
    x = mlp_ref.bf16_bits_to_f64(xb)
    t = rng.uniform(0, 20, 200).astype(np.float32)
    loss, g = M.mlp_gradient(p, xb, t)
    lr, gr = mlp_ref.loss_and_grad(p.astype(np.float64), x, t.astype(np.float64))
    assert abs(loss - lr) <= 1e-3 * (1 + lr)
    o = 0
    for name, n in mlp_ref.SIZES:
        a, b = g[o:o + n], gr[o:o + n]
        scale = np.max(np.abs(b)) + 1e-12
        assert np.max(np.abs(a - b)) <= 2e-2 * scale, (name, float(np.max(np.abs(a - b))), float(scale))
        o += n


def learned_stream():
    return gen.rmat_stream(10, 26000, 0.57, 0.19, 0.19, 4, 1.2, 2, 100, seed=4242)


def learned_queries():
    return [gen.q_path(3, labels=[0, 1, 0], vmask=[0, 1, 0, 2], iso=True, temporal="chain"),
            gen.q_cycle(4, labels=[0, 0, 1, 0], vmask=[1, 0, 2, 0], iso=True, temporal="none"),
            gen.q_tree6(labels=[0, 1, 2, 0, 1], vmask=[0, 1, 0, 2, 1, 2], iso=True, temporal="chain")]


def run(policy_schedule, s, qs, W=8000, B=3000, keep=()):
    """Insert the stream batch by batch; policy per batch index from the
    schedule (a callable k -> policy or 'train'); returns rows of kept batches
    and the work counters per batch."""
    g = M.Graph(s["num_vertices"], s["num_edge_labels"], vmask=s["vmask"], window=W, max_batch=B,
                max_queries=len(qs))
    rows, work, losses = {}, {}, []
    try:
        for lo in range(0, W, B):
            g.insert(M.edges_from_stream(s, lo, min(W, lo + B)), count_only=True)
        for q in qs:
            g.register_query(q)
        k = 0
        for lo in range(W, len(s["src"]) - B + 1, B):
            pol = policy_schedule(k)
            if pol == "train":
                losses.append(g.train_order_model(epochs=300, lr=2e-3))
                pol = "learned"
            g.set_order_policy(pol)
            g.reset_stats()
            r = g.insert(M.edges_from_stream(s, lo, lo + B))
            st = g.stats()
            work[k] = st["entries_scanned"] + st["binds"]
            if k in keep:
                rows[k] = [(g.fetch_rows(qi, +1), g.fetch_rows(qi, -1)) for qi in range(len(qs))]
            k += 1
    finally:
        g.close()
    return rows, work, losses


def test_every_candidate_order_gives_the_oracle_sets():
    s = learned_stream()
    qs = learned_queries()
    W, B = 8000, 3000
    rows, _, _ = run(lambda k: "explore", s, qs, keep={0, 3})
    for k in (0, 3):
        lo_b = W + k * B
        lo_w = lo_b + B - W - B          # window start after preload expiry
        for qi, q in enumerate(qs):
            pos = oracle.delta(s, lo_w, lo_b + B, lo_b, lo_b + B, q)
            neg = oracle.delta(s, lo_w, lo_b + B, lo_w, lo_w + B, q)
            assert_rows_equal(rows[k][qi][0], pos, f"explore batch {k} q{qi} dS+")
            assert_rows_equal(rows[k][qi][1], neg, f"explore batch {k} q{qi} dS-")


def test_learned_policy_exact_and_reported_gain(capsys):
    s = learned_stream()
    qs = learned_queries()
    n_train = 3
    eval_ks = set(range(n_train, 6))
    paper_rows, paper_work, _ = run(lambda k: "paper", s, qs, keep=eval_ks)
    sched = lambda k: "explore" if k < n_train else ("train" if k == n_train else "learned")
    learned_rows, learned_work, losses = run(sched, s, qs, keep=eval_ks)
    for k in eval_ks:
        for qi in range(len(qs)):
            for sign in (0, 1):
                assert_rows_equal(learned_rows[k][qi][sign], paper_rows[k][qi][sign],
                                  f"batch {k} q{qi} sign {sign}")
    (l0, l1), = losses
    assert l1 < l0, (l0, l1)
    pw = sum(paper_work[k] for k in eval_ks)
    lw = sum(learned_work[k] for k in eval_ks)
    with capsys.disabled():
        print(f"\nlearned-order gain: paper order work {pw}, learned {lw}, ratio {pw / max(lw, 1):.3f}; "
              f"training loss {l0:.3f} -> {l1:.3f}")
    # the trained model must pay for itself on the held-out batches
    assert lw < pw, (pw, lw)
