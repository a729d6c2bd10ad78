"""Pins of the seeded input generators (the synthetic stand-ins for the
paper's NetFlow / LSBench / LANL streams, Sec. VII-A) against closed forms of
the distributions they are meant to draw, so that a generator bug (a swapped
quadrant, a wrong label law, a broken role split) cannot pass unnoticed into
every workload.  The generators hold none of the matching arithmetic; these
tests check only the inputs.

R-MAT (Chakrabarti et al. 2004): every bit of (src, dst) picks quadrant
(0,0), (0,1), (1,0), (1,1) with probabilities a, b, c, d independently, so
quantities that a vertex relabelling cannot change have product closed forms:
  P(two edges share a source)      = ((a + b)^2 + (c + d)^2)^scale
  P(two edges share a destination) = ((a + c)^2 + (b + d)^2)^scale
  P(two edges share (src, dst))    = (a^2 + b^2 + c^2 + d^2)^scale
  P(an edge is a self-loop)        = (a + d)^scale
"""
import numpy as np
import pytest

from paper_2206_09983_b300 import gen, workloads

A, B, C = 0.57, 0.19, 0.19
D = 1.0 - A - B - C


def collision_rate(x, m):
    cnt = np.bincount(np.asarray(x, dtype=np.int64))
    return float((cnt * (cnt - 1)).sum()) / (m * (m - 1))


@pytest.mark.parametrize("scale,m", [(10, 200_000), (12, 400_000)])
def test_rmat_collision_rates_follow_the_quadrant_products(scale, m):
    s = gen.rmat_stream(scale, m, A, B, C, 8, 1.2, 4, 1000, seed=0x4D4E00F0 + scale)
    src = s["src"].astype(np.int64)
    dst = s["dst"].astype(np.int64)
    assert src.max() < (1 << scale) and dst.max() < (1 << scale)
    want = {
        "src": ((A + B) ** 2 + (C + D) ** 2) ** scale,
        "dst": ((A + C) ** 2 + (B + D) ** 2) ** scale,
        "pair": (A * A + B * B + C * C + D * D) ** scale,
    }
    got = {"src": collision_rate(src, m), "dst": collision_rate(dst, m),
           "pair": collision_rate(src * (1 << scale) + dst, m)}
    for k in want:
        assert abs(got[k] / want[k] - 1.0) < 0.06, (k, got[k], want[k])
    loops = float((src == dst).mean())
    p = (A + D) ** scale
    assert abs(loops - p) < 5 * np.sqrt(p * (1 - p) / m), (loops, p)


def test_rmat_swapped_quadrants_would_be_caught():
    """The destination rate with b and c exchanged equals the source rate:
    the test above tells the two apart only when b != c, so check a
    generator with b != c as well."""
    scale, m, a, b, c = 10, 200_000, 0.55, 0.25, 0.10
    d = 1.0 - a - b - c
    s = gen.rmat_stream(scale, m, a, b, c, 4, 1.2, 2, 10, seed=0x4D4E00F9)
    want_src = ((a + b) ** 2 + (c + d) ** 2) ** scale
    want_dst = ((a + c) ** 2 + (b + d) ** 2) ** scale
    assert abs(want_src / want_dst - 1.0) > 0.5
    assert abs(collision_rate(s["src"], m) / want_src - 1.0) < 0.06
    assert abs(collision_rate(s["dst"], m) / want_dst - 1.0) < 0.06


def test_zipf_label_frequencies():
    """P(label = r) proportional to (r + 1)^-s, within 5 standard errors."""
    rng = np.random.Generator(np.random.PCG64(11))
    for k, s_exp, m in ((8, 1.2, 400_000), (6, 1.1, 400_000)):
        lab = gen.zipf_labels(rng, m, k, s_exp)
        p = np.arange(1, k + 1, dtype=np.float64) ** -s_exp
        p /= p.sum()
        f = np.bincount(lab, minlength=k) / m
        assert len(f) == k
        assert (np.abs(f - p) < 5 * np.sqrt(p * (1 - p) / m)).all(), (f, p)


def test_stream_fields_ranges_and_timestamps():
    s = gen.rmat_stream(10, 50_000, A, B, C, 8, 1.2, 4, 1000, seed=5)
    u = gen.uniform_stream(2000, 20_000, 3, 4, seed=0x4D4E0001, self_loops=False)
    for st, nl, nv_lab, ar in ((s, 8, 4, 1000), (u, 4, 3, 1)):
        assert st["src"].dtype == np.uint32 and st["dst"].dtype == np.uint32
        assert st["label"].dtype == np.uint8 and st["attr"].dtype == np.int32 and st["ts"].dtype == np.int64
        assert st["label"].max() < nl
        assert st["attr"].min() >= 0 and st["attr"].max() < ar
        gaps = np.diff(st["ts"])
        assert gaps.min() >= 1 and gaps.max() <= 4, "timestamps strictly increasing, gaps in [1, 4]"
        vm = st["vmask"]
        assert len(vm) == st["num_vertices"]
        # one vertex label per vertex: exactly one bit, below num_vlabels
        assert (vm != 0).all() and ((vm & (vm - 1)) == 0).all() and vm.max() < (1 << nv_lab)
    assert (u["src"] != u["dst"]).all(), "self_loops=False leaves no self-loop"
    # vertex labels uniform over the 4 labels of the R-MAT recipe
    f = np.bincount(np.log2(s["vmask"]).astype(np.int64), minlength=4) / len(s["vmask"])
    assert (np.abs(f - 0.25) < 0.05).all()


def test_multi_label_masks_are_supersets():
    s0 = gen.uniform_stream(3000, 10, 4, 2, seed=9)
    s1 = gen.uniform_stream(3000, 10, 4, 2, seed=9, multi_label_p=0.3)
    assert ((s1["vmask"] & s0["vmask"]) == s0["vmask"]).all()
    extra = np.array([bin(int(v)).count("1") for v in s1["vmask"]]) - 1
    # each of the 3 other bits is added with probability 0.3
    assert abs(extra.mean() - 3 * 0.3) < 0.05
    assert (s1["vmask"] < 16).all()


def test_generators_are_seeded():
    a1 = gen.rmat_stream(8, 1000, A, B, C, 4, 1.2, 2, 10, seed=1)
    a2 = gen.rmat_stream(8, 1000, A, B, C, 4, 1.2, 2, 10, seed=1)
    a3 = gen.rmat_stream(8, 1000, A, B, C, 4, 1.2, 2, 10, seed=2)
    for k in ("src", "dst", "label", "attr", "ts", "vmask"):
        assert (a1[k] == a2[k]).all()
    assert not (a1["src"] == a3["src"]).all()


def test_flow_roles_bipartite_when_every_flow_is_client_to_server():
    """With every flow client -> server, sources and destinations are
    disjoint host sets, at most n_srv destinations and n_cli sources."""
    hosts, m = 5000, 100_000
    f = gen.flow_stream(hosts, m, 6, seed=21, client_server=1.0)
    srcs, dsts = np.unique(f["src"]), np.unique(f["dst"])
    assert len(np.intersect1d(srcs, dsts)) == 0
    assert len(dsts) <= hosts // 10 and len(srcs) <= hosts - hosts // 10
    assert (f["vmask"] == 1).all() and len(f["vmask"]) == hosts
    assert len(f["src"]) == m and np.diff(f["ts"]).min() >= 1
    # the default mix: 10% uniform background flows make the sets overlap
    g = gen.flow_stream(hosts, m, 6, seed=21)
    assert len(np.intersect1d(np.unique(g["src"]), np.unique(g["dst"]))) > 0


def test_flow_parallel_edges_per_pair():
    """Each drawn pair repeats Geometric(1/8) times; a chunk is then cut to
    its size by a random subset of its flows (about 4/5 survive), which
    leaves a geometric count with mean 1 / (1 - r), r = (1 - p) q / (p + q - p q)
    (p = 1/8, q the surviving fraction): about 6.6 edges per distinct pair
    when pairs practically never recur (hosts drawn uniformly from 10^7)."""
    m = 300_000
    f = gen.flow_stream(10 ** 7, m, 6, seed=3, client_server=0.0)
    pairs = f["src"].astype(np.int64) * 10 ** 7 + f["dst"].astype(np.int64)
    _, cnt = np.unique(pairs, return_counts=True)
    p, q = 1.0 / 8.0, 0.8
    r = (1 - p) * q / (p + q - p * q)
    assert abs(cnt.mean() - 1.0 / (1.0 - r)) < 0.35, cnt.mean()
    # chunked generation continues the same stream
    parts = list(gen.flow_chunks(10 ** 7, m, 6, 3, client_server=0.0, chunk=1 << 17))
    assert sum(len(x["src"]) for x in parts) == m
    ts = np.concatenate([x["ts"] for x in parts])
    assert np.diff(ts).min() >= 1


def test_benchmark_query_shapes():
    """Shapes of the benchmark queries: 4-vertex path (3 edges), 4-cycle,
    5-star (centre with 4 out-edges), the 6-vertex tree, isomorphism under
    the temporal chain."""
    qp, qc, qs, qt = workloads.rmat20_queries()
    es = lambda q: [(e[0], e[1]) for e in q["edges"]]
    assert qp["nv"] == 4 and es(qp) == [(0, 1), (1, 2), (2, 3)]
    assert qc["nv"] == 4 and es(qc) == [(0, 1), (1, 2), (2, 3), (3, 0)]
    assert qs["nv"] == 5 and es(qs) == [(0, 1), (0, 2), (0, 3), (0, 4)]
    assert qt["nv"] == 6 and es(qt) == [(0, 1), (0, 2), (1, 3), (1, 4), (2, 5)]
    for q in (qp, qc, qs, qt):
        assert q["iso"] and q["temporal"] == "chain"


def connected(nv, edges):
    seen, todo = {0}, [0]
    while todo:
        v = todo.pop()
        for a, b in edges:
            for x, y in ((a, b), (b, a)):
                if x == v and y not in seen:
                    seen.add(y)
                    todo.append(y)
    return len(seen) == nv


def test_uneven_queries_are_trees_and_chorded_cycles():
    """The 32 batched queries: 3-8 vertices; even index a tree (n - 1 edges,
    connected), odd index the directed cycle u0 -> ... -> u_{n-1} -> u0 plus
    1-2 chords between non-adjacent vertices (none for a triangle); no two
    query edges join the same pair; all of them plus the four benchmark
    queries in one workload."""
    qs = workloads.rmat20_c3_queries()
    assert len(qs) == 32 and len(workloads.WORKLOADS["rmat20_uneven"]["queries"]()) == 36
    sizes = set()
    for i, q in enumerate(qs):
        nv, E = q["nv"], [(e[0], e[1]) for e in q["edges"]]
        sizes.add(nv)
        assert 3 <= nv <= 8 and connected(nv, E)
        assert len({frozenset(e) for e in E}) == len(E) and all(a != b for a, b in E)
        if i % 2 == 0:
            assert len(E) == nv - 1
        else:
            assert E[:nv] == [(k, (k + 1) % nv) for k in range(nv)]
            chords = len(E) - nv
            assert (chords == 0) if nv == 3 else (1 <= chords <= 2)
        assert q["iso"] and q["temporal"] == "chain"
    assert sizes == set(range(3, 9))


def test_serving_queries_are_paths_and_forked_paths():
    """The 8 standing queries of the serving stream: directed paths and
    forked paths (trees in which every vertex has in-degree at most 1) of
    4-6 vertices, protocol labels in range or any."""
    qs = workloads.flow_queries()
    assert len(qs) == 8
    for q in qs:
        nv, E = q["nv"], [(e[0], e[1]) for e in q["edges"]]
        assert 4 <= nv <= 6 and len(E) == nv - 1 and connected(nv, E)
        indeg = np.bincount([b for _, b in E], minlength=nv)
        assert indeg[0] == 0 and (indeg[1:] == 1).all()
        assert all(-1 <= e[2] < workloads.FLOW["elabels"] for e in q["edges"])
