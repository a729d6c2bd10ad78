"""Pins of the DEBI-filtering reference (oracle/debi_filter.py) against facts
that do not come from it:

* soundness (the property the paper's filtering must keep, Sec. V-A): every
  embedding found by brute force over all vertex maps maps each query vertex
  into BU of it and uses only edges whose filtered bits are set;
* TD(u) by brute force: the vertices reached by some image of the root-to-u
  tree path whose edges match and whose vertices pass f2/f3;
* BU(u) by brute force: the v in TD(u) at which the query subtree of u has a
  homomorphic image whose every vertex c lands in TD(c);
* f2 / f3 on a hand fixture with parallel edges (edge count vs distinct
  neighbours), and their absence under homomorphism;
* the root rule on a hand fixture.
"""
import itertools

import numpy as np
import pytest

from oracle import debi_filter as F
from oracle import oracle as O
from paper_2206_09983_b300 import gen

from test_oracle_pins import random_tiny_query, tiny_stream


def edge_ok(s, q, e, i):
    """edgeMatcher of query edge e at data edge i, restated."""
    a, b, lab, alo, ahi, tlo, thi = q["edges"][e]
    ms, md = np.uint32(q["vmask"][a]), np.uint32(q["vmask"][b])
    return ((lab < 0 or s["label"][i] == lab) and (s["vmask"][s["src"][i]] & ms) == ms
            and (s["vmask"][s["dst"][i]] & md) == md and alo <= s["attr"][i] < ahi
            and tlo <= s["ts"][i] < thi)


def has_edge(s, q, e, x, y, lo, hi, want_src_first):
    """Some live edge in [lo, hi) matching query edge e from x to y (or y to x)."""
    for i in range(lo, hi):
        a, b = (x, y) if want_src_first else (y, x)
        if s["src"][i] == a and s["dst"][i] == b and edge_ok(s, q, e, i):
            return True
    return False


def path_to_root(parent, u):
    p = [u]
    while parent[p[-1]] >= 0:
        p.append(parent[p[-1]])
    return p[::-1]


def subtree(parent, order, u):
    out = [u]
    for w in order:
        if w != u and u in path_to_root(parent, w):
            out.append(w)
    return out


@pytest.mark.parametrize("seed", range(24))
def test_filter_is_sound_and_td_bu_match_brute_force(seed):
    rng = np.random.default_rng(7000 + seed)
    s = tiny_stream(1600 + seed, n=int(rng.integers(4, 6)), m=int(rng.integers(12, 24)))
    q = random_tiny_query(rng, nv_max=4)
    n = len(s["src"])
    V = s["num_vertices"]
    TD, BU, (root, parent, tedge, order) = F.filter_sets(s, 0, n, q)
    dok = F.degree_ok(s, 0, n, q)
    # TD by brute force over images of the root-to-u path
    for u in range(q["nv"]):
        path = path_to_root(parent, u)
        want = np.zeros(V, dtype=bool)
        for img in itertools.product(range(V), repeat=len(path)):
            m = np.uint32(q["vmask"][root])
            if (s["vmask"][img[0]] & m) != m:
                continue
            if not all(dok[w][x] for w, x in zip(path, img)):
                continue
            ok = True
            for k in range(1, len(path)):
                w, e = path[k], tedge[path[k]]
                src_first = q["edges"][e][0] == path[k - 1]
                if not has_edge(s, q, e, img[k - 1], img[k], 0, n, src_first):
                    ok = False
                    break
            if ok:
                want[img[-1]] = True
        assert (TD[u] == want).all(), (u, TD[u], want)
    # BU by brute force over homomorphic images of the subtree of u
    for u in range(q["nv"]):
        sub = subtree(parent, order, u)
        want = np.zeros(V, dtype=bool)
        for img in itertools.product(range(V), repeat=len(sub)):
            h = dict(zip(sub, img))
            if not all(TD[c][h[c]] for c in sub):
                continue
            if all(has_edge(s, q, tedge[c], h[parent[c]], h[c], 0, n, q["edges"][tedge[c]][0] == parent[c])
                   for c in sub if c != u):
                want[h[u]] = True
        assert (BU[u] == want).all(), (u, BU[u], want)
    # soundness against every embedding
    words = F.filtered_words(s, 0, n, q)
    seq_index = {int(x): i for i, x in enumerate(range(n))}
    for row in O.brute_force(s, 0, n, q):
        f = [int(x) for x in row[:q["nv"]]]
        g = [int(x) for x in row[q["nv"]:]]
        for u in range(q["nv"]):
            assert BU[u][f[u]], ("embedding vertex outside BU", u, f)
        for e, sq in enumerate(g):
            assert (words[seq_index[sq]] >> e) & 1, ("embedding edge lost its bit", e, sq)


def test_degree_filter_counts_edges_and_distinct_neighbours():
    """Vertex 0 has two parallel out-edges (label 0) to vertex 1 and one to
    vertex 2 (label 1).  A query vertex with two out-edges of label 0 needs two
    such edges (f2: 2 >= 2) and two distinct neighbours over them (f3: 1 < 2):
    rejected under isomorphism, accepted under homomorphism."""
    s = {
        "src": np.array([0, 0, 0, 3], dtype=np.uint32),
        "dst": np.array([1, 1, 2, 0], dtype=np.uint32),
        "label": np.array([0, 0, 1, 0], dtype=np.uint8),
        "attr": np.zeros(4, dtype=np.int32),
        "ts": np.arange(1, 5, dtype=np.int64),
        "vmask": np.ones(4, dtype=np.uint32),
        "num_vertices": 4, "num_edge_labels": 2,
    }
    q = gen.make_query(3, [(0, 1, 0), (0, 2, 0)], iso=True)
    ok = F.degree_ok(s, 0, 4, q)
    assert not ok[0][0]                 # f3 fails at vertex 0
    assert not ok[0][3]                 # vertex 3 has a single out-edge
    assert ok[1][1] and ok[2][1]        # leaves need one in-edge of label 0 ...
    assert not ok[2][2]                 # ... and vertex 2's only in-edge has label 1
    q1 = gen.make_query(3, [(0, 1, 0), (0, 2, 1)], iso=True)
    assert F.degree_ok(s, 0, 4, q1)[0][0]     # one label-0 and one label-1 out-edge: fine
    qh = dict(q, iso=False)
    assert F.degree_ok(s, 0, 4, qh).all()
    # and the filter then empties TD of the star's centre under isomorphism
    TD, BU, _ = F.filter_sets(s, 0, 4, q)
    assert not BU[0].any()
    assert len(O.brute_force(s, 0, 4, q)) == 0


def test_root_rule_hand_fixture():
    """Labels: vertices 0-3 carry label 0, vertex 4 label 1.  Path query
    u0 -(e0)-> u1 -(e1)-> u2 with u1 of label 1: u1 has 1 candidate over
    degree 2 (0.5), u0 and u2 have 4 over degree 1, so u1 is the root and the
    tree is u1 -> u0 (e0), u1 -> u2 (e1)."""
    vm = np.array([1, 1, 1, 1, 2], dtype=np.uint32)
    q = gen.q_path(2, vmask=[1, 2, 1], iso=True)
    root, parent, tedge, order = F.query_tree(q, vm)
    assert root == 1 and parent == [1, -1, 1] and tedge == [0, -1, 1] and order == [1, 0, 2]
    # a tie (equal ratios) goes to the smaller id
    q2 = gen.q_path(2, vmask=[0, 0, 0], iso=True)
    root, *_ = F.query_tree(q2, vm)
    assert root == 1                    # 5/2 < 5/1
    q3 = gen.q_cycle(3, vmask=[0, 0, 0], iso=True)
    assert F.query_tree(q3, vm)[0] == 0


@pytest.mark.parametrize("seed", range(6))
def test_filtered_words_only_clear_tree_bits_and_keep_embeddings(seed):
    """On a small R-MAT window: filtered words are a subset of the
    edgeMatcher's, non-tree bits are untouched, and the embeddings of the
    window (seed oracle) all keep their bits."""
    s = gen.rmat_stream(7, 1500, 0.57, 0.19, 0.19, 3, 1.2, 2, 5, seed=8000 + seed)
    rng = np.random.default_rng(seed)
    q = gen.random_query(rng, int(rng.integers(3, 6)), "tree" if seed % 2 else "cycle", 3, 2,
                         chords=1 if seed % 2 == 0 else 0, iso=bool(seed % 3))
    n = len(s["src"])
    w0 = O.debi_words(s, 0, n, q)
    wf = F.filtered_words(s, 0, n, q)
    assert ((wf & ~w0) == 0).all()
    _, _, (root, parent, tedge, order) = F.filter_sets(s, 0, n, q)
    tree_bits = 0
    for u in order[1:]:
        tree_bits |= 1 << tedge[u]
    assert ((wf & ~np.uint32(tree_bits)) == (w0 & ~np.uint32(tree_bits))).all()
    rows = O.list_static(s, 0, n, q)
    for row in rows:
        for e, sq in enumerate(row[q["nv"]:]):
            assert (wf[int(sq)] >> e) & 1
