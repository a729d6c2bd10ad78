"""Plain reference of the DEBI neighbourhood filtering (test infrastructure
only: imported by the tests, never by the product path; shares no code with
the CUDA path).

Reading of Sec. V-A ("Batch Processing") and Sec. IV-A taken here, on the
live graph G (the window's edges minus deleted ones):

* Query tree (Sec. III preprocessing): root = the most selective query vertex,
  the one minimising (#data vertices whose label set contains u's labels) /
  (query degree of u), ties to the smaller id; the tree is the BFS tree from
  the root, neighbours visited in ascending (vertex id, query edge id) order;
  each non-root u has a parent p(u) and a tree edge e(u).
* f2 / f3 (isomorphism only; under homomorphism two query edges may share a
  data edge, so the counts do not bind): for every edge label l and both
  directions, v has at least as many live edges with label l, and at least as
  many distinct neighbours over such edges, as u has query edges with label
  l; likewise over all labels together.
* Top-down (f1 + f2/f3), in BFS order: TD(root) = {v : labels(u) in labels(v),
  f2/f3(v, root)}; TD(u) = {v : f2/f3(v, u) and some live edge x matching e(u)
  (the edgeMatcher) joins a vertex of TD(p(u)) (as p(u)) to v (as u)}.
* Bottom-up (f4), in reverse BFS order: BU(u) = {v in TD(u) : for every child
  c of u, some live edge matching e(c) joins v (as u) to a vertex of BU(c)
  (as c)}.  roots = BU(root).
* Filtered DEBI word of a live edge x: bit j = the edgeMatcher's bit j, and
  for a tree edge j = e(u) also: x's p(u)-side endpoint is in TD(p(u)) and its
  u-side endpoint is in BU(u).  Non-tree bits are left to the enumerator
  (Sec. IV-A).

One top-down and one bottom-up pass (the paper's single-pass filtering, not
a fixpoint): the sets are a function of the graph alone, so an incremental
maintenance of them must reach exactly these sets.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import oracle as O


def query_tree(q: dict, vmask: np.ndarray):
    """(root, parent, tree_edge, bfs order) of the query by the rule above."""
    nv = q["nv"]
    edges = q["edges"]
    cand = []
    for u in range(nv):
        m = np.uint32(q["vmask"][u])
        cand.append(int(np.count_nonzero((vmask & m) == m)))
    deg = [0] * nv
    adj = [[] for _ in range(nv)]
    for e, (a, b, *_rest) in enumerate(edges):
        deg[a] += 1
        deg[b] += 1
        adj[a].append((b, e))
        adj[b].append((a, e))
    for a in adj:
        a.sort()
    root = 0
    for u in range(1, nv):
        # cand[u] / deg[u] < cand[root] / deg[root], exactly
        if cand[u] * deg[root] < cand[root] * deg[u]:
            root = u
    parent = [-1] * nv
    tedge = [-1] * nv
    seen = [False] * nv
    seen[root] = True
    order = [root]
    dq = deque([root])
    while dq:
        u = dq.popleft()
        for w, e in adj[u]:
            if not seen[w]:
                seen[w] = True
                parent[w] = u
                tedge[w] = e
                order.append(w)
                dq.append(w)
    assert len(order) == nv, "query not connected"
    return root, parent, tedge, order


def _live_edges(stream, lo, hi, alive):
    idx = np.arange(lo, hi)
    if alive is not None:
        idx = idx[np.asarray(alive, dtype=bool)]
    return idx


def degree_ok(stream, lo, hi, q, alive=None):
    """ok[u][v]: f2 and f3 of query vertex u at data vertex v (all True under
    homomorphism)."""
    nv = q["nv"]
    V = stream["num_vertices"]
    ok = np.ones((nv, V), dtype=bool)
    if not q["iso"]:
        return ok
    idx = _live_edges(stream, lo, hi, alive)
    src = stream["src"][idx].astype(np.int64)
    dst = stream["dst"][idx].astype(np.int64)
    lab = stream["label"][idx].astype(np.int64)
    labels = sorted({e[2] for e in q["edges"] if e[2] >= 0})
    for side in ("out", "in"):
        v_of = src if side == "out" else dst
        w_of = dst if side == "out" else src
        # per (v, label) edge counts and distinct-neighbour counts; label -1 = all
        for l in [-1] + labels:
            sel = np.ones(len(idx), dtype=bool) if l < 0 else (lab == l)
            cnt = np.bincount(v_of[sel], minlength=V)
            pairs = np.unique(np.stack([v_of[sel], w_of[sel]], axis=1), axis=0) if sel.any() \
                else np.zeros((0, 2), dtype=np.int64)
            dist = np.bincount(pairs[:, 0], minlength=V) if len(pairs) else np.zeros(V, dtype=np.int64)
            for u in range(nv):
                need = 0
                for (a, b, el, *_r) in q["edges"]:
                    end = a if side == "out" else b
                    if end == u and (l < 0 or el == l):
                        need += 1
                if need:
                    ok[u] &= (cnt >= need) & (dist >= need)
    return ok


def filter_sets(stream, lo, hi, q, alive=None):
    """TD, BU (bool [nv][V]) and the tree of the query on the live edges of
    [lo, hi) (alive: optional per-edge flags)."""
    V = stream["num_vertices"]
    nv = q["nv"]
    vmask = np.asarray(stream["vmask"], dtype=np.uint32)
    root, parent, tedge, order = query_tree(q, vmask)
    dok = degree_ok(stream, lo, hi, q, alive)
    words = O.debi_words(stream, lo, hi, q)                 # edgeMatcher bits per edge of [lo, hi)
    if alive is not None:
        words = np.where(np.asarray(alive, dtype=bool), words, 0)
    src = stream["src"][lo:hi].astype(np.int64)
    dst = stream["dst"][lo:hi].astype(np.int64)
    TD = np.zeros((nv, V), dtype=bool)
    m = np.uint32(q["vmask"][root])
    TD[root] = ((vmask & m) == m) & dok[root]
    for u in order[1:]:
        e = tedge[u]
        p = parent[u]
        a_src = q["edges"][e][0] == p                       # p(u) is the source of query edge e
        pv = src if a_src else dst
        uv = dst if a_src else src
        for i in np.nonzero((words >> e) & 1)[0]:
            if TD[p][pv[i]] and dok[u][uv[i]]:
                TD[u][uv[i]] = True
    BU = np.zeros((nv, V), dtype=bool)
    children = [[] for _ in range(nv)]
    for u in order[1:]:
        children[parent[u]].append(u)
    for u in reversed(order):
        good = TD[u].copy()
        for c in children[u]:
            e = tedge[c]
            a_src = q["edges"][e][0] == u
            uvv = src if a_src else dst
            cv = dst if a_src else src
            sup = np.zeros(V, dtype=bool)
            for i in np.nonzero((words >> e) & 1)[0]:
                if BU[c][cv[i]]:
                    sup[uvv[i]] = True
            good &= sup
        BU[u] = good
    return TD, BU, (root, parent, tedge, order)


def filtered_words(stream, lo, hi, q, alive=None):
    """Filtered DEBI word of every edge of [lo, hi) (0 for edges not live)."""
    TD, BU, (root, parent, tedge, order) = filter_sets(stream, lo, hi, q, alive)
    words = O.debi_words(stream, lo, hi, q).astype(np.uint32)
    if alive is not None:
        words = np.where(np.asarray(alive, dtype=bool), words, np.uint32(0)).astype(np.uint32)
    src = stream["src"][lo:hi].astype(np.int64)
    dst = stream["dst"][lo:hi].astype(np.int64)
    for u in order[1:]:
        e = tedge[u]
        p = parent[u]
        a_src = q["edges"][e][0] == p
        pv = src if a_src else dst
        uv = dst if a_src else src
        keep = TD[p][pv] & BU[u][uv]
        words = np.where(keep, words, words & np.uint32(~(1 << e) & 0xFFFFFFFF)).astype(np.uint32)
    return words
