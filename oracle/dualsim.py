"""Plain CPU oracle for dual simulation over the live window.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path;
it shares no code with the CUDA path.

Definition (the dual simulation of Ma et al. that the paper names as a
matching variant the index supports, Sec. III; evaluated per snapshot in
Sec. VII-C): a relation S between query vertices and data vertices is a dual
simulation if for every (u, v) in S
  * v carries u's vertex labels (qmask(u) subset of vmask(v)),
  * for every query edge e = (u, u') there is a live data edge (v, w) that
    matches e (the edgeMatcher: label, attribute and timestamp ranges, both
    endpoints' labels) with (u', w) in S, and
  * for every query edge e = (u'', u) there is a live data edge (w, v) that
    matches e with (u'', w) in S.
The union of dual simulations is one, so a largest exists; the query matches
only if that largest relation relates every query vertex to some data vertex,
else the result is empty.  Temporal precedence between query edges is not
part of a simulation (it relates vertices, not edge instances) and is
ignored.

The largest relation is computed by the textbook refinement: start from all
label-compatible pairs and remove pairs that violate a condition until none
does.  Result: one uint32 per data vertex, bit u set iff (u, v) in S.
"""
from __future__ import annotations

import numpy as np

from . import oracle


def _live_edges(stream: dict, lo: int, hi: int, q: dict, alive=None):
    """(src, dst, word) of the live edges of [lo, hi) whose edgeMatcher word
    is non-zero; deleted edges (alive == 0) are left out."""
    words = oracle.debi_words(stream, lo, hi, q)
    keep = words != 0
    if alive is not None:
        keep &= np.asarray(alive, dtype=bool)
    src = np.asarray(stream["src"][lo:hi])[keep]
    dst = np.asarray(stream["dst"][lo:hi])[keep]
    return src, dst, words[keep]


def dual_simulation(stream: dict, lo: int, hi: int, q: dict, alive=None) -> np.ndarray:
    nv, edges, qmask = q["nv"], q["edges"], q["vmask"]
    V = stream["num_vertices"]
    vmask = np.asarray(stream["vmask"], dtype=np.uint32)
    src, dst, words = _live_edges(stream, lo, hi, q, alive)
    # start: every label-compatible pair
    sim = np.zeros(V, dtype=np.uint32)
    for u in range(nv):
        qm = np.uint32(qmask[u])
        sim |= np.where((vmask & qm) == qm, np.uint32(1 << u), np.uint32(0))
    out_e = [[e for e, ed in enumerate(edges) if ed[0] == u] for u in range(nv)]
    in_e = [[e for e, ed in enumerate(edges) if ed[1] == u] for u in range(nv)]
    changed = True
    while changed:
        changed = False
        # sat_out[v] bit e: some live (v, w) matches e with (dst(e), w) in S;
        # sat_in[v] bit e: some live (w, v) matches e with (src(e), w) in S
        sat_out = np.zeros(V, dtype=np.uint32)
        sat_in = np.zeros(V, dtype=np.uint32)
        for e, ed in enumerate(edges):
            bit = np.uint32(1 << e)
            has = (words & bit) != 0
            ok_out = has & (((sim[dst] >> np.uint32(ed[1])) & 1) == 1)
            np.bitwise_or.at(sat_out, src[ok_out], bit)
            ok_in = has & (((sim[src] >> np.uint32(ed[0])) & 1) == 1)
            np.bitwise_or.at(sat_in, dst[ok_in], bit)
        new = sim.copy()
        for u in range(nv):
            need_out = np.uint32(sum(1 << e for e in out_e[u]))
            need_in = np.uint32(sum(1 << e for e in in_e[u]))
            bad = ((sat_out & need_out) != need_out) | ((sat_in & need_in) != need_in)
            new[bad] &= np.uint32(~(1 << u) & 0xFFFFFFFF)
        if not np.array_equal(new, sim):
            sim = new
            changed = True
    present = np.bitwise_or.reduce(sim) if V else np.uint32(0)
    if int(present) != (1 << nv) - 1:
        sim[:] = 0
    return sim


def is_dual_simulation(stream: dict, lo: int, hi: int, q: dict, rel: set, alive=None) -> bool:
    """Check the definition directly for a relation given as a set of
    (u, v) pairs (tiny inputs only)."""
    vmask = stream["vmask"]
    src, dst, words = _live_edges(stream, lo, hi, q, alive)
    for (u, v) in rel:
        if (int(vmask[v]) & q["vmask"][u]) != q["vmask"][u]:
            return False
        for e, (a, b, *_) in enumerate(q["edges"]):
            if a == u and not any(int(s) == v and (b, int(d)) in rel and (int(w) >> e) & 1
                                  for s, d, w in zip(src, dst, words)):
                return False
            if b == u and not any(int(d) == v and (a, int(s)) in rel and (int(w) >> e) & 1
                                  for s, d, w in zip(src, dst, words)):
                return False
    return True
