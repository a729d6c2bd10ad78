"""Seeded synthetic edge streams and query graphs.

This module only produces inputs: edge streams shaped like the workloads of
the Mnemonic evaluation (Sec. VII: power-law flow graphs, insert-only and
sliding-window streams, labelled tree and cyclic queries) and the query graphs
matched against them.  It holds none of the matching arithmetic, so both the
CPU oracle and the CUDA path can draw their inputs from it.

A stream is a dict of numpy arrays in arrival order:
  src, dst  uint32   endpoint vertex ids
  label     uint8    edge label (relationship type)
  attr      int32    edge attribute
  ts        int64    strictly increasing timestamp
plus ``vmask`` (uint32 per vertex, a bitmask of vertex labels) and
``num_vertices`` / ``num_edge_labels``.

A query is a dict:
  nv        number of query vertices
  vmask     list of uint32 label masks per query vertex (0 = any)
  edges     list of (src, dst, label, attr_lo, attr_hi, ts_lo, ts_hi);
            label -1 = any label
  iso       True for isomorphism, False for homomorphism
  temporal  'none' | 'chain' | 'pairs'
  prec      list of (a, b) query-edge pairs with ts(a) < ts(b) ('pairs')
"""
from __future__ import annotations

import numpy as np

INT32_MIN = -(2 ** 31)
INT32_MAX = 2 ** 31 - 1
INT64_MIN = -(2 ** 63)
INT64_MAX = 2 ** 63 - 1


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _timestamps(rng: np.random.Generator, n: int, t0: int = 1000) -> np.ndarray:
    """Strictly increasing int64 timestamps with random gaps in [1, 4]."""
    gaps = rng.integers(1, 5, size=n, dtype=np.int64)
    return t0 + np.cumsum(gaps)


def zipf_labels(rng: np.random.Generator, n: int, k: int, s: float) -> np.ndarray:
    """Labels 0..k-1 with P(label = r) proportional to (r + 1) ** -s."""
    p = (np.arange(1, k + 1, dtype=np.float64)) ** (-s)
    p /= p.sum()
    return rng.choice(k, size=n, p=p).astype(np.uint8)


def extra_vertex_labels(rng: np.random.Generator, vmask: np.ndarray, num_vlabels: int,
                        p: float) -> np.ndarray:
    """Multi-label vertices: to each vertex's mask add every label bit
    independently with probability p (Sec. II-A: a vertex carries a set of
    labels)."""
    out = vmask.copy()
    for b in range(num_vlabels):
        out |= (rng.random(len(vmask)) < p).astype(np.uint32) << np.uint32(b)
    return out


def uniform_stream(num_vertices: int, num_edges: int, num_vlabels: int,
                   num_elabels: int, seed: int, attr_range: int = 1,
                   self_loops: bool = True, multi_label_p: float = 0.0) -> dict:
    """Uniform random directed multigraph stream (parallel edges allowed).
    multi_label_p > 0 gives vertices extra label bits (extra_vertex_labels)."""
    rng = _rng(seed)
    src = rng.integers(0, num_vertices, size=num_edges, dtype=np.int64)
    dst = rng.integers(0, num_vertices, size=num_edges, dtype=np.int64)
    if not self_loops:
        loop = src == dst
        while loop.any():
            dst[loop] = rng.integers(0, num_vertices, size=int(loop.sum()))
            loop = src == dst
    vlab = rng.integers(0, num_vlabels, size=num_vertices)
    out = {
        "src": src.astype(np.uint32),
        "dst": dst.astype(np.uint32),
        "label": rng.integers(0, num_elabels, size=num_edges).astype(np.uint8),
        "attr": rng.integers(0, attr_range, size=num_edges).astype(np.int32),
        "ts": _timestamps(rng, num_edges),
        "vmask": (np.uint32(1) << vlab.astype(np.uint32)).astype(np.uint32),
        "num_vertices": int(num_vertices),
        "num_edge_labels": int(num_elabels),
    }
    if multi_label_p > 0:
        out["vmask"] = extra_vertex_labels(rng, out["vmask"], num_vlabels, multi_label_p)
    return out


def rmat_stream(scale: int, num_edges: int, a: float, b: float, c: float,
                num_elabels: int, label_zipf: float, num_vlabels: int,
                attr_range: int, seed: int, multi_label_p: float = 0.0) -> dict:
    """R-MAT power-law directed multigraph (Chakrabarti et al. 2004).

    Each edge picks one quadrant per bit level with probabilities (a, b, c, d);
    vertex ids are then permuted by a seeded shuffle so hubs are not the low ids.
    Self-loops and parallel edges are kept.
    """
    rng = _rng(seed)
    n = 1 << scale
    src = np.zeros(num_edges, dtype=np.int64)
    dst = np.zeros(num_edges, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    chunk = 1 << 22
    for lo in range(0, num_edges, chunk):
        hi = min(num_edges, lo + chunk)
        m = hi - lo
        s = np.zeros(m, dtype=np.int64)
        d = np.zeros(m, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(m)
            s = (s << 1) | (r >= ab)
            d = (d << 1) | (((r >= a) & (r < ab)) | (r >= abc))
        src[lo:hi] = s
        dst[lo:hi] = d
    perm = rng.permutation(n)
    src = perm[src]
    dst = perm[dst]
    vlab = rng.integers(0, num_vlabels, size=n)
    out = {
        "src": src.astype(np.uint32),
        "dst": dst.astype(np.uint32),
        "label": zipf_labels(rng, num_edges, num_elabels, label_zipf),
        "attr": rng.integers(0, attr_range, size=num_edges).astype(np.int32),
        "ts": _timestamps(rng, num_edges),
        "vmask": (np.uint32(1) << vlab.astype(np.uint32)).astype(np.uint32),
        "num_vertices": n,
        "num_edge_labels": int(num_elabels),
    }
    if multi_label_p > 0:
        out["vmask"] = extra_vertex_labels(rng, out["vmask"], num_vlabels, multi_label_p)
    return out


def flow_chunks(num_hosts: int, num_edges: int, num_elabels: int, seed: int,
                server_frac: float = 0.1, zipf_s: float = 1.1, mean_repeat: float = 8.0,
                client_server: float = 0.9, attr_range: int = 1000, chunk: int = 1 << 22):
    """Bipartite-heavy network-flow multigraph (NetFlow-like, Sec. VII), in
    arrival order, as chunks of at most `chunk` edges.

    Hosts [0, n_srv) are servers, the rest clients (before a seeded shuffle of
    the host ids).  A fraction `client_server` of the flows go from a client
    to a server: the client drawn by Zipf(zipf_s) over the clients' ranks
    (source activity), the server by Zipf(zipf_s) over the servers' ranks
    (popularity).  The other flows join two hosts drawn uniformly (background
    traffic).  Each (src, dst) pair repeats a geometric number of times (mean
    `mean_repeat`): timestamped parallel edges.  Protocol labels Zipf(zipf_s)
    over num_elabels; attribute uniform in [0, attr_range); one vertex label.
    """
    rng = _rng(seed)
    n_srv = max(1, int(num_hosts * server_frac))
    n_cli = max(1, num_hosts - n_srv)
    perm = rng.permutation(num_hosts)
    t0 = 1000
    done = 0
    while done < num_edges:
        m = min(chunk, num_edges - done)
        ss_parts, dd_parts, have = [], [], 0
        while have < m:                       # pairs until their repeats cover the chunk
            npairs = max(16, int((m - have) / mean_repeat * 1.25) + 16)
            cs = rng.random(npairs) < client_server
            cli = n_srv + (rng.zipf(zipf_s + 1e-9, size=npairs) - 1) % n_cli
            srv = (rng.zipf(zipf_s + 1e-9, size=npairs) - 1) % n_srv
            us = rng.integers(0, num_hosts, size=npairs)
            ud = rng.integers(0, num_hosts, size=npairs)
            s = np.where(cs, cli, us).astype(np.int64)
            d = np.where(cs, srv, ud).astype(np.int64)
            rep = rng.geometric(1.0 / mean_repeat, size=npairs)
            ss_parts.append(np.repeat(s, rep))
            dd_parts.append(np.repeat(d, rep))
            have += int(rep.sum())
        ss = np.concatenate(ss_parts)
        dd = np.concatenate(dd_parts)
        order = rng.permutation(len(ss))[:m]
        ts = _timestamps(rng, m, t0)
        t0 = int(ts[-1])
        yield {
            "src": perm[ss[order]].astype(np.uint32),
            "dst": perm[dd[order]].astype(np.uint32),
            "label": zipf_labels(rng, m, num_elabels, zipf_s),
            "attr": rng.integers(0, attr_range, size=m).astype(np.int32),
            "ts": ts,
        }
        done += m


def flow_stream(num_hosts: int, num_edges: int, num_elabels: int, seed: int, **kw) -> dict:
    """The whole flow stream of flow_chunks as one stream dict."""
    parts = list(flow_chunks(num_hosts, num_edges, num_elabels, seed, **kw))
    out = {k: np.concatenate([p[k] for p in parts]) for k in ("src", "dst", "label", "attr", "ts")}
    out["vmask"] = np.ones(num_hosts, dtype=np.uint32)
    out["num_vertices"] = int(num_hosts)
    out["num_edge_labels"] = int(num_elabels)
    return out


def slice_stream(stream: dict, lo: int, hi: int) -> dict:
    """Edges [lo, hi) of a stream, with the vertex table kept whole."""
    out = {k: v[lo:hi] for k, v in stream.items()
           if isinstance(v, np.ndarray) and k != "vmask"}
    out["vmask"] = stream["vmask"]
    out["num_vertices"] = stream["num_vertices"]
    out["num_edge_labels"] = stream["num_edge_labels"]
    return out


# ---------------------------------------------------------------- queries

def _qedge(s, d, label=-1, attr=(INT32_MIN, INT32_MAX), ts=(INT64_MIN, INT64_MAX)):
    return (int(s), int(d), int(label), int(attr[0]), int(attr[1]), int(ts[0]), int(ts[1]))


def make_query(nv, edges, vmask=None, iso=True, temporal="none", prec=()):
    """Build a query dict; ``edges`` holds (src, dst[, label[, attr[, ts]]])."""
    es = []
    for e in edges:
        s, d = e[0], e[1]
        label = e[2] if len(e) > 2 else -1
        attr = e[3] if len(e) > 3 else (INT32_MIN, INT32_MAX)
        ts = e[4] if len(e) > 4 else (INT64_MIN, INT64_MAX)
        es.append(_qedge(s, d, label, attr, ts))
    return {
        "nv": int(nv),
        "vmask": [int(m) for m in (vmask if vmask is not None else [0] * nv)],
        "edges": es,
        "iso": bool(iso),
        "temporal": temporal,
        "prec": [tuple(map(int, p)) for p in prec],
    }


def q_cycle(k, labels=None, vmask=None, **kw):
    """Directed k-cycle u0->u1->...->u_{k-1}->u0."""
    labels = labels if labels is not None else [-1] * k
    return make_query(k, [(i, (i + 1) % k, labels[i]) for i in range(k)], vmask, **kw)


def q_path(k_edges, labels=None, vmask=None, **kw):
    """Directed path u0->u1->...->u_k with k edges."""
    labels = labels if labels is not None else [-1] * k_edges
    return make_query(k_edges + 1, [(i, i + 1, labels[i]) for i in range(k_edges)], vmask, **kw)


def q_out_star(leaves, labels=None, vmask=None, **kw):
    """Centre u0 with out-edges to u1..u_leaves."""
    labels = labels if labels is not None else [-1] * leaves
    return make_query(leaves + 1, [(0, i + 1, labels[i]) for i in range(leaves)], vmask, **kw)


def q_tree6(labels=None, vmask=None, **kw):
    """6-vertex tree u0->u1, u0->u2, u1->u3, u1->u4, u2->u5."""
    E = [(0, 1), (0, 2), (1, 3), (1, 4), (2, 5)]
    labels = labels if labels is not None else [-1] * len(E)
    return make_query(6, [(s, d, labels[i]) for i, (s, d) in enumerate(E)], vmask, **kw)


def random_shape(rng: np.random.Generator, nv: int, kind: str, chords: int = 0):
    """Edge list (src, dst) of a random tree on nv vertices (random
    attachment, random directions) or of the directed cycle u0->...->u_{nv-1}->u0
    plus ``chords`` extra edges between non-adjacent vertices (random
    directions)."""
    edges = []
    if kind == "tree":
        for v in range(1, nv):
            p = int(rng.integers(0, v))
            edges.append((p, v) if rng.random() < 0.5 else (v, p))
    else:
        for i in range(nv):
            edges.append((i, (i + 1) % nv))
        have = {frozenset(e) for e in edges}
        tries = 0
        while chords > 0 and tries < 100:
            tries += 1
            a, b = map(int, rng.choice(nv, size=2, replace=False))
            if frozenset((a, b)) in have:
                continue
            have.add(frozenset((a, b)))
            edges.append((a, b) if rng.random() < 0.5 else (b, a))
            chords -= 1
    return edges


def random_query(rng: np.random.Generator, nv: int, kind: str, num_elabels: int,
                 num_vlabels: int, chords: int = 0, label_p=None, **kw):
    """Random labelled tree (random attachment, random directions) or a cycle
    of length nv with ``chords`` extra edges between non-adjacent vertices."""
    edges = random_shape(rng, nv, kind, chords)
    labels = rng.choice(num_elabels, size=len(edges), p=label_p)
    vm = [int(1 << int(rng.integers(0, num_vlabels))) for _ in range(nv)]
    return make_query(nv, [(s, d, int(l)) for (s, d), l in zip(edges, labels)], vm, **kw)
