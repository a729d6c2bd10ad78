"""ctypes front end of the plain C oracle (mn_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the product path.  It shares no
code with the CUDA path; its inputs come from the seeded generators.

The Python side only marshals arrays and drives the stream window:
per batch it applies the order of Alg. 1 (insertions first, then deletions),
asks the C oracle for dS+ on G1 = G + ins and for dS- on G1 with the expiring
edges as the batch (Sec. V-A, "Batching Deletions": enumeration runs on the
index before the deletion is applied).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OR_MAXV = 16
OR_MAXE = 16
OR_MAXP = 256


def build(force: bool = False, out: str | None = None, defines=()) -> str:
    """Compile mn_oracle.c with gcc into a shared library; returns its path."""
    out = out or _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", out, _SRC]
        cmd += [f"-D{d}" for d in defines]
        subprocess.check_call(cmd)
    return out


class _Query(C.Structure):
    _fields_ = [
        ("nv", C.c_int32), ("ne", C.c_int32),
        ("vmask", C.c_uint32 * OR_MAXV),
        ("esrc", C.c_int32 * OR_MAXE), ("edst", C.c_int32 * OR_MAXE),
        ("elabel", C.c_int32 * OR_MAXE),
        ("attr_lo", C.c_int32 * OR_MAXE), ("attr_hi", C.c_int32 * OR_MAXE),
        ("ts_lo", C.c_int64 * OR_MAXE), ("ts_hi", C.c_int64 * OR_MAXE),
        ("iso", C.c_int32), ("nprec", C.c_int32),
        ("prec_a", C.c_int32 * OR_MAXP), ("prec_b", C.c_int32 * OR_MAXP),
    ]


class _Result(C.Structure):
    _fields_ = [("n", C.c_uint64), ("cap", C.c_uint64), ("width", C.c_int32),
                ("rows", C.POINTER(C.c_uint64))]


class _Graph(C.Structure):
    _fields_ = [
        ("nV", C.c_uint32), ("vmask", C.c_void_p), ("m", C.c_uint64),
        ("src", C.c_void_p), ("dst", C.c_void_p), ("label", C.c_void_p),
        ("attr", C.c_void_p), ("ts", C.c_void_p), ("seq", C.c_void_p),
        ("alive", C.c_void_p), ("in_batch", C.c_void_p),
    ]


_lib = None


def _load(path: str | None = None):
    global _lib
    if path is not None:
        lib = C.CDLL(path)
    else:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
    for name in ("or_brute_force", "or_delta", "or_list_static"):
        fn = getattr(lib, name)
        fn.restype = C.POINTER(_Result)
        fn.argtypes = [C.POINTER(_Graph), C.POINTER(_Query)]
    for name in ("or_count_static", "or_delta_count"):
        fn = getattr(lib, name)
        fn.restype = C.c_uint64
        fn.argtypes = [C.POINTER(_Graph), C.POINTER(_Query)]
    lib.or_delta_count_omp.restype = C.c_uint64
    lib.or_delta_count_omp.argtypes = [C.POINTER(_Graph), C.POINTER(_Query), C.c_int]
    lib.or_max_threads.restype = C.c_int
    lib.or_max_threads.argtypes = []
    lib.or_delta_count_budget.restype = C.c_int
    lib.or_delta_count_budget.argtypes = [C.POINTER(_Graph), C.POINTER(_Query), C.c_uint64,
                                          C.POINTER(C.c_uint64)]
    lib.or_debi_words.restype = None
    lib.or_debi_words.argtypes = [C.POINTER(_Graph), C.POINTER(_Query), C.c_void_p]
    lib.or_result_free.restype = None
    lib.or_result_free.argtypes = [C.POINTER(_Result)]
    if path is None:
        _lib = lib
    return lib


def precedence_pairs(q: dict):
    """Expand a query's temporal constraint into (a, b) pairs: ts(a) < ts(b)."""
    if q["temporal"] == "chain":
        return [(i, i + 1) for i in range(len(q["edges"]) - 1)]
    if q["temporal"] == "pairs":
        return list(q["prec"])
    return []


def _query_struct(q: dict) -> _Query:
    s = _Query()
    s.nv = q["nv"]
    s.ne = len(q["edges"])
    assert s.nv <= OR_MAXV and s.ne <= OR_MAXE
    for u, m in enumerate(q["vmask"]):
        s.vmask[u] = m
    for e, (a, b, lab, alo, ahi, tlo, thi) in enumerate(q["edges"]):
        s.esrc[e], s.edst[e], s.elabel[e] = a, b, lab
        s.attr_lo[e], s.attr_hi[e] = alo, ahi
        s.ts_lo[e], s.ts_hi[e] = tlo, thi
    s.iso = 1 if q["iso"] else 0
    pairs = precedence_pairs(q)
    s.nprec = len(pairs)
    for p, (a, b) in enumerate(pairs):
        s.prec_a[p], s.prec_b[p] = a, b
    return s


class _GraphView:
    """Keeps the numpy arrays alive while the C struct points into them."""

    def __init__(self, stream: dict, lo: int, hi: int, alive=None, in_batch=None):
        self.arrs = {
            "vmask": np.ascontiguousarray(stream["vmask"], dtype=np.uint32),
            "src": np.ascontiguousarray(stream["src"][lo:hi], dtype=np.uint32),
            "dst": np.ascontiguousarray(stream["dst"][lo:hi], dtype=np.uint32),
            "label": np.ascontiguousarray(stream["label"][lo:hi], dtype=np.uint8),
            "attr": np.ascontiguousarray(stream["attr"][lo:hi], dtype=np.int32),
            "ts": np.ascontiguousarray(stream["ts"][lo:hi], dtype=np.int64),
            "seq": np.arange(lo, hi, dtype=np.uint64),
        }
        if alive is not None:
            self.arrs["alive"] = np.ascontiguousarray(alive, dtype=np.uint8)
        if in_batch is not None:
            self.arrs["in_batch"] = np.ascontiguousarray(in_batch, dtype=np.uint8)
        g = _Graph()
        g.nV = int(stream["num_vertices"])
        g.m = hi - lo
        for k, a in self.arrs.items():
            setattr(g, k, a.ctypes.data)
        if alive is None:
            g.alive = None
        if in_batch is None:
            g.in_batch = None
        self.g = g


def _take(res_ptr, nv: int, ne: int, lib) -> np.ndarray:
    r = res_ptr.contents
    n, w = int(r.n), int(r.width)
    if n:
        rows = np.ctypeslib.as_array(r.rows, shape=(n * w,)).reshape(n, w).copy()
    else:
        rows = np.zeros((0, w), dtype=np.uint64)
    lib.or_result_free(res_ptr)
    return rows


def delta(stream: dict, lo: int, hi: int, batch_lo: int, batch_hi: int, q: dict,
          alive=None, batch_mask=None, lib_path=None) -> np.ndarray:
    """Sorted rows (f..., seq...) of every embedding of the live edges
    [lo, hi) that uses at least one edge with seq in [batch_lo, batch_hi)
    (or, if ``batch_mask`` is given, one flagged edge)."""
    lib = _load(lib_path)
    if batch_mask is None:
        ib = np.zeros(hi - lo, dtype=np.uint8)
        ib[batch_lo - lo:batch_hi - lo] = 1
    else:
        ib = batch_mask
    gv = _GraphView(stream, lo, hi, alive, ib)
    qs = _query_struct(q)
    return _take(lib.or_delta(C.byref(gv.g), C.byref(qs)), q["nv"], len(q["edges"]), lib)


def delta_count_first_edge(stream, lo, hi, batch_lo, batch_hi, q, lib_path=None) -> int:
    """|dS| counted by keeping each embedding only at its first batch edge."""
    lib = _load(lib_path)
    ib = np.zeros(hi - lo, dtype=np.uint8)
    ib[batch_lo - lo:batch_hi - lo] = 1
    gv = _GraphView(stream, lo, hi, None, ib)
    qs = _query_struct(q)
    return int(lib.or_delta_count(C.byref(gv.g), C.byref(qs)))


def delta_count_parallel(stream, lo, hi, q, batch_mask, threads=0, lib_path=None) -> int:
    """|dS| for the flagged batch edges (first-edge rule), with the seeds
    spread over OpenMP threads (0 = all cores)."""
    lib = _load(lib_path)
    gv = _GraphView(stream, lo, hi, None, batch_mask)
    qs = _query_struct(q)
    return int(lib.or_delta_count_omp(C.byref(gv.g), C.byref(qs), int(threads)))


def max_threads(lib_path=None) -> int:
    """Threads the parallel count uses when asked for all cores."""
    return int(_load(lib_path).or_max_threads())


def delta_count_budget(stream, lo, hi, q, batch_mask, max_nodes, lib_path=None):
    """(count, complete): |dS| for the flagged batch edges, or a partial count
    with complete=False when the DFS node budget ran out."""
    lib = _load(lib_path)
    gv = _GraphView(stream, lo, hi, None, batch_mask)
    qs = _query_struct(q)
    cnt = C.c_uint64()
    aborted = lib.or_delta_count_budget(C.byref(gv.g), C.byref(qs), max_nodes, C.byref(cnt))
    return int(cnt.value), not aborted


def brute_force(stream: dict, lo: int, hi: int, q: dict, batch_lo=None, batch_hi=None,
                alive=None, lib_path=None) -> np.ndarray:
    """All embeddings by exhaustive vertex maps (tiny graphs only)."""
    lib = _load(lib_path)
    ib = None
    if batch_lo is not None:
        ib = np.zeros(hi - lo, dtype=np.uint8)
        ib[batch_lo - lo:batch_hi - lo] = 1
    gv = _GraphView(stream, lo, hi, alive, ib)
    qs = _query_struct(q)
    return _take(lib.or_brute_force(C.byref(gv.g), C.byref(qs)), q["nv"], len(q["edges"]), lib)


def list_static(stream: dict, lo: int, hi: int, q: dict, alive=None, lib_path=None) -> np.ndarray:
    lib = _load(lib_path)
    gv = _GraphView(stream, lo, hi, alive)
    qs = _query_struct(q)
    return _take(lib.or_list_static(C.byref(gv.g), C.byref(qs)), q["nv"], len(q["edges"]), lib)


def count_static(stream: dict, lo: int, hi: int, q: dict, alive=None, lib_path=None) -> int:
    lib = _load(lib_path)
    gv = _GraphView(stream, lo, hi, alive)
    qs = _query_struct(q)
    return int(lib.or_count_static(C.byref(gv.g), C.byref(qs)))


def debi_words(stream: dict, lo: int, hi: int, q: dict, lib_path=None) -> np.ndarray:
    """Match-level DEBI word per edge of [lo, hi): bit e = edgeMatcher(edge, e)."""
    lib = _load(lib_path)
    gv = _GraphView(stream, lo, hi)
    qs = _query_struct(q)
    out = np.zeros(hi - lo, dtype=np.uint32)
    lib.or_debi_words(C.byref(gv.g), C.byref(qs), out.ctypes.data)
    return out


def window_batches(num_edges: int, batch: int, window: int, preload: int = 0):
    """The count-window snapshot schedule: yields (lo, hi_old, hi_new, x)
    per batch, where [lo, hi_new) is G1 = G + ins and the x oldest live
    edges [lo, lo + x) expire after the batch (window = 0: insert-only)."""
    lo, hi = 0, preload
    while hi < num_edges:
        hi_new = min(num_edges, hi + batch)
        x = 0
        if window and hi_new - lo > window:
            x = hi_new - lo - window
        yield lo, hi, hi_new, x
        lo += x
        hi = hi_new


def stream_deltas(stream: dict, q: dict, batch: int, window: int = 0, preload: int = 0,
                  only=None, lib_path=None):
    """Per batch k (optionally only those in ``only``): (k, dS+, dS-) rows."""
    n = len(stream["src"])
    for k, (lo, hi, hi_new, x) in enumerate(window_batches(n, batch, window, preload)):
        if only is not None and k not in only:
            continue
        pos = delta(stream, lo, hi_new, hi, hi_new, q, lib_path=lib_path)
        neg = delta(stream, lo, hi_new, lo, lo + x, q, lib_path=lib_path) if x else \
            np.zeros((0, q["nv"] + len(q["edges"])), dtype=np.uint64)
        yield k, pos, neg
