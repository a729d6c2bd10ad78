"""Python binding of the C ABI in include/mnemonic.h (ctypes; marshalling only).

Every step of the matching path runs in the CUDA library libmnemonic.so built
from csrc/; this module only converts arguments.  If the library has not been
built, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmnemonic.so")

MN_OK = 0
MN_ERR_STATE = -9
STATUS_NAMES = {
    -1: "MN_ERR_INVALID_ARG", -2: "MN_ERR_INVALID_VERTEX", -3: "MN_ERR_TS_ORDER",
    -4: "MN_ERR_OOM", -5: "MN_ERR_ADMISSION", -6: "MN_ERR_OUTPUT_OVERFLOW",
    -7: "MN_ERR_TIMEOUT", -8: "MN_ERR_DEVICE", -9: "MN_ERR_STATE",
}
MN_ISO, MN_HOMO = 0, 1
MN_TEMPORAL = {"none": 0, "chain": 1, "pairs": 2}
MN_DEVICE_PTR = 0x1
MN_COUNT_ONLY = 0x2
MN_ASYNC = 0x4
MN_DST_DEVICE = 0x1
MN_FETCH_SORTED = 0x2
MN_MAX_QV = 16
MN_MAX_QE = 16

EDGE_DTYPE = np.dtype([("src", "<u4"), ("dst", "<u4"), ("label", "<u4"),
                       ("attr", "<i4"), ("ts", "<i8")])

EXPORTS = [
    "mn_create_graph", "mn_destroy_graph", "mn_register_query", "mn_insert_batch",
    "mn_delete_batch", "mn_fetch_embeddings", "mn_record_layout", "mn_count_static",
    "mn_read_debi", "mn_read_adjacency", "mn_graph_info", "mn_set_work_budget",
    "mn_set_timing", "mn_get_stats", "mn_reset_stats", "mn_count_static_noalloc",
    "mn_set_order_policy", "mn_train_order_model", "mn_order_model_params", "mn_mlp_forward",
    "mn_mlp_gradient", "mn_set_tuning", "mn_get_tuning", "mn_autotune", "mn_autotune_state",
    "mn_batch_wait", "mn_set_shard", "mn_set_time_window", "mn_memory_info", "mn_reset_index",
    "mn_dual_simulation", "mn_set_wait_limit", "mn_set_presplit", "mn_get_presplit",
    "mn_autotune_candidates", "mn_autotune_results", "mn_set_filtering", "mn_read_filter",
    "mn_set_graph_capture", "mn_set_spill", "mn_read_spill", "mn_set_slice_staging",
    "mn_get_slice_staging", "mn_autotune_filter_result", "mn_last_error", "mn_set_order_margin",
    "mn_get_order_margin", "mn_autotune_margin_result", "mn_set_query_margin",
]
MN_WAIT_HOLD = 0x1
MN_ORDER = {"paper": 0, "explore": 1, "learned": 2}
MLP_PARAMS = 18817


class MnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Config(C.Structure):
    _fields_ = [("num_vertices", C.c_uint32), ("num_edge_labels", C.c_uint32),
                ("vertex_label_mask", C.c_void_p), ("window_edges", C.c_uint64),
                ("max_batch", C.c_uint64), ("edge_capacity", C.c_uint64),
                ("out_capacity", C.c_uint64), ("mem_budget_bytes", C.c_uint64),
                ("max_queries", C.c_uint32), ("device", C.c_int32), ("cuda_stream", C.c_void_p)]


class _QEdge(C.Structure):
    _fields_ = [("src", C.c_uint32), ("dst", C.c_uint32), ("label", C.c_int32),
                ("attr_lo", C.c_int32), ("attr_hi", C.c_int32), ("pad_", C.c_int32),
                ("ts_lo", C.c_int64), ("ts_hi", C.c_int64)]


class _QueryDesc(C.Structure):
    _fields_ = [("nv", C.c_uint32), ("ne", C.c_uint32), ("vlabel_mask", C.c_void_p),
                ("edges", C.POINTER(_QEdge)), ("semantics", C.c_uint32),
                ("temporal", C.c_uint32), ("n_prec", C.c_uint32), ("prec", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("batches", C.c_uint64),
                ("enumerate_launches", C.c_uint64), ("ms_ingest", C.c_double),
                ("ms_adjacency", C.c_double), ("ms_seeds", C.c_double),
                ("ms_enumerate", C.c_double), ("ms_expire", C.c_double),
                ("seeds", C.c_uint64), ("entries_scanned", C.c_uint64),
                ("binds", C.c_uint64), ("records", C.c_uint64), ("busy_cycles", C.c_uint64), ("tasks_split", C.c_uint64),
                ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("rerun_launches", C.c_uint64), ("dualsim_passes", C.c_uint64),
                ("ms_filter", C.c_double), ("seeds_filtered", C.c_uint64), ("filter_changes", C.c_uint64),
                ("graph_launches", C.c_uint64), ("graph_instantiations", C.c_uint64),
                ("spill_bytes", C.c_uint64), ("entries_staged", C.c_uint64),
                ("ms_model", C.c_double), ("model_launches", C.c_uint64),
                ("ms_train", C.c_double), ("train_rows", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _TuneConfig(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_uint32), ("split_min", C.c_uint32), ("split_depth", C.c_uint32),
                ("presplit_log2", C.c_float), ("slice_min", C.c_uint32)]


class _TuneResult(C.Structure):
    _fields_ = [("config", _TuneConfig), ("enumerate_ms", C.c_double), ("work", C.c_double)]


class _BatchResult(C.Structure):
    _fields_ = [("batch_id", C.c_uint64), ("seq_lo", C.c_uint64), ("seq_hi", C.c_uint64),
                ("expired_lo", C.c_uint64), ("expired_hi", C.c_uint64),
                ("num_queries", C.c_uint32), ("count_pos", C.POINTER(C.c_uint64)),
                ("count_neg", C.POINTER(C.c_uint64))]


assert C.sizeof(_QEdge) == 40 and EDGE_DTYPE.itemsize == 24

_lib = None


def load(path: str | None = None):
    """Load libmnemonic.so (raises if it is missing: no CPU fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is not built; run paper_2206_09983_b300.build.build()")
    lib = C.CDLL(p)
    S = C.c_int32
    P = C.c_void_p
    U64 = C.c_uint64
    sig = {
        "mn_create_graph": (S, [C.POINTER(_Config), C.POINTER(P)]),
        "mn_destroy_graph": (None, [P]),
        "mn_register_query": (S, [P, C.POINTER(_QueryDesc), C.POINTER(C.c_uint32)]),
        "mn_insert_batch": (S, [P, P, U64, C.c_uint32, C.POINTER(_BatchResult)]),
        "mn_batch_wait": (S, [P, U64, C.POINTER(_BatchResult)]),
        "mn_set_shard": (S, [P, C.c_uint32, C.c_uint32]),
        "mn_set_time_window": (S, [P, C.c_int64]),
        "mn_memory_info": (S, [P, C.POINTER(U64), C.POINTER(U64), C.POINTER(U64)]),
        "mn_reset_index": (S, [P]),
        "mn_dual_simulation": (S, [P, C.c_uint32, P, C.c_uint32, C.POINTER(U64)]),
        "mn_delete_batch": (S, [P, P, U64, C.c_uint32, C.POINTER(_BatchResult)]),
        "mn_fetch_embeddings": (S, [P, U64, C.c_uint32, C.c_int32, U64, U64, P, C.c_uint32,
                                    C.POINTER(U64)]),
        "mn_record_layout": (S, [P, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                 C.POINTER(C.c_uint32)]),
        "mn_count_static": (S, [P, C.c_uint32, C.POINTER(U64)]),
        "mn_count_static_noalloc": (S, [P, C.c_uint32, C.POINTER(U64)]),
        "mn_set_order_policy": (S, [P, C.c_uint32]),
        "mn_train_order_model": (S, [P, C.c_uint32, C.c_float, C.POINTER(C.c_float),
                                     C.POINTER(C.c_float)]),
        "mn_order_model_params": (S, [P, P, P]),
        "mn_mlp_forward": (S, [C.c_int32, P, P, U64, P]),
        "mn_set_tuning": (S, [P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int32]),
        "mn_autotune": (S, [P, C.c_uint32]),
        "mn_autotune_state": (S, [P, C.POINTER(C.c_int32), C.POINTER(C.c_uint32)]),
        "mn_get_tuning": (S, [P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                              C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_int32)]),
        "mn_mlp_gradient": (S, [C.c_int32, P, P, P, U64, P, C.POINTER(C.c_float)]),
        "mn_read_debi": (S, [P, C.c_uint32, U64, U64, P]),
        "mn_read_adjacency": (S, [P, C.c_uint32, U64, P, P, P, C.POINTER(U64)]),
        "mn_graph_info": (S, [P, C.POINTER(U64), C.POINTER(U64), C.POINTER(C.c_uint32)]),
        "mn_set_work_budget": (S, [P, U64]),
        "mn_set_wait_limit": (S, [P, C.c_uint32, C.c_uint32]),
        "mn_set_presplit": (S, [P, C.c_float]),
        "mn_set_filtering": (S, [P, C.c_int32]),
        "mn_set_graph_capture": (S, [P, C.c_int32]),
        "mn_set_spill": (S, [P, U64]),
        "mn_read_spill": (S, [P, U64, U64, P, P, C.POINTER(U64), C.POINTER(U64)]),
        "mn_read_filter": (S, [P, C.c_uint32, P, P, C.POINTER(C.c_int32), P, P]),
        "mn_get_presplit": (S, [P, C.POINTER(C.c_float)]),
        "mn_set_slice_staging": (S, [P, C.c_uint32]),
        "mn_autotune_filter_result": (S, [P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_int32)]),
        "mn_get_slice_staging": (S, [P, C.POINTER(C.c_uint32)]),
        "mn_set_order_margin": (S, [P, C.c_float]),
        "mn_set_query_margin": (S, [P, C.c_uint32, C.c_float]),
        "mn_get_order_margin": (S, [P, C.c_uint32, C.POINTER(C.c_float)]),
        "mn_autotune_margin_result": (S, [P, C.c_uint32, P, P, P, C.POINTER(C.c_uint32), C.POINTER(C.c_float)]),
        "mn_autotune_candidates": (S, [P, C.c_uint32, P, C.POINTER(C.c_uint32)]),
        "mn_autotune_results": (S, [P, C.c_uint32, P, C.POINTER(C.c_uint32)]),
        "mn_set_timing": (S, [P, C.c_int32]),
        "mn_get_stats": (S, [P, C.POINTER(Stats)]),
        "mn_reset_stats": (S, [P]),
        "mn_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def edges_from_stream(stream: dict, lo: int, hi: int) -> np.ndarray:
    """Pack stream edges [lo, hi) into the C ABI's 24-byte mn_edge records."""
    a = np.empty(hi - lo, dtype=EDGE_DTYPE)
    a["src"] = stream["src"][lo:hi]
    a["dst"] = stream["dst"][lo:hi]
    a["label"] = stream["label"][lo:hi]
    a["attr"] = stream["attr"][lo:hi]
    a["ts"] = stream["ts"][lo:hi]
    return a


@dataclass
class BatchResult:
    batch_id: int
    seq_lo: int
    seq_hi: int
    expired_lo: int
    expired_hi: int
    count_pos: list
    count_neg: list


class Graph:
    """One streaming data graph on one CUDA device (mn_graph handle)."""

    def __init__(self, num_vertices: int, num_edge_labels: int, vmask=None, window: int = 0,
                 max_batch: int = 1 << 16, edge_capacity: int = 0, out_capacity: int = 0,
                 mem_budget: int = 0, max_queries: int = 8, device: int = 0, stream: int = 0):
        self._lib = load()
        self._vmask = None if vmask is None else np.ascontiguousarray(vmask, dtype=np.uint32)
        cfg = _Config(num_vertices, num_edge_labels,
                      None if self._vmask is None else self._vmask.ctypes.data,
                      window, max_batch, edge_capacity, out_capacity, mem_budget, max_queries,
                      device, stream or None)
        h = C.c_void_p()
        st = self._lib.mn_create_graph(C.byref(cfg), C.byref(h))
        if st != MN_OK:
            raise MnError(st, self._lib.mn_last_error(None).decode())
        self._h = h
        self._num_vertices = num_vertices
        self.layouts = []
        self.last = None

    # -------------------------------------------------------------- helpers
    def _check(self, st):
        if st != MN_OK:
            raise MnError(st, self._lib.mn_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mn_destroy_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- queries
    def register_query(self, q: dict) -> int:
        ne = len(q["edges"])
        edges = (_QEdge * ne)()
        for i, (s, d, lab, alo, ahi, tlo, thi) in enumerate(q["edges"]):
            edges[i] = _QEdge(s, d, lab, alo, ahi, 0, tlo, thi)
        vm = np.ascontiguousarray(q["vmask"], dtype=np.uint32)
        prec = np.ascontiguousarray(np.array(q.get("prec", []), dtype=np.uint32).reshape(-1))
        desc = _QueryDesc(q["nv"], ne, vm.ctypes.data, edges, MN_ISO if q["iso"] else MN_HOMO,
                          MN_TEMPORAL[q["temporal"]], len(q.get("prec", [])),
                          prec.ctypes.data if prec.size else None)
        qid = C.c_uint32()
        self._check(self._lib.mn_register_query(self._h, C.byref(desc), C.byref(qid)))
        nv, nee, rb = C.c_uint32(), C.c_uint32(), C.c_uint32()
        self._check(self._lib.mn_record_layout(self._h, qid.value, C.byref(nv), C.byref(nee),
                                               C.byref(rb)))
        self.layouts.append((nv.value, nee.value, rb.value))
        return qid.value

    # -------------------------------------------------------------- batches
    def _result(self, r: _BatchResult) -> BatchResult:
        nq = r.num_queries
        res = BatchResult(r.batch_id, r.seq_lo, r.seq_hi, r.expired_lo, r.expired_hi,
                          [r.count_pos[i] for i in range(nq)], [r.count_neg[i] for i in range(nq)])
        self.last = res
        return res

    def insert(self, edges, count_only: bool = False, device_ptr: int | None = None,
               n: int | None = None) -> BatchResult:
        """Insert a batch: a numpy EDGE_DTYPE array (host), or a device pointer
        to n packed mn_edge records (device_ptr, n)."""
        flags = MN_COUNT_ONLY if count_only else 0
        r = _BatchResult()
        if device_ptr is not None:
            st = self._lib.mn_insert_batch(self._h, C.c_void_p(device_ptr), n, flags | MN_DEVICE_PTR,
                                           C.byref(r))
        else:
            a = np.ascontiguousarray(edges, dtype=EDGE_DTYPE)
            st = self._lib.mn_insert_batch(self._h, a.ctypes.data if len(a) else None, len(a),
                                           flags, C.byref(r))
        self._check(st)
        return self._result(r)

    def dual_simulation(self, qid: int) -> np.ndarray:
        """Dual simulation over the live window: uint32 per data vertex, bit u
        set iff query vertex u is related to it (mn_dual_simulation)."""
        V = self._num_vertices
        out = np.zeros(V, dtype=np.uint32)
        pairs = C.c_uint64()
        self._check(self._lib.mn_dual_simulation(self._h, qid, out.ctypes.data, 0, C.byref(pairs)))
        return out

    def memory_info(self) -> dict:
        """Device bytes held now, the peak, and the budget (0 = none)."""
        u, p, b = C.c_uint64(), C.c_uint64(), C.c_uint64()
        self._check(self._lib.mn_memory_info(self._h, C.byref(u), C.byref(p), C.byref(b)))
        return {"used": u.value, "peak": p.value, "budget": b.value}

    def reset_index(self):
        """Clear and rebuild every query's DEBI words over the live window."""
        self._check(self._lib.mn_reset_index(self._h))

    def set_time_window(self, window: int):
        """Expire by timestamp: keep edges newer than newest - window."""
        self._check(self._lib.mn_set_time_window(self._h, window))

    def set_shard(self, index: int, count: int):
        """Enumerate only this shard's seeds of the stream (mn_set_shard)."""
        self._check(self._lib.mn_set_shard(self._h, index, count))

    def insert_async(self, edges=None, count_only: bool = False, device_ptr: int | None = None,
                     n: int | None = None) -> int:
        """Queue a batch (MN_ASYNC) and return its id; wait(id) completes it.
        A host array is kept referenced until then."""
        flags = MN_ASYNC | (MN_COUNT_ONLY if count_only else 0)
        r = _BatchResult()
        if device_ptr is not None:
            st = self._lib.mn_insert_batch(self._h, C.c_void_p(device_ptr), n, flags | MN_DEVICE_PTR,
                                           C.byref(r))
            self._async_keep = None
        else:
            a = np.ascontiguousarray(edges, dtype=EDGE_DTYPE)
            st = self._lib.mn_insert_batch(self._h, a.ctypes.data if len(a) else None, len(a),
                                           flags, C.byref(r))
            self._async_keep = a
        self._check(st)
        return r.batch_id

    def wait(self, batch_id: int) -> BatchResult:
        """Complete the batch queued by insert_async (mn_batch_wait)."""
        r = _BatchResult()
        try:
            self._check(self._lib.mn_batch_wait(self._h, batch_id, C.byref(r)))
        finally:
            self._async_keep = None
        return self._result(r)

    def insert_ptr(self, ptr: int, n: int, flags: int = 0) -> BatchResult:
        """Insert n packed mn_edge records at host address ptr (e.g. pinned)."""
        r = _BatchResult()
        self._check(self._lib.mn_insert_batch(self._h, C.c_void_p(ptr), n, flags, C.byref(r)))
        return self._result(r)

    def delete(self, seqs, count_only: bool = False) -> BatchResult:
        a = np.ascontiguousarray(seqs, dtype=np.uint64)
        r = _BatchResult()
        flags = MN_COUNT_ONLY if count_only else 0
        self._check(self._lib.mn_delete_batch(self._h, a.ctypes.data if len(a) else None, len(a),
                                              flags, C.byref(r)))
        return self._result(r)

    def fetch(self, qid: int, sign: int, offset: int = 0, max_records: int | None = None,
              sorted: bool = False):
        """Records of the last batch as (vertices [n, nv] uint32, seqs [n, ne] uint64);
        sorted=True asks the device for ascending (vertices, seqs) order."""
        nv, ne, rb = self.layouts[qid]
        total = (self.last.count_pos if sign > 0 else self.last.count_neg)[qid]
        m = total - offset if max_records is None else max_records
        m = max(0, min(m, total - offset))
        buf = np.empty(m * rb, dtype=np.uint8)
        nw = C.c_uint64()
        self._check(self._lib.mn_fetch_embeddings(self._h, self.last.batch_id, qid, sign, offset, m,
                                                  buf.ctypes.data if m else None,
                                                  MN_FETCH_SORTED if sorted else 0, C.byref(nw)))
        n = nw.value
        goff = (4 * nv + 7) // 8 * 8
        rows = buf[: n * rb].reshape(n, rb)
        verts = rows[:, : 4 * nv].copy().view(np.uint32).reshape(n, nv)
        seqs = rows[:, goff: goff + 8 * ne].copy().view(np.uint64).reshape(n, ne)
        return verts, seqs

    def fetch_rows(self, qid: int, sign: int) -> np.ndarray:
        """Sorted uint64 rows (f..., seq...) -- the oracle's row format."""
        v, s = self.fetch(qid, sign)
        rows = np.concatenate([v.astype(np.uint64), s], axis=1)
        if len(rows):
            rows = rows[np.lexsort(rows.T[::-1])]
        return rows

    def fetch_device(self, qid: int, sign: int, dst_ptr: int, offset: int = 0,
                     max_records: int = 0) -> int:
        nw = C.c_uint64()
        self._check(self._lib.mn_fetch_embeddings(self._h, self.last.batch_id, qid, sign, offset,
                                                  max_records, C.c_void_p(dst_ptr), MN_DST_DEVICE,
                                                  C.byref(nw)))
        return nw.value

    # -------------------------------------------------------------- inspection
    def count_static(self, qid: int) -> int:
        c = C.c_uint64()
        self._check(self._lib.mn_count_static(self._h, qid, C.byref(c)))
        return c.value

    def count_static_noalloc(self, qid: int) -> int:
        """mn_count_static_noalloc: the static count without any device allocation."""
        c = C.c_uint64()
        self._check(self._lib.mn_count_static_noalloc(self._h, qid, C.byref(c)))
        return c.value

    def read_debi(self, qid: int, lo: int, hi: int) -> np.ndarray:
        out = np.zeros(hi - lo, dtype=np.uint32)
        self._check(self._lib.mn_read_debi(self._h, qid, lo, hi,
                                           out.ctypes.data if hi > lo else None))
        return out

    def read_adjacency(self, direction: int):
        n = C.c_uint64()
        st = self._lib.mn_read_adjacency(self._h, direction, 0, None, None, None, C.byref(n))
        if st != MN_OK and n.value == 0:
            self._check(st)
        m = n.value
        k = np.zeros(m, dtype=np.uint32)
        b = np.zeros(m, dtype=np.uint32)
        s = np.zeros(m, dtype=np.uint64)
        self._check(self._lib.mn_read_adjacency(self._h, direction, m, k.ctypes.data, b.ctypes.data,
                                                s.ctypes.data, C.byref(n)))
        return k, b, s

    def info(self):
        lo, hi, nq = C.c_uint64(), C.c_uint64(), C.c_uint32()
        self._check(self._lib.mn_graph_info(self._h, C.byref(lo), C.byref(hi), C.byref(nq)))
        return lo.value, hi.value, nq.value

    def set_work_budget(self, max_iters: int):
        self._check(self._lib.mn_set_work_budget(self._h, max_iters))

    def set_wait_limit(self, max_polls: int = 0, hold: bool = False):
        """Bound of the enumerator's idle wait (mn_set_wait_limit); hold is a
        test hook that makes every idle wait run to its bound."""
        self._check(self._lib.mn_set_wait_limit(self._h, max_polls, MN_WAIT_HOLD if hold else 0))

    def set_timing(self, on: bool):
        self._check(self._lib.mn_set_timing(self._h, 1 if on else 0))

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.mn_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    def set_order_policy(self, policy: str):
        self._check(self._lib.mn_set_order_policy(self._h, MN_ORDER[policy]))

    def train_order_model(self, epochs: int = 200, lr: float = 1e-3):
        l0, l1 = C.c_float(), C.c_float()
        self._check(self._lib.mn_train_order_model(self._h, epochs, lr, C.byref(l0), C.byref(l1)))
        return l0.value, l1.value

    def model_params(self, new=None) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        src = None if new is None else np.ascontiguousarray(new, dtype=np.float32)
        self._check(self._lib.mn_order_model_params(self._h, out.ctypes.data,
                                                    None if src is None else src.ctypes.data))
        return out

    def set_tuning(self, blocks_per_sm: int = 0, split_min: int = 0, split_depth: int = 0,
                   smem_carveout: int = -1):
        self._check(self._lib.mn_set_tuning(self._h, blocks_per_sm, split_min, split_depth,
                                            smem_carveout))

    def autotune(self, batches_per_config: int = 1):
        self._check(self._lib.mn_autotune(self._h, batches_per_config))

    def set_spill(self, capacity_edges: int):
        """Spill expired edges with their DEBI words to a pinned host FIFO (mn_set_spill)."""
        self._check(self._lib.mn_set_spill(self._h, capacity_edges))

    def read_spill(self, lo: int, hi: int, nq: int):
        """(edges EDGE_DTYPE[hi - lo], words uint32[nq][hi - lo], (held_lo, held_hi))."""
        e = np.zeros(max(0, hi - lo), dtype=EDGE_DTYPE)
        w = np.zeros((nq, max(0, hi - lo)), dtype=np.uint32)
        a, b = C.c_uint64(), C.c_uint64()
        self._check(self._lib.mn_read_spill(self._h, lo, hi, e.ctypes.data if hi > lo else None,
                                            w.ctypes.data if hi > lo and nq else None, C.byref(a), C.byref(b)))
        return e, w, (a.value, b.value)

    def set_graph_capture(self, on: bool):
        """Launch each eligible insert batch as one CUDA graph (mn_set_graph_capture)."""
        self._check(self._lib.mn_set_graph_capture(self._h, 1 if on else 0))

    def set_filtering(self, on: bool):
        """DEBI neighbourhood filtering on or off (mn_set_filtering)."""
        self._check(self._lib.mn_set_filtering(self._h, 1 if on else 0))

    def read_filter(self, qid: int, sets: bool = True):
        """(root, parent[], tree_edge[], TD, BU) of query qid; TD / BU are bool
        arrays [nv][num_vertices] (None with sets=False)."""
        nv = self.layouts[qid][0]
        V = self._num_vertices
        w32 = (V + 31) // 32
        root = C.c_int32()
        par = np.zeros(nv, dtype=np.int32)
        ted = np.zeros(nv, dtype=np.int32)
        td = bu = None
        if sets:
            td = np.zeros(nv * w32, dtype=np.uint32)
            bu = np.zeros(nv * w32, dtype=np.uint32)
        self._check(self._lib.mn_read_filter(self._h, qid, None if td is None else td.ctypes.data,
                                             None if bu is None else bu.ctypes.data, C.byref(root),
                                             par.ctypes.data, ted.ctypes.data))

        def unpack(a):
            if a is None:
                return None
            bits = np.unpackbits(a.view(np.uint8), bitorder="little").reshape(nv, w32 * 32)
            return bits[:, :V].astype(bool)
        return root.value, par.tolist(), ted.tolist(), unpack(td), unpack(bu)

    def set_presplit(self, log2_cycles: float):
        """Learned pre-splitting threshold in log2 predicted SM cycles (0 = off)."""
        self._check(self._lib.mn_set_presplit(self._h, log2_cycles))

    def get_presplit(self) -> float:
        v = C.c_float()
        self._check(self._lib.mn_get_presplit(self._h, C.byref(v)))
        return v.value

    def set_slice_staging(self, min_entries: int):
        """Staged shared-memory windows for last-depth ranges of at least min_entries (0 = off)."""
        self._check(self._lib.mn_set_slice_staging(self._h, min_entries))

    def get_slice_staging(self) -> int:
        v = C.c_uint32()
        self._check(self._lib.mn_get_slice_staging(self._h, C.byref(v)))
        return v.value

    def autotune_candidates(self):
        """The autotuner's candidates: (blocks_per_sm, split_min, split_depth, presplit_log2, slice_min)."""
        n = C.c_uint32()
        self._check(self._lib.mn_autotune_candidates(self._h, 0, None, C.byref(n)))
        arr = (_TuneConfig * max(1, n.value))()
        self._check(self._lib.mn_autotune_candidates(self._h, n.value, arr, C.byref(n)))
        return [(c.blocks_per_sm, c.split_min, c.split_depth, c.presplit_log2, c.slice_min) for c in arr[:n.value]]

    def autotune_results(self):
        """Per autotuner candidate: (blocks_per_sm, split_min, split_depth,
        presplit_log2, slice_min, enumerate_ms, work) as measured on live batches."""
        n = C.c_uint32()
        self._check(self._lib.mn_autotune_results(self._h, 0, None, C.byref(n)))
        arr = (_TuneResult * max(1, n.value))()
        self._check(self._lib.mn_autotune_results(self._h, n.value, arr, C.byref(n)))
        return [(r.config.blocks_per_sm, r.config.split_min, r.config.split_depth, r.config.presplit_log2,
                 r.config.slice_min, r.enumerate_ms, r.work) for r in arr[:n.value]]

    def autotune_filter_result(self):
        """The autotuner's filtering trial: ms per 1,000 inserted edges with the
        filtering off and on, and whether it was kept; None before a trial."""
        off, on, kept = C.c_double(), C.c_double(), C.c_int32()
        st = self._lib.mn_autotune_filter_result(self._h, C.byref(off), C.byref(on), C.byref(kept))
        if st == MN_ERR_STATE:
            return None
        self._check(st)
        return {"ms_per_kedge_off": off.value, "ms_per_kedge_on": on.value, "filtering_kept": bool(kept.value)}

    def autotune_margin_result(self):
        """The autotuner's margin trial of the learned order: the candidate
        margins (log2 units), the SM cycles per seed under each (all queries),
        per registered query the SM cycles per seed under each (0: no seed of
        it drew that margin), and the default margin kept; None before a
        trial."""
        cap = 16
        n, kept = C.c_uint32(), C.c_float()
        m = (C.c_float * cap)()
        cs = (C.c_double * cap)()
        nq = len(self.layouts)
        qc = np.zeros((max(1, nq), cap), dtype=np.float64)
        st = self._lib.mn_autotune_margin_result(self._h, cap, m, cs, qc.ctypes.data, C.byref(n), C.byref(kept))
        if st == MN_ERR_STATE:
            return None
        self._check(st)
        k = n.value
        return {"margins": list(m[:k]), "cycles_per_seed": list(cs[:k]),
                "query_cycles_per_seed": qc[:nq, :k].tolist(), "kept": kept.value}

    def set_order_margin(self, log2_margin: float):
        """Every query's margin (log2 units of predicted cost) by which a
        learned pick must beat the paper's order (mn_set_order_margin)."""
        self._check(self._lib.mn_set_order_margin(self._h, log2_margin))

    def set_query_margin(self, qid: int, log2_margin: float):
        self._check(self._lib.mn_set_query_margin(self._h, qid, log2_margin))

    def get_order_margin(self, qid: int = None) -> float:
        """One query's margin; qid None: the default for queries registered later."""
        v = C.c_float()
        self._check(self._lib.mn_get_order_margin(self._h, 0xFFFFFFFF if qid is None else qid, C.byref(v)))
        return v.value

    def autotune_state(self):
        a, left = C.c_int32(), C.c_uint32()
        self._check(self._lib.mn_autotune_state(self._h, C.byref(a), C.byref(left)))
        return bool(a.value), left.value

    def get_tuning(self) -> dict:
        v = [C.c_uint32() for _ in range(4)] + [C.c_int32()]
        self._check(self._lib.mn_get_tuning(self._h, *[C.byref(x) for x in v]))
        d = dict(zip(("blocks_per_sm", "max_blocks_per_sm", "split_min", "split_depth",
                      "smem_carveout"), [x.value for x in v]))
        d["presplit_log2"] = self.get_presplit()
        d["slice_min"] = self.get_slice_staging()
        d["order_margin"] = self.get_order_margin()
        d["query_margins"] = [self.get_order_margin(q) for q in range(len(self.layouts))]
        return d

    def reset_stats(self):
        self._check(self._lib.mn_reset_stats(self._h))


def mlp_forward(params: np.ndarray, x_bf16_bits: np.ndarray, device: int = 0) -> np.ndarray:
    """Tensor-core forward pass of the work model (test hook)."""
    lib = load()
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x_bf16_bits, dtype=np.uint16)
    n = x.shape[0]
    y = np.zeros(n, dtype=np.float32)
    st = lib.mn_mlp_forward(device, p.ctypes.data, x.ctypes.data, n, y.ctypes.data)
    if st != MN_OK:
        raise MnError(st, lib.mn_last_error(None).decode())
    return y


def mlp_gradient(params, x_bf16_bits, targets, device: int = 0):
    """Loss and FP32 gradient of the work model on the device (test hook)."""
    lib = load()
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x_bf16_bits, dtype=np.uint16)
    t = np.ascontiguousarray(targets, dtype=np.float32)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = C.c_float()
    st = lib.mn_mlp_gradient(device, p.ctypes.data, x.ctypes.data, t.ctypes.data, len(t),
                             g.ctypes.data, C.byref(loss))
    if st != MN_OK:
        raise MnError(st, lib.mn_last_error(None).decode())
    return loss.value, g
