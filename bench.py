#!/usr/bin/env python
"""Benchmark of the incremental matching hot path (Mnemonic, arXiv 2206.09983).

Metric: inserted edges per second (and p50/p99 batch latency) at exact counts
on the sliding-window R-MAT workload: 2^20 vertices, 2^24 edges, window 2^22,
batches of 65,536 insertions each expiring 65,536 edges, four standing queries
(4-vertex path, 4-cycle, 5-star, 6-vertex tree; isomorphism; increasing
timestamps).  One step = one batch through the whole path: ingest and
edgeMatcher, adjacency update, work units, enumeration of new embeddings,
enumeration of expired embeddings, DEBI clear.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun): seed sharding -- every rank ingests the same stream
and enumerates only its shard of the seeds (mn_set_shard(rank, N)); the
shards' counts are summed on the host after the timed region.  Total work per
batch is fixed (strong scaling); value = stream edges / max time over ranks.
--impl reference times the CPU oracle on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "inserted edges/sec and p99 batch latency at exact counts"
UNIT = "edges/s"
CTRL_NOTE = "working set > 126 MB L2 (edge ring 176 MB, adjacency 2 x 2 x 96 MB); no flush"


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per k_enumerate
# launch, the mean of the learned arm's first two timed launches (one per batch) in
# one ncu capture (profiles/k_enumerate_rmat20_window.md).  It holds only for the
# enumerator code it was taken on (enum_source_sha1): null once that changed.
ENUM_TRAFFIC = {"source_sha1": "fea350eeb68150b8a130d732c83384fdbb4f1c7e", "bytes_per_launch": 883.8e6}


def enum_source_sha1() -> str:
    """sha1 of the enumerator's source code (mn_device.cuh from its launch
    constants to the end of k_enumerate): comments and blank space removed, so
    that only a change of the enumerator's code makes the stored traffic
    stale."""
    src = open(os.path.join(ROOT, "paper_2206_09983_b300", "csrc", "mn_device.cuh")).read()
    a = src.index("constexpr int ENUM_WARPS")
    b = src.index("// ------------------------------------------------------------------ expiry / deletion")
    src = src[a:b]
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha1(" ".join(src.split()).encode()).hexdigest()


def enum_traffic():
    return ENUM_TRAFFIC["bytes_per_launch"] if enum_source_sha1() == ENUM_TRAFFIC["source_sha1"] else None


ENUM_WARPS_PER_BLOCK = 4           # k_enumerate's block: 128 threads


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    return 6400.0, "fallback"


def measured_bf16_peak(sustained=False):
    """Dense BF16 tensor throughput in TFLOP/s (cuBLAS, MEASURED_PEAKS.json):
    the burst figure for a kernel timed alone, the sustained one for a kernel
    inside a long loop."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        k = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        if k in d:
            return float(d[k]), "measured"
    return (1400.0 if sustained else 1800.0), "fallback"


# tensor-core flops per row of the work model (16 -> 128 -> 128 -> 1): the
# forward's two MMAs, and the gradient's forward plus dW2, dH1 and dW1
MLP_FWD_FLOPS = 2 * (16 * 128 + 128 * 128)
MLP_GRAD_FLOPS = 2 * (2 * 16 * 128 + 3 * 128 * 128)
NCAND = 4                          # candidate matching orders scored per seed


# ------------------------------------------------------------------ CPU oracle sample

def oracle_sample(stream, queries, W, B, batch_index, sample, seed=7):
    """Time the CPU oracle on `sample` edges of one batch of the window
    stream: |dS+| (embeddings containing a sampled new edge, each counted at
    its first sampled edge) of every query, the seeds spread over all host
    cores with OpenMP (the paper's CPU design point).  Returns (seconds,
    embeddings, threads)."""
    from oracle import oracle
    lo = batch_index * B
    hi_new = lo + W + B
    rng = np.random.default_rng(seed + batch_index)
    pick = rng.choice(B, size=sample, replace=False)
    mask = np.zeros(hi_new - lo, dtype=np.uint8)
    mask[W + pick] = 1
    threads = oracle.max_threads()
    t = time.perf_counter()
    rows = 0
    for q in queries:
        rows += oracle.delta_count_parallel(stream, lo, hi_new, q, mask, 0)
    return time.perf_counter() - t, rows, threads


def oracle_sample_size(B):
    """Sampled edges per batch: 256 per host core, so a step takes a few
    seconds whatever the core count."""
    from oracle import oracle
    return min(B, 256 * oracle.max_threads())


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2206_09983_b300 import workloads
    w = workloads.RMAT20
    W, B = w["window"], w["batch"]
    stream = workloads.rmat20_stream()
    qs = workloads.rmat20_queries()
    sample = args.ref_sample or oracle_sample_size(B)
    times, edges, threads = [], 0, 1
    for k in range(args.warmup + args.steps):
        dt, _, threads = oracle_sample(stream, qs, W, B, k, sample)
        if k >= args.warmup:
            times.append(dt)
            edges += sample
    total = sum(times)
    value = edges / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": w["name"], "vertices": 1 << w["scale"], "edges": w["num_edges"],
                   "window": W, "batch": B, "queries": list(workloads.QUERY_NAMES),
                   "semantics": "isomorphism, increasing timestamps",
                   "parallelism": f"host CPU, {threads} OpenMP threads",
                   "path": "CPU oracle: seed DFS over sampled inserted edges of every timed batch"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{sample} random inserted edges per batch (|dS+| of all 4 queries, "
                                   f"seeds over {threads} OpenMP threads, adjacency rebuild included), "
                                   f"batches {args.warmup}..{args.warmup + args.steps - 1} of the window stream"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving mode

def run_serve(args, local):
    """Serving on the NetFlow-like stream (workloads.FLOW: 10M hosts, 6
    protocol labels, window 2^24, 8 standing queries): Poisson arrivals of
    log-uniform batches in [2^10, 2^18] edges; requests that queue while the
    GPU is busy are admitted together (continuous batching under a device
    memory budget).  First the maximum sustained rate is measured closed-loop
    (a backlog of requests), then the offered load is set to 50 / 80 / 95% of
    it.  Latency is arrival -> counts on the host.  Sampled parity: on device
    batches 0, 1, 2, 3 and every 16th of each load level, the records that
    contain one of 24 sampled edges equal the CPU oracle's."""
    import torch
    from oracle import oracle
    from paper_2206_09983_b300 import build, workloads
    from paper_2206_09983_b300 import mnemonic as M
    from paper_2206_09983_b300.serve import Server, poisson_batches

    build.build()
    torch.cuda.set_device(local)
    w = workloads.FLOW
    W, MB = w["window"], w["max_batch"]
    levels = [0.5, 0.8, 0.95]
    per_level = args.serve_edges
    n_total = W + (3 + 60) * (1 << 16) + (1 + len(levels)) * per_level    # warm-up, tuning, levels
    assert n_total <= w["num_edges"], "serve run longer than the stream"
    t0 = time.perf_counter()
    stream = workloads.flow_prefix(n_total)
    packed = M.edges_from_stream(stream, 0, n_total)
    gen_s = time.perf_counter() - t0
    qs = workloads.flow_queries()
    g = M.Graph(stream["num_vertices"], stream["num_edge_labels"], vmask=stream["vmask"], window=W,
                max_batch=MB, max_queries=len(qs), device=local, out_capacity=1 << 18)
    for lo in range(0, W, MB):
        g.insert(packed[lo:lo + MB], count_only=True)
    for q in qs:
        g.register_query(q)
    pos = W
    if args.serve_order == "learned":
        g.set_order_policy("explore")
    for _ in range(3):                                             # warm-up
        g.insert(packed[pos:pos + (1 << 16)])
        pos += 1 << 16
    tune = None
    if args.serve_order == "learned":
        g.train_order_model(epochs=args.train_epochs, lr=2e-3)
        g.set_order_policy("learned")
        # the learned + batched form: online autotuning of the launch and of
        # the filtering on live 65,536-edge batches before serving
        g.autotune(1)
        nt = 0
        while g.autotune_state()[0] and nt < 60:
            g.insert(packed[pos:pos + (1 << 16)])
            pos += 1 << 16
            nt += 1
        tune = {"batches": nt, "tuning": g.get_tuning(), "filter_trial": g.autotune_filter_result(),
                "margin_trial": g.autotune_margin_result()}
    rng = np.random.default_rng(0x5E4E)
    rec_bytes = [(4 * q["nv"] + 7) // 8 * 8 + 8 * len(q["edges"]) for q in qs]

    def one_level(rate, edges):
        """Serve `edges` edges; rate None = closed loop (all requests at t=0)."""
        nonlocal pos
        if rate is None:
            sizes = poisson_batches(rng, edges, 1 << 10, MB, 1e12)
        else:
            sizes = poisson_batches(rng, edges, 1 << 10, MB, rate)
        srv = Server(mem_budget_bytes=16 << 30, merge=True, max_batch=MB)
        ten = srv.add_tenant("flow", g, keep_rows=False, count_only=False)
        g.set_timing(True)
        g.reset_stats()
        reqs, spans = [], []
        t_start = time.perf_counter()
        for t, size in sizes:
            if rate is not None:
                now = time.perf_counter() - t_start
                if t > now:
                    time.sleep(t - now)
            reqs.append(srv.submit("flow", packed[pos:pos + size],
                                   t_arrival=t_start + (t if rate is not None else 0.0)))
            spans.append((pos, pos + size))
            pos += size
        srv.drain(timeout=3600)
        t_end = max(r.t_done for r in reqs)
        srv.close()
        lat = np.array([1e3 * r.latency for r in reqs])
        n_edges = sum(len(r.edges) for r in reqs)
        st = g.stats()
        g.set_timing(False)
        nb = max(1, len(ten.batches))
        ins = np.array([1e3 * b[2] for b in ten.batches])
        dev = {"batches": len(ten.batches), "mean_edges": float(np.mean([b[0] for b in ten.batches])),
               "insert_ms": {"mean": float(ins.mean()), "p50": float(np.percentile(ins, 50)),
                             "p99": float(np.percentile(ins, 99))},
               "stage_ms_per_batch": {k: st["ms_" + k] / nb for k in ("ingest", "adjacency", "seeds", "filter",
                                                                      "enumerate", "expire")},
               "rerun_launches": st["rerun_launches"]}
        return {"offered_edges_per_s": rate, "value": n_edges / (t_end - t_start), "requests": len(reqs),
                "edges": n_edges, "device": dev,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "max": float(lat.max())},
                "mean_requests_per_batch": float(np.mean([r.merged_with for r in reqs])),
                "errors": sum(1 for r in reqs if r.error)}, reqs, spans

    out = {"mode": "serve", "metric": METRIC, "unit": UNIT,
           "config": {"workload": w["name"], "hosts": w["hosts"], "window": W, "max_batch": MB,
                      "queries": len(qs), "arrivals": "Poisson, batch sizes log-uniform in [1024, 262144]",
                      "path": (("learned matching order, autotuned launch and filtering"
                                if args.serve_order == "learned" else
                                "paper's matching order") + ", continuous batching (queued requests merged)"),
                      "stream_generation_s": gen_s},
           "tuning": tune}
    mx, _, _ = one_level(None, per_level)
    out["max_sustained"] = mx
    out["levels"] = []
    for f in levels:
        r, reqs, spans = one_level(f * mx["value"], per_level)
        r["fraction_of_max"] = f
        out["levels"].append(r)
    out["value"] = out["levels"][-1]["value"]
    out["device_memory"] = g.memory_info()
    g.close()
    # sampled parity on a fresh replay of device batches (the serve run kept
    # no lists): a second graph replays the same edges as the same batches
    out["parity"] = None if args.no_serve_parity else serve_parity(args, local, stream, packed, qs, W, MB)
    return out


def serve_parity(args, local, stream, packed, qs, W, MB):
    """Replay the serving stream's first device batches (sizes log-uniform in
    [2^10, 2^18]) on a fresh graph keeping lists; on batches 0, 1, 2, 3, 16
    and 32, compare the records that contain one of 24 sampled
    batch edges (plus the 4 edges with the highest-degree endpoints) with the
    CPU oracle's, for every query."""
    from oracle import oracle
    from paper_2206_09983_b300 import mnemonic as M
    rng = np.random.default_rng(0x5E4F)
    g = M.Graph(stream["num_vertices"], stream["num_edge_labels"], vmask=stream["vmask"], window=W,
                max_batch=MB, max_queries=len(qs), device=local, out_capacity=1 << 18)
    for lo in range(0, W, MB):
        g.insert(packed[lo:lo + MB], count_only=True)
    for q in qs:
        g.register_query(q)
    pos, lo_w, checked, rows_checked = W, 0, [], 0
    for k in range(33):
        size = int(np.exp(rng.uniform(np.log(1 << 10), np.log(MB))))
        r = g.insert(packed[pos:pos + size])
        hi, hi_new = pos, pos + size
        x = max(0, hi_new - lo_w - W)
        if k in (0, 1, 2, 3) or k % 16 == 0:
            deg = np.bincount(stream["src"][lo_w:hi_new], minlength=stream["num_vertices"])
            for sign, base, n in ((+1, hi, size), (-1, lo_w, x)):
                if n == 0:
                    continue
                pick = base + rng.choice(n, size=min(n, 24), replace=False)
                bs = np.arange(base, base + n)
                hub = bs[np.argsort(-deg[stream["src"][bs]], kind="stable")[:4]]
                pick = np.unique(np.concatenate([pick, hub]))
                mask = np.zeros(hi_new - lo_w, dtype=np.uint8)
                mask[pick - lo_w] = 1
                for qi, q in enumerate(qs):
                    got = g.fetch_rows(qi, sign)
                    sel = np.isin(got[:, q["nv"]:], pick.astype(np.uint64)).any(axis=1)
                    want = oracle.delta(stream, lo_w, hi_new, 0, 0, q, batch_mask=mask)
                    assert got[sel].shape == want.shape and (got[sel] == want).all(), \
                        f"serve parity: batch {k} query {qi} sign {sign}"
                    rows_checked += len(want)
            checked.append(k)
        pos = hi_new
        lo_w += x
    g.close()
    return {"batches_checked": checked, "rows_checked": rows_checked, "ok": True,
            "sample": "24 random + 4 highest-degree batch edges per sign and checked batch, every query"}


# ------------------------------------------------------------------ GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-sample", type=int, default=0, help="edges per batch (0: 256 per core)")
    ap.add_argument("--cpu-sample", type=int, default=0, help="edges (0: 256 per core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--train-epochs", type=int, default=300)
    ap.add_argument("--plain-only", action="store_true", help="time only the plain arm (diagnostics)")
    ap.add_argument("--tuning", default="", help="blocks_per_sm,split_min,split_depth for both arms")
    ap.add_argument("--mode", default="bench", choices=["bench", "serve"])
    ap.add_argument("--workload", default="rmat20_window", choices=["rmat20_window", "rmat20_uneven"])
    ap.add_argument("--with-uneven", dest="with_uneven", action="store_true", default=True,
                    help="also time the 36-query batched workload on the same stream (the default)")
    ap.add_argument("--no-uneven", dest="with_uneven", action="store_false")
    ap.add_argument("--no-graph-probe", dest="graph_probe", action="store_false", default=True,
                    help="skip the CUDA-graph launch-overhead probe")
    ap.add_argument("--no-filter-arm", dest="filter_arm", action="store_false", default=True,
                    help="skip the plain arm with DEBI filtering")
    ap.add_argument("--serve-edges", type=int, default=30_000_000, help="edges per load level")
    ap.add_argument("--no-serve-parity", action="store_true", help="skip the sampled parity replay")
    ap.add_argument("--serve-order", default="learned", choices=["learned", "paper"])
    args = ap.parse_args()
    rank, world, local = env_rank()

    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)

    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc

    if args.mode == "serve":
        if rank == 0:
            print(json.dumps(run_serve(args, local)), flush=True)
        return 0

    import torch
    from paper_2206_09983_b300 import build, workloads
    from paper_2206_09983_b300 import mnemonic as M

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = workloads.rmat20_stream()
    packed = M.edges_from_stream(stream, 0, len(stream["src"]))
    d_edges = torch.from_numpy(packed.view(np.uint8)).to(dev)
    ctx = dict(torch=torch, M=M, dev=dev, local=local, rank=rank, world=world, stream=stream,
               packed=packed, base_ptr=d_edges.data_ptr(), cur_stream=torch.cuda.current_stream(dev))
    main_wl = workloads.WORKLOADS[args.workload]
    res = run_workload(args, ctx, main_wl, with_e2e=not args.no_e2e)
    line = res["line"]
    if args.graph_probe and world == 1:
        line["graph_capture"] = graph_probe(ctx, main_wl, res["pos"])
    if args.with_uneven and args.workload != "rmat20_uneven":
        # the batched-uneven-queries workload on the same stream, both arms
        extra = run_workload(args, ctx, workloads.WORKLOADS["rmat20_uneven"], with_e2e=False)["line"]
        line["batched_uneven"] = {k: extra[k] for k in (
            "value", "unit", "ms_per_step", "config", "plain", "learned_vs_plain", "latency_ms",
            "embeddings_per_step", "stage_ms_per_step", "work_per_step", "roofline", "tuning", "train",
            "clocks", "filtered", "presplit_gain", "model_roofline", "filter_trial", "margin_trial")}
        line["gpu_launches"] += extra["gpu_launches"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        W, B = main_wl["window"], main_wl["batch"]
        qs = main_wl["queries"]()
        sample = args.cpu_sample or oracle_sample_size(B) * 4 // max(4, len(qs))
        bi = (res["pos"] - W) // B - 1
        dt, rows, threads = oracle_sample(stream, qs, W, B, bi, sample)
        line["cpu_baseline"] = {
            "value": sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{sample} random inserted edges of batch {bi}, |dS+| of all {len(qs)} queries on the "
                      f"{W}-edge window (adjacency rebuild included), C oracle with the seeds over "
                      f"{threads} OpenMP threads; {rows} embeddings, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def graph_probe(ctx, wl, pos, small=4096, steps=40):
    """Launch overhead of the batch chain: batches of `small` edges on the
    same window and queries (paper order), kernel by kernel and then each as
    one CUDA graph (mn_set_graph_capture); CUDA-event time per batch."""
    torch, M, local = ctx["torch"], ctx["M"], ctx["local"]
    stream, base_ptr, cur_stream = ctx["stream"], ctx["base_ptr"], ctx["cur_stream"]
    W = wl["window"]
    qs = wl["queries"]()
    g = M.Graph(stream["num_vertices"], stream["num_edge_labels"], vmask=stream["vmask"], window=W,
                max_batch=wl["batch"], max_queries=len(qs), device=local, stream=cur_stream.cuda_stream,
                out_capacity=wl["out_capacity"])
    B0 = wl["batch"]
    for lo in range(0, W, B0):
        g.insert(None, device_ptr=base_ptr + 24 * lo, n=B0, count_only=True)
    for q in qs:
        g.register_query(q)
    out = {"batch": small}
    p = pos
    for mode in ("kernels", "graph"):
        g.set_graph_capture(mode == "graph")
        for _ in range(4):
            g.insert(None, device_ptr=base_ptr + 24 * p, n=small)
            p += small
        st0 = g.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur_stream)
        for _ in range(steps):
            g.insert(None, device_ptr=base_ptr + 24 * p, n=small)
            p += small
        e1.record(cur_stream)
        torch.cuda.synchronize()
        st1 = g.stats()
        out[mode] = {"ms_per_batch": e0.elapsed_time(e1) / steps,
                     "kernel_launches_per_batch": (st1["kernel_launches"] - st0["kernel_launches"]) / steps,
                     "graph_launches_per_batch": (st1["graph_launches"] - st0["graph_launches"]) / steps}
    g.close()
    out["speedup"] = out["kernels"]["ms_per_batch"] / out["graph"]["ms_per_batch"]
    return out


def presplit_gain(results):
    """Best enumeration time per unit of work among the autotuner's
    candidates with learned pre-splitting off and on, and the speed ratio of
    shared-memory slice staging against the same split without it (each
    candidate ran on a different live batch, so times are normalised by
    work)."""
    if not results:
        return None
    def best(sel):
        c = [(ms / w, cfg) for (*cfg, ms, w) in results if sel(cfg) and w > 1]
        return min(c) if c else None
    out = {}
    # learned pre-splitting: candidates without slice staging, threshold off vs on
    off, on = best(lambda c: c[3] == 0.0 and c[4] == 0), best(lambda c: c[3] != 0.0 and c[4] == 0)
    if off and on:
        out = {"ms_per_gwork_off": off[0] * 1e9, "ms_per_gwork_on": on[0] * 1e9, "ratio": off[0] / on[0],
               "best_off": list(off[1]), "best_on": list(on[1])}
    # shared-memory slice staging at the default split: off vs each threshold
    base = best(lambda c: c[1] == 40 and c[2] == 16 and c[3] == 0.0 and c[4] == 0)
    if base:
        out["slice_staging"] = {str(c[4]): base[0] / (ms / w) for (*c, ms, w) in results if c[4] and w > 1}
    return out or None


def run_workload(args, ctx, wl, with_e2e):
    """Both arms of one workload on the shared device-resident stream: the
    learned + autotuned arm (timed first; its end-to-end leg through host
    memory) and the plain GPU path (paper order, default launch parameters)
    on the same batches.  Returns the bench line of the learned arm with the
    plain arm beside it."""
    torch, M, dev, local = ctx["torch"], ctx["M"], ctx["dev"], ctx["local"]
    rank, world, stream, packed = ctx["rank"], ctx["world"], ctx["stream"], ctx["packed"]
    base_ptr, cur_stream = ctx["base_ptr"], ctx["cur_stream"]
    W, B = wl["window"], wl["batch"]
    K, WU = args.steps, max(3, args.warmup)
    qs = wl["queries"]()
    names = wl["query_names"]()
    n = len(stream["src"])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def arm(policy: str, with_e2e: bool, skip: int = 0, filtering: bool = False):
        """One arm on the same stream batches: preload, register, WU warm-up
        batches (under exploration for the learned arm, then training), K
        timed batches, then the end-to-end run."""
        g = M.Graph(stream["num_vertices"], stream["num_edge_labels"], vmask=stream["vmask"],
                    window=W, max_batch=B, max_queries=len(qs), device=local,
                    stream=cur_stream.cuda_stream, out_capacity=wl["out_capacity"])
        if world > 1:
            g.set_shard(rank, world)                             # this rank's part of the seeds
        res = {}
        if args.tuning:
            g.set_tuning(*[int(x) for x in args.tuning.split(",")])
        for lo in range(0, W, B):                               # preload the window
            g.insert(None, device_ptr=base_ptr + 24 * lo, n=B, count_only=True)
        for q in qs:
            g.register_query(q)
        if filtering:
            g.set_filtering(True)
        pos = W
        g.set_order_policy("explore" if policy == "learned" else "paper")
        for _ in range(WU):
            g.insert(None, device_ptr=base_ptr + 24 * pos, n=B)
            pos += B
        if policy == "learned":
            t0 = time.perf_counter()
            l0, l1 = g.train_order_model(epochs=args.train_epochs, lr=2e-3)
            ts = g.stats()
            res["train"] = {"loss_first": l0, "loss_last": l1, "epochs": args.train_epochs,
                            "seconds": time.perf_counter() - t0, "device_ms": ts["ms_train"],
                            "rows": ts["train_rows"]}
            g.set_order_policy("learned")
            if not args.tuning:                                  # online autotuning on live batches
                g.autotune(1)
                res["tune_batches"] = g.autotune_state()[1]
                while g.autotune_state()[0]:
                    g.insert(None, device_ptr=base_ptr + 24 * pos, n=B)
                    pos += B
                res["autotune"] = g.autotune_results()
                res["filter_trial"] = g.autotune_filter_result()
                res["margin_trial"] = g.autotune_margin_result()
        else:
            for _ in range(skip):                                # same batches as the learned arm
                g.insert(None, device_ptr=base_ptr + 24 * pos, n=B)
                pos += B
        assert pos + B * (K + (WU + K if with_e2e else 0)) <= n, "stream too short for the requested steps"
        g.set_timing(True)
        g.reset_stats()
        barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lat, counts, per_q = [], [], []
        torch.cuda.profiler.start()                  # ncu --profile-from-start off: timed batches only
        ev0.record(cur_stream)
        for _ in range(K):
            t0 = time.perf_counter()
            r = g.insert(None, device_ptr=base_ptr + 24 * pos, n=B)
            lat.append(time.perf_counter() - t0)
            counts.append((sum(r.count_pos), sum(r.count_neg)))
            per_q.append((list(r.count_pos), list(r.count_neg)))
            pos += B
        ev1.record(cur_stream)
        torch.cuda.profiler.stop()
        torch.cuda.synchronize()
        res["clocks"] = clk.stop()
        barrier()
        res.update(dev_ms=ev0.elapsed_time(ev1), lat=lat, counts=counts, per_q=per_q, st=g.stats())
        g.set_timing(False)
        res["e2e"] = None
        if with_e2e:
            host = torch.from_numpy(packed.view(np.uint8)[24 * pos: 24 * (pos + B * (WU + K))].copy())
            host = host.pin_memory()
            hp = host.data_ptr()
            for k in range(WU):
                g.insert_ptr(hp + 24 * B * k, B)
            st0 = g.stats()
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            elat = []
            for k in range(WU, WU + K):
                t1 = time.perf_counter()
                g.insert_ptr(hp + 24 * B * k, B)
                elat.append(time.perf_counter() - t1)
            torch.cuda.synchronize()
            e2e_s = time.perf_counter() - t0
            st1 = g.stats()
            if world > 1:
                import torch.distributed as dist
                t = torch.tensor([e2e_s], device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                e2e_s = float(t.item())
            res["e2e"] = {"value": K * B / e2e_s, "unit": UNIT,
                          "h2d_bytes_per_step": (st1["h2d_bytes"] - st0["h2d_bytes"]) // K,
                          "d2h_bytes_per_step": (st1["d2h_bytes"] - st0["d2h_bytes"]) // K,
                          "p50_ms": 1e3 * statistics.median(elat),
                          "p99_ms": 1e3 * float(np.percentile(elat, 99))}
        res["pos"] = pos
        res["tuning_used"] = g.get_tuning()
        g.close()
        return res

    filtered = None
    if args.plain_only:
        plain = learned = arm("paper", with_e2e=with_e2e)
    else:
        learned = arm("learned", with_e2e=with_e2e)
        plain = arm("paper", with_e2e=False, skip=learned.get("tune_batches", 0))
        if args.filter_arm:
            filtered = arm("paper", with_e2e=False, skip=learned.get("tune_batches", 0), filtering=True)
    for k in range(K):                                  # exact counts: the arms agree
        assert plain["per_q"][k] == learned["per_q"][k], "learned and plain counts differ"
        assert filtered is None or filtered["per_q"][k] == plain["per_q"][k], "filtered counts differ"
    dev_ms, lat, counts, per_q, st = (learned[k] for k in ("dev_ms", "lat", "counts", "per_q", "st"))
    clocks, e2e = learned["clocks"], learned["e2e"]

    # ---- aggregate over ranks (max time)
    dev_s = dev_ms / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([dev_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_s = float(t.item())
    value = K * B / dev_s                               # the stream's edges, once per job
    if world > 1:                                       # the job's counts: the shards' sum
        import torch.distributed as dist
        gl = dist.new_group(backend="gloo")
        for arm_res in (learned, plain) if plain is not learned else (learned,):
            pq = torch.tensor(arm_res["per_q"], dtype=torch.int64)
            dist.all_reduce(pq, group=gl)
            arm_res["per_q"] = pq.tolist()
            arm_res["counts"] = [(sum(a), sum(b)) for a, b in arm_res["per_q"]]
        counts, per_q = learned["counts"], learned["per_q"]

    # ---- roofline of the dominant stage, from the live event timings
    peak, peak_kind = measured_peaks()
    stage_ms = {"enumerate": st["ms_enumerate"], "adjacency": st["ms_adjacency"],
                "ingest": st["ms_ingest"], "seeds": st["ms_seeds"], "expire": st["ms_expire"],
                "model": st["ms_model"], "filter": st["ms_filter"]}
    # Algorithmic bytes of the enumerator (the method's traffic, counted from
    # the device work counters): per tested adjacency entry 8 B (neighbour,
    # seq) + 4 B DEBI word + 8 B timestamp when the query is temporal; per
    # record 4 n_q + 8 k_q; per seed 8 B seed word + 8 B ring endpoints.
    temporal = all(q["temporal"] != "none" for q in qs)
    entry_bytes = 20 if temporal else 12
    rec_alg = [4 * q["nv"] + 8 * len(q["edges"]) for q in qs]
    rec_layout = [(4 * q["nv"] + 7) // 8 * 8 + 8 * len(q["edges"]) for q in qs]
    rec_sum_alg = sum(sum((a[i] + b[i]) * rec_alg[i] for i in range(len(qs))) for a, b in per_q)
    rec_sum_layout = sum(sum((a[i] + b[i]) * rec_layout[i] for i in range(len(qs))) for a, b in per_q)
    launches = max(1, st["enumerate_launches"])
    enum_bytes = st["entries_scanned"] * entry_bytes + rec_sum_alg + st["seeds"] * 16
    enum_ms_per = st["ms_enumerate"] / launches
    roof = {"kernel": "k_enumerate", "bound": "hbm",
            "achieved": (enum_bytes / launches) / (enum_ms_per / 1e3) / 1e9 if enum_ms_per else None,
            "peak": peak, "unit": "GB/s", "traffic": enum_traffic() if wl["name"] == "rmat20_window" else None,
            "peak_source": f"{peak_kind} HBM copy bandwidth (burst figure: the kernel is timed alone per launch)",
            "bytes_per_launch": enum_bytes / launches, "ms_per_launch": enum_ms_per,
            "entry_bytes": entry_bytes,
            "launches_per_batch": st["enumerate_launches"] / K,
            "rerun_launches_per_batch": st.get("rerun_launches", 0) / K,
            "counting": (f"entries tested x {entry_bytes} B (8 B entry + 4 B DEBI word"
                         f"{' + 8 B timestamp: every query is temporal' if temporal else ''}) + records x "
                         f"(4 n_q + 8 k_q) + seeds x 16 B")}
    roof["frac"] = roof["achieved"] / peak if roof["achieved"] else None
    # the same with the device's own layout (12 B per entry: neighbour, seq32,
    # DEBI word; records padded to 8 bytes), for comparison
    layout_bytes = st["entries_scanned"] * 12 + rec_sum_layout + st["seeds"] * 16
    roof["layout_bytes_per_launch"] = layout_bytes / launches
    # sector-granular variant: every random touch rounded up to a 32-byte
    # sector (an upper estimate: each tested entry's DEBI word as one touch,
    # each seed's ring endpoints as two)
    sector_bytes = st["entries_scanned"] * (8 + 32) + rec_sum_layout + st["seeds"] * (8 + 64)
    roof["sector_bytes_per_launch"] = sector_bytes / launches
    roof["sector_achieved"] = ((sector_bytes / launches) / (enum_ms_per / 1e3) / 1e9
                               if enum_ms_per else None)
    tu = learned.get("tuning_used") or {}
    enum_warps = (torch.cuda.get_device_properties(dev).multi_processor_count * ENUM_WARPS_PER_BLOCK
                  * max(1, tu.get("blocks_per_sm", 2)))
    # adjacency update: the method's bytes are 2 x 8 B per inserted edge (one
    # entry per direction); the implementation rewrites the live window's
    # four sorted orders (out/in x by neighbour/by arrival, 12 B per entry),
    # read and written once per batch
    adj_alg = 16 * B
    adj_layout = 4 * 2 * (W + B) * 12
    adj = {"kernel": "adjacency update (delta sort + one-pass merge + offsets)",
           "ms_per_batch": st["ms_adjacency"] / K,
           "achieved_layout": adj_layout / (st["ms_adjacency"] / K / 1e3) / 1e9 if st["ms_adjacency"] else None,
           "unit": "GB/s", "algorithmic_bytes_per_batch": adj_alg, "layout_bytes_per_batch": adj_layout}

    # the work model's tensor-core kernels: the forward in every timed batch
    # (seeds x NCAND rows), the gradient kernel over the training passes
    bf16_burst, bf16_kind = measured_bf16_peak()
    model_roof = None
    if st.get("ms_model"):
        fl = st["seeds"] * NCAND * MLP_FWD_FLOPS / max(1, st["model_launches"])
        ms = st["ms_model"] / max(1, st["model_launches"])
        model_roof = {"kernel": "k_mlp_forward_tc", "bound": "tensor", "unit": "TFLOP/s",
                      "achieved": fl / (ms / 1e3) / 1e12, "peak": bf16_burst, "ms_per_launch": ms,
                      "flops_per_launch": fl, "peak_source": f"{bf16_kind} dense BF16 (cuBLAS burst)"}
        model_roof["frac"] = model_roof["achieved"] / bf16_burst
    tr = learned.get("train") or {}
    if tr.get("device_ms"):
        fl = tr["rows"] * MLP_GRAD_FLOPS
        tr["roofline"] = {"kernel": "k_mlp_grad_tc (+ k_adam)", "bound": "tensor", "unit": "TFLOP/s",
                          "achieved": fl / (tr["device_ms"] / 1e3) / 1e12, "peak": bf16_burst,
                          "peak_source": f"{bf16_kind} dense BF16 (cuBLAS burst)"}
        tr["roofline"]["frac"] = tr["roofline"]["achieved"] / bf16_burst

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": WU,
        "ms_per_step": 1e3 * dev_s / K, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": wl["name"], "vertices": stream["num_vertices"], "edges": n,
                   "window": W, "batch": B, "queries": names if len(names) <= 8 else f"{len(names)} queries",
                   "semantics": "isomorphism, increasing timestamps", "l2": CTRL_NOTE,
                   "parallelism": (f"seed-sharded over {world} GPUs (each ingests the whole stream)"
                                   if world > 1 else "1 GPU"),
                   "path": "learned matching order + learned splits + autotuned launch (value) vs plain "
                           "GPU path with the paper's order"},
        "plain": {"value": K * B / (plain["dev_ms"] / 1e3), "unit": UNIT,
                  "ms_per_step": plain["dev_ms"] / K,
                  "latency_ms": {"p50": 1e3 * statistics.median(plain["lat"]),
                                 "p99": 1e3 * float(np.percentile(plain["lat"], 99))},
                  "work_per_step": {k: plain["st"][k] / K for k in ("entries_scanned", "binds", "tasks_split")},
                  "stage_ms_per_step": {"enumerate": plain["st"]["ms_enumerate"] / K,
                                        "adjacency": plain["st"]["ms_adjacency"] / K},
                  "clocks": plain["clocks"]},
        "learned_vs_plain": (plain["dev_ms"] / dev_ms) if dev_ms else None,
        # the plain path with the DEBI neighbourhood filtering on (same
        # batches, same counts): pass time and seeds it removed
        "filtered": None if filtered is None else {
            "ms_per_step": filtered["dev_ms"] / K,
            "stage_ms_per_step": {"filter": filtered["st"]["ms_filter"] / K,
                                  "enumerate": filtered["st"]["ms_enumerate"] / K},
            "seeds_per_step": filtered["st"]["seeds"] / K,
            "seeds_filtered_per_step": filtered["st"]["seeds_filtered"] / K,
            "filter_changes_per_step": filtered["st"]["filter_changes"] / K,
            "work_per_step": {k: filtered["st"][k] / K for k in ("entries_scanned", "binds")}},
        "train": learned.get("train"),
        "tuning": {"plain": plain.get("tuning_used"), "learned": learned.get("tuning_used")},
        # the autotuner's trial of the DEBI filtering on the learned arm (kept
        # for the timed batches when it was faster per inserted edge)
        "filter_trial": learned.get("filter_trial"),
        # the autotuner's trial of the learned order's margin (log2 units by
        # which a pick must beat the paper's order), run first
        "margin_trial": learned.get("margin_trial"),
        # the autotuner's live measurements (one batch per candidate, learned
        # order): the best configuration with and without learned pre-splitting
        "presplit_gain": presplit_gain(learned.get("autotune")),
        "latency_ms": {"p50": 1e3 * statistics.median(lat), "p99": 1e3 * float(np.percentile(lat, 99)),
                       "max": 1e3 * max(lat)},
        "embeddings_per_step": {"new": float(np.mean([c[0] for c in counts])),
                                "removed": float(np.mean([c[1] for c in counts]))},
        "embeddings_per_step_by_query": {
            name: {"new": float(np.mean([c[0][i] for c in per_q])),
                   "removed": float(np.mean([c[1][i] for c in per_q]))}
            for i, name in enumerate(names)},
        "stage_ms_per_step": {k: v / K for k, v in stage_ms.items()},
        "work_per_step": {k: st[k] / K for k in ("seeds", "entries_scanned", "binds", "records",
                                                  "tasks_split")},
        # share of the enumerator's warp-time spent inside work units (the rest
        # is waiting for work at the end of a launch: load imbalance)
        "enum_warp_utilization": (st["busy_cycles"] / (st["ms_enumerate"] * 1e-3 * clocks["sm_mhz"] * 1e6
                                                        * enum_warps)
                                  if st["ms_enumerate"] and clocks.get("sm_mhz") else None),
        "gpu_launches": st["kernel_launches"],
        "roofline": roof,
        "adjacency_roofline": adj,
        "model_roofline": model_roof,
        "clocks": clocks,
        "e2e": e2e,
    }
    return {"line": line, "pos": learned["pos"]}


if __name__ == "__main__":
    sys.exit(main())
