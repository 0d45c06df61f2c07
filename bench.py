#!/usr/bin/env python
"""Throughput of the plain generator on the paper-scale workload.

One step = one call of the C-ABI entry point rhg_generate_pairs: the whole hot
path (R solve, band boundaries, Philox sampling, band assignment, radix sort,
gather, range query count, scan, range query emit) for n = 10^7, k = 200,
alpha = 1, seed 3 (~1.05e9 undirected edges written as uint32 pairs, ~8.4 GB).
The metric is edges per second; the working set (~9 GB) is far larger than L2,
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank generates its own graph (seed 3 + rank):
replicas, weak scaling, no collective on the data path.  --impl reference times
the CPU oracle on a bounded vertex sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s on 1 GB300 (plain vs batched/served, exact edge set); p50/p99 latency"
WORKLOAD = {"n": 10_000_000, "k": 200.0, "alpha": 1.0, "seed": 3}
WORKLOAD_NAME = "plain large graph: n=1e7, k=200, alpha=1.0, seed 3, uint32 pairs (~1G edges)"

# per-unit algorithmic bytes of the range query: every point is read once from
# the sorted arrays (sort key 8 B, angle key 4 B, angle hi/lo 8 B, P/M/S/gamma
# 16 B, id 4 B) and every edge is written once as two uint32; candidate reads are
# served by L1/L2 reuse inside a band window.
QUERY_BYTES_PER_POINT = 40
QUERY_BYTES_PER_EDGE = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-workload measurement")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--no-served", action="store_true", help="skip the served-workload measurement")
    ap.add_argument("--no-dynamic", action="store_true", help="skip the dynamic-model measurement")
    ap.add_argument("--no-configs", action="store_true", help="skip the small-pairs and CSR configurations")
    ap.add_argument("--moved", type=float, default=0.12, help="fraction of vertices moved per dynamic step")
    ap.add_argument("--served-requests", type=int, default=400, help="requests per arrival rate")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--k", type=float, default=WORKLOAD["k"])
    ap.add_argument("--alpha", type=float, default=WORKLOAD["alpha"])
    ap.add_argument("--seed", type=int, default=WORKLOAD["seed"])
    ap.add_argument("--bands", type=int, default=0, help="number of bands (0: ceil(log2 n))")
    ap.add_argument("--band-ratio", type=float, default=0.0, help="geometric band ratio p (0: 0.9)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


TRAFFIC_SOURCES = ("paper_1606_09481_gb300/csrc/query.cu", "paper_1606_09481_gb300/csrc/common.cuh",
                   "paper_1606_09481_gb300/csrc/kernels.h", "paper_1606_09481_gb300/csrc/detmath.cuh",
                   "paper_1606_09481_gb300/csrc/stages.cuh", "include/rhg.h")


def sources_digest(paths=TRAFFIC_SOURCES) -> str:
    """sha256 (16 hex digits) over the listed sources, in order: every file the
    range query kernels are compiled from."""
    h = hashlib.sha256()
    for rel in paths:
        h.update(rel.encode())
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def kernel_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if none of the
    sources the kernel is compiled from has changed since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or "sources_sha256_16" not in e:
        return None
    return e["dram_bytes_per_launch"] if sources_digest() == e["sources_sha256_16"] else None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if smax and s >= 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def cpu_baseline(args, budget_s: float = 20.0, steps: int = 1):
    """The oracle (plain C, FP64) on this host: all points, the band structure,
    and the outward range queries of a vertex sample.  The O(n log n) set-up
    (points and bands) runs once and is charged once, in full when the samples
    cover at least n vertices, else pro rata to the vertices queried.
    Returns (edges/s, info)."""
    import numpy as np

    import oracle
    n, k, alpha, seed = args.n, args.k, args.alpha, args.seed
    R = oracle.target_radius(n, k, alpha)
    B = oracle.default_bands(n)
    t0 = time.perf_counter()
    phi, r = oracle.sample_points(n, alpha, R, seed)
    t_points = time.perf_counter() - t0
    t0 = time.perf_counter()
    prep = oracle.Prepared(phi, r, R, B, 0.9)
    t_bands = time.perf_counter() - t0
    # probe the per-vertex query cost on a small sample, then size the real one
    rng = np.random.default_rng(12345)
    probe = np.sort(rng.choice(n, size=2000, replace=False)).astype(np.uint32)
    t0 = time.perf_counter()
    prep.count_edges(probe)
    per_vertex = max((time.perf_counter() - t0) / len(probe), 1e-8)
    size = int(min(n, max(2000, budget_s / steps / per_vertex)))
    total_edges, query_time, threads = 0, 0.0, 1
    diag = None
    for step in range(steps):
        ids = np.sort(rng.choice(n, size=size, replace=False)).astype(np.uint32)
        t0 = time.perf_counter()
        m_s, threads, st = prep.count_edges(ids, with_stats=True)
        query_time += max(time.perf_counter() - t0, 1e-9)
        total_edges += m_s
        diag = diag or st
    setup_charged = (t_points + t_bands) * min(1.0, steps * size / n)
    total_time = query_time + setup_charged
    value = total_edges / total_time
    # the same queries on one thread, on a sample sized for about a tenth of the budget
    size1 = int(min(n, max(500, 0.1 * budget_s / max(per_vertex * threads, 1e-8))))
    ids1 = np.sort(rng.choice(n, size=size1, replace=False)).astype(np.uint32)
    t0 = time.perf_counter()
    m1, _ = prep.count_edges(ids1, threads=1)
    t1 = time.perf_counter() - t0 + (t_points + t_bands) * size1 / n
    prep.close()
    # the O(n^2) all-pairs definition on the small plain graph (n = 10^4, k = 6, alpha = 1, seed 1)
    R1 = oracle.target_radius(10_000, 6, 1.0)
    phi1, r1 = oracle.sample_points(10_000, 1.0, R1, 1)
    t0 = time.perf_counter()
    mb = len(oracle.brute_edges(phi1, r1, R1))
    tb = time.perf_counter() - t0
    info = {"value": value, "unit": "edges/s", "cores": threads, "kind": "oracle",
            "sample": (f"outward range queries of {size} random vertices per step x {steps} step(s) on the full "
                       f"n={n} point set ({total_edges} edges); point sampling ({t_points:.1f} s, 1 thread) and "
                       f"band build ({t_bands:.1f} s, 1 thread) run once, charged once "
                       f"({min(1.0, steps * size / n):.3f} of it: the fraction of n queried)"),
            "seconds": total_time, "setup_seconds_charged": setup_charged, "query_seconds": query_time,
            "diagnostics_first_step": diag,
            "single_thread": {"value": m1 / t1, "unit": "edges/s", "cores": 1,
                              "sample": f"outward range queries of {size1} random vertices ({m1} edges), set-up "
                                        f"charged pro rata"},
            "all_pairs_small": {"value": mb / tb, "unit": "edges/s", "cores": 1, "seconds": tb,
                                "sample": f"O(n^2) all pairs of n=10000, k=6, alpha=1, seed 1 ({mb} edges)"}}
    return value, info


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    steps = max(1, args.steps)
    budget = min(150.0, 12.0 * steps)
    value, info = cpu_baseline(args, budget_s=budget, steps=steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000 * info["seconds"] / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "n": args.n, "k": args.k,
                                             "alpha": args.alpha, "seed": args.seed},
            "cpu_baseline": info,
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_configs(args, rhg, torch, stream, reps1: int = 200, reps2: int = 20):
    """The two other plain configurations, each with its own throughput and the
    roofline of its range query:
    - small pairs graph: n = 1e4, k = 6, alpha = 1, seed 1 (uint32 pairs);
    - CSR graph: n = 1e6, k = 16, alpha = 0.75, seed 2 (row_ptr u64[n+1] +
      col u32[2m]); its CSR stage (radix sort of the 2m directed keys the query
      writes, then the row pointers) is timed on its own, with algorithmic bytes
      = 16 B per directed key written and read by the query/sort boundary plus
      the sort's passes (8 B read + 8 B written per key and pass) + 4 B per column
      entry + 8 B per row pointer."""
    import ctypes
    L = rhg.load()
    peak, peak_kind = measured_peaks()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sptr = ctypes.c_void_p(stream.cuda_stream)
    out = {}

    def timed(call, reps):
        for _ in range(5):
            call()
        torch.cuda.synchronize()
        timer = rhg.StageTimer()
        with timer:
            e0.record(stream)
            for _ in range(reps):
                timer.reset_marks()
                res = call()
                timer.accumulate()
            e1.record(stream)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, {s_: timer.totals[s_] / reps for s_ in rhg.STAGES}, res

    # small pairs graph
    n, k, a, sd = 10_000, 6.0, 1.0, 1
    p = rhg.make_params(n, k, a, sd)
    wsp = rhg.allocate_pairs(p)
    ms, st, res = timed(lambda: rhg.generate_pairs(n, k, a, sd, workspace=wsp, stream=stream)[1], reps1)
    m = int(res.m)
    alg = n * QUERY_BYTES_PER_POINT + m * QUERY_BYTES_PER_EDGE
    out["small_pairs"] = {
        "workload": "plain single graph: n=1e4, k=6, alpha=1.0, seed 1, uint32 pairs", "edges": m,
        "value": m / (ms / 1e3), "unit": "edges/s", "ms_per_step": ms, "stages_ms": st, "reps": reps1,
        "roofline": {"kernel": "range query", "bound": "hbm", "achieved": alg / (st["query"] / 1e3) / 1e9,
                     "peak": peak, "unit": "GB/s", "frac": alg / (st["query"] / 1e3) / 1e9 / peak,
                     "algorithmic_bytes_per_launch": alg, "peak_source": f"{peak_kind} hbm_gbs"},
        "note": "launch- and latency-bound: ~28 kernel launches and one host synchronisation per call"}
    del wsp
    # CSR graph
    n, k, a, sd = 10**6, 16.0, 0.75, 2
    p = rhg.make_params(n, k, a, sd)
    row_ptr, col, res0 = rhg.generate_csr(n, k, a, sd, stream=stream)
    cap = int(col.numel()) + 4096
    nb = ctypes.c_size_t(0)
    L.rhg_workspace_bytes(ctypes.byref(p), cap, ctypes.byref(nb))
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    colbuf = torch.empty(cap, dtype=torch.int32, device="cuda")
    res = rhg.Result()

    def csr_call():
        rc = L.rhg_generate_csr(ctypes.byref(p), ws.data_ptr(), ws.numel(), row_ptr.data_ptr(), colbuf.data_ptr(),
                                cap, sptr, ctypes.byref(res))
        rhg._check(rc, "rhg_generate_csr", res)
        return res

    ms, st, res = timed(csr_call, reps2)
    m = int(res.m)
    q_alg = n * QUERY_BYTES_PER_POINT + m * 16
    passes = 2 * ((max(n - 1, 1).bit_length() + 7) // 8)
    csr_alg = 2 * m * (16 * passes + 8 + 4) + 8 * (n + 1)
    out["csr"] = {
        "workload": "plain single graph: n=1e6, k=16, alpha=0.75, seed 2, CSR (row_ptr u64[n+1], col u32[2m])",
        "edges": m, "value": m / (ms / 1e3), "unit": "edges/s", "ms_per_step": ms, "stages_ms": st, "reps": reps2,
        "roofline": {"kernel": "range query", "bound": "hbm", "achieved": q_alg / (st["query"] / 1e3) / 1e9,
                     "peak": peak, "unit": "GB/s", "frac": q_alg / (st["query"] / 1e3) / 1e9 / peak,
                     "algorithmic_bytes_per_launch": q_alg, "peak_source": f"{peak_kind} hbm_gbs",
                     "bytes_note": "40 B per point read + 16 B per edge written (two 8-byte directed keys)"},
        "csr_stage_roofline": {"kernel": f"radix sort of 2m keys ({passes} passes) + row pointers", "bound": "hbm",
                               "achieved": csr_alg / (st["csr"] / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                               "frac": csr_alg / (st["csr"] / 1e3) / 1e9 / peak,
                               "algorithmic_bytes_per_launch": csr_alg}}
    del ws, colbuf, row_ptr, col
    return out


def batched_specs(count: int = 4096):
    """The batched workload: graph j has seed 1000 + j, n = floor(10^U(3, 5)),
    k uniform in 6..32, alpha uniform in [0.55, 1.5], drawn by numpy's PCG64 with
    seed 4096 (the same list on every run)."""
    import numpy as np
    rng = np.random.default_rng(4096)
    return [(int(10 ** rng.uniform(3, 5)), int(rng.integers(6, 33)), float(rng.uniform(0.55, 1.5)), 1000 + j)
            for j in range(count)]


def bench_batched(args, rhg, torch, stream):
    """Edges/s of the batched path (one rhg_generate_batch call per step for all
    graphs) against the plain path called once per graph on the same graphs."""
    specs = batched_specs(args.batch_graphs)
    params = rhg.batch_params(specs)
    buf = rhg.allocate_batch(params)
    rc, res, tot = rhg.run_batch(buf, stream)
    if rc == rhg.OVERFLOW:
        caps = [max(int(res[g].m), int(buf.offsets[g + 1] - buf.offsets[g])) for g in range(len(params))]
        del buf
        buf = rhg.allocate_batch(params, caps)
        rc, res, tot = rhg.run_batch(buf, stream)
    if rc != rhg.OK:
        raise rhg.RhgError(rc, "rhg_generate_batch", tot)
    for _ in range(max(args.warmup - 1, 0)):
        rhg.run_batch(buf, stream)
    timer = rhg.StageTimer()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with timer:
        e0.record(stream)
        for _ in range(args.steps):
            timer.reset_marks()
            rc, res, tot = rhg.run_batch(buf, stream)
            timer.accumulate()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    m = int(tot.m)
    points = sum(sp[0] for sp in specs)
    # the same batch prepared once and captured in a CUDA graph, then replayed
    plan = rhg.batch_prepare(buf, stream)
    graph = rhg.capture_batch(plan, buf)
    with torch.cuda.stream(stream):
        graph.replay()
    grc, _, gtot = rhg.batch_read_results(plan, buf, stream)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup - 1, 0)):
            graph.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / args.steps
    graph_replay = {"value": int(gtot.m) / (graph_ms / 1000.0), "ms_per_step": graph_ms,
                    "edges_equal_default": grc == rhg.OK and int(gtot.m) == m}
    device_stages = rhg.batch_stage_times(plan, buf, stream)  # of the last replay
    del graph
    del buf
    # the plain path, one call per graph, reusing one workspace sized for the most
    # demanding graph (the largest n, or a graph that may run in FP64 mode)
    cap = max(int(r.m) for r in res) + 4096
    ws_bytes = max(rhg.workspace_bytes(rhg.make_params(*sp)) for sp in specs)
    wsp = rhg.Workspace(torch.empty(ws_bytes, dtype=torch.uint8, device="cuda"),
                        torch.empty(2 * cap, dtype=torch.int32, device="cuda"), cap)
    for sp in specs[:64]:
        rhg.generate_pairs(*sp, workspace=wsp)
    torch.cuda.synchronize()
    e0.record(stream)
    plain_m = 0
    for sp in specs:
        _, r = rhg.generate_pairs(*sp, workspace=wsp)
        plain_m += int(r.m)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    del wsp
    value = m / (ms / 1000.0)
    plain = plain_m / (plain_ms / 1000.0)
    # the band count per size class chosen by the autotuner, then the same timing
    from paper_1606_09481_gb300.autotune import gpu_runner, tune
    table = tune(specs, gpu_runner(stream))

    def tuned_one(n, kk, a, sd):
        b, bb, ch, fl = table.params(n)
        return rhg.make_params(n, kk, a, sd, b, batch_budget=bb, core_heavy=ch, fringe_limit=fl)

    tuned_params = (rhg.Params * len(specs))(*[tuned_one(*sp) for sp in specs])
    tbuf = rhg.allocate_batch(tuned_params)
    rc, tres, ttot = rhg.run_batch(tbuf, stream)
    if rc == rhg.OVERFLOW:
        caps = [max(int(tres[g].m), int(tbuf.offsets[g + 1] - tbuf.offsets[g])) for g in range(len(specs))]
        del tbuf
        tbuf = rhg.allocate_batch(tuned_params, caps)
        rc, tres, ttot = rhg.run_batch(tbuf, stream)
    for _ in range(max(args.warmup - 1, 0)):
        rhg.run_batch(tbuf, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        rc, tres, ttot = rhg.run_batch(tbuf, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    tuned_ms = e0.elapsed_time(e1) / args.steps
    del tbuf
    tuned = {"value": int(ttot.m) / (tuned_ms / 1000.0), "ms_per_step": tuned_ms,
             "edges_equal_default": int(ttot.m) == m,
             "tuned_per_size_class": table.describe()}
    peak, peak_kind = measured_peaks()
    q_ms = sum(v for s_, v in device_stages.items() if s_.startswith(("query", "heavy", "recheck")))
    alg = points * QUERY_BYTES_PER_POINT + m * QUERY_BYTES_PER_EDGE
    roof = {"kernel": "batched range query (all graphs)", "bound": "hbm", "achieved": alg / (q_ms / 1e3) / 1e9,
            "peak": peak, "unit": "GB/s", "frac": alg / (q_ms / 1e3) / 1e9 / peak, "algorithmic_bytes_per_launch": alg,
            "avg_launch_ms": q_ms, "peak_source": f"{peak_kind} hbm_gbs",
            "whole_call_frac": (alg / (ms / 1e3) / 1e9) / peak}
    return {"value": value, "unit": "edges/s", "ms_per_step": ms, "graphs": len(specs), "points": points,
            "roofline": roof,
            "autotuned": tuned, "graph_replay": graph_replay,
            "edges": m, "exact_edges_equal_plain": plain_m == m, "plain_per_graph_value": plain,
            "plain_per_graph_ms": plain_ms, "speedup_vs_plain": value / plain,
            "stages_ms": device_stages, "launches_per_call": "1 (persistent, cooperative)",
            "workload": "batched: 4096 graphs, n log-uniform in [1e3, 1e5], k uniform in 6..32, alpha uniform "
                        "in [0.55, 1.5], seeds 1000..5095 (numpy PCG64 seed 4096), FP32 filter + FP64 recheck, "
                        "B = ceil(log2 n) per graph"}


def bench_served(args, rhg, torch):
    """Served workload: the plain path's capacity (requests one after another on
    one stream), then Poisson arrivals at multiples of it through the serving
    loop (4 workers, 120 GB admission budget, grouping of requests with n <= 1e5);
    p50/p99 latency (arrival to edges ready on the device) and edges/s."""
    from paper_1606_09481_gb300.serve import Server, percentile, poisson_requests, replay
    sample = poisson_requests(args.served_requests, rate=1.0, seed=5)
    for r in sample[:8]:  # warm-up: caching allocator, module load
        rhg.generate_pairs(r.n, r.k, r.alpha, r.seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_m = 0
    for r in sample:
        _, res = rhg.generate_pairs(r.n, r.k, r.alpha, r.seed)
        plain_m += int(res.m)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    cap = len(sample) / plain_s
    rates = []
    for mult in (0.25, 0.5, 1.0, 2.0, 4.0):
        reqs = poisson_requests(args.served_requests, rate=mult * cap, seed=5)
        srv = Server(budget_bytes=120 * 10**9, workers=4)
        done = replay(srv, reqs)
        lat = [1000.0 * c.latency for c in done]
        span = max(c.end for c in done) - min(c.arrival for c in done)
        m = sum(c.m for c in done)
        rates.append({"multiple_of_plain_capacity": mult, "rate_rps": mult * cap, "requests": len(done),
                      "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99), "edges_per_s": m / span,
                      "batched_fraction": sum(c.batch_size > 1 for c in done) / len(done),
                      "peak_reserved_gb": srv.peak_reserved / 1e9})
    peak, _ = measured_peaks()
    for r in rates:  # bytes the generations write (pairs) and read (sorted points) per second, vs the peak
        r["hbm_frac_of_output_and_points"] = (r["edges_per_s"] * QUERY_BYTES_PER_EDGE) / 1e9 / peak
    best = max(r["edges_per_s"] for r in rates)
    return {"plain_capacity_rps": cap, "plain_edges_per_s": plain_m / plain_s, "best_edges_per_s": best,
            "speedup_vs_plain": best / (plain_m / plain_s), "rates": rates,
            "workload": f"served: {args.served_requests} requests per rate, n = floor(10^U(4,7)), k uniform in "
                        "8..64, alpha uniform in [0.6, 1.2], seeds 10^6 + request, Poisson arrivals (numpy PCG64 "
                        "seed 5) at 0.25..4x the plain path's capacity; 120 GB admission budget, 4 workers"}


def bench_dynamic(args, rhg, torch, stream):
    """Dynamic model at the plain workload's size: one step = move a fraction of
    the vertices (rotation + Algorithm 2) and update the edge list from the
    previous one (rhg_update_edges), against generating the graph of the moved
    points again (rhg_edges_from_points).  Buffers are allocated once."""
    L = rhg.load()
    n, k, alpha = args.n, args.k, args.alpha
    phi, r, R = rhg.sample_points(n, k, alpha, args.seed)
    cap = rhg.estimate_capacity(n, k)
    nb = ctypes.c_size_t(0)
    L.rhg_workspace_bytes_points(n, 0, ctypes.byref(nb))
    ws_full = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    cnt = int(args.moved * n)
    L.rhg_workspace_bytes_update(n, cnt, 0, ctypes.byref(nb))
    ws_upd = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    bufs = [torch.empty(2 * cap, dtype=torch.int32, device="cuda") for _ in range(2)]
    sptr = ctypes.c_void_p(stream.cuda_stream)
    res = rhg.Result()

    def full(out):
        rc = L.rhg_edges_from_points(phi.data_ptr(), r.data_ptr(), n, R, 0, 0.0, 0, ws_full.data_ptr(),
                                     ws_full.numel(), out.data_ptr(), cap, sptr, ctypes.byref(res))
        rhg._check(rc, "rhg_edges_from_points", res)
        return int(res.m)

    m = full(bufs[0])
    tphi, tr = rhg.draw_movement(n, args.seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed)
    steps = []
    for _ in range(args.warmup + args.steps):
        steps.append(torch.sort(torch.randperm(n, device="cuda", generator=gen)[:cnt]).values.to(torch.int32))
    cur = 0

    def update(ids, src, dst, m_old):
        L.rhg_move_points(ids.data_ptr(), cnt, n, phi.data_ptr(), r.data_ptr(), tphi.data_ptr(), tr.data_ptr(), R,
                          alpha, sptr)
        rc = L.rhg_update_edges(phi.data_ptr(), r.data_ptr(), n, R, 0, 0.0, 0, ids.data_ptr(), cnt, src.data_ptr(),
                                m_old, ws_upd.data_ptr(), ws_upd.numel(), dst.data_ptr(), cap, sptr,
                                ctypes.byref(res))
        rhg._check(rc, "rhg_update_edges", res)
        return int(res.m)

    for i in range(args.warmup):
        m = update(steps[i], bufs[cur], bufs[1 - cur], m)
        cur = 1 - cur
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        m = update(steps[args.warmup + i], bufs[cur], bufs[1 - cur], m)
        cur = 1 - cur
    e1.record(stream)
    torch.cuda.synchronize()
    upd_ms = e0.elapsed_time(e1) / args.steps
    # the same final positions generated from scratch
    e0.record(stream)
    for _ in range(args.steps):
        m_full = full(bufs[1 - cur])
    e1.record(stream)
    torch.cuda.synchronize()
    full_ms = e0.elapsed_time(e1) / args.steps
    same = m_full == m
    del ws_full, ws_upd, bufs
    peak, peak_kind = measured_peaks()
    # per update, the bytes an update cannot avoid: the old pairs read once, the
    # new pairs written once, the points' FP64 coordinates read once (16 B)
    upd_alg = 8 * m + 8 * m + 16 * n
    return {"moved_fraction": args.moved, "moved_per_step": cnt, "edges": m, "update_ms": upd_ms,
            "regenerate_ms": full_ms, "update_edges_per_s": m / (upd_ms / 1000.0),
            "speedup_vs_regenerate": full_ms / upd_ms, "edge_count_equals_regeneration": same,
            "roofline": {"kernel": "update step (keep old pairs, re-query moved vertices)", "bound": "hbm",
                         "achieved": upd_alg / (upd_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": upd_alg / (upd_ms / 1e3) / 1e9 / peak, "algorithmic_bytes_per_launch": upd_alg,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "workload": f"dynamic: n={n}, k={k}, alpha={alpha}, seed {args.seed}; per step {args.moved:.0%} of the "
                        "vertices (uniform random, torch generator) move with tau_phi in (-1, 1), tau_r in (-10, 1) "
                        "(Philox); step = move + update of the previous edge list"}


def replica_seed(seed: int, rank: int) -> int:
    """Replicas (one per GPU, no exchange) generate independent graphs: rank r
    uses seed + r."""
    return seed + rank


def combine_ranks(elapsed_ms: float, edges: int, world: int, device: str):
    """Whole-job figures over the replicas: the slowest rank's time (MAX) and the
    edges of all ranks (SUM).  A no-op at world size 1."""
    if world <= 1:
        return elapsed_ms, edges
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    mm = torch.tensor([edges], dtype=torch.int64, device=device)
    dist.all_reduce(mm)
    return float(t.item()), int(mm.item())


def run_ours(args):
    import torch

    import paper_1606_09481_gb300 as rhg
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    rhg.build()
    seed = replica_seed(args.seed, rank)
    n, k, alpha = args.n, args.k, args.alpha
    params = rhg.make_params(n, k, alpha, seed, args.bands, args.band_ratio)
    wsp = rhg.allocate_pairs(params)
    stream = torch.cuda.current_stream()

    def step():
        return rhg.generate_pairs(n, k, alpha, seed, args.bands, args.band_ratio, workspace=wsp)

    pairs, res = step()
    if res.m > wsp.capacity:  # the n k / 2 estimate was short: size the output exactly
        del pairs
        wsp = rhg.allocate_pairs(params, int(res.m))
        pairs, res = step()
    for _ in range(max(args.warmup - 1, 0)):
        step()
    torch.cuda.synchronize()

    timer = rhg.StageTimer()
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[0].strip().isdigit():
        gpu_index = int(vis.split(",")[local].strip()) if local < len(vis.split(",")) else local
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = rhg.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index) as clocks, timer:
        ev0.record(stream)
        for _ in range(args.steps):
            timer.reset_marks()
            _, res = step()
            timer.accumulate()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = rhg.launch_count() - launches0
    elapsed_ms = ev0.elapsed_time(ev1)
    m = int(res.m)
    elapsed_ms, total_m = combine_ranks(elapsed_ms, m, world, "cuda")
    ms_per_step = elapsed_ms / args.steps
    value = total_m / (ms_per_step / 1000.0)

    # roofline of the dominant stage: the range query (batch, heavy-chunk and
    # recheck kernels), which writes the output
    stages = {s: timer.totals[s] / max(args.steps, 1) for s in rhg.STAGES}
    q_ms = stages["query"]
    alg_bytes = n * QUERY_BYTES_PER_POINT + m * QUERY_BYTES_PER_EDGE
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (q_ms / 1000.0) / 1e9 if q_ms > 0 else 0.0
    roofline = {"kernel": "range query (batch_kernel + heavy_kernel + recheck_kernel)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": kernel_traffic("query"), "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_ms": q_ms, "peak_source": f"{peak_kind} hbm_gbs"}

    line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "n": n, "k": k, "alpha": alpha, "seed": args.seed,
                       "num_bands": int(res.num_bands), "output": "uint32 pairs",
                       "l2": "working set ~9 GB > 129 MB L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "edges": m, "R": res.R, "candidates": int(res.candidates),
            "near_threshold": int(res.near_threshold), "rechecks": int(res.rechecks), "heavy_chunks": int(res.heavy_chunks),
            "mode": "fp32 filter + fp64 recheck" if res.mode else "fp64",
            "stages_ms": stages, "roofline": roofline,
            "gpu_launches": launches, "clocks": clocks.summary()}

    if not args.no_e2e:
        # end to end through the host-buffer entry point: pairs copied to pinned memory
        host = torch.empty(2 * wsp.capacity, dtype=torch.int32).pin_memory()
        rhg.generate_pairs_host(n, k, alpha, seed, host, wsp, args.bands, args.band_ratio)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r2 = rhg.generate_pairs_host(n, k, alpha, seed, host, wsp, args.bands, args.band_ratio)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e_s, _ = combine_ranks(e2e_s, 0, world, "cuda")
        line["e2e"] = {"value": total_m / e2e_s, "unit": "edges/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": int(r2.m) * 8 + 2 * rhg.plan_workspace_bytes(),
                       "ms_per_step": 1000 * e2e_s,
                       "note": "parameters in, pairs out to pinned host memory; two metadata reads per call"}
        del host

    if not args.no_configs:
        line["configs"] = bench_configs(args, rhg, torch, stream)

    if not args.no_batched:
        del pairs
        pairs = None
        line["batched"] = bench_batched(args, rhg, torch, stream)

    if not args.no_dynamic:
        pairs = None
        line["dynamic"] = bench_dynamic(args, rhg, torch, stream)

    if not args.no_served:
        pairs = None
        line["served"] = bench_served(args, rhg, torch)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        del pairs
        _, info = cpu_baseline(args)
        line["cpu_baseline"] = info
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
