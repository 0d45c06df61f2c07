"""GB300 generator of threshold random hyperbolic graphs (arXiv:1606.09481).

Thin ctypes binding over the C ABI declared in ``include/rhg.h``: argument
marshalling only.  Every step of the method runs in the CUDA kernels of
``librhg.so``; PyTorch provides device memory and the current stream.  There is
no fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

from .build import LIB, build

__all__ = [
    "RhgError", "Params", "Result", "BatchGraph", "load", "status_str", "target_radius", "plan", "workspace_bytes",
    "sample_points", "generate_pairs", "generate_pairs_host", "generate_pairs_static", "generate_csr",
    "edges_from_points", "batch_params", "batch_workspace_bytes", "allocate_batch", "run_batch", "generate_batch",
    "BatchPlan", "batch_prepare", "batch_launch", "batch_read_results", "capture_batch",
    "draw_movement", "move_points", "update_edges", "dm_eval", "default_bands", "make_params", "estimate_capacity",
    "batch_stage_times", "grid_barrier_test",
    "StageTimer", "launch_count", "FLAG_FP64_ONLY", "FLAG_VERIFY", "MAX_BANDS", "STATIC_MAX_POINTS", "build",
]

OK, INVALID_ARG, NO_SOLUTION, OOM, CUDA_ERROR, TIMEOUT, OVERFLOW = range(7)
FLAG_FP64_ONLY = 0x1
FLAG_VERIFY = 0x2
MAX_BANDS = 64
DM_FUNCS = {"exp": 0, "log": 1, "cos": 2, "cosh": 3, "sinh": 4, "asinh": 5}

_c_u64, _c_u32, _c_dbl, _c_size, _p = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                       ctypes.c_size_t, ctypes.c_void_p)


class Params(ctypes.Structure):
    _fields_ = [("n", _c_u64), ("k", _c_dbl), ("alpha", _c_dbl), ("seed", _c_u64),
                ("num_bands", _c_u32), ("flags", _c_u32), ("band_ratio", _c_dbl),
                ("R_override", _c_dbl), ("batch_budget", _c_u32), ("core_heavy", _c_u32),
                ("fringe_limit", _c_u32), ("reserved", _c_u32)]


class Result(ctypes.Structure):
    _fields_ = [("m", _c_u64), ("R", _c_dbl), ("num_bands", _c_u32), ("cuda_error", ctypes.c_int32),
                ("candidates", _c_u64), ("near_threshold", _c_u64), ("rechecks", _c_u64),
                ("verify_failures", _c_u64), ("mode", _c_u32), ("heavy_chunks", _c_u32),
                ("rounding_band", _c_u64)]

    def asdict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchGraph(ctypes.Structure):
    """rhg_batch_graph: one graph's outcome in rhg_generate_batch."""
    _fields_ = [("m", _c_u64), ("R", _c_dbl), ("num_bands", _c_u32), ("status", ctypes.c_int32),
                ("mode", _c_u32), ("reserved", _c_u32)]


class BatchPlan(ctypes.Structure):
    """rhg_batch_plan: the counts rhg_batch_prepare records for rhg_batch_launch."""
    _fields_ = [("count", _c_u32), ("verify", _c_u32), ("num_tiles", _c_u64), ("points", _c_u64),
                ("index_entries", _c_u64), ("pair_capacity", _c_u64), ("workspace_bytes", _c_u64),
                ("chunk_extra", _c_u64)]


class RhgError(RuntimeError):
    def __init__(self, status: int, where: str, result: Result | None = None):
        self.status = status
        self.result = result
        super().__init__(f"{where}: {status_str(status)} ({status})")


_lib = None


_load_lock = threading.Lock()


def load() -> ctypes.CDLL:
    """Load librhg.so (built by build()); raises if it is missing.  Thread-safe."""
    if _lib is not None:
        return _lib
    with _load_lock:
        return _load_locked()


def _load_locked() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"CUDA library {LIB} is not built; run paper_1606_09481_gb300.build()")
    L = ctypes.CDLL(LIB)
    L.rhg_status_str.restype = ctypes.c_char_p
    L.rhg_status_str.argtypes = [ctypes.c_int]
    L.rhg_version.restype = ctypes.c_int
    L.rhg_plan_workspace_bytes.restype = _c_size
    L.rhg_plan_workspace_bytes.argtypes = []
    L.rhg_target_radius.argtypes = [_c_u64, _c_dbl, _c_dbl, _p, _c_size, _p, ctypes.POINTER(_c_dbl)]
    L.rhg_plan.argtypes = [ctypes.POINTER(Params), _p, _c_size, _p, ctypes.POINTER(_c_dbl), _p,
                           ctypes.POINTER(_c_u32)]
    L.rhg_workspace_bytes.argtypes = [ctypes.POINTER(Params), _c_u64, ctypes.POINTER(_c_size)]
    L.rhg_workspace_bytes_points.argtypes = [_c_u64, _c_u32, ctypes.POINTER(_c_size)]
    L.rhg_sample_points.argtypes = [ctypes.POINTER(Params), _p, _c_size, _p, _p, _p, ctypes.POINTER(_c_dbl)]
    L.rhg_generate_pairs.argtypes = [ctypes.POINTER(Params), _p, _c_size, _p, _c_u64, _p,
                                     ctypes.POINTER(Result)]
    L.rhg_generate_pairs_static.argtypes = [ctypes.POINTER(Params), _p, _c_u64, _p, ctypes.POINTER(Result)]
    L.rhg_batch_workspace_bytes.argtypes = [ctypes.POINTER(Params), _c_u32, ctypes.POINTER(_c_size)]
    L.rhg_generate_batch.argtypes = [ctypes.POINTER(Params), _c_u32, _p, _c_size, _p, ctypes.POINTER(_c_u64), _p,
                                     ctypes.POINTER(BatchGraph), ctypes.POINTER(Result)]
    L.rhg_batch_prepare.argtypes = [ctypes.POINTER(Params), _c_u32, ctypes.POINTER(_c_u64), _p, _c_size, _p,
                                    ctypes.POINTER(BatchPlan)]
    L.rhg_batch_launch.argtypes = [ctypes.POINTER(BatchPlan), _p, _p, _p]
    L.rhg_batch_read_results.argtypes = [ctypes.POINTER(BatchPlan), _p, _p, ctypes.POINTER(BatchGraph),
                                         ctypes.POINTER(Result)]
    L.rhg_batch_stage_times.argtypes = [ctypes.POINTER(BatchPlan), _p, _p, ctypes.POINTER(_c_dbl), _c_u32]
    L.rhg_grid_barrier_test.argtypes = [_c_u32, _c_u64, _p, _c_size, _p]
    L.rhg_draw_movement.argtypes = [_c_u64, _c_u64, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _p, _p, _p]
    L.rhg_move_points.argtypes = [_p, _c_u64, _c_u64, _p, _p, _p, _p, _c_dbl, _c_dbl, _p]
    L.rhg_workspace_bytes_update.argtypes = [_c_u64, _c_u64, _c_u32, ctypes.POINTER(_c_size)]
    L.rhg_update_edges.argtypes = [_p, _p, _c_u64, _c_dbl, _c_u32, _c_dbl, _c_u32, _p, _c_u64, _p, _c_u64, _p, _c_size,
                                   _p, _c_u64, _p, ctypes.POINTER(Result)]
    L.rhg_generate_pairs_host.argtypes = [ctypes.POINTER(Params), _p, _c_size, _p, _c_u64, _p, _c_u64, _p,
                                          ctypes.POINTER(Result)]
    L.rhg_generate_csr.argtypes = [ctypes.POINTER(Params), _p, _c_size, _p, _p, _c_u64, _p,
                                   ctypes.POINTER(Result)]
    L.rhg_edges_from_points.argtypes = [_p, _p, _c_u64, _c_dbl, _c_u32, _c_dbl, _c_u32, _p, _c_size, _p,
                                        _c_u64, _p, ctypes.POINTER(Result)]
    L.rhg_dm_eval.argtypes = [ctypes.c_int, _p, _p, _c_u64, _p]
    L.rhg_sort_keys_workspace_bytes.argtypes = [_c_u64, ctypes.c_uint32, _p, ctypes.POINTER(ctypes.c_size_t)]
    L.rhg_sort_keys.argtypes = [_p, _c_u64, ctypes.c_uint32, _p, _p, ctypes.c_size_t, _p, _p, _p]
    L.rhg_set_stage_events.argtypes = [_p, _c_u32]
    L.rhg_launch_count.restype = _c_u64
    L.rhg_launch_count.argtypes = []
    L.rhg_default_bands.restype = _c_u32
    L.rhg_default_bands.argtypes = [_c_u64]
    _lib = L
    return L


STAGES = ("plan", "sample", "sort", "gather", "query", "csr")


class StageTimer:
    """Per-stage CUDA events recorded by the library on its stream (profiling)."""

    def __init__(self):
        torch = _torch()
        self.events = [torch.cuda.Event(enable_timing=True) for _ in range(2 * len(STAGES))]
        for e in self.events:  # torch creates the CUDA event on first record
            e.record()
        torch.cuda.synchronize()
        self._arr = (ctypes.c_void_p * len(self.events))(*[e.cuda_event for e in self.events])
        self.totals = {s: 0.0 for s in STAGES}
        self.recorded = {s: 0 for s in STAGES}

    def __enter__(self):
        load().rhg_set_stage_events(self._arr, len(self.events))
        return self

    def __exit__(self, *exc):
        load().rhg_set_stage_events(None, 0)

    def reset_marks(self):
        """Re-record every event so that a stage that does not run reads ~0."""
        for e in self.events:
            e.record()

    def accumulate(self):
        """After a synchronised call: add each stage's elapsed ms to the totals."""
        for i, s in enumerate(STAGES):
            ms = self.events[2 * i].elapsed_time(self.events[2 * i + 1])
            if ms > 0:
                self.totals[s] += ms
                self.recorded[s] += 1


def launch_count() -> int:
    return int(load().rhg_launch_count())


def status_str(status: int) -> str:
    return load().rhg_status_str(status).decode()


def default_bands(n: int) -> int:
    """The library's default band count for n points (rhg_default_bands)."""
    return int(load().rhg_default_bands(int(n)))


def make_params(n, k=0.0, alpha=1.0, seed=0, num_bands=0, band_ratio=0.0, R_override=0.0, flags=0,
                batch_budget=0, core_heavy=0, fringe_limit=0):
    """rhg_params; the last three set the range query's work mapping (0: default)."""
    return Params(int(n), float(k), float(alpha), int(seed), int(num_bands), int(flags), float(band_ratio),
                  float(R_override), int(batch_budget), int(core_heavy), int(fringe_limit), 0)


# ---------------------------------------------------------------- torch plumbing
def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _empty_bytes(nbytes: int, device=None):
    torch = _torch()
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


def _check(rc: int, where: str, result: Result | None = None):
    if rc != OK:
        raise RhgError(rc, where, result)


# ------------------------------------------------------------------- entry points
def plan_workspace_bytes() -> int:
    return int(load().rhg_plan_workspace_bytes())


def target_radius(n: int, k: float, alpha: float, stream=None) -> float:
    ws = _empty_bytes(plan_workspace_bytes())
    R = _c_dbl(0.0)
    _check(load().rhg_target_radius(n, k, alpha, ws.data_ptr(), ws.numel(), _stream(stream), ctypes.byref(R)),
           "rhg_target_radius")
    return R.value


def plan(n, k, alpha, seed=0, num_bands=0, band_ratio=0.0, R_override=0.0, stream=None):
    p = make_params(n, k, alpha, seed, num_bands, band_ratio, R_override)
    ws = _empty_bytes(plan_workspace_bytes())
    R = _c_dbl(0.0)
    B = _c_u32(0)
    c = (ctypes.c_double * (MAX_BANDS + 1))()
    _check(load().rhg_plan(ctypes.byref(p), ws.data_ptr(), ws.numel(), _stream(stream), ctypes.byref(R), c,
                           ctypes.byref(B)), "rhg_plan")
    return R.value, [c[j] for j in range(B.value + 1)]


def workspace_bytes(params: Params, capacity_entries: int = 0) -> int:
    out = _c_size(0)
    _check(load().rhg_workspace_bytes(ctypes.byref(params), capacity_entries, ctypes.byref(out)),
           "rhg_workspace_bytes")
    return int(out.value)


def sample_points(n, k, alpha, seed, R_override=0.0, stream=None):
    """Points by id as two float64 CUDA tensors (phi, r), and R."""
    torch = _torch()
    p = make_params(n, k, alpha, seed, R_override=R_override)
    ws = _empty_bytes(plan_workspace_bytes())
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    R = _c_dbl(0.0)
    _check(load().rhg_sample_points(ctypes.byref(p), ws.data_ptr(), ws.numel(), phi.data_ptr(), r.data_ptr(),
                                    _stream(stream), ctypes.byref(R)), "rhg_sample_points")
    return phi, r, R.value


def estimate_capacity(n: int, k: float) -> int:
    """Pairs buffer size from the expected edge count n k / 2, with slack."""
    return int(math.ceil(n * k / 2 * 1.25)) + 4096


@dataclass
class Workspace:
    """Reusable device buffers for repeated calls with the same parameters."""
    ws: object
    out: object
    capacity: int


def allocate_pairs(params: Params, capacity: int | None = None) -> Workspace:
    torch = _torch()
    cap = capacity if capacity is not None else estimate_capacity(params.n, params.k or 8.0)
    ws = _empty_bytes(workspace_bytes(params, 0))
    out = torch.empty(max(2 * cap, 2), dtype=torch.int32, device="cuda")
    return Workspace(ws, out, cap)


def generate_pairs(n, k, alpha, seed, num_bands=0, band_ratio=0.0, flags=0, R_override=0.0,
                   workspace: Workspace | None = None, stream=None, overflow_retry: bool = True):
    """Edges as an (m, 2) int32 CUDA tensor of uint32 ids (u < v), and the Result.

    Allocates the output from n k / 2 with slack.  On RHG_ERR_OVERFLOW (more
    edges than room) it keeps the workspace, replaces the output by one of the
    exact size reported and calls again; with overflow_retry=False it raises
    RhgError(OVERFLOW) instead, whose result.m is the exact edge count."""
    p = make_params(n, k, alpha, seed, num_bands, band_ratio, R_override, flags)
    wsp = workspace or allocate_pairs(p)
    res = Result()
    L = load()
    rc = L.rhg_generate_pairs(ctypes.byref(p), wsp.ws.data_ptr(), wsp.ws.numel(), wsp.out.data_ptr(),
                              wsp.capacity, _stream(stream), ctypes.byref(res))
    if rc == OVERFLOW and overflow_retry:
        m = int(res.m)
        out = wsp.out
        if workspace is None:
            wsp.out = None  # our own buffer: released before the larger one is made
        del out
        wsp = Workspace(wsp.ws, _torch().empty(max(2 * m, 2), dtype=_torch().int32, device="cuda"), m)
        rc = L.rhg_generate_pairs(ctypes.byref(p), wsp.ws.data_ptr(), wsp.ws.numel(), wsp.out.data_ptr(),
                                  wsp.capacity, _stream(stream), ctypes.byref(res))
    _check(rc, "rhg_generate_pairs", res)
    return wsp.out[: 2 * res.m].view(-1, 2), res


def batch_params(specs, flags=0, num_bands=0, band_ratio=0.0):
    """A ctypes array of Params from (n, k, alpha, seed) tuples (or Params)."""
    ps = [sp if isinstance(sp, Params) else make_params(sp[0], sp[1], sp[2], sp[3], num_bands, band_ratio, 0.0, flags)
          for sp in specs]
    return (Params * len(ps))(*ps)


def batch_workspace_bytes(params_array) -> int:
    b = _c_size(0)
    _check(load().rhg_batch_workspace_bytes(params_array, len(params_array), ctypes.byref(b)),
           "rhg_batch_workspace_bytes")
    return int(b.value)


@dataclass
class BatchBuffers:
    """Device buffers of a batch: workspace, pairs, and the host pair offsets."""
    params: object
    ws: object
    out: object
    offsets: object  # ctypes uint64 array, count + 1


def allocate_batch(params_array, capacities=None) -> BatchBuffers:
    torch = _torch()
    caps = capacities or [estimate_capacity(p.n, p.k or 8.0) for p in params_array]
    offs = (_c_u64 * (len(caps) + 1))()
    for g, c in enumerate(caps):
        offs[g + 1] = offs[g] + int(c)
    ws = _empty_bytes(batch_workspace_bytes(params_array))
    out = torch.empty(max(2 * int(offs[len(caps)]), 2), dtype=torch.int32, device="cuda")
    return BatchBuffers(params_array, ws, out, offs)


def run_batch(buf: BatchBuffers, stream=None):
    """One rhg_generate_batch call on prepared buffers: (status, [BatchGraph], totals)."""
    G = len(buf.params)
    res = (BatchGraph * G)()
    tot = Result()
    rc = load().rhg_generate_batch(buf.params, G, buf.ws.data_ptr(), buf.ws.numel(), buf.out.data_ptr(),
                                   buf.offsets, _stream(stream), res, ctypes.byref(tot))
    return rc, res, tot


def batch_prepare(buf: BatchBuffers, stream=None) -> BatchPlan:
    """rhg_batch_prepare: check the graphs of `buf` and copy their tables into its
    workspace; the plan is what rhg_batch_launch needs."""
    plan = BatchPlan()
    _check(load().rhg_batch_prepare(buf.params, len(buf.params), buf.offsets, buf.ws.data_ptr(), buf.ws.numel(),
                                    _stream(stream), ctypes.byref(plan)), "rhg_batch_prepare")
    return plan


def batch_launch(plan: BatchPlan, buf: BatchBuffers, stream=None) -> None:
    """rhg_batch_launch: enqueue the prepared batch (kernel launches only; may be
    captured into a CUDA graph)."""
    _check(load().rhg_batch_launch(ctypes.byref(plan), buf.ws.data_ptr(), buf.out.data_ptr(), _stream(stream)),
           "rhg_batch_launch")


def batch_read_results(plan: BatchPlan, buf: BatchBuffers, stream=None):
    """rhg_batch_read_results after a launch or replay: (status, [BatchGraph], totals)."""
    res = (BatchGraph * plan.count)()
    tot = Result()
    rc = load().rhg_batch_read_results(ctypes.byref(plan), buf.ws.data_ptr(), _stream(stream), res,
                                       ctypes.byref(tot))
    return rc, res, tot


BATCH_STAGES = ("plan", "sample", "bucket_scan", "bucket_scatter", "bucket_sort_gather", "bucket_index",
                "query_filter", "heavy_filter", "recheck", "phase_reset", "query_fp64", "heavy_fp64", "results")


def batch_stage_times(plan: BatchPlan, buf: BatchBuffers, stream=None) -> dict:
    """rhg_batch_stage_times: device time (ms) of each stage of the last launch."""
    arr = (_c_dbl * len(BATCH_STAGES))()
    _check(load().rhg_batch_stage_times(ctypes.byref(plan), buf.ws.data_ptr(), _stream(stream), arr,
                                        len(BATCH_STAGES)), "rhg_batch_stage_times")
    return dict(zip(BATCH_STAGES, (float(v) for v in arr)))


def grid_barrier_test(missing: int, timeout_ns: int, stream=None) -> int:
    """rhg_grid_barrier_test: the persistent launch's grid barrier with `missing`
    CTAs that never arrive; returns the status (OK or TIMEOUT)."""
    ws = _empty_bytes(plan_workspace_bytes() + 256)
    return int(load().rhg_grid_barrier_test(int(missing), int(timeout_ns), ws.data_ptr(), ws.numel(),
                                            _stream(stream)))


def capture_batch(plan: BatchPlan, buf: BatchBuffers):
    """A torch.cuda.CUDAGraph holding one rhg_batch_launch of the prepared batch;
    graph.replay() regenerates the batch into buf.out."""
    torch = _torch()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch_launch(plan, buf)
    return graph


def generate_batch(specs, flags=0, num_bands=0, band_ratio=0.0, stream=None):
    """Graphs from (n, k, alpha, seed) tuples in one rhg_generate_batch call.

    Returns ([(m_g, 2) int32 CUDA views], [BatchGraph], totals Result).  Graphs
    that overflowed their estimated room are generated again with exact room."""
    params = batch_params(specs, flags, num_bands, band_ratio)
    buf = allocate_batch(params)
    rc, res, tot = run_batch(buf, stream)
    if rc == OVERFLOW:
        caps = [max(int(res[g].m), int(buf.offsets[g + 1] - buf.offsets[g])) for g in range(len(params))]
        buf = allocate_batch(params, caps)
        rc, res, tot = run_batch(buf, stream)
    if rc != OK:
        raise RhgError(rc, "rhg_generate_batch", tot)
    views = [buf.out[2 * buf.offsets[g]: 2 * (buf.offsets[g] + res[g].m)].view(-1, 2) for g in range(len(params))]
    return views, list(res), tot


STATIC_MAX_POINTS = 131072  # RHG_STATIC_MAX_POINTS


def generate_pairs_static(n, k, alpha, seed, out, num_bands=0, band_ratio=0.0, flags=0, R_override=0.0,
                          stream=None):
    """rhg_generate_pairs_static: the edges into `out` (a CUDA int32 tensor of at
    least 2 words per edge) with the library's fixed device scratch instead of a
    workspace; n <= STATIC_MAX_POINTS.  Returns the (m, 2) view of `out` and the
    Result.  Calls on one device must not overlap in time."""
    p = make_params(n, k, alpha, seed, num_bands, band_ratio, R_override, flags)
    res = Result()
    rc = load().rhg_generate_pairs_static(ctypes.byref(p), out.data_ptr(), out.numel() // 2, _stream(stream),
                                          ctypes.byref(res))
    _check(rc, "rhg_generate_pairs_static", res)
    return out[: 2 * res.m].view(-1, 2), res


def generate_pairs_host(n, k, alpha, seed, host_out, workspace: Workspace, num_bands=0, band_ratio=0.0,
                        flags=0, stream=None):
    """Generate into device buffers and copy the pairs to host_out (a pinned
    int32 CPU tensor with room for 2 * capacity words); returns the Result."""
    p = make_params(n, k, alpha, seed, num_bands, band_ratio, 0.0, flags)
    res = Result()
    rc = load().rhg_generate_pairs_host(ctypes.byref(p), workspace.ws.data_ptr(), workspace.ws.numel(),
                                        workspace.out.data_ptr(), workspace.capacity, host_out.data_ptr(),
                                        host_out.numel() // 2, _stream(stream), ctypes.byref(res))
    _check(rc, "rhg_generate_pairs_host", res)
    return res


def generate_csr(n, k, alpha, seed, num_bands=0, band_ratio=0.0, flags=0, capacity_entries=None,
                 stream=None):
    """Symmetric CSR: (row_ptr int64[n+1], col int32[2m]) CUDA tensors, and the Result."""
    torch = _torch()
    p = make_params(n, k, alpha, seed, num_bands, band_ratio, 0.0, flags)
    cap = capacity_entries if capacity_entries is not None else 2 * estimate_capacity(n, k)
    L = load()
    for _ in range(2):
        ws = _empty_bytes(workspace_bytes(p, cap))
        row_ptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
        res = Result()
        rc = L.rhg_generate_csr(ctypes.byref(p), ws.data_ptr(), ws.numel(), row_ptr.data_ptr(), col.data_ptr(),
                                cap, _stream(stream), ctypes.byref(res))
        if rc != OVERFLOW:
            break
        cap = 2 * int(res.m)
    _check(rc, "rhg_generate_csr", res)
    return row_ptr, col[: 2 * res.m], res


def edges_from_points(phi, r, R, num_bands=0, band_ratio=0.0, flags=0, capacity=None, stream=None):
    """Edges among caller points (float64 CUDA tensors by id), as generate_pairs."""
    torch = _torch()
    n = int(phi.numel())
    phi = phi.contiguous()
    r = r.contiguous()
    nb = _c_size(0)
    L = load()
    _check(L.rhg_workspace_bytes_points(n, num_bands, ctypes.byref(nb)), "rhg_workspace_bytes_points")
    ws = _empty_bytes(nb.value)
    cap = capacity if capacity is not None else max(4 * n, 4096)
    for _ in range(2):
        out = torch.empty(max(2 * cap, 2), dtype=torch.int32, device="cuda")
        res = Result()
        rc = L.rhg_edges_from_points(phi.data_ptr(), r.data_ptr(), n, float(R), num_bands, float(band_ratio),
                                     flags, ws.data_ptr(), ws.numel(), out.data_ptr(), cap, _stream(stream),
                                     ctypes.byref(res))
        if rc != OVERFLOW:
            break
        cap = int(res.m)
    _check(rc, "rhg_edges_from_points", res)
    return out[: 2 * res.m].view(-1, 2), res


# ------------------------------------------------------------------- dynamic model
def draw_movement(n, seed, phi_range=(-1.0, 1.0), r_range=(-10.0, 1.0), stream=None):
    """Step values (tau_phi, tau_r) of vertices 0..n-1 as float64 CUDA tensors;
    the default ranges are the paper's experiment."""
    torch = _torch()
    tphi = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    tr = torch.empty_like(tphi)
    _check(load().rhg_draw_movement(n, seed, float(phi_range[0]), float(phi_range[1]), float(r_range[0]),
                                    float(r_range[1]), tphi.data_ptr(), tr.data_ptr(), _stream(stream)),
           "rhg_draw_movement")
    return tphi[:n], tr[:n]


def move_points(ids, phi, r, tau_phi, tau_r, R, alpha, stream=None):
    """One movement step of the vertices `ids` (int32 CUDA tensor of distinct ids),
    in place on the float64 CUDA tensors phi, r and tau_r."""
    n = int(phi.numel())
    _check(load().rhg_move_points(ids.data_ptr(), int(ids.numel()), n, phi.data_ptr(), r.data_ptr(),
                                  tau_phi.data_ptr(), tau_r.data_ptr(), float(R), float(alpha), _stream(stream)),
           "rhg_move_points")


def update_edges(phi, r, R, moved_ids, old_pairs, num_bands=0, band_ratio=0.0, flags=0, capacity=None,
                 stream=None):
    """The edge list after a movement step (rhg_update_edges): old_pairs is the
    (m, 2) int32 CUDA tensor of the graph before the step, phi / r the positions
    after it, moved_ids the moved vertices.  Returns ((m', 2) pairs, Result)."""
    torch = _torch()
    n = int(phi.numel())
    cnt = int(moved_ids.numel())
    nb = _c_size(0)
    L = load()
    _check(L.rhg_workspace_bytes_update(n, cnt, num_bands, ctypes.byref(nb)), "rhg_workspace_bytes_update")
    ws = _empty_bytes(nb.value)
    old = old_pairs.contiguous()
    m_old = int(old.shape[0]) if old.numel() else 0
    cap = capacity if capacity is not None else m_old + m_old // 4 + 4096
    for _ in range(2):
        out = torch.empty(max(2 * cap, 2), dtype=torch.int32, device="cuda")
        res = Result()
        rc = L.rhg_update_edges(phi.data_ptr(), r.data_ptr(), n, float(R), num_bands, float(band_ratio), flags,
                                moved_ids.data_ptr() if cnt else None, cnt, old.data_ptr() if m_old else None, m_old,
                                ws.data_ptr(), ws.numel(), out.data_ptr(), cap, _stream(stream), ctypes.byref(res))
        if rc != OVERFLOW:
            break
        cap = int(res.m)
    _check(rc, "rhg_update_edges", res)
    return out[: 2 * res.m].view(-1, 2), res


def sort_keys(keys, num_bands: int, bucket_bits):
    """rhg_sort_keys: keys (int64 CUDA tensor of (band << 32) | angle key) sorted
    by (key, index) through the generator's bucket sort; bucket_bits[j] = the
    top angle-key bits that cut band j into buckets.  Returns (sorted keys,
    indices) as int64 / int32 CUDA tensors."""
    torch = _torch()
    keys = keys.contiguous()
    n = keys.numel()
    bits = (ctypes.c_uint32 * len(bucket_bits))(*[int(b) for b in bucket_bits])
    nbytes = ctypes.c_size_t(0)
    _check(load().rhg_sort_keys_workspace_bytes(n, num_bands, bits, ctypes.byref(nbytes)),
           "rhg_sort_keys_workspace_bytes")
    ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=keys.device)
    base = ws.data_ptr()
    ptr = (base + 255) // 256 * 256
    out_k = torch.empty(n, dtype=torch.int64, device=keys.device)
    out_i = torch.empty(n, dtype=torch.int32, device=keys.device)
    _check(load().rhg_sort_keys(keys.data_ptr(), n, num_bands, bits, ptr, nbytes.value, out_k.data_ptr(),
                                out_i.data_ptr(), _stream()), "rhg_sort_keys")
    return out_k, out_i


def dm_eval(fn: str, x):
    """The library's deterministic FP64 function `fn` on a float64 CUDA tensor."""
    torch = _torch()
    x = x.contiguous()
    out = torch.empty_like(x)
    _check(load().rhg_dm_eval(DM_FUNCS[fn], x.data_ptr(), out.data_ptr(), x.numel(), _stream()), "rhg_dm_eval")
    return out
