"""Autotuner for batched generation: the band count per graph-size class.

The band count B changes how the range query splits its work (how many bands a
point's windows visit against how many fringe candidates each band leaves) but
never the edge set, so it is a free performance parameter.  For each size class
(a range of n) the tuner times rhg_generate_batch on sample graphs of that class
with B = ceil(log2 n) + d for a few offsets d, and keeps the fastest offset.
The warp-to-point mapping of the query (warp batches of 32 consecutive sorted
points, claimed dynamically) is fixed and not tuned.
"""
from __future__ import annotations

from dataclasses import dataclass, field

DEFAULT_CLASSES = ((1_000, 10_000), (10_000, 100_000), (100_000, 10_000_000))
DEFAULT_OFFSETS = (-8, -6, -4, -2, 0, 2)


def default_bands(n: int) -> int:
    """The library's default band count (rhg_default_bands), so that the tuner's
    offsets are relative to what the library would use."""
    from . import default_bands as lib_default_bands
    return lib_default_bands(n)


@dataclass
class BandTable:
    """Band-count offset per size class [lo, hi)."""
    classes: tuple = DEFAULT_CLASSES
    offsets: dict = field(default_factory=dict)  # class index -> offset
    timings: dict = field(default_factory=dict)  # (class index, offset) -> seconds

    def bands(self, n: int) -> int:
        for c, (lo, hi) in enumerate(self.classes):
            if lo <= n < hi:
                return min(64, max(1, default_bands(n) + self.offsets.get(c, 0)))
        return default_bands(n)


def tune(specs, run, classes=DEFAULT_CLASSES, offsets=DEFAULT_OFFSETS, per_class: int = 256,
         repeats: int = 3) -> BandTable:
    """specs: (n, k, alpha, seed) tuples like the workload; run(list of (n, k, alpha,
    seed, num_bands)) -> seconds for one batched generation of those graphs.
    Each class is timed on up to per_class of its graphs, the best of `repeats`."""
    table = BandTable(classes=tuple(classes))
    for c, (lo, hi) in enumerate(classes):
        members = [sp for sp in specs if lo <= sp[0] < hi][:per_class]
        if not members:
            continue
        best = None
        for d in offsets:
            graphs = [(n, k, a, s, min(64, max(1, default_bands(n) + d))) for (n, k, a, s) in members]
            t = min(run(graphs) for _ in range(repeats))
            table.timings[(c, d)] = t
            if best is None or t < best[1]:
                best = (d, t)
        table.offsets[c] = best[0]
    return table


def gpu_runner(stream=None):
    """A `run` for tune(): one rhg_generate_batch call on the device, timed with
    CUDA events (buffers allocated outside the timed region)."""
    import torch

    from . import allocate_batch, make_params, run_batch, Params, OK, RhgError

    def run(graphs):
        params = (Params * len(graphs))(*[make_params(n, k, a, s, b) for (n, k, a, s, b) in graphs])
        buf = allocate_batch(params)
        rc, res, tot = run_batch(buf, stream)  # warm-up and size check
        if rc != OK:
            raise RhgError(rc, "rhg_generate_batch", tot)
        s = stream if stream is not None else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        run_batch(buf, stream)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0

    return run
