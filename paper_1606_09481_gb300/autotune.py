"""Autotuner for batched generation: band count and work mapping per graph-size class.

Neither the band count B nor the range query's work mapping changes the edge set;
both only change how the work is split, so they are free performance parameters:
- B: how many bands a point's windows visit against how many fringe candidates
  each band leaves;
- batch_budget: candidates a warp batch of 32 points keeps before its longer
  ranges go to the chunk list that all warps share;
- core_heavy: the longest certain range a warp batch writes itself;
- fringe_limit: the longest tested range a lane tests itself.
For each size class (a range of n) the tuner times rhg_generate_batch on sample
graphs of that class and picks the parameters by coordinate descent: the band
offset d (B = default + d) first, then the budget, the core limit and the fringe
limit, each with the others at their best so far.
"""
from __future__ import annotations

from dataclasses import dataclass, field

DEFAULT_CLASSES = ((1_000, 10_000), (10_000, 100_000), (100_000, 10_000_000))
DEFAULT_OFFSETS = (-8, -6, -4, -2, 0, 2)
DEFAULT_BUDGETS = (16_384, 65_536, 262_144)
DEFAULT_CORE = (1_024, 4_096, 16_384)
DEFAULT_FRINGE = (16, 32)
LIBRARY_MAPPING = (65_536, 4_096, 32)  # the library's defaults (batch_budget, core_heavy, fringe_limit)


def default_bands(n: int) -> int:
    """The library's default band count (rhg_default_bands), so that the tuner's
    offsets are relative to what the library would use."""
    from . import default_bands as lib_default_bands
    return lib_default_bands(n)


@dataclass
class BandTable:
    """Tuned parameters per size class [lo, hi): band offset and work mapping."""
    classes: tuple = DEFAULT_CLASSES
    offsets: dict = field(default_factory=dict)   # class index -> band offset
    mapping: dict = field(default_factory=dict)   # class index -> (batch_budget, core_heavy, fringe_limit)
    timings: dict = field(default_factory=dict)   # (class index, parameter, value) -> seconds

    def _class(self, n: int):
        for c, (lo, hi) in enumerate(self.classes):
            if lo <= n < hi:
                return c
        return None

    def bands(self, n: int) -> int:
        c = self._class(n)
        d = self.offsets.get(c, 0) if c is not None else 0
        return min(64, max(1, default_bands(n) + d))

    def params(self, n: int):
        """(num_bands, batch_budget, core_heavy, fringe_limit) for a graph of n points."""
        c = self._class(n)
        m = self.mapping.get(c, LIBRARY_MAPPING) if c is not None else LIBRARY_MAPPING
        return (self.bands(n),) + tuple(m)

    def describe(self) -> dict:
        return {f"{lo}-{hi}": {"band_offset": self.offsets.get(c, 0),
                               "batch_budget": self.mapping.get(c, LIBRARY_MAPPING)[0],
                               "core_heavy": self.mapping.get(c, LIBRARY_MAPPING)[1],
                               "fringe_limit": self.mapping.get(c, LIBRARY_MAPPING)[2]}
                for c, (lo, hi) in enumerate(self.classes)}


def tune(specs, run, classes=DEFAULT_CLASSES, offsets=DEFAULT_OFFSETS, budgets=DEFAULT_BUDGETS,
         cores=DEFAULT_CORE, fringes=DEFAULT_FRINGE, per_class: int = 256, repeats: int = 3) -> BandTable:
    """specs: (n, k, alpha, seed) tuples like the workload; run(list of (n, k, alpha,
    seed, num_bands, batch_budget, core_heavy, fringe_limit)) -> seconds for one
    batched generation of those graphs.  Each class is timed on up to per_class of
    its graphs, the best of `repeats`; empty parameter lists keep the default."""
    table = BandTable(classes=tuple(classes))
    for c, (lo, hi) in enumerate(classes):
        members = [sp for sp in specs if lo <= sp[0] < hi][:per_class]
        if not members:
            continue
        best = {"offset": 0, "budget": LIBRARY_MAPPING[0], "core": LIBRARY_MAPPING[1], "fringe": LIBRARY_MAPPING[2]}

        def timed(name, value):
            cur = dict(best, **{name: value})
            graphs = [(n, k, a, s, min(64, max(1, default_bands(n) + cur["offset"])), cur["budget"], cur["core"],
                       cur["fringe"]) for (n, k, a, s) in members]
            t = min(run(graphs) for _ in range(repeats))
            table.timings[(c, name, value)] = t
            return t

        for name, values in (("offset", offsets), ("budget", budgets), ("core", cores), ("fringe", fringes)):
            if not values:
                continue
            scored = [(timed(name, v), v) for v in values]
            best[name] = min(scored)[1]
        table.offsets[c] = best["offset"]
        table.mapping[c] = (best["budget"], best["core"], best["fringe"])
    return table


def gpu_runner(stream=None):
    """A `run` for tune(): one rhg_generate_batch call on the device, timed with
    CUDA events (buffers allocated outside the timed region)."""
    import torch

    from . import allocate_batch, make_params, run_batch, Params, OK, RhgError

    def run(graphs):
        params = (Params * len(graphs))(*[make_params(n, k, a, s, b, batch_budget=bb, core_heavy=ch, fringe_limit=fl)
                                          for (n, k, a, s, b, bb, ch, fl) in graphs])
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
