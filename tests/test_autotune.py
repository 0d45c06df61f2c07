"""The autotuner's selection logic (band offset and work mapping per size class),
with a fake timer (no GPU)."""
from paper_1606_09481_gb300.autotune import LIBRARY_MAPPING, BandTable, default_bands, tune


def test_picks_the_fastest_parameters_per_class():
    """A planted optimum per class in each of the four parameters (a separable
    cost): coordinate descent finds it."""
    specs = [(2_000, 8, 1.0, 1), (5_000, 8, 1.0, 2), (20_000, 8, 1.0, 3), (90_000, 8, 1.0, 4)]
    calls = []
    planted = {0: (-2, 16_384, 1_024, 16), 1: (2, 262_144, 16_384, 32)}

    def run(graphs):
        calls.append(graphs)
        n, _, _, _, b, bb, ch, fl = graphs[0]
        d, pb, pc, pf = planted[0 if n < 10_000 else 1]
        return 1.0 + abs(b - (default_bands(n) + d)) + (bb != pb) + (ch != pc) + (fl != pf)

    t = tune(specs, run, offsets=(-4, -2, 0, 2), repeats=2)
    assert t.offsets == {0: -2, 1: 2}
    assert t.mapping == {0: (16_384, 1_024, 16), 1: (262_144, 16_384, 32)}
    assert t.bands(3_000) == default_bands(3_000) - 2 and t.bands(50_000) == default_bands(50_000) + 2
    assert t.params(3_000) == (default_bands(3_000) - 2, 16_384, 1_024, 16)
    assert t.bands(5_000_000) == default_bands(5_000_000)  # class without samples: default
    assert t.params(5_000_000) == (default_bands(5_000_000),) + LIBRARY_MAPPING
    assert len(calls) == 2 * (4 + 3 + 3 + 2) * 2
    # every call of a class holds only that class's graphs
    assert all(all(1_000 <= g[0] < 10_000 for g in c) or all(10_000 <= g[0] < 100_000 for g in c) for c in calls)
    desc = t.describe()
    assert desc["1000-10000"] == {"band_offset": -2, "batch_budget": 16_384, "core_heavy": 1_024, "fringe_limit": 16}


def test_band_counts_stay_in_range():
    t = BandTable(offsets={0: -40, 1: 70})
    assert t.bands(1_500) == 1 and t.bands(20_000) == 64
    assert default_bands(2) == 1 and default_bands(1024) == 10 and default_bands(1025) == 11
