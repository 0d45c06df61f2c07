"""The band-count autotuner's selection logic, with a fake timer (no GPU)."""
from paper_1606_09481_gb300.autotune import BandTable, default_bands, tune


def test_picks_the_fastest_offset_per_class():
    specs = [(2_000, 8, 1.0, 1), (5_000, 8, 1.0, 2), (20_000, 8, 1.0, 3), (90_000, 8, 1.0, 4)]
    calls = []

    def run(graphs):
        calls.append(graphs)
        n = graphs[0][0]
        b = graphs[0][4]
        best = default_bands(n) - 2 if n < 10_000 else default_bands(n) + 2
        return 1.0 + abs(b - best)  # fastest at the planted band count

    t = tune(specs, run, offsets=(-4, -2, 0, 2), repeats=2)
    assert t.offsets == {0: -2, 1: 2}
    assert t.bands(3_000) == default_bands(3_000) - 2 and t.bands(50_000) == default_bands(50_000) + 2
    assert t.bands(5_000_000) == default_bands(5_000_000)  # class without samples: default
    assert len(calls) == 2 * 4 * 2
    # every call of a class holds only that class's graphs
    assert all(all(1_000 <= g[0] < 10_000 for g in c) or all(10_000 <= g[0] < 100_000 for g in c) for c in calls)


def test_band_counts_stay_in_range():
    t = BandTable(offsets={0: -40, 1: 70})
    assert t.bands(1_500) == 1 and t.bands(20_000) == 64
    assert default_bands(2) == 1 and default_bands(1024) == 10 and default_bands(1025) == 11
