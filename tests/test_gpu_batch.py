"""rhg_generate_batch: every graph of a batch equals the graph the single-graph
path gives for the same parameters (itself equal to the oracle), and small ones
equal the oracle's all-pairs definition directly; per-graph statuses."""
import numpy as np
import pytest

from gpu_util import assert_valid_pairs, require_gpu, sorted_pairs

pytestmark = pytest.mark.gpu

MIXED = [(2, 0.5, 1.0, 1), (3, 1, 1.0, 2), (17, 4, 0.8, 3), (100, 6, 1.0, 4), (1000, 30, 0.6, 6),
         (2047, 6, 1.0, 7), (2048, 8, 0.75, 8), (2049, 6, 1.0, 9), (4097, 12, 0.75, 10), (5000, 3, 3.0, 11),
         (3000, 60, 1.5, 12), (20000, 16, 0.75, 13), (60000, 24, 1.2, 14), (1500, 32, 0.55, 15),
         (9000, 10, 1.0, 2**40 + 3)]


def _single(rhg, p):
    pairs, res = rhg.generate_pairs(p.n, p.k, p.alpha, p.seed, p.num_bands, p.band_ratio, p.flags, p.R_override)
    return sorted_pairs(pairs), res


def _check_against_single(rhg, params, views, results):
    for g, p in enumerate(params):
        got = sorted_pairs(views[g])
        assert_valid_pairs(got, p.n)
        want, res = _single(rhg, p)
        assert results[g].status == 0
        assert results[g].R == res.R and results[g].num_bands == res.num_bands and results[g].mode == res.mode
        assert results[g].m == res.m == len(want), g
        assert np.array_equal(got, want), g


def test_mixed_batch_equals_single_graphs_and_oracle(O):
    rhg = require_gpu()
    params = rhg.batch_params(MIXED)
    views, results, tot = rhg.generate_batch(params)
    _check_against_single(rhg, params, views, results)
    assert tot.m == sum(r.m for r in results)
    for g, (n, k, alpha, seed) in enumerate(MIXED):
        if n <= 5000:
            R = O.target_radius(n, k, alpha)
            phi, r = O.sample_points(n, alpha, R, seed)
            assert np.array_equal(sorted_pairs(views[g]), O.brute_edges(phi, r, R)), g


def test_batch_modes_and_flags():
    """FP64-only graphs, a graph whose R (> 32) rules the filter out, custom bands,
    and verification mode, all in one batch."""
    rhg = require_gpu()
    ps = [rhg.make_params(3000, 10, 1.0, 21), rhg.make_params(3000, 10, 1.0, 21, flags=rhg.FLAG_FP64_ONLY),
          rhg.make_params(2500, 0.0, 0.8, 22, R_override=33.0), rhg.make_params(8000, 20, 0.9, 23, num_bands=5),
          rhg.make_params(8000, 20, 0.9, 23, num_bands=1), rhg.make_params(7000, 16, 1.1, 24, band_ratio=1.0),
          rhg.make_params(12000, 12, 0.7, 25, flags=rhg.FLAG_VERIFY)]
    params = rhg.batch_params(ps)
    views, results, tot = rhg.generate_batch(params)
    _check_against_single(rhg, params, views, results)
    assert [r.mode for r in results] == [1, 0, 0, 1, 1, 1, 1]
    assert np.array_equal(sorted_pairs(views[0]), sorted_pairs(views[1]))
    assert np.array_equal(sorted_pairs(views[3]), sorted_pairs(views[4]))
    assert tot.verify_failures == 0


def test_per_graph_status_no_solution_and_overflow():
    rhg = require_gpu()
    ps = rhg.batch_params([(3000, 8, 1.0, 31), (100, 1e6, 1.0, 32), (4000, 12, 0.8, 33)])
    # graph 2 gets room for 10 pairs only
    caps = [rhg.estimate_capacity(3000, 8), 16, 10]
    buf = rhg.allocate_batch(ps, caps)
    rc, res, tot = rhg.run_batch(buf)
    assert rc == rhg.NO_SOLUTION  # the first failing graph
    assert [r.status for r in res] == [rhg.OK, rhg.NO_SOLUTION, rhg.OVERFLOW]
    _, single = rhg.generate_pairs(4000, 12, 0.8, 33)
    assert res[2].m == single.m  # exact count on overflow
    want0, _ = _single(rhg, ps[0])
    got0 = sorted_pairs(buf.out[2 * buf.offsets[0]: 2 * (buf.offsets[0] + res[0].m)].view(-1, 2))
    assert np.array_equal(got0, want0)
    assert tot.m == res[0].m


def test_p4_shaped_batch_sample():
    """256 graphs drawn like the batched workload (n log-uniform in [1e3, 1e5], k in
    6..32, alpha in [0.55, 1.5]); every 16th graph against the single-graph path,
    invariants on all."""
    rhg = require_gpu()
    rng = np.random.default_rng(4096)
    specs = [(int(10 ** rng.uniform(3, 5)), int(rng.integers(6, 33)), float(rng.uniform(0.55, 1.5)), 1000 + j)
             for j in range(256)]
    params = rhg.batch_params(specs)
    views, results, tot = rhg.generate_batch(params)
    for g, (n, k, alpha, seed) in enumerate(specs):
        got = sorted_pairs(views[g])
        assert_valid_pairs(got, n)
        if g % 16 == 0:
            want, res = _single(rhg, params[g])
            assert np.array_equal(got, want), g
    assert tot.m == sum(r.m for r in results)


def test_autotuned_parameters_give_the_same_graphs():
    """The autotuner only changes band counts and the query's work mapping: every
    graph stays the same, also with extreme mappings (tiny budget, fringe limit 1)."""
    rhg = require_gpu()
    from paper_1606_09481_gb300.autotune import gpu_runner, tune
    rng = np.random.default_rng(77)
    specs = [(int(10 ** rng.uniform(3, 5)), int(rng.integers(6, 33)), float(rng.uniform(0.55, 1.5)), 3000 + j)
             for j in range(48)]
    table = tune(specs, gpu_runner(), per_class=16, repeats=1, offsets=(-2, 0), budgets=(16_384, 65_536),
                 cores=(1_024, 4_096), fringes=(16, 32))
    assert set(table.offsets) <= {0, 1}

    def tuned_one(n, k, a, s):
        b, bb, ch, fl = table.params(n)
        return rhg.make_params(n, k, a, s, b, batch_budget=bb, core_heavy=ch, fringe_limit=fl)

    v1, r1, _ = rhg.generate_batch(rhg.batch_params(specs))
    v2, r2, _ = rhg.generate_batch(rhg.batch_params([tuned_one(*sp) for sp in specs]))
    extreme = rhg.batch_params([rhg.make_params(n, k, a, s, batch_budget=1024, core_heavy=64, fringe_limit=1)
                                for (n, k, a, s) in specs])
    v3, r3, _ = rhg.generate_batch(extreme)
    for g in range(len(specs)):
        assert r2[g].num_bands == table.bands(specs[g][0])
        assert np.array_equal(sorted_pairs(v1[g]), sorted_pairs(v2[g])), g
        assert np.array_equal(sorted_pairs(v1[g]), sorted_pairs(v3[g])), g


def test_captured_batch_replays_the_same_graphs():
    """rhg_batch_prepare once, rhg_batch_launch captured in a CUDA graph: the
    direct launch and every replay give exactly the graphs of rhg_generate_batch."""
    rhg = require_gpu()
    import torch
    want, wres, wtot = rhg.generate_batch(MIXED)
    params = rhg.batch_params(MIXED)
    buf = rhg.allocate_batch(params, [max(int(r.m), 1) + 7 for r in wres])
    plan = rhg.batch_prepare(buf)
    assert plan.count == len(MIXED) and plan.points == sum(sp[0] for sp in MIXED)
    assert plan.workspace_bytes == rhg.batch_workspace_bytes(params)

    def check():
        rc, res, tot = rhg.batch_read_results(plan, buf)
        assert rc == rhg.OK and tot.m == wtot.m
        for g in range(len(MIXED)):
            assert res[g].m == wres[g].m and res[g].R == wres[g].R and res[g].status == rhg.OK
            got = buf.out[2 * buf.offsets[g]: 2 * (buf.offsets[g] + res[g].m)].view(-1, 2)
            assert np.array_equal(sorted_pairs(got), sorted_pairs(want[g])), g

    rhg.batch_launch(plan, buf)
    check()
    graph = rhg.capture_batch(plan, buf)
    for _ in range(2):
        buf.out.fill_(-1)
        graph.replay()
        check()


def test_persistent_barrier_gives_up_and_the_device_stays_usable():
    """The persistent batch launch's grid barrier: it completes when every CTA
    arrives; when one never does (the test asks for one CTA more than the launch
    has), every wait gives up after its limit and the call reports
    RHG_ERR_TIMEOUT, and the device runs the next batch normally."""
    import time
    rhg = require_gpu()
    assert rhg.grid_barrier_test(0, 10**9) == rhg.OK
    t0 = time.perf_counter()
    assert rhg.grid_barrier_test(1, 20 * 10**6) == rhg.TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    params = rhg.batch_params(MIXED[:9])
    views, results, _ = rhg.generate_batch(params)
    _check_against_single(rhg, params, views, results)


def test_batch_stage_times():
    """The persistent launch records the device time of each of its stages."""
    rhg = require_gpu()
    import torch
    params = rhg.batch_params(MIXED)
    buf = rhg.allocate_batch(params)
    plan = rhg.batch_prepare(buf)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rhg.batch_launch(plan, buf)
    e1.record()
    torch.cuda.synchronize()
    st = rhg.batch_stage_times(plan, buf)
    assert list(st) == list(rhg.BATCH_STAGES) and len(st) == 13
    assert all(v >= 0.0 for v in st.values())
    total = sum(st.values())
    assert 0.0 < total <= e0.elapsed_time(e1) * 1.05 + 0.05
