"""Edge sets from the device equal the oracle's, exactly (Alg. 1 range query vs the
all-pairs definition and the oracle's own Alg. 1)."""
import numpy as np
import pytest

from gpu_util import assert_valid_pairs, require_gpu, sorted_pairs

pytestmark = pytest.mark.gpu


def test_config1_equals_brute_force(O):
    """n = 10^4, k = 6, alpha = 1, seed 1: uint32 pairs == O(n^2) all pairs."""
    rhg = require_gpu()
    n, k, alpha, seed = 10_000, 6, 1.0, 1
    pairs, res = rhg.generate_pairs(n, k, alpha, seed)
    got = sorted_pairs(pairs)
    assert_valid_pairs(got, n)
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    ref = O.brute_edges(phi, r, R)
    assert res.R == R and res.m == len(ref)
    assert np.array_equal(got, ref)
    _, st = O.band_edges(phi, r, R, O.default_bands(n), with_stats=True)
    assert res.near_threshold == st["near_threshold"]


SMALL = [(2, 0.5, 1.0, 1), (3, 1, 1.0, 2), (17, 4, 0.8, 3), (100, 6, 1.0, 4), (257, 10, 0.55, 5),
         (1000, 30, 0.6, 6), (2047, 6, 1.0, 7), (2049, 6, 1.0, 8), (4097, 12, 0.75, 9), (5000, 3, 3.0, 10),
         (3000, 60, 1.5, 11), (6000, 1, 1.0, 12), (8191, 8, 0.9, 2**40 + 3),
         # dense graphs with small R (core and fringe chunks of the heavy kernel), a
         # steep radial density, and the largest seed
         (500, 200, 1.0, 13), (2000, 600, 0.6, 16), (8000, 1000, 0.7, 15), (3000, 8, 10.0, 14),
         (4000, 10, 1.0, 2**64 - 1)]


@pytest.mark.parametrize("n,k,alpha,seed", SMALL)
def test_small_graphs_equal_brute_force(O, n, k, alpha, seed):
    rhg = require_gpu()
    pairs, res = rhg.generate_pairs(n, k, alpha, seed)
    got = sorted_pairs(pairs)
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    assert np.array_equal(got, O.brute_edges(phi, r, R))


@pytest.mark.parametrize("B,p,flags", [(1, 0.9, 0), (2, 0.9, 0), (7, 0.5, 0), (30, 0.9, 0), (64, 0.97, 0),
                                       (14, 1.0, 0), (14, 0.9, 1)])
def test_band_structure_does_not_change_edges(O, B, p, flags):
    rhg = require_gpu()
    n, k, alpha, seed = 10_000, 6, 1.0, 1
    base, _ = rhg.generate_pairs(n, k, alpha, seed)
    other, _ = rhg.generate_pairs(n, k, alpha, seed, num_bands=B, band_ratio=p, flags=flags)
    assert np.array_equal(sorted_pairs(base), sorted_pairs(other))


def test_config2_csr_equals_oracle(O):
    """n = 10^6, k = 16, alpha = 0.75, seed 2: CSR (row_ptr, sorted columns) ==
    the oracle's Alg. 1 edge set in CSR form."""
    rhg = require_gpu()
    n, k, alpha, seed = 10**6, 16, 0.75, 2
    row_ptr, col, res = rhg.generate_csr(n, k, alpha, seed)
    g = O.generate(n, k, alpha, seed, with_stats=True)
    ref_rp, ref_col = O.pairs_to_csr(g["pairs"], n)
    assert res.m == len(g["pairs"])
    assert np.array_equal(row_ptr.cpu().numpy().astype(np.uint64), ref_rp)
    assert np.array_equal(col.cpu().numpy().astype(np.uint32), ref_col)
    assert res.near_threshold == g["stats"]["near_threshold"]


def test_pairs_to_host_matches_device(O):
    rhg = require_gpu()
    import torch
    n, k, alpha, seed = 20_000, 10, 0.8, 4
    dev, res = rhg.generate_pairs(n, k, alpha, seed)
    p = rhg.make_params(n, k, alpha, seed)
    wsp = rhg.allocate_pairs(p)
    host = torch.empty(2 * wsp.capacity, dtype=torch.int32).pin_memory()
    res2 = rhg.generate_pairs_host(n, k, alpha, seed, host, wsp)
    assert res2.m == res.m
    assert np.array_equal(sorted_pairs(host[: 2 * res2.m].view(-1, 2)), sorted_pairs(dev))


@pytest.mark.parametrize("flags", [0, 1])
def test_pairs_to_host_in_phases(O, flags):
    """A graph large enough for several query phases whose copies overlap the
    later phases (pinned host memory): the same pairs as the device output, in
    filter and FP64-only mode; a pageable host buffer takes the plain path and
    gives them too; a host buffer one pair short reports OVERFLOW with the exact m."""
    rhg = require_gpu()
    import ctypes
    import torch
    n, k, alpha, seed = 10**6, 64, 0.75, 8
    fl = rhg.FLAG_FP64_ONLY if flags else 0
    dev, res = rhg.generate_pairs(n, k, alpha, seed, flags=fl)
    assert res.m > 3 * 2**23  # three phases or more
    p = rhg.make_params(n, k, alpha, seed, flags=fl)
    wsp = rhg.allocate_pairs(p, capacity=res.m + 1000)
    ref = sorted_pairs(dev)
    for pin in (True, False):
        host = torch.empty(2 * wsp.capacity, dtype=torch.int32)
        if pin:
            host = host.pin_memory()
        res2 = rhg.generate_pairs_host(n, k, alpha, seed, host, wsp, flags=fl)
        assert res2.m == res.m
        assert np.array_equal(sorted_pairs(host[: 2 * res2.m].view(-1, 2)), ref)
    host = torch.empty(2 * (res.m - 1), dtype=torch.int32).pin_memory()
    r3 = rhg.Result()
    rc = rhg.load().rhg_generate_pairs_host(ctypes.byref(p), wsp.ws.data_ptr(), wsp.ws.numel(), wsp.out.data_ptr(),
                                            wsp.capacity, host.data_ptr(), res.m - 1, rhg._stream(),
                                            ctypes.byref(r3))
    assert rc == rhg.OVERFLOW and r3.m == res.m


def test_overflow_reports_exact_count(O):
    rhg = require_gpu()
    import ctypes
    n, k, alpha, seed = 10_000, 6, 1.0, 1
    p = rhg.make_params(n, k, alpha, seed)
    wsp = rhg.allocate_pairs(p, capacity=1000)
    res = rhg.Result()
    rc = rhg.load().rhg_generate_pairs(ctypes.byref(p), wsp.ws.data_ptr(), wsp.ws.numel(), wsp.out.data_ptr(),
                                       wsp.capacity, rhg._stream(), ctypes.byref(res))
    assert rc == rhg.OVERFLOW
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    assert res.m == len(O.brute_edges(phi, r, R))
    # the retrying wrapper then succeeds
    pairs, res2 = rhg.generate_pairs(n, k, alpha, seed, workspace=wsp)
    assert res2.m == res.m and len(pairs) == res.m


def test_no_solution_and_invalid():
    rhg = require_gpu()
    with pytest.raises(rhg.RhgError) as e:
        rhg.generate_pairs(100, 1e6, 1.0, 1)
    assert e.value.status == rhg.NO_SOLUTION
    with pytest.raises(rhg.RhgError) as e:
        rhg.generate_pairs(1, 6, 1.0, 1)
    assert e.value.status == rhg.INVALID_ARG


@pytest.mark.parametrize("n,k,alpha,seed,mode", [(5000, 3, 3.0, 21, 1), (5000, 2, 3.0, 22, 0), (4000, 3, 4.0, 23, 0),
                                                  (3000, 2, 5.0, 24, 0)])
def test_steep_density_near_the_filter_range(O, n, k, alpha, seed, mode):
    """alpha R just below 44 runs the FP32 filter; above it (where the FP32-assisted
    sampler radius would overflow) the graph runs in FP64 mode; both equal all pairs."""
    rhg = require_gpu()
    pairs, res = rhg.generate_pairs(n, k, alpha, seed)
    R = O.target_radius(n, k, alpha)
    assert res.mode == mode, (alpha * R, res.mode)
    phi, r = O.sample_points(n, alpha, R, seed)
    assert np.array_equal(sorted_pairs(pairs), O.brute_edges(phi, r, R))


def test_dense_graphs_in_fp64_mode(O):
    """Dense graphs in FP64 mode (no core, every window tested, one chunk per long
    piece): the chunk list, sized for FP64 mode from n k, holds them.  The
    FP64-only flag gives the default mode's graph, and a dense graph with
    alpha R > 44 equals the oracle's Algorithm 1."""
    rhg = require_gpu()
    n, k, alpha, seed = 20000, 1500, 0.7, 41
    a, ra = rhg.generate_pairs(n, k, alpha, seed)
    b, rb = rhg.generate_pairs(n, k, alpha, seed, flags=rhg.FLAG_FP64_ONLY)
    assert ra.mode == 1 and rb.mode == 0
    assert rb.heavy_chunks > n // 4 + 65536  # more than the list holds without the FP64 sizing
    assert np.array_equal(sorted_pairs(a), sorted_pairs(b))
    n, k, alpha, seed = 100_000, 200, 4.0, 31
    pairs, res = rhg.generate_pairs(n, k, alpha, seed)
    R = O.target_radius(n, k, alpha)
    assert res.mode == 0 and alpha * R > 44
    phi, r = O.sample_points(n, alpha, R, seed)
    assert np.array_equal(sorted_pairs(pairs), O.band_edges(phi, r, R, O.default_bands(n)))


@pytest.mark.parametrize("n,k,alpha,seed", [(20_000, 30, 0.8, 5), (3000, 200, 1.0, 6)])
def test_output_buffer_at_odd_slot(O, n, k, alpha, seed):
    """The C ABI asks only for an 8-byte aligned pair buffer: a buffer that starts
    8 bytes past a 16-byte boundary gives the same edges (the core writer's
    16-byte stores align themselves to the buffer's address)."""
    import ctypes

    import torch
    rhg = require_gpu()
    p = rhg.make_params(n, k, alpha, seed)
    wsp = rhg.allocate_pairs(p)
    out = torch.empty(2 * wsp.capacity + 4, dtype=torch.int32, device="cuda")
    assert out.data_ptr() % 16 == 0
    res = rhg.Result()
    rc = rhg.load().rhg_generate_pairs(ctypes.byref(p), wsp.ws.data_ptr(), wsp.ws.numel(), out.data_ptr() + 8,
                                       wsp.capacity, None, ctypes.byref(res))
    assert rc == rhg.OK
    torch.cuda.synchronize()
    got = sorted_pairs(out[2: 2 + 2 * res.m].view(-1, 2))
    R = O.target_radius(n, k, alpha)
    phi, r = O.sample_points(n, alpha, R, seed)
    assert np.array_equal(got, O.brute_edges(phi, r, R))
    assert res.m > 0


@pytest.mark.parametrize("budget,core,fringe", [(1024, 64, 1), (1024, 65536, 32), (1 << 24, 64, 16)])
def test_work_mapping_does_not_change_edges(O, budget, core, fringe):
    """The range query's work mapping (batch budget, core chunk limit, fringe
    limit) moves work between the batch and the heavy-chunk kernels, never changes
    the edges."""
    import ctypes

    import torch
    rhg = require_gpu()
    n, k, alpha, seed = 30_000, 120, 0.9, 41
    base, res0 = rhg.generate_pairs(n, k, alpha, seed)
    want = sorted_pairs(base)
    p = rhg.make_params(n, k, alpha, seed, batch_budget=budget, core_heavy=core, fringe_limit=fringe)
    wsp = rhg.allocate_pairs(p, int(res0.m) + 16)
    res = rhg.Result()
    rc = rhg.load().rhg_generate_pairs(ctypes.byref(p), wsp.ws.data_ptr(), wsp.ws.numel(), wsp.out.data_ptr(),
                                       wsp.capacity, None, ctypes.byref(res))
    assert rc == rhg.OK
    torch.cuda.synchronize()
    assert np.array_equal(sorted_pairs(wsp.out[: 2 * res.m].view(-1, 2)), want)
    if fringe == 1:
        assert res.heavy_chunks > res0.heavy_chunks
