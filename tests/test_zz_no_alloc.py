"""rhg_generate_pairs_static (fixed device scratch, no allocation) gives the same
edges as rhg_generate_pairs, call after call.  Collected last on purpose: the
scratch array is shared process-wide, so this also runs after every other test
has used the library."""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_valid_pairs, require_gpu, sorted_pairs

CASES = [(10_000, 6, 1.0, 1), (131_072, 20, 0.75, 5)]


def test_rejects_n_beyond_scratch():
    """n above the stated maximum fails on the host, before any device work."""
    import paper_1606_09481_gb300 as rhg
    L = rhg.load()
    p = rhg.make_params(rhg.STATIC_MAX_POINTS + 1, 10, 1.0, 1)
    res = rhg.Result()
    rc = L.rhg_generate_pairs_static(ctypes.byref(p), None, 0, None, ctypes.byref(res))
    assert rc == rhg.INVALID_ARG
    assert L.rhg_generate_pairs_static(None, None, 0, None, ctypes.byref(res)) == rhg.INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("n,k,alpha,seed", CASES)
def test_static_equals_workspace_entry_point(n, k, alpha, seed):
    rhg = require_gpu()
    import torch
    ref_pairs, ref = rhg.generate_pairs(n, k, alpha, seed)
    want = sorted_pairs(ref_pairs)
    out = torch.empty(2 * rhg.estimate_capacity(n, k), dtype=torch.int32, device="cuda")
    for _ in range(2):  # two calls in a row on the same scratch
        out.fill_(-1)
        pairs, res = rhg.generate_pairs_static(n, k, alpha, seed, out)
        torch.cuda.synchronize()
        got = sorted_pairs(pairs)
        assert_valid_pairs(got, n)
        assert res.R == ref.R and res.m == ref.m and res.num_bands == ref.num_bands
        assert np.array_equal(got, want)


@pytest.mark.gpu
def test_static_overflow_reports_exact_m():
    rhg = require_gpu()
    import torch
    n, k, alpha, seed = 10_000, 6, 1.0, 1
    _, ref = rhg.generate_pairs(n, k, alpha, seed)
    out = torch.empty(2 * 100, dtype=torch.int32, device="cuda")
    with pytest.raises(rhg.RhgError) as e:
        rhg.generate_pairs_static(n, k, alpha, seed, out)
    assert e.value.status == rhg.OVERFLOW and e.value.result.m == ref.m
