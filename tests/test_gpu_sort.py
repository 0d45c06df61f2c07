"""The generator's bucket sort (rhg_sort_keys): (band, angle key) order with ties by
index, against numpy's lexsort, on uniform keys (the shared-memory path) and on
skewed keys that force the global-memory path (a bucket above 2048 keys, a
sub-bucket above 32 keys), plus its argument checks."""
import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _expected(keys):
    order = np.lexsort((np.arange(keys.size), keys))  # by key, then index
    return keys[order], order.astype(np.int32)


def _run(rhg, keys, num_bands, bits):
    import torch
    k = torch.from_numpy(keys.view(np.int64)).cuda()
    sk, si = rhg.sort_keys(k, num_bands, bits)
    torch.cuda.synchronize()
    return sk.cpu().numpy().view(np.uint64), si.cpu().numpy()


def _keys(rng, n, num_bands, weights=None):
    band = rng.choice(num_bands, n, p=weights).astype(np.uint64)
    akey = rng.integers(0, 2**32, n, dtype=np.uint64)
    return (band << np.uint64(32)) | akey


@pytest.mark.parametrize("n,num_bands", [(1, 1), (5, 3), (4097, 4), (300_000, 18), (2_000_001, 22)])
def test_uniform_keys_sorted_like_lexsort(n, num_bands):
    rhg = require_gpu()
    rng = np.random.default_rng(n)
    w = 0.9 ** np.arange(num_bands)[::-1]
    keys = _keys(rng, n, num_bands, w / w.sum())
    # bucket bits as the plan sets them: about 512..1024 keys per bucket
    counts = np.bincount((keys >> np.uint64(32)).astype(np.int64), minlength=num_bands)
    bits = [int(max(0, np.floor(np.log2(max(c, 1) / 512)))) for c in counts]
    sk, si = _run(rhg, keys, num_bands, bits)
    ek, ei = _expected(keys)
    assert np.array_equal(sk, ek) and np.array_equal(si, ei)


def test_equal_angle_keys_keep_index_order():
    """Many equal keys in one bucket (a sub-bucket far above 32: global path) and
    equal keys spread over buckets: ties come out in index order."""
    rhg = require_gpu()
    rng = np.random.default_rng(3)
    keys = _keys(rng, 20_000, 2)
    keys[rng.choice(keys.size, 500, replace=False)] = (np.uint64(1) << np.uint64(32)) | np.uint64(12345)
    sk, si = _run(rhg, keys, 2, [3, 3])
    ek, ei = _expected(keys)
    assert np.array_equal(sk, ek) and np.array_equal(si, ei)


@pytest.mark.parametrize("n", [2049, 70_000])
def test_one_bucket_beyond_the_shared_memory_path(n):
    """Every key in one bucket of more than 2048: the bucket's LSD radix sort in
    global memory (several tiles, all 8 digit passes)."""
    rhg = require_gpu()
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2**32, n, dtype=np.uint64)  # band 0
    keys[: n // 3] = keys[n // 3: 2 * (n // 3)]  # duplicates: ties by index
    sk, si = _run(rhg, keys, 1, [0])
    ek, ei = _expected(keys)
    assert np.array_equal(sk, ek) and np.array_equal(si, ei)


def test_band_out_of_range_is_an_argument_error():
    rhg = require_gpu()
    keys = np.array([(5 << 32) | 7, 1], dtype=np.uint64)
    with pytest.raises(rhg.RhgError) as e:
        _run(rhg, keys, 2, [0, 0])
    assert e.value.status == rhg.INVALID_ARG


def test_argument_checks():
    rhg = require_gpu()
    import torch
    k = torch.zeros(4, dtype=torch.int64, device="cuda")
    for nb, bits in ((0, []), (65, [0] * 65), (1, [25])):
        with pytest.raises(rhg.RhgError):
            rhg.sort_keys(k, nb, bits)
