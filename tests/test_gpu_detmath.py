"""The device's deterministic FP64 functions give the same bits as the oracle's
independent implementation of the same definition."""
import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _inputs(fn, seed=0):
    rng = np.random.default_rng(seed)
    if fn == "exp":
        return np.concatenate([rng.uniform(-60, 60, 40000), rng.uniform(-1, 1, 10000), np.linspace(-30, 30, 1001)])
    if fn == "log":
        return np.concatenate([np.exp(rng.uniform(-40, 80, 40000)), 1 + rng.uniform(0, 1e-3, 5000),
                               1 + rng.uniform(0, 1e-12, 1000), [1.0, 2.0, 0.5, 1e300]])
    if fn == "cos":
        return np.concatenate([rng.uniform(0, 2 * np.pi, 50000), rng.uniform(0, 1e-6, 2000),
                               np.linspace(0, 2 * np.pi, 4097)])
    if fn == "asinh":
        return np.concatenate([10.0 ** rng.uniform(-8, 35, 40000), rng.uniform(0, 10, 10000), [0.0, 1.0, 1e-300]])
    return np.concatenate([rng.uniform(0, 60, 40000), rng.uniform(0, 0.6, 10000), [0.0, 0.5, 0.4999999999]])


@pytest.mark.parametrize("fn", ["exp", "log", "cos", "cosh", "sinh", "asinh"])
def test_dm_bitwise(O, fn):
    rhg = require_gpu()
    import torch
    x = _inputs(fn)
    got = rhg.dm_eval(fn, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.dm(fn, x)
    bad = np.flatnonzero(got.view(np.uint64) != ref.view(np.uint64))
    assert len(bad) == 0, (fn, x[bad[:5]], got[bad[:5]], ref[bad[:5]])
