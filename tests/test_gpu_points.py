"""R, band boundaries and sampled points on the device are bit-identical to the
oracle's (Sec. III-B getTargetRadius, Sec. III-A boundaries, Alg. 1 sampling)."""
import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

PLANS = [(10**4, 6, 1.0, 0, 0.9), (10**6, 16, 0.75, 0, 0.9), (10**7, 200, 1.0, 0, 0.9),
         (1000, 30, 0.55, 0, 0.9), (10**5, 10, 3.0, 7, 0.5), (10**5, 10, 1.2, 33, 1.0), (500, 3, 0.8, 1, 1.3),
         (2, 0.5, 1.0, 1, 0.9), (2**32 - 1, 10, 1.0, 64, 0.9)]


@pytest.mark.parametrize("n,k,alpha,B,p", PLANS)
def test_plan_bitwise(O, n, k, alpha, B, p):
    rhg = require_gpu()
    R, c = rhg.plan(n, k, alpha, num_bands=B, band_ratio=p)
    assert R == O.target_radius(n, k, alpha)
    Bref = B or O.default_bands(n)
    assert np.array_equal(np.array(c), O.boundaries(R, Bref, p))
    assert rhg.target_radius(n, k, alpha) == R


def test_plan_errors():
    rhg = require_gpu()
    with pytest.raises(rhg.RhgError) as e:
        rhg.plan(100, 1e6, 1.0)
    assert e.value.status == rhg.NO_SOLUTION
    with pytest.raises(rhg.RhgError) as e:
        rhg.plan(100, 6, 0.5)
    assert e.value.status == rhg.INVALID_ARG


@pytest.mark.parametrize("n,k,alpha,seed", [(100_000, 6, 1.0, 1), (100_000, 16, 0.75, 2), (50_001, 10, 0.55, 9),
                                            (50_000, 10, 3.0, 2**63 + 5), (3, 1, 1.0, 0)])
def test_points_bitwise(O, n, k, alpha, seed):
    rhg = require_gpu()
    phi, r, R = rhg.sample_points(n, k, alpha, seed)
    phi_ref, r_ref = O.sample_points(n, alpha, R, seed)
    assert R == O.target_radius(n, k, alpha)
    assert np.array_equal(phi.cpu().numpy().view(np.uint64), phi_ref.view(np.uint64))
    assert np.array_equal(r.cpu().numpy().view(np.uint64), r_ref.view(np.uint64))


def test_points_config3_sampled(O):
    """n = 10^7, k = 200, alpha = 1, seed 3: random ids and both ends match."""
    rhg = require_gpu()
    n, k, alpha, seed = 10**7, 200, 1.0, 3
    phi, r, R = rhg.sample_points(n, k, alpha, seed)
    phi, r = phi.cpu().numpy(), r.cpu().numpy()
    rng = np.random.default_rng(0)
    ids = np.concatenate([[0, 1, n - 2, n - 1], rng.integers(0, n, 2000)])
    for i in ids:
        p1, r1 = O.sample_points(1, alpha, R, seed, first=int(i))
        assert phi[i] == p1[0] and r[i] == r1[0], i
