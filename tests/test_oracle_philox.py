"""Pins for the oracle's Philox4x64-10 (Salmon et al., SC'11) against numpy's
independent implementation, and for the angular coordinate of Alg. 1 (phi ~ U[0,2pi))."""
import numpy as np
import pytest

M64 = (1 << 64) - 1


def _numpy_block(counter, key):
    # numpy's Philox increments its 256-bit counter before producing a block, so a
    # generator started at counter c - 1 yields the block of counter c.
    c = list(counter)
    i = 0
    while True:  # subtract 1 with borrow
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = M64
        i += 1
        if i == 4:
            break
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("key", [(0, 0), (1, 0), (2, 0), (3, 0), (0xDEADBEEF, 0),
                                 (M64, M64), (12345678901234567, 987654321)])
def test_philox_matches_numpy(O, key):
    rng = np.random.default_rng(7)
    counters = [(0, 0, 0, 0), (1, 0, 0, 0), (9999, 0, 0, 0), (M64, 0, 0, 0), (5, 7, 0, 0),
                (0, 0, 0, 1)]
    counters += [tuple(int(x) for x in rng.integers(0, 2**63, 4)) for _ in range(20)]
    for c in counters:
        assert np.array_equal(O.philox4x64(c, key), _numpy_block(c, key)), (c, key)


def test_philox_batch_is_per_counter(O):
    b = O.philox4x64_batch(64, (100, 0, 0, 0), (42, 0))
    for i in range(64):
        assert np.array_equal(b[i], _numpy_block((100 + i, 0, 0, 0), (42, 0)))


def test_phi_is_u53_times_scaled_two_pi(O):
    """phi_i = fl((x0 >> 11) * 2pi * 2^-53) with x0 from counter (i,0,0,0), key (seed,0)."""
    seed, n = 1, 4096
    phi, _ = O.sample_points(n, 1.0, 16.0, seed)
    x = np.array([_numpy_block((i, 0, 0, 0), (seed, 0)) for i in range(n)], dtype=np.uint64)
    u53 = (x[:, 0] >> np.uint64(11)).astype(np.float64)
    S = np.float64(2 * np.pi) * np.float64(2.0 ** -53)
    assert S == np.ldexp(np.float64(2 * np.pi), -53)
    assert np.array_equal(phi, u53 * S)
    assert phi.min() >= 0.0 and phi.max() < 2 * np.pi


def test_first_offset(O):
    a, ra = O.sample_points(100, 0.8, 20.0, 9)
    b, rb = O.sample_points(60, 0.8, 20.0, 9, first=40)
    assert np.array_equal(a[40:], b) and np.array_equal(ra[40:], rb)
