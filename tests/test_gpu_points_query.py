"""The range query on caller-given points (rhg_edges_from_points) against the
oracle's all-pairs edge set, on adversarial point sets: ties in angle, points on
band boundaries, at the origin, on both sides of the 0 / 2pi seam, duplicates."""
import math

import numpy as np
import pytest

from gpu_util import assert_valid_pairs, require_gpu, sorted_pairs

pytestmark = pytest.mark.gpu


def _run(O, rhg, phi, r, R, **kw):
    import torch
    pairs, res = rhg.edges_from_points(torch.from_numpy(phi).cuda(), torch.from_numpy(r).cuda(), R, **kw)
    got = sorted_pairs(pairs)
    assert_valid_pairs(got, len(phi))
    ref = O.brute_edges(phi, r, R)
    assert np.array_equal(got, ref), (len(got), len(ref))
    return res


def _cases(O):
    rng = np.random.default_rng(5)
    R = 12.0
    n = 3000
    cases = {}
    cases["same_angle"] = (np.full(n, 1.2345), rng.uniform(0, R, n), R)
    cases["origin"] = (rng.uniform(0, 2 * math.pi, n), np.where(rng.random(n) < 0.1, 0.0, rng.uniform(0, R, n)), R)
    c = O.boundaries(R, 12, 0.9)
    cases["on_boundaries"] = (rng.uniform(0, 2 * math.pi, n), c[rng.integers(0, 13, n)], R)
    seam = np.concatenate([rng.uniform(0, 1e-6, n // 2), np.nextafter(2 * math.pi, 0) - rng.uniform(0, 1e-6, n // 2)])
    cases["seam"] = (seam, rng.uniform(R - 1, R, n), R)
    base_phi, base_r = rng.uniform(0, 2 * math.pi, n // 3), rng.uniform(R / 2, R, n // 3)
    cases["duplicates"] = (np.repeat(base_phi, 3), np.repeat(base_r, 3), R)
    cases["outer_rim"] = (rng.uniform(0, 2 * math.pi, n), np.full(n, R), R)
    cases["two_points"] = (np.array([0.0, math.pi]), np.array([R / 2, R / 2]), R)
    cases["one_point"] = (np.array([3.0]), np.array([1.0]), R)
    phi, r = O.sample_points(n, 1.0, 30.0, 9)
    cases["large_R"] = (phi, r, 30.0)
    return cases


@pytest.mark.parametrize("name", ["same_angle", "origin", "on_boundaries", "seam", "duplicates", "outer_rim",
                                  "two_points", "one_point", "large_R"])
def test_adversarial_points(O, name):
    rhg = require_gpu()
    phi, r, R = _cases(O)[name]
    _run(O, rhg, phi.astype(np.float64), r.astype(np.float64), R)
    _run(O, rhg, phi.astype(np.float64), r.astype(np.float64), R, num_bands=3, band_ratio=0.5)


@pytest.mark.parametrize("bad", ["phi_2pi", "phi_neg", "r_gt_R", "nan"])
def test_points_outside_domain_rejected(O, bad):
    rhg = require_gpu()
    import torch
    phi = np.linspace(0, 6, 100)
    r = np.linspace(0, 10, 100)
    if bad == "phi_2pi":
        phi[3] = 2 * math.pi
    elif bad == "phi_neg":
        phi[3] = -1e-300
    elif bad == "r_gt_R":
        r[5] = 10.5
    else:
        r[7] = float("nan")
    with pytest.raises(rhg.RhgError) as e:
        rhg.edges_from_points(torch.from_numpy(phi).cuda(), torch.from_numpy(r).cuda(), 10.0)
    assert e.value.status == rhg.INVALID_ARG
