"""Dynamic model on the GPU: step values and movement bit-identical to the
oracle's; the updated edge list equals the graph of the moved points (the
library's own full query and the oracle's all pairs), over several steps."""
import numpy as np
import pytest

from gpu_util import assert_valid_pairs, require_gpu, sorted_pairs

pytestmark = pytest.mark.gpu


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def test_draw_and_move_bitwise(O):
    rhg = require_gpu()
    import torch
    n, alpha = 50_000, 0.8
    R = O.target_radius(n, 12, alpha)
    tphi, tr = rhg.draw_movement(n, 17)
    ophi, otr = O.draw_movement(n, 17)
    assert np.array_equal(_bits(tphi.cpu().numpy()), _bits(ophi)) and np.array_equal(_bits(tr.cpu().numpy()),
                                                                                    _bits(otr))
    phi, r, _ = rhg.sample_points(n, 12, alpha, 17)
    hphi, hr = phi.cpu().numpy(), r.cpu().numpy()
    ids = np.sort(np.random.default_rng(1).choice(n, n // 3, replace=False)).astype(np.int32)
    # large steps too, so that reflections at 0 and R happen
    big = torch.tensor(np.where(np.arange(n) % 7 == 0, 1e9, 1.0), dtype=torch.float64, device="cuda")
    tr = tr * big
    otr = otr * big.cpu().numpy()
    rhg.move_points(torch.from_numpy(ids).cuda(), phi, r, tphi, tr, R, alpha)
    p2, r2, tr2 = O.move(ids.astype(np.uint32), hphi, hr, ophi, otr, R, alpha)
    assert np.array_equal(_bits(phi.cpu().numpy()), _bits(p2))
    assert np.array_equal(_bits(r.cpu().numpy()), _bits(r2))
    assert np.array_equal(_bits(tr.cpu().numpy()), _bits(tr2))
    assert np.any(tr2 != otr)  # some vertices bounced


@pytest.mark.parametrize("n,k,alpha,frac,flags", [(20_000, 10, 1.0, 0.12, 0), (6_000, 30, 0.7, 0.5, 0),
                                                  (9_000, 8, 1.2, 0.12, 1), (3_000, 6, 1.0, 1.0, 0),
                                                  (3_000, 6, 1.0, 0.0, 0)])
def test_update_equals_regeneration(O, n, k, alpha, frac, flags):
    rhg = require_gpu()
    import torch
    R = O.target_radius(n, k, alpha)
    phi, r, _ = rhg.sample_points(n, k, alpha, 5)
    pairs, _ = rhg.edges_from_points(phi, r, R, flags=flags)
    tphi, tr = rhg.draw_movement(n, 5)
    rng = np.random.default_rng(2)
    for step in range(3):
        ids = np.sort(rng.choice(n, int(frac * n), replace=False)).astype(np.int32)
        tid = torch.from_numpy(ids).cuda()
        rhg.move_points(tid, phi, r, tphi, tr, R, alpha)
        upd, res = rhg.update_edges(phi, r, R, tid, pairs, flags=flags)
        want, _ = rhg.edges_from_points(phi, r, R, flags=flags)
        got = sorted_pairs(upd)
        assert_valid_pairs(got, n)
        assert np.array_equal(got, sorted_pairs(want)), step
        pairs = upd
    if n <= 6000:  # and the oracle's all pairs on the oracle's own moved points
        ophi, orr = O.sample_points(n, alpha, R, 5)
        otp, otr = O.draw_movement(n, 5)
        rng = np.random.default_rng(2)
        for step in range(3):
            ids = np.sort(rng.choice(n, int(frac * n), replace=False)).astype(np.uint32)
            ophi, orr, otr = O.move(ids, ophi, orr, otp, otr, R, alpha)
        assert np.array_equal(sorted_pairs(pairs), O.brute_edges(ophi, orr, R))


def test_update_rejects_repeated_ids():
    rhg = require_gpu()
    import torch
    n = 2000
    phi, r, _ = rhg.sample_points(n, 8, 1.0, 3)
    R = rhg.target_radius(n, 8, 1.0)
    pairs, _ = rhg.edges_from_points(phi, r, R)
    ids = torch.tensor([5, 9, 5, 700], dtype=torch.int32, device="cuda")
    with pytest.raises(rhg.RhgError) as e:
        rhg.update_edges(phi, r, R, ids, pairs)
    assert e.value.status == rhg.INVALID_ARG
