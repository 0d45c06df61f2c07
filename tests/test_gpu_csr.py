"""CSR output (rhg_generate_csr): row pointers and the columns of every row in
ascending order equal the oracle's Algorithm 1 edge set in CSR form, on graphs
from one vertex pair to power-law graphs whose largest rows hold 10^5 entries
(alpha = 0.55 at n = 2*10^5), and in FP64-only mode."""
import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,k,alpha,seed", [(2, 1.0, 1.0, 1), (3000, 8, 1.0, 5), (50_000, 20, 0.75, 6),
                                            (200_000, 64, 0.55, 7)])
def test_csr_equals_oracle(O, n, k, alpha, seed):
    rhg = require_gpu()
    row_ptr, col, res = rhg.generate_csr(n, k, alpha, seed)
    g = O.generate(n, k, alpha, seed)
    ref_rp, ref_col = O.pairs_to_csr(g["pairs"], n)
    assert res.m == len(g["pairs"])
    assert np.array_equal(row_ptr.cpu().numpy().astype(np.uint64), ref_rp)
    assert np.array_equal(col.cpu().numpy().astype(np.uint32), ref_col)
    if n == 200_000:  # rows of every size class, up to beyond 2048 entries
        deg = np.diff(ref_rp.astype(np.int64))
        for lo, hi in ((1, 32), (32, 256), (256, 2048), (2048, None)):
            assert ((deg > lo) & (deg <= (hi or deg.max()))).any(), (lo, hi)


def test_csr_fp64_mode_equals_oracle(O):
    """The FP64-only mode (no FP32 filter) gives the same CSR."""
    rhg = require_gpu()
    n, k, alpha, seed = 40_000, 12, 0.9, 11
    row_ptr, col, res = rhg.generate_csr(n, k, alpha, seed, flags=rhg.FLAG_FP64_ONLY)
    ref_rp, ref_col = O.pairs_to_csr(O.generate(n, k, alpha, seed)["pairs"], n)
    assert np.array_equal(row_ptr.cpu().numpy().astype(np.uint64), ref_rp)
    assert np.array_equal(col.cpu().numpy().astype(np.uint32), ref_col)
