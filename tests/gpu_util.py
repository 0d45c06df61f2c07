"""Helpers shared by the GPU tests (no method arithmetic here)."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_09481_gb300 as rhg
    rhg.build()
    return rhg


def sorted_pairs(pairs) -> np.ndarray:
    """(m, 2) pairs from the device as int64, lexicographically sorted."""
    a = pairs.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    if len(a) == 0:
        return a.reshape(0, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def assert_valid_pairs(a: np.ndarray, n: int):
    if len(a):
        assert np.all(a[:, 0] < a[:, 1]), "pairs must satisfy u < v (no self-loops)"
        assert a.max() < n
        key = a[:, 0] * n + a[:, 1]
        assert len(np.unique(key)) == len(a), "duplicate pairs"
