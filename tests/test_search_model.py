"""The range query's integer search logic restated in Python and checked against
numpy's searchsorted on adversarial key sets: the per-band bucket index (2^b
buckets of the top key bits, b the largest with 2^b <= the band's count, at
least 1; entry j = the first position whose bucket is >= j, entry 2^b = the
band's end), the four lock-step searches through it, and the wrap-around split
of a window that crosses key 0.  Keys are the 32-bit angle keys of one band,
sorted; duplicates, empty buckets and the extreme keys 0 and 2^32 - 1 included.
"""
import numpy as np
import pytest

M32 = (1 << 32) - 1


def bucket_bits(count):
    b = 1
    while b < 31 and (2 << b) <= count:
        b += 1
    return b


def build_index(keys, s):
    """Index entries of one band whose sorted keys sit at positions s .. s + len - 1,
    written the way each position writes them (its own bucket and the empty ones
    before it; the last position also the ones after it, up to the sentinel)."""
    count = len(keys)
    b = bucket_bits(count)
    sh = 32 - b
    nb = 1 << b
    idx = np.full(nb + 1, -1, dtype=np.int64)
    e = s + count
    for q in range(count):
        p = s + q
        cur = int(keys[q]) >> sh
        first = 0 if q == 0 else (int(keys[q - 1]) >> sh) + 1
        for j in range(first, cur + 1):
            idx[j] = p
        if q == count - 1:
            for j in range(cur + 1, nb + 1):
                idx[j] = e
    return idx, sh


def search(keys_abs, idx, sh, x, upper):
    """First position with key >= x (upper: > x) through the index, then bisection."""
    j = x >> sh
    lo, hi = int(idx[j]), int(idx[j + 1])
    while lo < hi:
        mid = lo + ((hi - lo) >> 1)
        k = int(keys_abs[mid])
        if (k <= x) if upper else (k < x):
            lo = mid + 1
        else:
            hi = mid
    return lo


def key_ranges(keys_abs, s, e, a, W):
    """The two candidate ranges of a window that may cross key 0."""
    if W >= 0x80000000:
        return (s, e), (0, 0)
    lo, hi = (a - W) & M32, (a + W) & M32
    band = keys_abs[s:e]
    if W <= a and a + W <= M32:
        return (s + int(np.searchsorted(band, lo, "left")), s + int(np.searchsorted(band, hi, "right"))), (0, 0)
    return (s + int(np.searchsorted(band, lo, "left")), e), (s, s + int(np.searchsorted(band, hi, "right")))


KEYSETS = {
    "uniform": lambda rng: rng.integers(0, 2**32, 3000),
    "duplicates": lambda rng: rng.choice(rng.integers(0, 2**32, 40), 2000),
    "all_equal": lambda rng: np.full(500, 123456789),
    "extremes": lambda rng: np.concatenate([np.zeros(50, np.int64), np.full(50, M32), rng.integers(0, 2**32, 100)]),
    "clustered": lambda rng: (rng.integers(0, 2**20, 3000) + 2**31),
    "one": lambda rng: np.array([7]),
    "two": lambda rng: np.array([0, M32]),
}


@pytest.mark.parametrize("name", sorted(KEYSETS))
def test_index_search_equals_searchsorted(name):
    rng = np.random.default_rng(len(name))
    keys = np.sort(KEYSETS[name](rng).astype(np.int64))
    s = 1000  # the band starts at a nonzero position
    keys_abs = np.concatenate([np.zeros(s, np.int64), keys])
    idx, sh = build_index(keys, s)
    assert (idx >= s).all() and (idx <= s + len(keys)).all() and (np.diff(idx) >= 0).all()
    xs = np.concatenate([rng.integers(0, 2**32, 400), keys[rng.integers(0, len(keys), 100)],
                         np.array([0, 1, M32 - 1, M32]), keys[:5] - 1, keys[-5:] + 1]) & M32
    for x in xs:
        x = int(x)
        assert search(keys_abs, idx, sh, x, False) == s + int(np.searchsorted(keys, x, "left"))
        assert search(keys_abs, idx, sh, x, True) == s + int(np.searchsorted(keys, x, "right"))


@pytest.mark.parametrize("name", ["uniform", "extremes", "duplicates"])
def test_window_ranges_cover_exactly_the_keys_in_the_window(name):
    """Every key within circular distance W of a lies in one of the two ranges,
    and no other key does."""
    rng = np.random.default_rng(99)
    keys = np.sort(KEYSETS[name](rng).astype(np.int64))
    s, e = 0, len(keys)
    for _ in range(300):
        a = int(rng.integers(0, 2**32))
        W = int(rng.choice([0, 1, 2**10, 2**20, 2**30, 2**31 - 1, int(rng.integers(0, 2**31))]))
        if rng.random() < 0.3:
            a = int(rng.choice([0, 1, M32, M32 - 5]))
        (r0, r1), (r2, r3) = key_ranges(keys, s, e, a, W)
        got = np.zeros(len(keys), bool)
        got[r0:r1] = True
        got[r2:r3] = True
        d = np.abs(keys - a)
        want = np.minimum(d, 2**32 - d) <= W
        assert np.array_equal(got, want), (a, W)
