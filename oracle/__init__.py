"""CPU oracle for threshold random hyperbolic graphs (arXiv:1606.09481).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product library never loads it, and it never loads the product library.

The arithmetic lives in ``rhg_oracle.c`` (plain C, FP64, FMA contraction off);
this module compiles it with gcc and wraps it with ctypes and numpy.  See the
header of ``rhg_oracle.c`` for what each function follows in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rhg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librhg_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OK = 0
STATUS_INVALID_ARG = 1
STATUS_NO_SOLUTION = 2

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc; OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-Wall", "-Wno-unused-function", _SRC, "-lm"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:-2] + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base[:-1] + ["-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.ro_philox4x64.argtypes = [_p, _p, _p]
            L.ro_philox4x64_batch.argtypes = [_u64, _p, _p, _p]
            for f in ("ro_exp", "ro_log", "ro_cos", "ro_cosh", "ro_sinh"):
                getattr(L, f).argtypes = [_dbl]
                getattr(L, f).restype = _dbl
            L.ro_kbar.argtypes = [_dbl, _u64, _dbl]
            L.ro_kbar.restype = _dbl
            L.ro_target_radius.argtypes = [_u64, _dbl, _dbl, _p]
            L.ro_default_bands.argtypes = [_u64]
            L.ro_default_bands.restype = _u32
            L.ro_boundaries.argtypes = [_dbl, _u32, _dbl, _p]
            L.ro_sample_points.argtypes = [_u64, _dbl, _dbl, _u64, _u64, _p, _p]
            L.ro_radius_from_u53.argtypes = [_p, _u64, _dbl, _dbl, _p]
            L.ro_edge.argtypes = [_dbl, _dbl, _dbl, _dbl, _dbl]
            L.ro_edge_L.argtypes = [_dbl, _dbl, _dbl, _dbl]
            L.ro_edge_L.restype = _dbl
            L.ro_brute_edges.argtypes = [_u64, _p, _p, _dbl, _p, _u64]
            L.ro_brute_edges.restype = _i64
            L.ro_neighbors.argtypes = [_u64, _u64, _p, _p, _dbl, _p, _u64]
            L.ro_neighbors.restype = _i64
            L.ro_band_edges.argtypes = [_u64, _p, _p, _dbl, _u32, _dbl, _p, _u64, _p]
            L.ro_band_edges.restype = _i64
            L.ro_band_assign.argtypes = [_u64, _p, _dbl, _u32, _dbl, _p]
            L.ro_band_count_subset.argtypes = [_u64, _p, _p, _dbl, _u32, _dbl, _p, _u64, _p, _p]
            L.ro_band_count_subset.restype = _i64
            L.ro_openmp_threads.restype = ctypes.c_int
            L.ro_constants.argtypes = [_p]
            L.ro_prepare.argtypes = [_u64, _p, _p, _dbl, _u32, _dbl]
            L.ro_prepare.restype = _p
            L.ro_prepared_count.argtypes = [_p, _p, _u64, _p, _p]
            L.ro_prepared_count.restype = _i64
            L.ro_prepared_upper_pairs.argtypes = [_p, _u64, _u64, _p, _u64]
            L.ro_prepared_upper_pairs.restype = _i64
            L.ro_prepared_window_misses.argtypes = [_p, _p, _u64, _dbl, _p]
            L.ro_prepared_free.argtypes = [_p]
            L.ro_set_threads.argtypes = [ctypes.c_int32]
            L.ro_asinh.restype = _dbl
            L.ro_asinh.argtypes = [_dbl]
            L.ro_draw_movement.argtypes = [_u64, _u64, _dbl, _dbl, _dbl, _dbl, _p, _p]
            L.ro_move.argtypes = [_u64, _p, _p, _p, _p, _p, _dbl, _dbl, ctypes.c_int32]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_p)


NUM_STATS = 6
STAT_NAMES = ("candidates", "near_threshold", "windows", "rounding_band", "disagree_fp64_wellcond",
              "disagree_longdouble_wellcond")


def _stats_dict(stats) -> dict:
    """Counters of the examined pairs: near_threshold = |L - cosh R| <= 1e-12 cosh R;
    rounding_band = |L - cosh R| <= 8 u cosh r_v cosh r_w; disagree_* = pairs the
    cancellation-free form of Eq. 3 decides otherwise (FP64, long double)."""
    return {k: int(v) for k, v in zip(STAT_NAMES, stats)}


# --------------------------------------------------------------------------- Philox
def philox4x64(counter, key) -> np.ndarray:
    c = np.asarray(counter, dtype=np.uint64).reshape(4).copy()
    k = np.asarray(key, dtype=np.uint64).reshape(2).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib().ro_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox4x64_batch(count: int, counter0, key) -> np.ndarray:
    c = np.asarray(counter0, dtype=np.uint64).reshape(4).copy()
    k = np.asarray(key, dtype=np.uint64).reshape(2).copy()
    out = np.zeros((count, 4), dtype=np.uint64)
    lib().ro_philox4x64_batch(count, _ptr(c), _ptr(k), _ptr(out))
    return out


# --------------------------------------------------------------- deterministic math
def dm(fn: str, x) -> np.ndarray:
    """Evaluate one of exp/log/cos/cosh/sinh of the deterministic definition."""
    f = getattr(lib(), "ro_" + fn)
    xs = np.asarray(x, dtype=np.float64).ravel()
    return np.array([f(float(v)) for v in xs], dtype=np.float64)


CONSTANT_NAMES = ("PI", "TWO_PI", "INV_LN2", "LN2_HI", "LN2_LO", "TWO_OVER_PI", "PIO2_1",
                  "PIO2_2", "PIO2_3", "SQRT_HALF")


def constants() -> dict:
    out = np.zeros(len(CONSTANT_NAMES), dtype=np.float64)
    lib().ro_constants(_ptr(out))
    return dict(zip(CONSTANT_NAMES, (float(v) for v in out)))


# ----------------------------------------------------------------- model pieces
def kbar(R: float, n: int, alpha: float) -> float:
    return lib().ro_kbar(R, n, alpha)


def target_radius(n: int, k: float, alpha: float) -> float:
    out = _dbl(0.0)
    st = lib().ro_target_radius(n, k, alpha, ctypes.byref(out))
    if st != STATUS_OK:
        raise ValueError(f"target_radius(n={n}, k={k}, alpha={alpha}) status {st}")
    return out.value


def target_radius_status(n: int, k: float, alpha: float):
    out = _dbl(0.0)
    st = lib().ro_target_radius(n, k, alpha, ctypes.byref(out))
    return st, out.value


def default_bands(n: int) -> int:
    return int(lib().ro_default_bands(n))


def boundaries(R: float, B: int, p: float = 0.9) -> np.ndarray:
    c = np.zeros(B + 1, dtype=np.float64)
    st = lib().ro_boundaries(R, B, p, _ptr(c))
    if st != STATUS_OK:
        raise ValueError(f"boundaries status {st}")
    return c


def sample_points(n: int, alpha: float, R: float, seed: int, first: int = 0):
    phi = np.zeros(n, dtype=np.float64)
    r = np.zeros(n, dtype=np.float64)
    lib().ro_sample_points(n, alpha, R, seed, first, _ptr(phi), _ptr(r))
    return phi, r


def radius_from_u53(u, alpha: float, R: float) -> np.ndarray:
    """The sampler's radius (inverse CDF of Eq. 1, FP64 definition) of given
    53-bit variates: the radial step of sample_points alone."""
    u = np.ascontiguousarray(u, dtype=np.uint64)
    r = np.zeros(u.size, dtype=np.float64)
    st = lib().ro_radius_from_u53(_ptr(u), u.size, alpha, R, _ptr(r))
    if st != STATUS_OK:
        raise ValueError(f"radius_from_u53 status {st}")
    return r


def asinh(y: float) -> float:
    """The dynamic model's deterministic asinh (y >= 0)."""
    return lib().ro_asinh(float(y))


def draw_movement(n: int, seed: int, phi_range=(-1.0, 1.0), r_range=(-10.0, 1.0)):
    """Step values (tau_phi, tau_r) of nodes 0..n-1 (Sec. III-C); the default
    ranges are those of the paper's experiment."""
    tphi = np.zeros(n, dtype=np.float64)
    tr = np.zeros(n, dtype=np.float64)
    lib().ro_draw_movement(n, seed, float(phi_range[0]), float(phi_range[1]), float(r_range[0]),
                           float(r_range[1]), _ptr(tphi), _ptr(tr))
    return tphi, tr


COORD_UNIFORM = 0  # radial step in cosh(alpha r) - 1, uniform under Eq. 1 (Theorem 1 holds)
COORD_SINH = 1     # radial step in sinh(alpha r), as Algorithm 2 prints it


def move(ids, phi, r, tau_phi, tau_r, R: float, alpha: float, coord: int = COORD_UNIFORM):
    """One movement step (rotation + the radial movement of Algorithm 2 with
    reflection) of the nodes `ids`; returns new (phi, r, tau_r) arrays, the inputs
    unchanged.  `coord` selects the coordinate of the radial step (see the header
    of rhg_oracle.c)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    phi = np.array(phi, dtype=np.float64)
    r = np.array(r, dtype=np.float64)
    tau_r = np.array(tau_r, dtype=np.float64)
    tau_phi = np.ascontiguousarray(tau_phi, dtype=np.float64)
    lib().ro_move(len(ids), _ptr(ids), _ptr(phi), _ptr(r), _ptr(tau_phi), _ptr(tau_r), float(R), float(alpha),
                  int(coord))
    return phi, r, tau_r


def band_assign(r: np.ndarray, R: float, B: int, p: float = 0.9) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(len(r), dtype=np.uint32)
    st = lib().ro_band_assign(len(r), _ptr(r), R, B, p, _ptr(out))
    if st != STATUS_OK:
        raise ValueError(f"band_assign status {st}")
    return out


def edge(phv: float, rv: float, phw: float, rw: float, R: float) -> bool:
    return bool(lib().ro_edge(phv, rv, phw, rw, R))


def edge_L(phv: float, rv: float, phw: float, rw: float) -> float:
    return lib().ro_edge_L(phv, rv, phw, rw)


def _pts(phi, r):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    assert phi.shape == r.shape
    return phi, r


def brute_edges(phi, r, R: float) -> np.ndarray:
    """All pairs (u < v) with an edge, in (u, v) lexicographic order."""
    phi, r = _pts(phi, r)
    n = len(phi)
    m = lib().ro_brute_edges(n, _ptr(phi), _ptr(r), R, None, 0)
    out = np.zeros((max(m, 1), 2), dtype=np.uint32)
    m2 = lib().ro_brute_edges(n, _ptr(phi), _ptr(r), R, _ptr(out), m)
    assert m2 == m
    return out[:m]


def neighbors(v: int, phi, r, R: float) -> np.ndarray:
    phi, r = _pts(phi, r)
    n = len(phi)
    cap = 1024
    while True:
        out = np.zeros(cap, dtype=np.uint32)
        m = lib().ro_neighbors(v, n, _ptr(phi), _ptr(r), R, _ptr(out), cap)
        if m <= cap:
            return out[:m]
        cap = int(m)


def band_edges(phi, r, R: float, B: int, p: float = 0.9, with_stats: bool = False):
    """Alg. 1 range query; returns pairs (u < v) sorted lexicographically."""
    phi, r = _pts(phi, r)
    n = len(phi)
    stats = np.zeros(NUM_STATS, dtype=np.int64)
    cap = max(1024, 8 * n)
    while True:
        out = np.zeros((cap, 2), dtype=np.uint32)
        m = lib().ro_band_edges(n, _ptr(phi), _ptr(r), R, B, p, _ptr(out), cap, _ptr(stats))
        if m < 0:
            raise ValueError(f"band_edges status {-m}")
        if m <= cap:
            break
        cap = int(m)
    pairs = out[:m]
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    if with_stats:
        return pairs, _stats_dict(stats)
    return pairs


def band_count_subset(phi, r, R: float, B: int, p: float, ids: np.ndarray, with_stats: bool = False):
    """Edges found from the given vertices' outward queries, and threads used
    (and the diagnostics of the examined pairs with with_stats)."""
    phi, r = _pts(phi, r)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    nt = ctypes.c_int32(0)
    stats = np.zeros(NUM_STATS, dtype=np.int64)
    m = lib().ro_band_count_subset(len(phi), _ptr(phi), _ptr(r), R, B, p, _ptr(ids), len(ids),
                                   ctypes.byref(nt), _ptr(stats))
    if with_stats:
        return int(m), int(nt.value), _stats_dict(stats)
    return int(m), int(nt.value)


class Prepared:
    """Band structure of Alg. 1 built once over given points; count_edges(ids)
    runs the outward range queries of those vertices (OpenMP when available)."""

    def __init__(self, phi, r, R: float, B: int, p: float = 0.9):
        self.phi, self.r = _pts(phi, r)
        self.h = lib().ro_prepare(len(self.phi), _ptr(self.phi), _ptr(self.r), R, B, p)
        if not self.h:
            raise MemoryError("ro_prepare failed")

    def count_edges(self, ids, threads: int = 0, with_stats: bool = False):
        """(edges, threads used[, diagnostics]); threads > 0 caps the OpenMP threads
        for this call."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        nt = ctypes.c_int32(0)
        stats = np.zeros(NUM_STATS, dtype=np.int64)
        if threads > 0:
            lib().ro_set_threads(threads)
        try:
            m = lib().ro_prepared_count(self.h, _ptr(ids), len(ids), ctypes.byref(nt), _ptr(stats))
        finally:
            if threads > 0:
                lib().ro_set_threads(0)
        if with_stats:
            return int(m), int(nt.value), _stats_dict(stats)
        return int(m), int(nt.value)

    def upper_pairs(self, u0: int, u1: int, capacity: int = 0) -> np.ndarray:
        """Every edge (u, w) with u0 <= u < u1 and u < w, in lexicographic order
        (uint32, shape (m, 2))."""
        cap = capacity or max(1 << 16, 64 * (u1 - u0))
        while True:
            out = np.empty((cap, 2), dtype=np.uint32)
            m = lib().ro_prepared_upper_pairs(self.h, u0, u1, _ptr(out), cap)
            if m < 0:
                raise MemoryError(f"ro_prepared_upper_pairs status {-m}")
            if m <= cap:
                return out[:m]
            cap = int(m)

    def window_misses(self, ids, theta_scale: float = 1.0) -> dict:
        """All-pairs edges of the listed vertices checked against their
        getMinMaxPhi windows (Sec. III-B); theta_scale < 1 narrows the windows
        (negative control)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        out = np.zeros(4, dtype=np.int64)
        st = lib().ro_prepared_window_misses(self.h, _ptr(ids), len(ids), float(theta_scale), _ptr(out))
        if st != STATUS_OK:
            raise ValueError(f"ro_prepared_window_misses status {st}")
        return {"edges": int(out[0]), "misses": int(out[1]), "alg1_edges": int(out[2]),
                "inner_endpoint_edges": int(out[3])}

    def close(self):
        if self.h:
            lib().ro_prepared_free(self.h)
            self.h = None

    def __del__(self):
        self.close()


def openmp_threads() -> int:
    return int(lib().ro_openmp_threads())


def generate(n: int, k: float, alpha: float, seed: int, num_bands: int = 0, p: float = 0.9,
             method: str = "band", with_stats: bool = False):
    """The whole oracle pipeline: R, points, then the edge set."""
    R = target_radius(n, k, alpha)
    B = num_bands or default_bands(n)
    phi, r = sample_points(n, alpha, R, seed)
    out = {"R": R, "B": B, "phi": phi, "r": r}
    if method == "brute":
        out["pairs"] = brute_edges(phi, r, R)
    else:
        res = band_edges(phi, r, R, B, p, with_stats=with_stats)
        if with_stats:
            out["pairs"], out["stats"] = res
        else:
            out["pairs"] = res
    return out


def pairs_to_csr(pairs: np.ndarray, n: int):
    """Symmetric CSR with ascending columns from undirected pairs (u < v)."""
    u = np.concatenate([pairs[:, 0], pairs[:, 1]]).astype(np.int64)
    v = np.concatenate([pairs[:, 1], pairs[:, 0]]).astype(np.int64)
    order = np.lexsort((v, u))
    u, v = u[order], v[order]
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    np.add.at(row_ptr, u + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.uint64)
    return row_ptr, v.astype(np.uint32)
