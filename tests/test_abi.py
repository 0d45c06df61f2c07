"""The C-ABI library builds, loads and exports every entry point that
include/rhg.h declares; host-side validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rhg():
    import paper_1606_09481_gb300 as rhg
    rhg.build()
    return rhg


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rhg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(rhg_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("rhg_generate_pairs", "rhg_generate_csr", "rhg_target_radius", "rhg_edges_from_points",
                 "rhg_sample_points", "rhg_status_str", "rhg_workspace_bytes"):
        assert must in names


def test_library_exports_every_declared_symbol(rhg):
    lib = ctypes.CDLL(rhg.LIB)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings_and_version(rhg):
    assert rhg.status_str(0) == "RHG_OK"
    assert rhg.status_str(6) == "RHG_ERR_OVERFLOW"
    assert rhg.status_str(99) == "RHG_ERR_UNKNOWN"
    assert rhg.load().rhg_version() == 4


def test_params_layout_matches_header(rhg):
    assert ctypes.sizeof(rhg.Params) == 72
    assert ctypes.sizeof(rhg.Result) == 72


def _ws_status(rhg, **kw):
    p = rhg.make_params(**kw)
    out = ctypes.c_size_t(0)
    return rhg.load().rhg_workspace_bytes(ctypes.byref(p), 0, ctypes.byref(out)), out.value


def test_host_validation(rhg):
    ok, nbytes = _ws_status(rhg, n=10_000_000, k=200, alpha=1.0)
    assert ok == 0 and nbytes > 10_000_000 * 80
    bad = [dict(n=1, k=6, alpha=1.0), dict(n=2**32, k=6, alpha=1.0), dict(n=100, k=6, alpha=0.5),
           dict(n=100, k=0, alpha=1.0), dict(n=100, k=-1, alpha=1.0), dict(n=100, k=6, alpha=101.0),
           dict(n=100, k=6, alpha=1.0, num_bands=65), dict(n=100, k=6, alpha=1.0, band_ratio=-0.5),
           dict(n=100, k=6, alpha=1.0, flags=0x80), dict(n=100, k=6, alpha=1.0, flags=0x4), dict(n=100, k=6, alpha=float("nan"))]
    for kw in bad:
        assert _ws_status(rhg, **kw)[0] == rhg.INVALID_ARG, kw
    # an R given directly replaces k
    assert _ws_status(rhg, n=100, k=0, alpha=1.0, R_override=12.0)[0] == 0
    # the range query's work mapping: 0 = default, else within its documented range
    for kw in (dict(batch_budget=1023), dict(batch_budget=(1 << 24) + 1), dict(core_heavy=63),
               dict(core_heavy=65537), dict(fringe_limit=33)):
        assert _ws_status(rhg, n=100, k=6, alpha=1.0, **kw)[0] == rhg.INVALID_ARG, kw
    for kw in (dict(batch_budget=1024), dict(batch_budget=1 << 24), dict(core_heavy=64), dict(core_heavy=65536),
               dict(fringe_limit=1), dict(fringe_limit=32)):
        assert _ws_status(rhg, n=100, k=6, alpha=1.0, **kw)[0] == 0, kw
    p = rhg.make_params(n=100, k=6, alpha=1.0)
    p.reserved = 1
    out = ctypes.c_size_t(0)
    assert rhg.load().rhg_workspace_bytes(ctypes.byref(p), 0, ctypes.byref(out)) == rhg.INVALID_ARG


def test_invalid_arguments_rejected_before_device_work(rhg):
    L = rhg.load()
    p = rhg.make_params(n=1, k=6, alpha=1.0)
    res = rhg.Result()
    assert L.rhg_generate_pairs(ctypes.byref(p), None, 0, None, 0, None, ctypes.byref(res)) == rhg.INVALID_ARG
    p = rhg.make_params(n=1000, k=6, alpha=1.0)
    assert L.rhg_generate_pairs(ctypes.byref(p), None, 0, None, 0, None, ctypes.byref(res)) == rhg.INVALID_ARG
    # workspace smaller than required: OOM, still before any device work
    assert L.rhg_generate_pairs(ctypes.byref(p), ctypes.c_void_p(256), 16, ctypes.c_void_p(256), 10, None,
                                ctypes.byref(res)) == rhg.OOM
    assert L.rhg_dm_eval(7, None, None, 0, None) == rhg.INVALID_ARG
    R = ctypes.c_double(0)
    assert L.rhg_target_radius(100, 6.0, 0.4, None, 0, None, ctypes.byref(R)) == rhg.INVALID_ARG


def test_product_package_does_not_touch_oracle():
    """The product path never imports, loads or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1606_09481_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "rhg_oracle", "librhg_oracle"):
                    assert bad not in txt, (f, bad)


def test_batch_plan_layout_and_validation(rhg):
    """rhg_batch_plan matches the header; plans that rhg_batch_prepare did not
    make, and missing buffers, are refused on the host."""
    assert ctypes.sizeof(rhg.BatchPlan) == 56
    L = rhg.load()
    params = rhg.batch_params([(1000, 8, 1.0, 1), (3000, 10, 0.8, 2)])
    offs = (ctypes.c_uint64 * 3)(0, 10_000, 30_000)
    plan = rhg.BatchPlan()
    assert L.rhg_batch_prepare(params, 2, offs, None, 1 << 30, None, ctypes.byref(plan)) == rhg.INVALID_ARG
    assert L.rhg_batch_prepare(params, 2, None, 256, 1 << 30, None, ctypes.byref(plan)) == rhg.INVALID_ARG
    assert L.rhg_batch_prepare(params, 0, offs, 256, 1 << 30, None, ctypes.byref(plan)) == rhg.INVALID_ARG
    assert L.rhg_batch_prepare(params, 2, offs, 256, 16, None, ctypes.byref(plan)) == rhg.OOM
    # a plan with counts that describe no workspace of its size
    fake = rhg.BatchPlan(count=2, verify=0, num_tiles=3, points=4000, index_entries=4000, pair_capacity=30_000,
                         workspace_bytes=12345)
    assert L.rhg_batch_launch(ctypes.byref(fake), 256, 256, None) == rhg.INVALID_ARG
    assert L.rhg_batch_launch(None, 256, 256, None) == rhg.INVALID_ARG
    zero = rhg.BatchPlan()
    assert L.rhg_batch_launch(ctypes.byref(zero), 256, 256, None) == rhg.INVALID_ARG
    res = (rhg.BatchGraph * 2)()
    assert L.rhg_batch_read_results(ctypes.byref(fake), 256, None, res, None) == rhg.INVALID_ARG


def test_library_loads_once_across_threads(rhg):
    """Serving threads that call into the binding at once share one library handle."""
    import threading
    saved = rhg._lib
    rhg._lib = None
    try:
        got = []
        threads = [threading.Thread(target=lambda: got.append(rhg.load())) for _ in range(8)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert len(got) == 8 and len({id(x) for x in got}) == 1
    finally:
        rhg._lib = saved if saved is not None else rhg._lib


def test_chunk_list_sized_for_fp64_mode_when_solved_R_exceeds_the_filter(rhg):
    """A graph whose R solved from Eq. 22 is above the filter's range runs in FP64
    mode on the device: its workspace is sized like an FP64-only graph's.  One
    whose R is well inside the range is sized like a filter graph."""
    fp64 = rhg.FLAG_FP64_ONLY
    # n = 5e6, k = 8, alpha = 0.6: R = 32.7 > 32
    assert _ws_status(rhg, n=5_000_000, k=8, alpha=0.6)[1] == _ws_status(rhg, n=5_000_000, k=8, alpha=0.6,
                                                                          flags=fp64)[1]
    # n = 5e6, k = 8, alpha = 1: R = 28.6, filter mode
    assert _ws_status(rhg, n=5_000_000, k=8, alpha=1.0)[1] < _ws_status(rhg, n=5_000_000, k=8, alpha=1.0,
                                                                         flags=fp64)[1]
