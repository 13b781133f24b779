"""The C-ABI library builds, loads and exports every symbol include/gbfit.h declares.

No compute calls here (no GPU): only symbol checks, the registry query and the
host-side argument checks that fail before any device work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2208_12187_gb300 import build, gbfit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gbfit.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gbfit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbfit_\w+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert _declared_functions() == sorted(gbfit.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_version_and_model_registry(lib):
    assert lib.gbfit_version() == 1
    n, xd = ctypes.c_int(), ctypes.c_int()
    expect = {0: (4, 1), 1: (5, 1), 2: (7, 2), 3: (3, 1)}
    for mid, (np_, xdim) in expect.items():
        assert lib.gbfit_model_info(mid, ctypes.byref(n), ctypes.byref(xd)) == 0
        assert (n.value, xd.value) == (np_, xdim)
    assert lib.gbfit_model_info(9, ctypes.byref(n), ctypes.byref(xd)) == gbfit.E_INVALID_ARG
    assert b"unknown model" in lib.gbfit_last_error()


def test_default_options(lib):
    o = gbfit.Options()
    assert lib.gbfit_default_options(ctypes.byref(o)) == 0
    assert o.ftol == o.xtol == o.gtol == 1e-8
    assert o.precision == gbfit.PREC_MIXED


@pytest.mark.parametrize("kw,code", [
    (dict(p0=[1.0, 0.0, 1.0, 0.0], lb=[0, -1, 0, -1], ub=[2, 1, 2, 1]), gbfit.E_INVALID_ARG),  # 1D model, 2D x
    (dict(p0=[1.0, np.nan, 1.0, 0.0]), gbfit.E_INVALID_ARG),
    (dict(p0=[1.0, 0.0, 1.0, 0.0], lb=[2, -1, 0, -1], ub=[3, 1, 2, 1]), gbfit.E_INFEASIBLE_X0),
    (dict(p0=[1.0, 0.0, 1.0, 0.0], lb=[1, -1, 0, -1], ub=[1, 1, 2, 1]), gbfit.E_INVALID_ARG),
])
def test_host_argument_checks(lib, kw, code):
    x = np.zeros((2, 10)) if "lb" in kw and kw["lb"][0] == 0 else np.zeros(10)
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.curve_fit(gbfit.MODEL_GAUSS1D, x, np.zeros(10), **kw)
    assert e.value.code == code


def test_too_few_points_rejected(lib):
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.curve_fit(gbfit.MODEL_GAUSS2D, None, np.zeros(6), [1, 0, 0, 1, 1, 0, 0], grid_wh=(2, 3))
    assert e.value.code == gbfit.E_INVALID_ARG
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.curve_fit(gbfit.MODEL_GAUSS1D, np.zeros(0), np.zeros(0), [1, 0, 1, 0])
    assert e.value.code == gbfit.E_INVALID_ARG


def test_tune_table_host_api():
    """Tile table: defaults, lookup by log2 bucket, one tile for small fits, validation."""
    saved = gbfit.tune_get()
    tp = saved["tile_points"]
    assert tp.shape == (4, 2, gbfit.TUNE_BUCKETS)
    assert gbfit.tune_shape(gbfit.MODEL_DEXP, "mixed", 1 << 20) == (int(tp[1, 1, 20]), int(saved["group_tiles"][1, 1, 20]))
    assert gbfit.tune_shape(gbfit.MODEL_DEXP, "mixed", 1000)[0] == 1024          # a fit smaller than its tile: one tile
    bad = {k: v.copy() for k, v in saved.items()}
    bad["tile_points"][0, 0, 5] = 1000                                            # not a multiple of 256
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.tune_set(bad)
    assert e.value.code == gbfit.E_INVALID_ARG
    assert np.array_equal(gbfit.tune_get()["tile_points"], tp)                    # unchanged after a refusal
    new = {k: v.copy() for k, v in saved.items()}
    new["tile_points"][2, 1, :] = 4096
    new["group_tiles"][2, 1, :] = 8
    try:
        gbfit.tune_set(new)
        assert gbfit.tune_shape(gbfit.MODEL_GAUSS2D, "mixed", 1 << 22) == (4096, 8)
        assert gbfit.tune_shape(gbfit.MODEL_GAUSS2D, "mixed", 3000) == (3072, 8)
    finally:
        gbfit.tune_set(saved)
    with pytest.raises(gbfit.GbfitError):
        gbfit.tune_shape(9, "mixed", 100)


def test_covariance_size_limit_checked_on_the_host():
    """m above GBFIT_COV_MAX_M is refused before any device work."""
    import ctypes
    import numpy as np
    from paper_2208_12187_gb300 import build, gbfit
    build.build()
    lib = gbfit.load()
    m = 8193
    x = np.zeros(m)
    y = np.zeros(m)
    C = np.zeros(1)            # never read: the size check comes first
    p0 = np.array([1.0, 0.0, 1.0, 0.0])
    out = np.zeros(4 + 16 + 1)
    ints = np.zeros(2, dtype=np.int32)
    a = out.ctypes.data
    rc = lib.gbfit_curve_fit_cov(0, x.ctypes.data, m, 0, None, y.ctypes.data, C.ctypes.data, 1, p0.ctypes.data,
                                 None, None, None, a, a + 32, a + 160, ints.ctypes.data, ints.ctypes.data + 4, None)
    assert rc == gbfit.E_INVALID_ARG
    assert b"m <=" in lib.gbfit_last_error()


@pytest.mark.parametrize("m,tile_points,refused", [
    (120_000_000, 0, False),          # the default tile grows so that 2048 tiles hold it
    (134_000_000, 0, False),
    (134_217_728, 0, False),          # 2048 tiles of 65536 points exactly
    (134_217_729, 0, True),
    (2048 * 256, 256, False),
    (2048 * 256 + 1, 256, True),
    (2048 * 2048 + 1, 2000, True),    # tile_points rounds up to 2048
])
def test_noalloc_size_limit_checked_on_the_host(lib, m, tile_points, refused):
    """The allocation-free entry point's tile limit (2048 tiles) is host
    arithmetic done before any CUDA call: sizes within it are not refused for
    size (the call then fails later on a CPU-only host, or on the fake data
    pointers, which are never read), sizes beyond it are."""
    out = np.zeros(4 + 10 + 1)
    p = np.array([1.0, 0.0, 1.0, 0.0])
    fake = ctypes.c_void_p(256)           # never dereferenced: every failing check comes first
    rc = lib.gbfit_evaluate_noalloc(gbfit.MODEL_GAUSS1D, fake, ctypes.c_int64(m), gbfit.X_VEC, None, fake, None,
                                    gbfit.F32, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), gbfit.PREC_MIXED,
                                    tile_points, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    msg = lib.gbfit_last_error()
    assert rc != 0
    size_refusal = rc == gbfit.E_INVALID_ARG and b"2048 tiles" in msg
    assert size_refusal == refused, msg


def test_guard_options_checked_on_the_host(lib):
    """NaN precision-guard thresholds are refused before any device work."""
    for kw in (dict(guard_cond=float("nan")), dict(guard_floor=float("nan"))):
        with pytest.raises(gbfit.GbfitError) as e:
            gbfit.curve_fit(gbfit.MODEL_GAUSS1D, np.zeros(10), np.zeros(10), [1.0, 0.0, 1.0, 0.0], **kw)
        assert e.value.code == gbfit.E_INVALID_ARG
        assert "guard" in str(e.value)
