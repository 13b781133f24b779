"""User-defined models on the host (no GPU): run-time compilation through
the C ABI, the registry, and argument / compile-error handling.

NVRTC compiles without a device, so the whole registration path runs here;
loading the code on a device happens at a model's first fit (GPU tests).
"""
import pytest

from paper_2208_12187_gb300 import build, gbfit
from user_model_defs import LORENTZ_SRC


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gbfit.load()


@pytest.fixture(scope="module")
def lorentz_id(lib):
    return gbfit.register_model(LORENTZ_SRC, 4)


def test_register_returns_a_user_id_with_its_shape(lib, lorentz_id):
    import ctypes
    assert lorentz_id >= gbfit.USER_MODEL_BASE
    n, d = ctypes.c_int(), ctypes.c_int()
    assert lib.gbfit_model_info(lorentz_id, ctypes.byref(n), ctypes.byref(d)) == 0
    assert (n.value, d.value) == (4, 1)
    assert gbfit.N_PARAMS[lorentz_id] == 4


def test_compile_error_is_reported_with_the_log(lib):
    bad = "template <class T, class S> __device__ T model(const T* p, S x, S x2) { return p[0] * no_such(x); }"
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.register_model(bad, 1)
    assert e.value.code == gbfit.E_INVALID_ARG
    assert "no_such" in str(e.value)
    assert "user_source" in gbfit.model_log()


@pytest.mark.parametrize("kw", [dict(n_params=0), dict(n_params=9), dict(x_dims=3), dict(func_name="1bad"),
                                dict(func_name="a b")])
def test_register_argument_checks(lib, kw):
    args = dict(source=LORENTZ_SRC, n_params=4, x_dims=1, func_name="model")
    args.update(kw)
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.register_model(**args)
    assert e.value.code == gbfit.E_INVALID_ARG


def test_unknown_ids_are_rejected(lib):
    import ctypes
    n, d = ctypes.c_int(), ctypes.c_int()
    for mid in (4, 99, gbfit.USER_MODEL_BASE + 63, -1):
        assert lib.gbfit_model_info(mid, ctypes.byref(n), ctypes.byref(d)) == gbfit.E_INVALID_ARG


def test_tile_table_takes_builtin_models_only(lib, lorentz_id):
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.tune_shape(lorentz_id, "mixed", 10_000)
    assert e.value.code == gbfit.E_INVALID_ARG
