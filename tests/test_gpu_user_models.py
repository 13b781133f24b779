"""User-defined models on the GPU: run-time compiled loop kernels (dual-number
partials) against the FP64 oracle with the same model written in NumPy.

Tolerances as for the built-in models:
  reductions at fixed p   plain 1e-12 relative to each entry's scale; mixed 2e-5
  whole fits              plain popt / cost 1e-8 with the same nfev and status;
                          mixed popt 1e-6
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reduce as red, trf
from paper_2208_12187_gb300 import build, gbfit, synth
from user_model_defs import (GAUSS1D_SRC, GAUSS2D_AXIS_SRC, LORENTZ_SRC, ZOO_P, ZOO_SRC, gauss2d_axis_np,
                             lorentz_np, zoo_np)

pytestmark = pytest.mark.gpu
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)


@pytest.fixture(scope="module")
def ids():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gbfit.load()
    return dict(lorentz=gbfit.register_model(LORENTZ_SRC, 4),
                gauss2d_axis=gbfit.register_model(GAUSS2D_AXIS_SRC, 6, x_dims=2, func_name="gauss_axis"),
                gauss1d=gbfit.register_model(GAUSS1D_SRC, 4),
                zoo=gbfit.register_model(ZOO_SRC, 8))


def dev(a, dtype):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


def gpu_fit(mid, pr, precision, **kw):
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = None if pr.layout == synth.LAYOUT_GRID else dev(pr.x, dt)
    return gbfit.curve_fit(mid, x, dev(pr.y, dt), pr.p0, sigma=dev(pr.sigma, dt), lb=pr.lb, ub=pr.ub,
                           grid_wh=pr.grid_wh, precision=precision, **kw)


def oracle_fit(fn, pr, **kw):
    return trf.curve_fit(fn, pr.coords(), pr.y, pr.sigma, pr.p0, pr.lb, pr.ub, **kw)


def check_reduction(mid, fn, pr, p, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    prc = pr.astype(np.float64 if precision == "fp64" else np.float32)
    f, g, B, _, _ = red.evaluate(fn, prc.coords(), prc.y.astype(np.float64), red.weights(prc.sigma, prc.m), p)
    x = None if prc.layout == synth.LAYOUT_GRID else dev(prc.x, dt)
    Bp, gg, cost = gbfit.evaluate(mid, x, dev(prc.y, dt), p, sigma=dev(prc.sigma, dt), grid_wh=prc.grid_wh,
                                  precision=precision, tile_points=2048)
    n = len(p)
    Bg = gbfit.unpack_upper(Bp, n)
    tol = 1e-12 if precision == "fp64" else 2e-5
    dscale = np.sqrt(np.outer(np.diag(B), np.diag(B)))
    assert np.max(np.abs(Bg - B) / np.maximum(dscale, 1e-300)) <= tol
    gscale = np.sqrt(np.diag(B) * 2 * f)
    assert np.max(np.abs(gg - g) / np.maximum(gscale, 1e-300)) <= tol
    assert abs(cost - f) <= tol * f


# ------------------------------------------------------------------ fixed-p reductions
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dual_number_partials_of_every_operation(ids, precision):
    """Every operation of the dual-number types, against complex-step partials."""
    rng = np.random.default_rng(0)
    m = 3 * 2048 + 77
    x = rng.uniform(0.1, 2.0, m)
    y = rng.normal(0.0, 1.0, m)
    pr = synth.Problem(ids["zoo"], x, synth.LAYOUT_VEC, None, y, None, ZOO_P.copy(), None, None, ZOO_P, n_user=8)
    check_reduction(ids["zoo"], zoo_np, pr, ZOO_P, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("layout", [synth.LAYOUT_GRID, synth.LAYOUT_SOA2])
def test_user_2d_reduction(ids, precision, layout):
    pr = synth.user_family("gauss2d_axis", 70 * 70, seed=1, layout=layout, with_sigma=True)
    check_reduction(ids["gauss2d_axis"], gauss2d_axis_np, pr, pr.p0, precision)


# ------------------------------------------------------------------ whole fits
@pytest.mark.parametrize("with_sigma", [False, True])
def test_user_fit_plain_matches_oracle(ids, with_sigma):
    pr = synth.user_family("lorentz1d", 20_000 + 13, seed=2, with_sigma=with_sigma)
    ref = oracle_fit(lorentz_np, pr, **TOL)
    out = gpu_fit(ids["lorentz"], pr, "fp64", **TOL)
    assert out["status"] == ref["status"] and out["nfev"] == ref["nfev"]
    assert relerr(out["popt"], ref["popt"]) <= 1e-8
    assert out["cost"] == pytest.approx(ref["cost"], rel=1e-8)
    np.testing.assert_allclose(out["pcov"], ref["pcov"], rtol=1e-6, atol=1e-12 * np.max(np.abs(ref["pcov"])))


def test_user_fit_mixed_matches_oracle(ids):
    pr = synth.user_family("lorentz1d", 200_000, seed=3).astype(np.float32)
    ref = oracle_fit(lorentz_np, pr, **TOL)
    out = gpu_fit(ids["lorentz"], pr, "mixed", **TOL)
    assert out["status"] > 0
    assert relerr(out["popt"], ref["popt"]) <= 1e-6
    assert out["cost"] == pytest.approx(ref["cost"], rel=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("layout", [synth.LAYOUT_GRID, synth.LAYOUT_SOA2])
def test_user_2d_fit_bounded(ids, precision, layout):
    pr = synth.user_family("gauss2d_axis", 120 * 120, seed=4, layout=layout)
    if precision == "mixed":
        pr = pr.astype(np.float32)
    ref = oracle_fit(gauss2d_axis_np, pr, **TOL)
    out = gpu_fit(ids["gauss2d_axis"], pr, precision, **TOL)
    if precision == "fp64":
        assert out["status"] == ref["status"] and out["nfev"] == ref["nfev"]
        assert relerr(out["popt"], ref["popt"]) <= 1e-8
    else:
        assert relerr(out["popt"], ref["popt"]) <= 1e-6


@pytest.mark.parametrize("precision,m", [("fp64", 30_000), ("mixed", 30_000), ("mixed", 4_000_000)])
def test_user_written_gaussian_equals_the_builtin(ids, precision, m):
    """The built-in 1D Gaussian written as a user model: same fit.  At 4M
    points the mixed steps near convergence fall below the FP32 resolution of
    the parameters; the carried rounding correction keeps the iteration count
    at the built-in's."""
    pr = synth.gauss1d(m, seed=6)
    if precision == "mixed":
        pr = pr.astype(np.float32)
    a = gpu_fit(gbfit.MODEL_GAUSS1D, pr, precision, **TOL)
    b = gpu_fit(ids["gauss1d"], pr, precision, **TOL)
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert relerr(b["popt"], a["popt"]) <= tol
    if precision == "fp64":
        assert a["nfev"] == b["nfev"]
    else:
        assert abs(a["nfev"] - b["nfev"]) <= 1


def test_user_model_batch(ids):
    rng = np.random.default_rng(7)
    probs = [synth.user_family("lorentz1d", int(m), seed=10 + k).astype(np.float32)
             for k, m in enumerate(rng.integers(500, 40_000, 6))]
    off = np.concatenate([[0], np.cumsum([p.m for p in probs])]).astype(np.int64)
    x = np.concatenate([p.x for p in probs])
    y = np.concatenate([p.y for p in probs])
    p0 = np.stack([p.p0 for p in probs])
    out = gbfit.curve_fit_batch(ids["lorentz"], off, dev(x, torch.float32), dev(y, torch.float32), p0,
                                precision="mixed", **TOL)
    for k, pr in enumerate(probs):
        ref = oracle_fit(lorentz_np, pr, **TOL)
        assert relerr(out["popt"][k], ref["popt"]) <= 1e-6, k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_user_model_robust_loss(ids, precision):
    pr = synth.user_family("lorentz1d", 30_000, seed=8)
    rng = np.random.default_rng(8)
    bad = rng.choice(pr.m, pr.m // 20, replace=False)
    pr.y[bad] += rng.normal(0, 3.0, bad.size)
    if precision == "mixed":
        pr = pr.astype(np.float32)
    ref = trf.curve_fit(lorentz_np, pr.coords(), pr.y, None, pr.p0, loss="soft_l1", f_scale=0.2, **TOL)
    out = gpu_fit(ids["lorentz"], pr, precision, loss="soft_l1", f_scale=0.2, **TOL)
    assert relerr(out["popt"], ref["popt"]) <= (1e-8 if precision == "fp64" else 1e-6)


def test_user_models_rejected_where_unsupported(ids):
    pr = synth.user_family("lorentz1d", 5000, seed=9).astype(np.float32)
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.evaluate_noalloc(ids["lorentz"], dev(pr.x, torch.float32), dev(pr.y, torch.float32), pr.p0,
                               precision="mixed")
    assert e.value.code == gbfit.E_UNSUPPORTED
