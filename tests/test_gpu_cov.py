"""Full-covariance fits on the GPU (Appendix C, Eqs. covariance, slsq1,
slsq2) against the FP64 oracle (Cholesky factor and triangular solves).

Tolerances:
  fixed-p whitened sums   plain 1e-10 relative to each entry's scale (the GPU
                          applies X = L^-1 formed by forward substitution, the
                          oracle solves with L: rounding differs by cond(L) eps);
                          mixed 5e-5 (FP32 X, FP32 row sums)
  whole fits              plain popt / cost 1e-8 with the same nfev and status,
                          pcov 1e-6; mixed popt 1e-6
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reduce as red, trf
from paper_2208_12187_gb300 import build, gbfit, synth

pytestmark = pytest.mark.gpu
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


def dev(a, dtype):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


def gpu_fit(pr, precision, cov_on_device=True, **kw):
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = None if pr.layout == synth.LAYOUT_GRID else dev(pr.x, dt)
    C = dev(pr.sigma, torch.float64) if cov_on_device else pr.sigma
    return gbfit.curve_fit(pr.model, x, dev(pr.y, dt), pr.p0, sigma=C, lb=pr.lb, ub=pr.ub, grid_wh=pr.grid_wh,
                           precision=precision, **kw)


CASES = [
    ("gauss1d_1000", lambda: synth.with_covariance(synth.gauss1d(1000, seed=1), 0.5, 0.1, seed=2)),
    ("gauss1d_2053_ragged", lambda: synth.with_covariance(synth.gauss1d(2053, seed=3), 0.7, 0.1, seed=4)),
    ("dexp_1500", lambda: synth.with_covariance(synth.dexp(1500, seed=21), 0.4, 0.05, seed=6)),
    ("gauss2d_grid_48", lambda: synth.with_covariance(
        synth.gauss2d_grid(48, seed=4, dtype=np.float64, truth=[980.0, 24.3, 23.1, 6.0, 4.0, 0.4, 20.0]),
        0.5, 5.0, seed=8)),
]


@pytest.mark.parametrize("name,make", CASES[:2] + CASES[3:])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_whitened_sums_match_oracle(name, make, precision):
    pr = make()
    if precision == "mixed":
        pr = pr.astype(np.float32)
    f, g, B, _, _ = red.evaluate(pr.model, pr.coords(), pr.y.astype(np.float64), red.weights(pr.sigma, pr.m), pr.p0)
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = None if pr.layout == synth.LAYOUT_GRID else dev(pr.x, dt)
    Bp, gg, cost = gbfit.evaluate(pr.model, x, dev(pr.y, dt), pr.p0, sigma=dev(pr.sigma, torch.float64),
                                  grid_wh=pr.grid_wh, precision=precision)
    Bg = gbfit.unpack_upper(Bp, pr.n)
    tol = 1e-10 if precision == "fp64" else 5e-5
    dscale = np.sqrt(np.outer(np.diag(B), np.diag(B)))
    assert np.max(np.abs(Bg - B) / np.maximum(dscale, 1e-300)) <= tol
    gscale = np.sqrt(np.diag(B) * 2 * f)
    assert np.max(np.abs(gg - g) / np.maximum(gscale, 1e-300)) <= tol
    assert abs(cost - f) <= tol * f


@pytest.mark.parametrize("name,make", CASES)
def test_plain_cov_fit_matches_oracle(name, make):
    pr = make()
    ref = trf.curve_fit(pr.model, pr.coords(), pr.y, pr.sigma, pr.p0, pr.lb, pr.ub, **TOL)
    out = gpu_fit(pr, "fp64", **TOL)
    assert out["status"] == ref["status"] and out["nfev"] == ref["nfev"]
    assert relerr(out["popt"], ref["popt"]) <= 1e-8
    assert out["cost"] == pytest.approx(ref["cost"], rel=1e-8)
    np.testing.assert_allclose(out["pcov"], ref["pcov"], rtol=1e-6, atol=1e-12 * np.max(np.abs(ref["pcov"])))


@pytest.mark.parametrize("name,make", CASES[:2] + CASES[3:])
def test_mixed_cov_fit_matches_oracle(name, make):
    pr = make().astype(np.float32)
    ref = trf.curve_fit(pr.model, pr.coords(), pr.y, pr.sigma, pr.p0, pr.lb, pr.ub, **TOL)
    out = gpu_fit(pr, "mixed", **TOL)
    assert out["status"] > 0
    assert relerr(out["popt"], ref["popt"]) <= 1e-6


def test_host_covariance_equals_device_covariance():
    pr = CASES[0][1]()
    a = gpu_fit(pr, "fp64", cov_on_device=True, **TOL)
    b = gpu_fit(pr, "fp64", cov_on_device=False, **TOL)
    np.testing.assert_array_equal(a["popt"], b["popt"])


def test_diagonal_covariance_equals_sigma_path():
    pr = synth.gauss1d(1500, seed=9)
    sig = np.random.default_rng(10).uniform(0.05, 0.2, pr.m)
    x, y = dev(pr.x, torch.float64), dev(pr.y, torch.float64)
    a = gbfit.curve_fit(pr.model, x, y, pr.p0, sigma=dev(sig, torch.float64), precision="fp64", **TOL)
    b = gbfit.curve_fit(pr.model, x, y, pr.p0, sigma=np.diag(sig ** 2), precision="fp64", **TOL)
    assert a["nfev"] == b["nfev"]
    assert relerr(b["popt"], a["popt"]) <= 1e-10
    np.testing.assert_allclose(b["pcov"], a["pcov"], rtol=1e-8)


def test_not_positive_definite_is_rejected():
    pr = synth.gauss1d(300, seed=11)
    C = np.eye(pr.m)
    C[5, 5] = -1.0
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.curve_fit(pr.model, dev(pr.x, torch.float64), dev(pr.y, torch.float64), pr.p0, sigma=C,
                        precision="fp64")
    assert e.value.code == gbfit.E_INVALID_ARG
    # the context stays usable
    out = gpu_fit(CASES[0][1](), "fp64", **TOL)
    assert out["status"] > 0


def test_cov_with_robust_loss_is_unsupported():
    pr = CASES[0][1]()
    with pytest.raises(gbfit.GbfitError) as e:
        gpu_fit(pr, "fp64", loss="soft_l1")
    assert e.value.code == gbfit.E_UNSUPPORTED
