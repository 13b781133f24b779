"""Pins of the oracle's full-covariance weighting (Appendix C, Eqs.
covariance, slsq1, slsq2), CPU.

The covariance path is fixed against: the diagonal special case (the sigma
path), the generalised-least-squares closed form of a model linear in p,
explicit whitening by the inverse Cholesky factor, and SciPy's curve_fit with
the same 2D sigma (a library run of the same problem).
"""
import numpy as np
import pytest

from oracle import reduce as red, trf
from paper_2208_12187_gb300 import synth

TOL = dict(ftol=1e-12, xtol=1e-12, gtol=1e-12)


def ar1_cov(m, rho, sig, seed=0):
    """C_ij = s_i s_j rho^|i-j| (a stationary exponential correlation) with per-point scales."""
    rng = np.random.default_rng(seed)
    s = sig * rng.uniform(0.5, 1.5, m)
    i = np.arange(m)
    return np.outer(s, s) * rho ** np.abs(i[:, None] - i[None, :])


def test_diagonal_covariance_is_the_sigma_path():
    pr = synth.gauss1d(600, seed=1)
    sig = np.random.default_rng(2).uniform(0.05, 0.2, pr.m)
    a = trf.curve_fit(pr.model, pr.coords(), pr.y, sig, pr.p0, **TOL)
    b = trf.curve_fit(pr.model, pr.coords(), pr.y, np.diag(sig ** 2), pr.p0, **TOL)
    assert a["nfev"] == b["nfev"] and a["status"] == b["status"]
    np.testing.assert_allclose(b["popt"], a["popt"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b["pcov"], a["pcov"], rtol=1e-9)
    assert b["cost"] == pytest.approx(a["cost"], rel=1e-12)


def test_linear_model_is_the_gls_solution():
    """poly2 with correlated errors: popt = (V^T C^-1 V)^-1 V^T C^-1 y, pcov = (V^T C^-1 V)^-1 (absolute)."""
    pr = synth.poly2(300, seed=3)
    x = pr.coords()[0]
    C = ar1_cov(pr.m, 0.6, 0.05, seed=4)
    out = trf.curve_fit(pr.model, pr.coords(), pr.y, C, pr.p0, absolute_sigma=True, **TOL)
    V = np.stack([np.ones_like(x), x, x * x], axis=1)
    Ci = np.linalg.inv(C)
    A = V.T @ Ci @ V
    beta = np.linalg.solve(A, V.T @ Ci @ pr.y)
    np.testing.assert_allclose(out["popt"], beta, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(out["pcov"], np.linalg.inv(A), rtol=1e-8)


def test_whitened_quantities_equal_explicit_inverse_factor():
    pr = synth.gauss1d(200, seed=5)
    C = ar1_cov(pr.m, 0.4, 0.1, seed=6)
    w = red.weights(C, pr.m)
    f, g, B, r, J = red.evaluate(pr.model, pr.coords(), pr.y, w, pr.p0)
    from oracle import models
    h, dh = models.value_and_jac(pr.model, pr.coords(), pr.p0)
    Li = np.linalg.inv(np.linalg.cholesky(C))
    rr = Li @ (h - pr.y)
    JJ = Li @ dh
    assert f == pytest.approx(0.5 * rr @ rr, rel=1e-10)
    np.testing.assert_allclose(g, JJ.T @ rr, rtol=1e-9)
    np.testing.assert_allclose(B, JJ.T @ JJ, rtol=1e-9)
    # the cost is the Mahalanobis form 1/2 r^T C^-1 r (Eq. covariance with W = C^-1)
    assert f == pytest.approx(0.5 * (h - pr.y) @ np.linalg.solve(C, h - pr.y), rel=1e-9)


def test_scipy_curve_fit_with_covariance():
    scipy_opt = pytest.importorskip("scipy.optimize")
    pr = synth.gauss1d(400, seed=7)
    C = ar1_cov(pr.m, 0.5, 0.1, seed=8)
    rng = np.random.default_rng(9)
    y = synth.forward_values(pr.model, pr.coords(), pr.truth) + np.linalg.cholesky(C) @ rng.normal(size=pr.m)
    out = trf.curve_fit(pr.model, pr.coords(), y, C, pr.p0, **TOL)
    f = lambda x, A, mu, s, c: A * np.exp(-(x - mu) ** 2 / (2 * s * s)) + c
    popt, pcov = scipy_opt.curve_fit(f, pr.coords()[0], y, p0=pr.p0, sigma=C, method="trf",
                                     ftol=1e-14, xtol=1e-14, gtol=1e-14)
    np.testing.assert_allclose(out["popt"], popt, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(out["pcov"], pcov, rtol=1e-5)


def test_covariance_scale_laws():
    """C -> k^2 C leaves popt unchanged; pcov scales by k^2 only with absolute_sigma."""
    pr = synth.gauss1d(300, seed=10)
    C = ar1_cov(pr.m, 0.3, 0.1, seed=11)
    a = trf.curve_fit(pr.model, pr.coords(), pr.y, C, pr.p0, **TOL)
    b = trf.curve_fit(pr.model, pr.coords(), pr.y, 9.0 * C, pr.p0, **TOL)
    np.testing.assert_allclose(b["popt"], a["popt"], rtol=1e-9)
    np.testing.assert_allclose(b["pcov"], a["pcov"], rtol=1e-8)
    aa = trf.curve_fit(pr.model, pr.coords(), pr.y, C, pr.p0, absolute_sigma=True, **TOL)
    bb = trf.curve_fit(pr.model, pr.coords(), pr.y, 9.0 * C, pr.p0, absolute_sigma=True, **TOL)
    np.testing.assert_allclose(bb["pcov"], 9.0 * aa["pcov"], rtol=1e-8)
