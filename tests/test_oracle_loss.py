"""Pins of the oracle's robust losses (reading R14; Section 5 names loss
functions without stating them).

- each rho' and rho'' equals central differences of rho (every loss);
- the rescaled rows give the exact gradient of the robust cost (central
  differences of f(p)) and its Gauss-Newton Hessian;
- linear loss == no loss; a very large f_scale reduces any loss to linear;
- gross outliers: every robust loss recovers the truth far better than the
  linear one;
- the fitted optimum equals SciPy least_squares with the same loss (a library
  run, different trust-region details, the same minimiser).
"""
import numpy as np
import pytest

from oracle import models, reduce as red, trf
from paper_2208_12187_gb300 import synth

TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)
ROBUST = ("soft_l1", "huber", "cauchy", "arctan")


@pytest.mark.parametrize("loss", red.LOSSES)
def test_rho_derivatives_central_differences(loss):
    z = np.array([0.01, 0.3, 0.9, 1.7, 4.0, 25.0])          # both sides of huber's knee
    h = 1e-6 * np.maximum(z, 1e-3)
    rho, r1, r2 = red.loss_rho(loss, z)
    rp, r1p, _ = red.loss_rho(loss, z + h)
    rm, r1m, _ = red.loss_rho(loss, z - h)
    np.testing.assert_allclose(r1, (rp - rm) / (2 * h), rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(r2, (r1p - r1m) / (2 * h), rtol=1e-5, atol=1e-9)
    assert np.all(r1 > 0)                                    # all losses increase


@pytest.mark.parametrize("loss", ROBUST)
def test_rescaled_rows_give_gradient_and_gn_hessian(loss):
    pr = synth.gauss1d(400, seed=3, noise=0.5)
    X, w = pr.coords(), red.weights(None, pr.m)
    C = 0.4
    p = pr.p0.copy()
    f, g, B, rt, Jt = red.evaluate(pr.model, X, pr.y, w, p, loss, C)
    cost = lambda q: red.evaluate(pr.model, X, pr.y, w, q, loss, C)[0]
    for j in range(pr.n):
        e = np.zeros(pr.n)
        e[j] = 1e-6 * max(abs(p[j]), 1.0)
        fd = (cost(p + e) - cost(p - e)) / (2 * e[j])
        assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    r, J = red.residual_and_jac(pr.model, X, pr.y, w, p)
    z = (r / C) ** 2
    _, r1, r2 = red.loss_rho(loss, z)
    s = np.maximum(r1 + 2 * z * r2, red.EPS)
    np.testing.assert_allclose(B, J.T @ (s[:, None] * J), rtol=1e-12, atol=1e-12 * np.abs(B).max())


def test_linear_loss_and_large_f_scale_reduce_to_plain_least_squares():
    pr = synth.dexp(3000, seed=4, dtype=np.float64)
    base = trf.curve_fit_problem(pr, **TOL)
    lin = trf.curve_fit_problem(pr, loss="linear", f_scale=3.0, **TOL)
    np.testing.assert_array_equal(base["popt"], lin["popt"])
    for loss in ROBUST:
        big = trf.curve_fit_problem(pr, loss=loss, f_scale=1e6, **TOL)
        rel = np.max(np.abs(big["popt"] - base["popt"]) / np.maximum(np.abs(base["popt"]), 1.0))
        assert rel <= 1e-6, loss


def _with_outliers(seed=7):
    pr = synth.gauss1d(2000, seed=seed, noise=0.05)
    rng = np.random.default_rng(seed)
    idx = rng.choice(pr.m, size=100, replace=False)          # 5 % gross outliers
    y = pr.y.copy()
    y[idx] += rng.uniform(2.0, 6.0, size=idx.size)
    pr.y = y
    return pr


@pytest.mark.parametrize("loss", ROBUST)
def test_robust_losses_resist_outliers(loss):
    pr = _with_outliers()
    lin = trf.curve_fit_problem(pr, **TOL)
    rob = trf.curve_fit_problem(pr, loss=loss, f_scale=0.1, **TOL)
    err = lambda p: np.max(np.abs(p - pr.truth) / np.abs(pr.truth))
    assert err(rob["popt"]) < 0.2 * err(lin["popt"]), (err(rob["popt"]), err(lin["popt"]))


@pytest.mark.parametrize("loss", ROBUST)
def test_matches_scipy_least_squares_with_loss(loss):
    scipy_opt = pytest.importorskip("scipy.optimize")
    pr = _with_outliers(11)
    X, w = pr.coords(), red.weights(None, pr.m)
    fun = lambda p: red.residual_and_jac(pr.model, X, pr.y, w, p)[0]
    jac = lambda p: red.residual_and_jac(pr.model, X, pr.y, w, p)[1]
    ref = scipy_opt.least_squares(fun, pr.p0, jac=jac, method="trf", loss=loss, f_scale=0.1, **TOL)
    out = trf.curve_fit_problem(pr, loss=loss, f_scale=0.1, **TOL)
    rel = np.abs(out["popt"] - ref.x) / np.maximum(np.abs(ref.x), 1.0)
    assert rel.max() <= 1e-6
    assert out["cost"] == pytest.approx(ref.cost, rel=1e-9)
