"""Pins of the oracle's user-defined-model path (CPU).

A user model reaches the oracle as a NumPy callable (X, p) -> (h, dh/dp).
These tests fix that path against things other than itself: central
differences for each test model's partials, the built-in model it repeats,
a model linear in p against its closed form, and noise-free data.
"""
import numpy as np
import pytest

from oracle import models, reduce as red, trf
from paper_2208_12187_gb300 import synth
from user_model_defs import gauss2d_axis_np, lorentz_np, zoo_np, zoo_value, ZOO_P

TOL = dict(ftol=1e-12, xtol=1e-12, gtol=1e-12)


def central_diff(f, X, p, rel=1e-6):
    p = np.asarray(p, dtype=np.float64)
    J = np.empty((X.shape[1], p.size))
    for j in range(p.size):
        h = rel * max(abs(p[j]), 1.0)
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        J[:, j] = (f(X, pp)[0] - f(X, pm)[0]) / (2 * h)
    return J


@pytest.mark.parametrize("fam,fn", [("lorentz1d", lorentz_np), ("gauss2d_axis", gauss2d_axis_np)])
def test_user_model_partials_match_central_differences(fam, fn):
    pr = synth.user_family(fam, 900, seed=3)
    X = pr.coords()
    for p in (pr.truth, pr.p0):
        h, J = fn(X, p)
        Jc = central_diff(fn, X, p)
        scale = np.maximum(np.abs(J).max(axis=0), 1e-12)
        assert np.max(np.abs(J - Jc) / scale) < 1e-7


def test_complex_step_partials_match_central_differences():
    """The zoo model's complex-step Jacobian (the oracle side of the dual-number test)."""
    X = np.linspace(0.1, 2.0, 301)[None, :]
    h, J = zoo_np(X, ZOO_P)
    Jc = central_diff(lambda X, p: (np.real(zoo_value(X, p)), None), X, ZOO_P)
    scale = np.maximum(np.abs(J).max(axis=0), 1e-12)
    assert np.max(np.abs(J - Jc) / scale) < 1e-7


def test_callable_equal_to_builtin_gives_the_builtin_fit():
    pr = synth.gauss1d(3000, seed=5)
    a = trf.curve_fit(pr.model, pr.coords(), pr.y, None, pr.p0, **TOL)
    b = trf.curve_fit(models.gauss1d, pr.coords(), pr.y, None, pr.p0, **TOL)
    assert a["nfev"] == b["nfev"] and a["status"] == b["status"]
    np.testing.assert_array_equal(a["popt"], b["popt"])
    assert a["cost"] == b["cost"]


def test_linear_user_model_is_the_weighted_least_squares_solution():
    """A cubic (linear in p) given as a callable: the fit is the normal-equations solution."""
    rng = np.random.default_rng(11)
    x = rng.uniform(-2, 2, 400)
    X = x[None, :]
    sig = rng.uniform(0.5, 2.0, 400)
    y = 1.0 - 0.5 * x + 0.25 * x ** 2 + 0.125 * x ** 3 + rng.normal(0, 0.05, 400) * sig

    def cubic(X, p):
        V = np.stack([np.ones_like(X[0]), X[0], X[0] ** 2, X[0] ** 3], axis=1)
        return V @ p, V

    out = trf.curve_fit(cubic, X, y, sig, np.zeros(4), **TOL)
    V = np.stack([np.ones_like(x), x, x ** 2, x ** 3], axis=1) / sig[:, None]
    ref = np.linalg.lstsq(V, y / sig, rcond=None)[0]
    np.testing.assert_allclose(out["popt"], ref, rtol=1e-10, atol=1e-12)


def test_noise_free_user_model_recovers_truth():
    pr = synth.user_family("lorentz1d", 2000, seed=2)
    X = pr.coords()
    y = lorentz_np(X, pr.truth)[0]
    out = trf.curve_fit(lorentz_np, X, y, None, pr.p0, **TOL)
    np.testing.assert_allclose(out["popt"], pr.truth, rtol=1e-8)


def test_user_model_reduction_follows_definitions():
    """f, g and B of a callable model equal their definitions from (h, J)."""
    pr = synth.user_family("gauss2d_axis", 1600, seed=4, with_sigma=True)
    X = pr.coords()
    w = red.weights(pr.sigma, pr.m)
    f, g, B, r, J = red.evaluate(gauss2d_axis_np, X, pr.y, w, pr.p0)
    h, dh = gauss2d_axis_np(X, pr.p0)
    rr = w * (h - pr.y)
    JJ = w[:, None] * dh
    assert f == pytest.approx(0.5 * rr @ rr, rel=1e-14)
    np.testing.assert_allclose(g, JJ.T @ rr, rtol=1e-12)
    np.testing.assert_allclose(B, JJ.T @ JJ, rtol=1e-12)
