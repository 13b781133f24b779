"""Pins for the oracle's variable scaling D (reading R7 of the paper's
"usually diagonal" D, Section 2 Eq. hat, and the Jacobian scaling named in
Section 5).

D enters the method in three places: the initial radius Delta0 = ||D x0||
(R6), the trust region ||D w|| <= Delta, and the damped step of Eq. lm,
which in unscaled variables reads (J^T J + alpha D^2) w = -J^T r.  These tests
recompute all three from the recorded trials with J evaluated independently of
the fit, so that an inverted D (x_scale where 1/x_scale belongs), a D that is
not a running maximum, or a zero column norm not read as 1 fails here.
"""
import math

import numpy as np
import pytest

from oracle import reduce as red, trf
from paper_2208_12187_gb300 import synth

TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)


def _jac(pr, p):
    """Jacobian at p by central differences of the oracle's residual
    (independent of the analytic partials the fit uses)."""
    X, w = pr.coords(), red.weights(pr.sigma, pr.m)
    r0 = red.residual_and_jac(pr.model, X, pr.y, w, p)[0]
    J = np.empty((r0.size, p.size))
    for j in range(p.size):
        h = 1e-6 * max(abs(p[j]), 1.0)
        e = np.zeros_like(p)
        e[j] = h
        rp = red.residual_and_jac(pr.model, X, pr.y, w, p + e)[0]
        rm = red.residual_and_jac(pr.model, X, pr.y, w, p - e)[0]
        J[:, j] = (rp - rm) / (2 * h)
    return J, r0


def test_jac_scale_inv_scripted_sequence():
    """Running maximum of column norms over the Jacobians seen, zeros read as 1 (R7)."""
    def cols(*norms):
        # a 4 x 3 Jacobian whose column j has norm norms[j] (entries 0.6 n, 0.8 n)
        J = np.zeros((4, 3))
        for j, nv in enumerate(norms):
            J[j, j], J[j + 1, j] = 0.6 * nv, 0.8 * nv
        return J
    s1 = trf.jac_scale_inv(cols(3.0, 0.0, 5.0))
    np.testing.assert_allclose(s1, [3.0, 1.0, 5.0], rtol=1e-15)
    s2 = trf.jac_scale_inv(cols(1.0, 2.0, 7.0), s1)
    np.testing.assert_allclose(s2, [3.0, 2.0, 7.0], rtol=1e-15)
    s3 = trf.jac_scale_inv(cols(4.0, 0.0, 0.0), s2)
    np.testing.assert_allclose(s3, [4.0, 2.0, 7.0], rtol=1e-15)
    # a column that was zero reads 1 afterwards; later norms below 1 keep it at 1
    s4 = trf.jac_scale_inv(cols(0.5, 0.25, 0.0), np.array([1.0, 1.0, 1.0]))
    np.testing.assert_allclose(s4, [1.0, 1.0, 1.0], rtol=1e-15)
    # the previous vector is not modified in place
    np.testing.assert_allclose(s1, [3.0, 1.0, 5.0], rtol=1e-15)


def _start(pr, p0):
    import dataclasses
    return dataclasses.replace(pr, p0=np.asarray(p0, dtype=np.float64))


def _check_damped_steps(pr, hist, dvec_of):
    """Every trial: ||D w|| <= (1 + 0.1) Delta (Algorithm 2 stops within
    sigma Delta of the boundary, R1); the damped steps (alpha > 0) solve
    (J^T J + alpha D^2) w = -g and sit on the boundary within that band.
    Returns the number of damped steps."""
    n_damped = 0
    for k, h in enumerate(hist):
        D = dvec_of(k)
        w = h["step"]
        assert np.linalg.norm(D * w) <= 1.1 * h["Delta"] * (1 + 1e-9)
        if h["alpha"] <= 0:
            continue
        n_damped += 1
        assert abs(np.linalg.norm(D * w) - h["Delta"]) <= 0.1 * h["Delta"] * (1 + 1e-9)
        J, r = _jac(pr, h["x"])
        Bw = J.T @ (J @ w)
        damp = h["alpha"] * D * D * w
        g = J.T @ r
        # scale of the three terms (difference Jacobian: ~1e-9 relative error)
        scale = np.linalg.norm(Bw) + np.linalg.norm(damp) + np.linalg.norm(g)
        assert np.linalg.norm(Bw + damp + g) <= 1e-6 * scale
        # the damping term is not negligible (so that D is really tested)
        assert np.linalg.norm(damp) >= 1e-3 * scale
    return n_damped


def test_numeric_x_scale_is_inverse_D():
    """x_scale = s gives D = diag(1/s): Delta0 = ||x0 / s||, region ||w / s|| <= Delta,
    damping alpha diag(1/s^2)."""
    # D = 1/x_scale is large on mu, whose start is close to 0 but 0.4 from the
    # optimum: the first steps are limited by the region (alpha > 0)
    pr = _start(synth.gauss1d(4000, seed=3), [6.5, -0.1, 0.96, 0.75])
    xs = np.array([100.0, 0.01, 100.0, 100.0])
    out = trf.curve_fit_problem(pr, x_scale=xs, record=True, **TOL)
    hist = out["history"]
    assert hist[0]["Delta"] == pytest.approx(np.linalg.norm(pr.p0 / xs), rel=1e-14)
    n_damped = _check_damped_steps(pr, hist, lambda k: 1.0 / xs)
    assert n_damped >= 2
    assert out["status"] in (1, 2, 3, 4)


def test_jac_x_scale_is_running_column_norm_max():
    """x_scale = 'jac' gives D_j = running max over accepted iterates of ||J_:j||."""
    # A and c start near 0 (Delta0 = ||D x0|| small), far from their optimum
    pr = _start(synth.gauss1d(3000, seed=5), [0.5, -0.1, 1.0, 0.05])
    out = trf.curve_fit_problem(pr, x_scale="jac", record=True, **TOL)
    hist = out["history"]
    # the test's own running maximum over the accepted iterates
    Ds, c = [], None
    for h in hist:
        if c is None:
            J, _ = _jac(pr, h["x"])
            c = np.sqrt(np.sum(J * J, axis=0))
            c[c == 0] = 1.0
        Ds.append(c.copy())
        if h["accepted"]:
            J, _ = _jac(pr, h["x_new"])
            c = np.maximum(c, np.sqrt(np.sum(J * J, axis=0)))
    assert hist[0]["Delta"] == pytest.approx(np.linalg.norm(Ds[0] * pr.p0), rel=1e-6)
    n_damped = _check_damped_steps(pr, hist, lambda k: Ds[k])
    assert n_damped >= 1
    assert out["status"] in (1, 2, 3, 4)


@pytest.mark.parametrize("x_scale", ["jac", "vec"])
def test_scaled_fit_invariants_bounded(x_scale):
    """Bounded double exponential with a scaled region: monotone cost over
    accepted steps, strict feasibility, the model-reduction bound of
    Algorithm 3, and the bound-constrained first-order conditions at the end."""
    pr = synth.dexp(4000, seed=8, dtype=np.float64)
    xs = "jac" if x_scale == "jac" else np.array([1.0, 0.1, 3.0, 10.0, 0.5])
    out = trf.curve_fit_problem(pr, x_scale=xs, record=True, **TOL)
    hist = out["history"]
    acc = [h for h in hist if h["accepted"]]
    costs = [hist[0]["f"]] + [h["f_new"] for h in acc]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    assert all(h["f"] - h["f_new"] >= 0.25 * h["predicted"] * (1 - 1e-12) for h in acc)
    assert all(np.all(h["x_new"] > pr.lb) and np.all(h["x_new"] < pr.ub) for h in hist)
    J = red.evaluate(pr.model, pr.coords(), pr.y, red.weights(pr.sigma, pr.m), out["popt"])[4]
    gscale = np.sqrt(np.sum(J * J, axis=0)) * math.sqrt(2 * out["cost"])
    assert np.all(np.abs(out["v"] * out["g"]) <= 1e-5 * gscale)
    assert out["status"] in (1, 2, 3, 4)


@pytest.mark.parametrize("x_scale", ["jac", "vec"])
def test_scaled_fit_matches_scipy_minimiser(x_scale):
    """SciPy's least_squares with the same x_scale reaches the same optimum
    (a library run; scaling changes the path, not the minimiser)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    pr = synth.gauss1d(5000, seed=9)
    xs = "jac" if x_scale == "jac" else np.array([10.0, 0.1, 1.0, 0.01])
    X, w = pr.coords(), red.weights(pr.sigma, pr.m)
    fun = lambda p: red.residual_and_jac(pr.model, X, pr.y, w, p)[0]
    jac = lambda p: red.residual_and_jac(pr.model, X, pr.y, w, p)[1]
    ref = scipy_opt.least_squares(fun, pr.p0, jac=jac, method="trf", x_scale=xs, **TOL)
    out = trf.curve_fit_problem(pr, x_scale=xs, **TOL)
    rel = np.abs(out["popt"] - ref.x) / np.maximum(np.abs(ref.x), 1.0)
    assert rel.max() <= 1e-7
    assert out["cost"] == pytest.approx(ref.cost, rel=1e-10)
