"""Pins for oracle/models.py: analytic partials against central differences.

Section 2 (Eq. jacobian) defines J_ij = d r_i / d x_j; the oracle writes the
partials out by hand, so each is checked against a numerical derivative of the
model value alone (which uses none of the partial formulas).
"""
import numpy as np
import pytest

from oracle import models

RNG = np.random.default_rng(1234)

CASES = [
    (models.GAUSS1D, np.array([5.0, 0.3, 1.2, 0.5]), lambda m: RNG.uniform(-4, 4, (1, m))),
    (models.DEXP, np.array([3.0, 0.7, 6.5, 4.0, 0.2]), lambda m: RNG.uniform(0, 10, (1, m))),
    (models.GAUSS2D, np.array([9.0, 1.3, -0.7, 2.0, 1.1, 0.4, 0.5]),
     lambda m: RNG.uniform(-4, 4, (2, m))),
    (models.POLY2, np.array([1.5, -0.7, 0.25]), lambda m: RNG.uniform(-3, 3, (1, m))),
]


@pytest.mark.parametrize("model,p,xgen", CASES)
def test_partials_match_central_differences(model, p, xgen):
    X = xgen(64)
    h, J = models.value_and_jac(model, X, p)
    assert J.shape == (64, p.size)
    for j in range(p.size):
        step = 1e-6 * max(1.0, abs(p[j]))
        pp, pm = p.copy(), p.copy()
        pp[j] += step
        pm[j] -= step
        fd = (models.value_and_jac(model, X, pp)[0] - models.value_and_jac(model, X, pm)[0]) / (2 * step)
        scale = max(1.0, np.max(np.abs(fd)))
        assert np.max(np.abs(fd - J[:, j])) <= 1e-7 * scale, (model, j)


def test_gauss2d_rotation_reduces_to_axis_aligned():
    """theta = 0: u = X-x0, v = Y-y0, a product of two 1D Gaussians."""
    X = RNG.uniform(-3, 3, (2, 50))
    p = np.array([2.0, 0.5, -0.25, 1.5, 0.8, 0.0, 0.1])
    h, _ = models.value_and_jac(models.GAUSS2D, X, p)
    ref = 2.0 * np.exp(-(X[0] - 0.5) ** 2 / (2 * 1.5 ** 2)) * np.exp(-(X[1] + 0.25) ** 2 / (2 * 0.8 ** 2)) + 0.1
    np.testing.assert_allclose(h, ref, rtol=1e-14)


def test_gauss2d_symmetry_swap_axes():
    """(sx, sy, th) and (sy, sx, th + pi/2) describe the same surface (two equivalent optima)."""
    X = RNG.uniform(-3, 3, (2, 50))
    p = np.array([2.0, 0.5, -0.25, 1.5, 0.8, 0.3, 0.1])
    q = p.copy()
    q[3], q[4], q[5] = p[4], p[3], p[5] + np.pi / 2
    np.testing.assert_allclose(models.value_and_jac(models.GAUSS2D, X, p)[0],
                               models.value_and_jac(models.GAUSS2D, X, q)[0], rtol=1e-13)


def test_gauss1d_peak_and_offset():
    """At x = mu the value is A + c and the mu-partial vanishes."""
    p = np.array([5.0, 0.3, 1.2, 0.5])
    h, J = models.value_and_jac(models.GAUSS1D, np.array([[0.3]]), p)
    assert h[0] == pytest.approx(5.5, rel=1e-15)
    assert J[0, 1] == 0.0 and J[0, 2] == 0.0 and J[0, 0] == 1.0 and J[0, 3] == 1.0


def test_poly2_exact():
    X = RNG.uniform(-3, 3, (1, 20))
    h, J = models.value_and_jac(models.POLY2, X, [1.0, 2.0, 3.0])
    np.testing.assert_array_equal(J[:, 0], 1.0)
    np.testing.assert_array_equal(J[:, 1], X[0])
    np.testing.assert_allclose(h, 1 + 2 * X[0] + 3 * X[0] ** 2, rtol=1e-15)


def test_dexp_limits():
    """x = 0: h = a1 + a2 + c and the t-partials vanish."""
    h, J = models.value_and_jac(models.DEXP, np.zeros((1, 1)), [3.0, 0.7, 6.5, 4.0, 0.2])
    assert h[0] == pytest.approx(9.7, rel=1e-15)
    assert J[0, 1] == 0.0 and J[0, 3] == 0.0
