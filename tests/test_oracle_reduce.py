"""Pins for oracle/reduce.py: cost, gradient and Gram from their definitions.

g = J^T r (Eq. gradient) is checked against a finite-difference gradient of
the cost f = r^T r / 2 (Eq. msqe), which uses no partials; B = J^T J (Eq.
hessian) is checked against the finite-difference Hessian of f on noise-free
data, where the dropped term sum r_i grad^2 r_i vanishes.  The 1/sigma
weighting (Appendix C) is checked through its scaling laws.
"""
import numpy as np
import pytest

from oracle import models, reduce as red
from paper_2208_12187_gb300 import synth


def _cost(model, X, y, w, p):
    h, _ = models.value_and_jac(model, X, p)
    r = w * (h - y)
    return 0.5 * float(r @ r)


PROBLEMS = [
    lambda: synth.gauss1d(200, seed=2),
    lambda: synth.dexp(200, seed=5, dtype=np.float64),
    lambda: synth.gauss2d_grid(16, seed=3, dtype=np.float64),
    lambda: synth.poly2(100, seed=4),
]


@pytest.mark.parametrize("make", PROBLEMS)
def test_gradient_is_finite_difference_of_cost(make):
    pr = make()
    X, w = pr.coords(), red.weights(pr.sigma, pr.m)
    p = pr.p0
    f, g, B, r, J = red.evaluate(pr.model, X, pr.y, w, p)
    assert f == pytest.approx(_cost(pr.model, X, pr.y, w, p), rel=1e-15)
    for j in range(pr.n):
        hstep = 1e-6 * max(1.0, abs(p[j]))
        pp, pm = p.copy(), p.copy()
        pp[j] += hstep
        pm[j] -= hstep
        fd = (_cost(pr.model, X, pr.y, w, pp) - _cost(pr.model, X, pr.y, w, pm)) / (2 * hstep)
        assert fd == pytest.approx(g[j], rel=1e-6, abs=1e-6 * max(1.0, f)), j


@pytest.mark.parametrize("make", PROBLEMS[:3])
def test_gram_is_hessian_on_noise_free_data(make):
    pr = make()
    X, w = pr.coords(), red.weights(pr.sigma, pr.m)
    p = pr.truth
    y0, _ = models.value_and_jac(pr.model, X, p)      # residual exactly zero at p
    _, _, B, _, _ = red.evaluate(pr.model, X, y0, w, p)
    n = pr.n
    H = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            hi = 1e-4 * max(1.0, abs(p[i]))
            hj = 1e-4 * max(1.0, abs(p[j]))
            def fpp(a, b):
                q = p.copy()
                q[i] += a
                q[j] += b
                return _cost(pr.model, X, y0, w, q)
            H[i, j] = (fpp(hi, hj) - fpp(hi, -hj) - fpp(-hi, hj) + fpp(-hi, -hj)) / (4 * hi * hj)
    scale = np.max(np.abs(B))
    assert np.max(np.abs(H - B)) <= 1e-5 * scale


def test_split_pieces_sum_to_whole():
    pr = synth.gauss1d(1001, seed=9)
    X, w = pr.coords(), red.weights(pr.sigma, pr.m)
    f, g, B, _, _ = red.evaluate(pr.model, X, pr.y, w, pr.p0)
    parts = [red.evaluate(pr.model, X[:, a:b], pr.y[a:b], w[a:b], pr.p0) for a, b in ((0, 333), (333, 1001))]
    assert f == pytest.approx(sum(q[0] for q in parts), rel=1e-13)
    np.testing.assert_allclose(g, sum(q[1] for q in parts), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(B, sum(q[2] for q in parts), rtol=1e-12)


def test_sigma_scaling_laws():
    """sigma -> k sigma scales f by 1/k^2, g by 1/k^2 and B by 1/k^2 (Eq. explicit)."""
    pr = synth.poly2(300, seed=1)
    X = pr.coords()
    k = 3.0
    f1, g1, B1, _, _ = red.evaluate(pr.model, X, pr.y, red.weights(pr.sigma, pr.m), pr.p0)
    f2, g2, B2, _, _ = red.evaluate(pr.model, X, pr.y, red.weights(k * pr.sigma, pr.m), pr.p0)
    assert f2 == pytest.approx(f1 / k ** 2, rel=1e-13)
    np.testing.assert_allclose(g2, g1 / k ** 2, rtol=1e-12)
    np.testing.assert_allclose(B2, B1 / k ** 2, rtol=1e-12)


def test_masked_points_contribute_nothing():
    """Appendix A: padded dummy points (weight 0) leave f, g, B unchanged."""
    pr = synth.gauss1d(500, seed=4)
    X, w = pr.coords(), red.weights(pr.sigma, pr.m)
    Xp = np.concatenate([X, np.full((1, 77), 123.0)], axis=1)
    yp = np.concatenate([pr.y, np.full(77, -5.0)])
    wp = np.concatenate([w, np.zeros(77)])
    a = red.evaluate(pr.model, X, pr.y, w, pr.p0)
    b = red.evaluate(pr.model, Xp, yp, wp, pr.p0)
    # equal up to the summation order of the library dot product
    assert a[0] == pytest.approx(b[0], rel=1e-14)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a[2], b[2], rtol=1e-13)


def test_packed_upper_layout():
    B = np.arange(16.0).reshape(4, 4)
    B = B + B.T
    pk = red.packed_upper(B)
    assert pk.size == 10
    assert list(pk[:4]) == list(B[0]) and pk[4] == B[1, 1] and pk[-1] == B[3, 3]
