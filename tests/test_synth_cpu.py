"""The seeded input generators follow their stated recipes.

The benchmarks and parity tests stand in synthetic data for the paper's
workloads (Section 4 draws its own synthetic 2D Gaussians; the configs add a
1D Gaussian sweep, a ragged double-exponential batch and a mixed serving
stream).  These checks pin each recipe: coordinate ranges, noise levels,
parameter ranges, the seed perturbation, bounds, size distributions and the
model mix, and that a seed fixes every array.  Observations are checked
against the oracle's own model values (written independently of the
generators' forward lines).
"""
import math

import numpy as np
import pytest

from oracle import models
from paper_2208_12187_gb300 import synth


def model_values(pr, p):
    return models.value_and_jac(pr.model, pr.coords(), p)[0]


def test_gauss1d_recipe():
    pr = synth.gauss1d(20_000, seed=0)
    assert pr.model == synth.MODEL_GAUSS1D and pr.m == 20_000 and pr.sigma is None
    assert pr.x.min() >= -10.0 and pr.x.max() <= 10.0
    np.testing.assert_array_equal(pr.truth, [5.0, 0.3, 1.2, 0.5])
    e = pr.y - model_values(pr, pr.truth)
    assert abs(e.std() - 0.1) < 0.005 and abs(e.mean()) < 0.005
    assert np.all(np.abs(pr.p0 / pr.truth - 1.0) <= 0.2)
    again = synth.gauss1d(20_000, seed=0)
    np.testing.assert_array_equal(again.x, pr.x)
    np.testing.assert_array_equal(again.y, pr.y)
    np.testing.assert_array_equal(again.p0, pr.p0)
    assert not np.array_equal(synth.gauss1d(20_000, seed=1).y, pr.y)
    f32 = synth.gauss1d(20_000, seed=0, dtype=np.float32)
    assert f32.x.dtype == np.float32 and f32.y.dtype == np.float32
    np.testing.assert_array_equal(f32.y, pr.y.astype(np.float32))
    assert np.all(synth.gauss1d(100, seed=0, with_sigma=True).sigma == 1.0)


def test_gauss2d_grid_recipe_1024():
    pr = synth.gauss2d_grid(1024, seed=0, dtype=np.float64)
    assert pr.layout == synth.LAYOUT_GRID and pr.grid_wh == (1024, 1024) and pr.m == 1024 * 1024
    A, x0, y0, sx, sy, th, c = pr.truth
    assert (A, c, sx, sy, th) == (980.0, 20.0, 60.0, 35.0, 0.4)
    # Poisson counts: integers, background 20 far from the centre, peak near 1000
    assert np.all(pr.y == np.round(pr.y)) and pr.y.min() >= 0
    X = pr.coords()
    far = np.hypot(X[0] - x0, X[1] - y0) > 8 * sx
    assert abs(pr.y[far].mean() - 20.0) < 0.2
    mu = model_values(pr, pr.truth)
    assert abs(mu.max() - 1000.0) < 1.0
    # Poisson: variance equals the mean
    z = (pr.y - mu) / np.sqrt(mu)
    assert abs(z.std() - 1.0) < 0.01 and abs(z.mean()) < 0.01
    np.testing.assert_array_equal(pr.sigma, np.sqrt(np.maximum(pr.y, 1.0)))
    np.testing.assert_array_equal(pr.lb, [-np.inf, -np.inf, -np.inf, 0.5, 0.5, -math.pi / 2, -np.inf])
    np.testing.assert_array_equal(pr.ub, [np.inf, np.inf, np.inf, 500.0, 500.0, math.pi / 2, np.inf])
    d = pr.p0 - pr.truth
    assert np.all(np.abs(pr.p0[[0, 3, 4, 6]] / pr.truth[[0, 3, 4, 6]] - 1) <= 0.2)
    assert np.all(np.abs(d[[1, 2]]) <= 5.0) and abs(d[5]) <= 0.1
    assert np.all(pr.p0 > pr.lb) and np.all(pr.p0 < pr.ub)
    soa = synth.gauss2d_grid(64, seed=3, layout=synth.LAYOUT_SOA2)
    grid = synth.gauss2d_grid(64, seed=3)
    np.testing.assert_array_equal(soa.coords(), grid.coords())
    np.testing.assert_array_equal(soa.y, grid.y)


def test_dexp_recipe():
    pr = synth.dexp(50_000, seed=21)
    a1, t1, a2, t2, c = pr.truth
    assert 0.1 <= min(t1, t2) and max(t1, t2) <= 100.0
    assert 1.0 <= min(a1, a2) and max(a1, a2) <= 10.0 and 0.0 <= c <= 1.0
    assert pr.x.min() >= 0.0 and pr.x.max() <= 5.0 * max(t1, t2)
    e = pr.y - model_values(pr, pr.truth)
    assert abs(e.std() / (0.01 * (a1 + a2 + c)) - 1.0) < 0.02
    np.testing.assert_array_equal(pr.lb, [-np.inf, 0.0, -np.inf, 0.0, -np.inf])
    assert np.all(np.isinf(pr.ub))
    assert np.all(np.abs(pr.p0 / pr.truth - 1.0) <= 0.2)


def test_dexp_batch_structure_and_size_distribution():
    bt = synth.dexp_batch(64, seed=7, m_lo=200, m_hi=20_000, dtype=np.float32)
    m = np.diff(bt.offsets)
    assert bt.offsets[0] == 0 and np.all(m >= 200) and np.all(m < 20_000)
    assert bt.x.shape == bt.y.shape == (bt.offsets[-1],) and bt.x.dtype == np.float32
    for k in (0, 31, 63):
        pr = bt.fit(k)
        assert pr.m == m[k] and pr.x.max() <= 5.0 * max(pr.truth[1], pr.truth[3]) * (1 + 1e-6)
        np.testing.assert_array_equal(pr.lb, [-np.inf, 0.0, -np.inf, 0.0, -np.inf])
    # log-uniform sizes: log m uniform on [log lo, log hi)
    rng = np.random.default_rng(0)
    s = synth.log_uniform_int(rng, 200, 200_000, 200_000)
    u = (np.log(s + 0.5) - math.log(200)) / math.log(1000)
    hist = np.histogram(u, bins=10, range=(0, 1))[0] / s.size
    assert np.all(np.abs(hist - 0.1) < 0.01)
    assert s.min() >= 200 and s.max() < 200_000


def test_serve_stream_mix_sizes_and_arrivals():
    st = synth.ServeStream(4000, seed=0, m_lo=1e3, m_hi=1e5, n_data=2)
    frac = {mdl: float(np.mean(st.models == mdl)) for mdl, _ in synth.SERVE_MIX}
    for mdl, w in synth.SERVE_MIX:
        assert abs(frac[mdl] - w) < 0.03
    assert np.all(st.m >= 1e3 * 0.8) and np.all(st.m <= 1e5 * 1.2)
    for k in range(0, 4000, 97):
        pr = st.request(k)
        assert pr.model == st.models[k] and pr.m == st.m[k]
        if pr.model == synth.MODEL_GAUSS2D:
            W = pr.grid_wh[0]
            assert W in st.ladder and pr.m == W * W
    t = synth.ServeStream.arrivals(20_000, 500.0, seed=1)
    assert np.all(np.diff(t) > 0) and abs(np.mean(np.diff(t)) * 500.0 - 1.0) < 0.03
    assert np.all(synth.ServeStream.arrivals(10, np.inf) == 0.0)


def test_correlated_errors_recipe():
    C = synth.ar1_covariance(400, 0.6, 0.2, seed=3)
    np.testing.assert_array_equal(C, C.T)
    s = np.sqrt(np.diag(C))
    assert np.all((s >= 0.1) & (s <= 0.3))
    np.testing.assert_allclose(C[np.arange(399), np.arange(1, 400)] / (s[:-1] * s[1:]), 0.6, rtol=1e-12)
    np.linalg.cholesky(C)                        # positive definite (raises otherwise)
    pr = synth.with_covariance(synth.gauss1d(3000, seed=4), 0.6, 0.2, seed=5)
    assert pr.sigma.shape == (3000, 3000)
    e = np.linalg.solve(np.linalg.cholesky(pr.sigma), pr.y - model_values(pr, pr.truth))
    assert abs(e.std() - 1.0) < 0.05 and abs(e.mean()) < 0.06
