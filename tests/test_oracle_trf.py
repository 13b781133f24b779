"""Pins for oracle/trf.py against what the paper and the mathematics fix.

Subproblem: the More-Sorensen conditions (Section 2, Eqs. lm and pbound), the
SVD identity of Appendix B (Eq. reducedlm against a direct linear solve), a
bisection root of phi (Eq. phi) and, for n = 2, brute-force minimisation of
the quadratic model over the disc.  Algorithm 3 by its table.  Whole fit: the
linear model's closed form (Section 2 notes linear problems solve
analytically), exact recovery on noise-free data, zero projected gradient,
monotone cost over accepted steps, feasibility, infinite bounds == unbounded,
and SciPy's least_squares minimiser (a library run that reaches the same
optimum by a different trust-region rule).
"""
import math

import numpy as np
import pytest

from oracle import models, reduce as red, trf
from paper_2208_12187_gb300 import synth

TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)


def _random_problem(rng, n, cond=1e3):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.exp(rng.uniform(0, math.log(cond), n))
    B = (Q * lam) @ Q.T
    g = rng.normal(size=n) * 10
    return B, g


def _eig_factors(B, g):
    lam, V = np.linalg.eigh(B)
    return lam, V, V.T @ g


# ------------------------------------------------------------- Algorithm 2
@pytest.mark.parametrize("seed", range(12))
def test_lm_parameter_more_sorensen(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    B, g = _random_problem(rng, n)
    lam, V, gV = _eig_factors(B, g)
    pt = -np.linalg.solve(B, g)
    Delta = np.linalg.norm(pt) * rng.uniform(0.05, 0.9)
    p, alpha = trf.tr_solve(lam, V, gV, np.linalg.norm(g), Delta, 0.0, True)
    assert alpha > 0
    # Eq. lm: (B + alpha I) p = -g, checked with a direct solve
    np.testing.assert_allclose(p, -np.linalg.solve(B + alpha * np.eye(n), g), rtol=1e-10, atol=1e-12)
    # Eq. pbound within Algorithm 2's accuracy sigma = 0.1
    assert abs(np.linalg.norm(p) - Delta) <= 0.1 * Delta
    # B + alpha I positive semidefinite
    assert np.linalg.eigvalsh(B + alpha * np.eye(n)).min() >= 0


@pytest.mark.parametrize("seed", range(6))
def test_lm_parameter_matches_bisection_root(seed):
    """alpha lies within the sigma-band around the exact root of phi."""
    rng = np.random.default_rng(100 + seed)
    n = 5
    B, g = _random_problem(rng, n)
    lam, V, gV = _eig_factors(B, g)
    Delta = np.linalg.norm(np.linalg.solve(B, g)) * 0.3

    def pnorm(a):
        return np.linalg.norm(np.linalg.solve(B + a * np.eye(n), g))
    lo, hi = 0.0, 1.0
    while pnorm(hi) > Delta:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if pnorm(mid) > Delta else (lo, mid)
    root = 0.5 * (lo + hi)
    alpha = trf.lm_parameter(lam, gV, np.linalg.norm(g), Delta, 0.0, True)
    # ||p|| is decreasing in alpha: the sigma-band maps to an alpha interval
    a_lo = root
    while pnorm(a_lo) < 1.1 * Delta and a_lo > 1e-300:
        a_lo *= 0.5
    assert pnorm(alpha) <= 1.1 * Delta + 1e-12 and pnorm(alpha) >= 0.9 * Delta - 1e-12
    assert alpha >= a_lo


def test_svd_identity_appendix_b():
    """p(alpha) from the thin SVD of J equals the normal-equation solution."""
    rng = np.random.default_rng(7)
    J = rng.normal(size=(50, 4))
    r = rng.normal(size=50)
    lam, V, gV, full = trf.scaled_svd(J, r, np.ones(4), None)
    assert full
    g = J.T @ r
    for a in (0.0, 0.3, 5.0):
        p = -V @ (gV / (lam + a))
        np.testing.assert_allclose(p, -np.linalg.solve(J.T @ J + a * np.eye(4), g), rtol=1e-11)


@pytest.mark.parametrize("seed", range(4))
def test_tr_step_is_disc_minimiser_n2(seed):
    """n = 2: the step minimises the model over the disc of its own radius."""
    rng = np.random.default_rng(200 + seed)
    B, g = _random_problem(rng, 2, cond=50)
    lam, V, gV = _eig_factors(B, g)
    Delta = np.linalg.norm(np.linalg.solve(B, g)) * 0.4
    p, _ = trf.tr_solve(lam, V, gV, np.linalg.norm(g), Delta, 0.0, True)
    q = lambda s: g @ s + 0.5 * s @ B @ s
    R = np.linalg.norm(p)
    t = np.linspace(0, 2 * np.pi, 20001)
    rad = np.linspace(0, R, 201)
    best = min(q(np.array([rr * math.cos(tt), rr * math.sin(tt)])) for rr in rad[::20] for tt in t[::50])
    ring = min(q(R * np.array([math.cos(tt), math.sin(tt)])) for tt in t)
    assert q(p) <= min(best, ring) + 1e-9 * abs(ring)


def test_rank_deficient_pseudo_inverse():
    """A null direction of J carries no step (R10)."""
    rng = np.random.default_rng(3)
    J = rng.normal(size=(40, 3))
    J[:, 2] = J[:, 0]                       # exact collinearity
    r = rng.normal(size=40)
    lam, V, gV, full = trf.scaled_svd(J, r, np.ones(3), None)
    assert not full and np.count_nonzero(lam) == 2
    p, _ = trf.tr_solve(lam, V, gV, np.linalg.norm(J.T @ r), 1e6, 0.0, full)
    np.testing.assert_allclose(p, -np.linalg.pinv(J) @ r, rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------- Algorithm 3
@pytest.mark.parametrize("gamma,acc,factor", [
    (0.9, True, 2.0), (0.76, True, 2.0), (0.75, True, 1.0), (0.5, True, 1.0),
    (0.25, True, 1.0), (0.2499, False, None), (-3.0, False, None), (float("nan"), False, None),
    (-math.inf, False, None)])
def test_radius_update_table(gamma, acc, factor):
    accepted, D = trf.tr_radius_update(gamma, 4.0, 2.0)
    assert accepted is acc
    assert D == (4.0 * factor if acc else 0.25 * 2.0)


# ------------------------------------------------------------- whole fits
def test_linear_model_closed_form():
    """poly2 is linear in p: the fit equals the weighted normal equations."""
    pr = synth.poly2(2000, seed=11)
    out = trf.curve_fit_problem(pr, **TOL)
    X = pr.coords()[0]
    A = np.stack([np.ones_like(X), X, X * X], axis=1) / pr.sigma[:, None]
    b = pr.y / pr.sigma
    ref = np.linalg.solve(A.T @ A, A.T @ b)
    np.testing.assert_allclose(out["popt"], ref, rtol=1e-10, atol=1e-12)
    assert out["status"] in (1, 2, 3, 4)
    # pcov of a linear problem: inv(A^T A) * 2f/(m-n)
    res = A @ ref - b
    cov = np.linalg.inv(A.T @ A) * (res @ res) / (pr.m - 3)
    np.testing.assert_allclose(out["pcov"], cov, rtol=1e-8)


@pytest.mark.parametrize("make", [
    lambda: synth.gauss1d(3000, seed=1, noise_free=True),
    lambda: synth.dexp(3000, seed=2, truth=[3.0, 0.5, 5.0, 4.0, 0.3], dtype=np.float64, noise_free=True),
    lambda: synth.gauss2d_grid(48, seed=5, dtype=np.float64, poisson=False),
])
def test_noise_free_recovers_truth(make):
    pr = make()
    out = trf.curve_fit_problem(pr, **TOL)
    np.testing.assert_allclose(out["popt"], pr.truth, rtol=1e-7, atol=1e-8)
    assert out["cost"] < 1e-12


@pytest.mark.parametrize("make", [
    lambda: synth.gauss1d(10_000, seed=0),
    lambda: synth.dexp(4000, seed=8, dtype=np.float64),
    lambda: synth.gauss2d_grid(64, seed=2, dtype=np.float64),
])
def test_invariants_along_the_fit(make):
    pr = make()
    out = trf.curve_fit_problem(pr, record=True, **TOL)
    hist = out["history"]
    acc = [h for h in hist if h["accepted"]]
    # monotone cost over accepted steps
    costs = [hist[0]["f"]] + [h["f_new"] for h in acc]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    # accepted steps really reduced the cost by >= 1/4 of the prediction
    assert all(h["f"] - h["f_new"] >= 0.25 * h["predicted"] * (1 - 1e-12) for h in acc)
    # feasibility of every trial point
    lb = pr.lb if pr.lb is not None else -np.inf
    ub = pr.ub if pr.ub is not None else np.inf
    assert all(np.all(h["x_new"] > lb) and np.all(h["x_new"] < ub) for h in hist)
    # projected (Coleman-Li scaled) gradient small at the end
    J = red.evaluate(pr.model, pr.coords(), pr.y, red.weights(pr.sigma, pr.m), out["popt"])[4]
    gscale = np.sqrt(np.sum(J * J, axis=0)) * math.sqrt(2 * out["cost"])
    assert np.all(np.abs(out["v"] * out["g"]) <= 1e-5 * gscale)
    assert out["status"] in (1, 2, 3, 4)


def test_infinite_bounds_equal_unbounded():
    pr = synth.gauss1d(2000, seed=6)
    a = trf.curve_fit_problem(pr, **TOL)
    b = trf.curve_fit(pr.model, pr.coords(), pr.y, pr.sigma, pr.p0,
                      np.full(4, -np.inf), np.full(4, np.inf), **TOL)
    np.testing.assert_array_equal(a["popt"], b["popt"])
    assert a["nfev"] == b["nfev"] and a["cost"] == b["cost"]


def test_sigma_ones_equals_none():
    pr = synth.gauss1d(2000, seed=6)
    a = trf.curve_fit_problem(pr, **TOL)
    b = trf.curve_fit(pr.model, pr.coords(), pr.y, np.ones(pr.m), pr.p0, **TOL)
    np.testing.assert_array_equal(a["popt"], b["popt"])


def test_sigma_scale_invariance():
    """sigma -> k sigma: same popt, cost / k^2, pcov unchanged unless absolute_sigma."""
    pr = synth.poly2(500, seed=3)
    a = trf.curve_fit_problem(pr, **TOL)
    b = trf.curve_fit(pr.model, pr.coords(), pr.y, 2.0 * pr.sigma, pr.p0, **TOL)
    np.testing.assert_allclose(a["popt"], b["popt"], rtol=1e-10)
    assert b["cost"] == pytest.approx(a["cost"] / 4, rel=1e-10)
    np.testing.assert_allclose(a["pcov"], b["pcov"], rtol=1e-8)


def test_active_bound_kkt():
    """Optimum on a bound: the fit stops there with the gradient pointing out."""
    pr = synth.gauss1d(4000, seed=12)
    lb = np.array([-np.inf, -np.inf, 0.2, -np.inf])
    ub = np.array([np.inf, np.inf, 1.0, np.inf])        # truth s = 1.2 lies outside
    p0 = pr.p0.copy()
    p0[2] = 0.8
    out = trf.curve_fit(pr.model, pr.coords(), pr.y, None, p0, lb, ub, **TOL)
    assert out["popt"][2] == pytest.approx(1.0, abs=1e-6)
    assert out["popt"][2] < 1.0
    assert out["g"][2] < 0                               # cost would fall past the bound
    free = [0, 1, 3]
    J = red.evaluate(pr.model, pr.coords(), pr.y, np.ones(pr.m), out["popt"])[4]
    gscale = np.sqrt(np.sum(J * J, axis=0)) * math.sqrt(2 * out["cost"])
    assert np.all(np.abs(out["g"][free]) <= 1e-5 * gscale[free])


@pytest.mark.parametrize("make,bounded", [
    (lambda: synth.gauss1d(10_000, seed=0), False),
    (lambda: synth.dexp(6000, seed=21, dtype=np.float64), True),
    (lambda: synth.gauss2d_grid(96, seed=4, dtype=np.float64), True),
    (lambda: synth.poly2(800, seed=2), False),
])
def test_matches_scipy_least_squares_minimiser(make, bounded):
    scipy_opt = pytest.importorskip("scipy.optimize")
    pr = make()
    X, w = pr.coords(), red.weights(pr.sigma, pr.m)
    fun = lambda p: red.residual_and_jac(pr.model, X, pr.y, w, p)[0]
    jac = lambda p: red.residual_and_jac(pr.model, X, pr.y, w, p)[1]
    lb = -np.inf if pr.lb is None else pr.lb
    ub = np.inf if pr.ub is None else pr.ub
    ref = scipy_opt.least_squares(fun, pr.p0, jac=jac, bounds=(lb, ub), method="trf", **TOL)
    out = trf.curve_fit_problem(pr, **TOL)
    rel = np.abs(out["popt"] - ref.x) / np.maximum(np.abs(ref.x), 1.0)
    assert rel.max() <= 1e-7
    assert out["cost"] == pytest.approx(ref.cost, rel=1e-10)


def _box_around_shifted_truth(pr, seed):
    """A box whose centre is shifted off the truth, so that the optimum may sit on a face."""
    rng = np.random.default_rng(seed)
    n = pr.n
    c = pr.truth + rng.normal(0, 0.3, n) * np.abs(pr.truth)
    lb = c - rng.uniform(0.02, 0.5, n) * np.abs(pr.truth)
    ub = c + rng.uniform(0.02, 0.5, n) * np.abs(pr.truth)
    p0 = lb + rng.uniform(0.01, 0.99, n) * (ub - lb)
    return lb, ub, p0


@pytest.mark.parametrize("make,seed", [
    (lambda: synth.dexp(2000, seed=2, dtype=np.float64), 2),
    (lambda: synth.gauss2d_grid(32, seed=1, dtype=np.float64, bounded=False), 1),
])
def test_reflective_steps_feasible_and_kkt(make, seed):
    """Fits whose full steps leave the box: truncated, reflected and gradient
    candidates are taken, every trial stays strictly inside, and the end point
    satisfies the bound-constrained first-order conditions."""
    pr = make()
    lb, ub, p0 = _box_around_shifted_truth(pr, seed)
    out = trf.curve_fit(pr.model, pr.coords(), pr.y, pr.sigma, p0, lb, ub, record=True,
                        max_nfev=2000, **TOL)
    hist = out["history"]
    assert all(np.all(h["x_new"] > lb) and np.all(h["x_new"] < ub) for h in hist)
    assert any(h["kind"] in ("A", "B", "C") for h in hist)
    assert out["status"] in (1, 2, 3, 4)
    x, g = out["popt"], out["g"]
    J = red.evaluate(pr.model, pr.coords(), pr.y, red.weights(pr.sigma, pr.m), x)[4]
    gscale = np.sqrt(np.sum(J * J, axis=0)) * math.sqrt(2 * out["cost"])
    at_lo = (x - lb) <= 1e-6 * (ub - lb)
    at_hi = (ub - x) <= 1e-6 * (ub - lb)
    free = ~(at_lo | at_hi)
    assert np.all(g[at_lo] >= -1e-5 * gscale[at_lo])
    assert np.all(g[at_hi] <= 1e-5 * gscale[at_hi])
    assert np.all(np.abs(g[free]) <= 1e-4 * gscale[free])


def test_max_nfev_and_status_codes():
    pr = synth.gauss2d_grid(32, seed=1, dtype=np.float64)
    out = trf.curve_fit_problem(pr, max_nfev=3, **TOL)
    assert out["status"] == trf.STATUS_MAX_NFEV and out["nfev"] == 3


def test_nonfinite_start_is_numerical_failure():
    pr = synth.gauss1d(100, seed=1)
    y = pr.y.copy()
    y[5] = np.nan
    out = trf.curve_fit(pr.model, pr.coords(), y, None, pr.p0, **TOL)
    assert out["status"] == trf.STATUS_NUMERICAL


def test_infeasible_start_rejected():
    pr = synth.gauss1d(100, seed=1)
    with pytest.raises(ValueError):
        trf.curve_fit(pr.model, pr.coords(), pr.y, None, pr.p0, np.full(4, 10.0), np.full(4, 20.0))


@pytest.mark.parametrize("absolute_sigma", [False, True])
@pytest.mark.parametrize("name", ["gauss1d_sigma", "gauss2d_grid_bounded", "dexp_bounded"])
def test_pcov_matches_scipy_curve_fit(name, absolute_sigma):
    """pcov (R13: SciPy's documented curve_fit covariance, the pseudo-inverse of
    J^T J at the solution scaled by 2f/(m-n) unless absolute_sigma) against
    scipy.optimize.curve_fit run on the oracle's own model function, per-point
    sigma, nonlinear models, with and without bounds (a library run)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    if name == "gauss1d_sigma":
        pr = synth.gauss1d(3000, seed=3)
        sigma = np.random.default_rng(4).uniform(0.05, 0.2, pr.m)
    elif name == "gauss2d_grid_bounded":
        pr = synth.gauss2d_grid(48, seed=5, dtype=np.float64, truth=[980.0, 24.3, 23.1, 6.0, 4.0, 0.4, 20.0])
        sigma = pr.sigma
    else:
        pr = synth.dexp(3000, seed=21, dtype=np.float64)
        sigma = np.random.default_rng(6).uniform(0.02, 0.1, pr.m)
    X = pr.coords()
    f = lambda _, *p: models.value_and_jac(pr.model, X, np.array(p))[0]
    jac = lambda _, *p: models.value_and_jac(pr.model, X, np.array(p))[1]
    lb = -np.inf if pr.lb is None else pr.lb
    ub = np.inf if pr.ub is None else pr.ub
    popt, pcov = scipy_opt.curve_fit(f, np.arange(pr.m), pr.y, p0=pr.p0, sigma=sigma, absolute_sigma=absolute_sigma,
                                     bounds=(lb, ub), method="trf", jac=jac, ftol=1e-14, xtol=1e-14, gtol=1e-14)
    out = trf.curve_fit(pr.model, X, pr.y, sigma, pr.p0, pr.lb, pr.ub, absolute_sigma=absolute_sigma, **TOL)
    # the two stop at the same optimum up to their tolerances: within 1e-3
    # standard errors (the double exponential's valley is flat: ~1e-6 relative)
    se = np.sqrt(np.diag(pcov))
    assert np.max(np.abs(out["popt"] - popt) / se) <= 1e-3
    np.testing.assert_allclose(out["pcov"], pcov, rtol=1e-4, atol=1e-12 * np.max(np.abs(pcov)))
