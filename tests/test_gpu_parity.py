"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances, stated per quantity:
  reductions at fixed p, plain FP64   relative 1e-12 of each entry's scale
                                      (summation order only)
  reductions at fixed p, mixed        relative 1e-5 (FP32 model/Jacobian rows,
                                      FP32 tile sums, FP64 combine)
  whole fits, plain FP64              popt, cost within 1e-8 relative
                                      (|dp| / max(|p|, 1)), same nfev
  whole fits, mixed                   popt within 1e-6 relative of the oracle
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle_checks
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


def dev(a, dtype=None):
    if a is None:
        return None
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


def gpu_fit(pr, precision, dtype=torch.float64, **kw):
    x = None if pr.layout == synth.LAYOUT_GRID else dev(pr.x, dtype)
    return gbfit.curve_fit(pr.model, x, dev(pr.y, dtype), pr.p0, sigma=dev(pr.sigma, dtype), lb=pr.lb,
                           ub=pr.ub, grid_wh=pr.grid_wh, precision=precision, **kw)


# ------------------------------------------------------------------ fixed-p reductions
REDUCE_CASES = [
    ("gauss1d", lambda: synth.gauss1d(3 * 2048 + 17, seed=1)),
    ("gauss1d_sigma", lambda: synth.gauss1d(2048 + 5, seed=2, with_sigma=True)),
    ("dexp", lambda: synth.dexp(4 * 2048 + 1000, seed=3, dtype=np.float64)),
    ("gauss2d_grid", lambda: synth.gauss2d_grid(97, seed=4, dtype=np.float64)),
    ("gauss2d_soa", lambda: synth.gauss2d_grid(75, seed=5, dtype=np.float64, layout=synth.LAYOUT_SOA2)),
    ("poly2", lambda: synth.poly2(2048 * 2 + 1, seed=6)),
    ("tiny", lambda: synth.gauss1d(7, seed=7)),
]


@pytest.mark.parametrize("name,make", REDUCE_CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_reduction_matches_definition(name, make, precision):
    pr = make()
    p = pr.p0
    f, g, B, _, _ = red.evaluate(pr.model, pr.coords(), pr.y, red.weights(pr.sigma, pr.m), p)
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = None if pr.layout == synth.LAYOUT_GRID else dev(pr.x, dt)
    Bp, gg, cost = gbfit.evaluate(pr.model, x, dev(pr.y, dt), p, sigma=dev(pr.sigma, dt), grid_wh=pr.grid_wh,
                                  precision=precision, tile_points=2048)
    Bg = gbfit.unpack_upper(Bp, pr.n)
    tol = 1e-12 if precision == "fp64" else 2e-5
    dscale = np.sqrt(np.outer(np.diag(B), np.diag(B)))
    assert np.max(np.abs(Bg - B) / np.maximum(dscale, 1e-300)) <= tol
    gscale = np.sqrt(np.diag(B) * 2 * f)
    assert np.max(np.abs(gg - g) / np.maximum(gscale, 1e-300)) <= tol
    assert abs(cost - f) <= tol * f


def test_reduction_tile_size_independent():
    """Ragged tails: different tilings give the same sums (FP64) to rounding."""
    pr = synth.gauss1d(50_001, seed=8)
    outs = [gbfit.evaluate(pr.model, dev(pr.x), dev(pr.y), pr.p0, precision="fp64", tile_points=t)
            for t in (256, 2048, 4096 + 256)]
    for B, g, c in outs[1:]:
        np.testing.assert_allclose(B, outs[0][0], rtol=1e-12)
        assert c == pytest.approx(outs[0][2], rel=1e-13)


# ------------------------------------------------------------------ subproblem
@pytest.mark.parametrize("seed", range(8))
def test_tr_subproblem_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.exp(rng.uniform(0, math.log(1e4), n))
    B = (Q * lam) @ Q.T
    g = rng.normal(size=n) * 10
    full = np.linalg.norm(np.linalg.solve(B, g))
    for frac in (0.1, 0.5, 2.0):
        Delta = full * frac
        p, alpha, lg = gbfit.tr_subproblem(B, g, Delta, 0.0)
        le, V = np.linalg.eigh(B)
        pe, ae = trf.tr_solve(le, V, V.T @ g, np.linalg.norm(g), Delta, 0.0, True)
        # FP64 results from FP32 rotations + FP64 refinement: eigenvalues to
        # 1e-12 of the largest, the step to 1e-9 of its norm
        np.testing.assert_allclose(np.sort(lg), le, rtol=0, atol=1e-12 * le.max())
        assert alpha == pytest.approx(ae, rel=1e-9, abs=1e-12)
        assert np.linalg.norm(p - pe) <= 1e-9 * np.linalg.norm(pe)


# ------------------------------------------------------------------ whole fits, plain FP64
PLAIN_FITS = [
    ("gauss1d_m1e4", lambda: synth.gauss1d(10_000, seed=0)),
    ("gauss1d_sigma_ones", lambda: synth.gauss1d(10_000, seed=0, with_sigma=True)),
    ("dexp_bounded", lambda: synth.dexp(6000, seed=21, dtype=np.float64)),
    ("gauss2d_grid_bounded", lambda: synth.gauss2d_grid(96, seed=4, dtype=np.float64)),
    ("poly2_linear", lambda: synth.poly2(3000, seed=2)),
]


@pytest.mark.parametrize("name,make", PLAIN_FITS)
def test_plain_fit_matches_oracle(name, make):
    pr = make()
    ref = trf.curve_fit_problem(pr, **TOL)
    out = gpu_fit(pr, "fp64", **TOL)
    assert out["status"] == ref["status"]
    assert out["nfev"] == ref["nfev"]
    assert relerr(out["popt"], ref["popt"]) <= 1e-8
    assert out["cost"] == pytest.approx(ref["cost"], rel=1e-8)
    np.testing.assert_allclose(out["pcov"], ref["pcov"], rtol=1e-6, atol=1e-12 * np.max(np.abs(ref["pcov"])))


def test_plain_fit_bounded_reflective_path():
    """A box that forces truncated/reflected/gradient steps (bounded path)."""
    pr = synth.dexp(2000, seed=2, dtype=np.float64)
    rng = np.random.default_rng(2)
    n = pr.n
    c = pr.truth + rng.normal(0, 0.3, n) * np.abs(pr.truth)
    lb = c - rng.uniform(0.02, 0.5, n) * np.abs(pr.truth)
    ub = c + rng.uniform(0.02, 0.5, n) * np.abs(pr.truth)
    p0 = lb + rng.uniform(0.01, 0.99, n) * (ub - lb)
    ref = trf.curve_fit(pr.model, pr.coords(), pr.y, None, p0, lb, ub, record=True, **TOL)
    assert any(h["kind"] != "full" for h in ref["history"])
    out = gbfit.curve_fit(pr.model, dev(pr.x), dev(pr.y), p0, lb=lb, ub=ub, precision="fp64", **TOL)
    assert out["status"] == ref["status"] and out["nfev"] == ref["nfev"]
    assert relerr(out["popt"], ref["popt"]) <= 1e-8
    assert np.all(out["popt"] > lb) and np.all(out["popt"] < ub)


def test_plain_max_nfev_and_linear_closed_form():
    pr = synth.poly2(5000, seed=9)
    out = gpu_fit(pr, "fp64", **TOL)
    X = pr.coords()[0]
    A = np.stack([np.ones_like(X), X, X * X], axis=1) / pr.sigma[:, None]
    ref = np.linalg.solve(A.T @ A, A.T @ (pr.y / pr.sigma))
    assert relerr(out["popt"], ref) <= 1e-10
    pr2 = synth.gauss2d_grid(40, seed=1, dtype=np.float64)
    out = gpu_fit(pr2, "fp64", max_nfev=3, **TOL)
    ref2 = trf.curve_fit_problem(pr2, max_nfev=3, **TOL)
    assert out["status"] == gbfit.FIT_MAX_NFEV and out["nfev"] == 3
    assert relerr(out["popt"], ref2["popt"]) <= 1e-8


def test_x_scale_jac_matches_oracle():
    pr = synth.gauss2d_grid(64, seed=7, dtype=np.float64)
    ref = trf.curve_fit_problem(pr, x_scale="jac", **TOL)
    out = gpu_fit(pr, "fp64", x_scale="jac", **TOL)
    assert out["nfev"] == ref["nfev"]
    assert relerr(out["popt"], ref["popt"]) <= 1e-8


def test_x_scale_vector_and_absolute_sigma_match_oracle():
    """R7 with a numeric x_scale (D = 1/x_scale) and R13 with absolute_sigma."""
    pr = synth.gauss1d(5000, seed=4, with_sigma=True)
    pr.sigma = np.random.default_rng(4).uniform(0.05, 0.2, pr.m)
    xs = np.array([2.0, 0.5, 0.25, 1.0])
    ref = trf.curve_fit_problem(pr, x_scale=xs, absolute_sigma=True, **TOL)
    out = gpu_fit(pr, "fp64", x_scale=xs, absolute_sigma=True, **TOL)
    assert out["nfev"] == ref["nfev"]
    assert relerr(out["popt"], ref["popt"]) <= 1e-8
    np.testing.assert_allclose(out["pcov"], ref["pcov"], rtol=1e-6, atol=1e-12 * np.max(np.abs(ref["pcov"])))


def test_batch_soa2_sigma_and_1d_sigma_match_oracle():
    """Batched fits through explicit 2D coordinates with sigma (mixed) and 1D
    fits with sigma (plain FP64): each fit against the oracle."""
    fits = [synth.gauss2d_grid(48 + 8 * k, seed=20 + k, dtype=np.float32, layout=synth.LAYOUT_SOA2) for k in range(5)]
    off = np.concatenate([[0], np.cumsum([f.m for f in fits])])
    X = np.concatenate([f.x for f in fits], axis=1).astype(np.float32)
    Y = np.concatenate([f.y for f in fits]).astype(np.float32)
    S = np.concatenate([f.sigma for f in fits]).astype(np.float32)
    P0 = np.stack([f.p0 for f in fits])
    out = gbfit.curve_fit_batch(gbfit.MODEL_GAUSS2D, off, dev(X), dev(Y), P0, sigma=dev(S), lb=fits[0].lb,
                                ub=fits[0].ub, precision="mixed", **TOL)
    for k, f in enumerate(fits):
        ref = trf.curve_fit_problem(f.astype(np.float64), **TOL)
        assert relerr(out["popt"][k], ref["popt"]) <= 1e-6, k
    fits = [synth.gauss1d(3000 + 1111 * k, seed=30 + k, with_sigma=True) for k in range(4)]
    for f in fits:
        f.sigma = np.random.default_rng(f.m).uniform(0.05, 0.3, f.m)
    off = np.concatenate([[0], np.cumsum([f.m for f in fits])])
    out = gbfit.curve_fit_batch(gbfit.MODEL_GAUSS1D, off, dev(np.concatenate([f.x for f in fits])),
                                dev(np.concatenate([f.y for f in fits])), np.stack([f.p0 for f in fits]),
                                sigma=dev(np.concatenate([f.sigma for f in fits])), precision="fp64", **TOL)
    for k, f in enumerate(fits):
        ref = trf.curve_fit_problem(f, **TOL)
        assert out["nfev"][k] == ref["nfev"]
        assert relerr(out["popt"][k], ref["popt"]) <= 1e-8, k


# ------------------------------------------------------------------ whole fits, mixed precision
MIXED_FITS = [
    ("gauss1d_m1e4", lambda: synth.gauss1d(10_000, seed=0), None),
    ("dexp", lambda: synth.dexp(20_000, seed=5, truth=[4.0, 0.8, 6.0, 9.0, 0.5], dtype=np.float64), None),
    ("gauss2d_256_grid", lambda: synth.gauss2d_grid(256, seed=1, dtype=np.float64), None),
    ("gauss2d_soa", lambda: synth.gauss2d_grid(128, seed=3, dtype=np.float64, layout=synth.LAYOUT_SOA2), None),
    ("gauss1d_sigma", lambda: with_sigma(synth.gauss1d(30_000, seed=6), 6), None),
    ("dexp_sigma", lambda: with_sigma(synth.dexp(20_000, seed=5, truth=[4.0, 0.8, 6.0, 9.0, 0.5],
                                                 dtype=np.float64), 7), None),
]


def with_sigma(pr, seed):
    """The same problem with per-point uncertainties U(0.05, 0.3) (App. C weighting)."""
    import dataclasses
    return dataclasses.replace(pr, sigma=np.random.default_rng(seed).uniform(0.05, 0.3, pr.m))


@pytest.mark.parametrize("name,make,_", MIXED_FITS)
def test_mixed_fit_matches_oracle(name, make, _):
    pr = make()
    ref = trf.curve_fit_problem(pr, **TOL)
    out = gpu_fit(pr, "mixed", dtype=torch.float32, **TOL)
    assert out["status"] in (1, 2, 3, 4)
    # the oracle sees the same FP32-rounded data
    pr32 = pr.astype(np.float32)
    ref32 = trf.curve_fit_problem(pr32, **TOL)
    assert relerr(out["popt"], ref32["popt"]) <= 1e-6
    assert out["cost"] == pytest.approx(ref32["cost"], rel=1e-6)


def test_mixed_degenerate_dexp_identifiable_part():
    """t1 ~ t2: only a1 + a2 and the curve are determined; the split is not.
    The precision guard moves this fit to FP64 passes (its Gram's equilibrated
    condition number is far above 1e3), so the mixed fit stops where the
    FP64 iteration does: cost within 1e-6 of the oracle's and not above it
    beyond 1e-9 (the oracle's FP64 cost at both points), and the same fitted
    curve."""
    pr = synth.dexp(20_000, seed=5, dtype=np.float64)
    assert abs(pr.truth[1] / pr.truth[3] - 1) < 0.1          # a near-degenerate draw
    pr32 = pr.astype(np.float32)
    ref = trf.curve_fit_problem(pr32, **TOL)
    out = gpu_fit(pr, "mixed", dtype=torch.float32, **TOL)
    assert out["cost"] == pytest.approx(ref["cost"], rel=1e-6)
    assert oracle_checks.oracle_cost(pr32, out["popt"]) <= ref["cost"] * (1 + 1e-9)
    from oracle import models
    X = pr.coords()
    hg = models.value_and_jac(pr.model, X, out["popt"])[0]
    ho = models.value_and_jac(pr.model, X, ref["popt"])[0]
    assert np.max(np.abs(hg - ho)) <= 1e-4 * np.max(np.abs(ho))


def test_mixed_config1_full_size_1024_grid():
    """Rotated 2D Gaussian on the 1024 x 1024 grid, Poisson data, bounds (full size)."""
    pr = synth.gauss2d_grid(1024, seed=0, dtype=np.float32)
    ref = trf.curve_fit_problem(pr, **TOL)
    out = gpu_fit(pr, "mixed", dtype=torch.float32, **TOL)
    assert out["status"] in (1, 2, 3, 4)
    assert relerr(out["popt"], ref["popt"]) <= 1e-6
    outp = gpu_fit(pr, "fp64", dtype=torch.float32, **TOL)
    assert relerr(outp["popt"], ref["popt"]) <= 1e-8
    assert outp["nfev"] == ref["nfev"]


def test_host_buffers_equal_device_buffers():
    pr = synth.gauss1d(5000, seed=4)
    a = gbfit.curve_fit(pr.model, pr.x, pr.y, pr.p0, precision="fp64", **TOL)
    b = gpu_fit(pr, "fp64", **TOL)
    np.testing.assert_array_equal(a["popt"], b["popt"])


# ------------------------------------------------------------------ batched
def test_batch_matches_alone_and_oracle():
    bt = synth.dexp_batch(48, seed=11, m_lo=200, m_hi=20_000, dtype=np.float64)
    out = gbfit.curve_fit_batch(bt.model, bt.offsets, dev(bt.x), dev(bt.y), bt.p0, lb=bt.lb, ub=bt.ub,
                                precision="fp64", **TOL)
    for k in (0, 7, 23, 47):
        pr = bt.fit(k)
        tp, gt = gbfit.tune_shape(pr.model, "fp64", pr.m)                # the shape the batch gave this fit
        alone = gbfit.curve_fit(pr.model, dev(pr.x), dev(pr.y), pr.p0, lb=pr.lb, ub=pr.ub, precision="fp64",
                                tile_points=tp, group_tiles=gt, **TOL)
        np.testing.assert_array_equal(out["popt"][k], alone["popt"])     # bit-identical in the mix
        ref = trf.curve_fit_problem(pr, **TOL)
        assert out["nfev"][k] == ref["nfev"]
        assert relerr(out["popt"][k], ref["popt"]) <= 1e-8


def test_batch_mixed_matches_oracle():
    """Every fit of a mixed batch against the oracle, per fit (oracle_checks:
    popt within 1e-6 where the oracle's popt is determined to that level,
    else no higher cost than the oracle's)."""
    bt = synth.dexp_batch(32, seed=12, m_lo=500, m_hi=50_000, dtype=np.float32)
    out = gbfit.curve_fit_batch(bt.model, bt.offsets, dev(bt.x, torch.float32), dev(bt.y, torch.float32), bt.p0,
                                lb=bt.lb, ub=bt.ub, precision="mixed", **TOL)
    assert np.all(out["status"] >= 0)
    for k in range(bt.nfits):
        pr = bt.fit(k).astype(np.float64)
        ref = trf.curve_fit_problem(pr, **TOL)
        oracle_checks.check_mixed(pr, out["popt"][k], ref, TOL)


def test_autotune_installs_valid_shapes_and_fits_still_match():
    saved = gbfit.tune_get()
    try:
        tab = gbfit.autotune(gbfit.MODEL_DEXP, "mixed", m_max=1 << 15, points_per_run=1 << 20)
        tp = tab["tile_points"][gbfit.MODEL_DEXP][gbfit.PREC_MIXED]
        gt = tab["group_tiles"][gbfit.MODEL_DEXP][gbfit.PREC_MIXED]
        assert np.all(tp % 256 == 0) and np.all(tp >= 256) and np.all((gt >= 1) & (gt <= 1024))
        # buckets above m_max and other models / precisions are untouched
        assert np.array_equal(tp[15:], saved["tile_points"][gbfit.MODEL_DEXP][gbfit.PREC_MIXED][15:])
        assert np.array_equal(tab["tile_points"][gbfit.MODEL_GAUSS1D], saved["tile_points"][gbfit.MODEL_GAUSS1D])
        assert gbfit.tune_shape(gbfit.MODEL_DEXP, "mixed", 3 << 13) == (min(int(tp[14]), 3 << 13), int(gt[14]))
        bt = synth.dexp_batch(16, seed=13, m_lo=1000, m_hi=30_000, dtype=np.float32)
        out = gbfit.curve_fit_batch(bt.model, bt.offsets, dev(bt.x, torch.float32), dev(bt.y, torch.float32), bt.p0,
                                    lb=bt.lb, ub=bt.ub, precision="mixed", **TOL)
        for k in range(bt.nfits):
            pr = bt.fit(k).astype(np.float64)
            oracle_checks.check_mixed(pr, out["popt"][k], trf.curve_fit_problem(pr, **TOL), TOL)
    finally:
        gbfit.tune_set(saved)
    assert np.array_equal(gbfit.tune_get()["tile_points"], saved["tile_points"])


def test_sigma_none_equals_sigma_ones():
    """Config 0 passes sigma = None and sigma = ones: Eqs. easy_jac / easy_res
    with S = I leave J and r unchanged, so the fits must agree exactly."""
    pr = synth.gauss1d(10_000, seed=0)
    ones = np.ones(pr.m)
    for prec, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
        a = gbfit.curve_fit(pr.model, dev(pr.x, dt), dev(pr.y, dt), pr.p0, precision=prec, **TOL)
        b = gbfit.curve_fit(pr.model, dev(pr.x, dt), dev(pr.y, dt), pr.p0, sigma=dev(ones, dt), precision=prec,
                            **TOL)
        assert relerr(a["popt"], b["popt"]) <= 1e-12
        assert a["nfev"] == b["nfev"]
        np.testing.assert_allclose(a["pcov"], b["pcov"], rtol=1e-10)


def test_explicit_coordinates_equal_implicit_grid():
    """Config 1's two layouts: pixel coordinates passed as x, y rows give the
    fit of the implicit grid (mixed: within the mixed tolerance of each other
    and of the oracle)."""
    pr = synth.gauss2d_grid(256, seed=8, dtype=np.float32)
    ref = trf.curve_fit_problem(pr.astype(np.float64), **TOL)
    g = gpu_fit(pr, "mixed", dtype=torch.float32, **TOL)
    Xc = pr.coords().astype(np.float32)
    e = gbfit.curve_fit(pr.model, dev(Xc), dev(pr.y, torch.float32), pr.p0, sigma=dev(pr.sigma, torch.float32),
                        lb=pr.lb, ub=pr.ub, precision="mixed", **TOL)
    assert relerr(g["popt"], ref["popt"]) <= 1e-6
    assert relerr(e["popt"], ref["popt"]) <= 1e-6


# ------------------------------------------------------------------ edge cases
def test_minimum_size_fit_m_equals_n():
    rng = np.random.default_rng(0)
    x = rng.uniform(-2, 2, 3)
    y = 1 + 2 * x - 0.5 * x * x
    out = gbfit.curve_fit(gbfit.MODEL_POLY2, dev(x), dev(y), [0.0, 0.0, 0.0], precision="fp64", **TOL)
    assert relerr(out["popt"], [1, 2, -0.5]) <= 1e-9
    assert np.all(np.isinf(out["pcov"]))


def test_invalid_data_rejected_on_device():
    pr = synth.gauss1d(3000, seed=1, with_sigma=True)
    sig = pr.sigma.copy()
    sig[1234] = 0.0
    for prec, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
        with pytest.raises(gbfit.GbfitError) as e:
            gbfit.curve_fit(pr.model, dev(pr.x, dt), dev(pr.y, dt), pr.p0, sigma=dev(sig, dt), precision=prec)
        assert e.value.code == gbfit.E_INVALID_ARG
    y = pr.y.copy()
    y[77] = np.nan
    with pytest.raises(gbfit.GbfitError):
        gbfit.curve_fit(pr.model, dev(pr.x), dev(y), pr.p0, precision="fp64")
