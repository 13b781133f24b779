"""Full-size parity at the largest workloads the benchmarks time, where the
whole oracle fit is too slow to run at every size: properties that hold at
any size, and whole oracle fits on a sample.

1D Gaussian + offset at 1e7 and 5e7 points (the size sweep's largest; FP64
data for the plain path, the same data rounded to FP32 for the mixed one):
  - fixed-p sums (Gram B, gradient g = J^T r, cost; Eq. gradient, B ~ J^T J)
    against the oracle's FP64 definition summed over chunks (the sum of the
    pieces equals the whole: pinned on the CPU).  Tolerance relative to each
    entry's scale: plain 1e-10 (two summation orders over up to 5e7 terms,
    typically ~sqrt(m) eps64 apart; a single dropped point moves a sum by
    ~1/m = 2e-8), mixed 1e-5 (FP32 rows and tile sums, as at small sizes).
  - whole fits: popt against the stationary point p* = popt - B^-1 g, one
    Gauss-Newton step from popt with the oracle's FP64 B and g on the data the
    fit saw (the exact optimum to second order in the step): plain within
    1e-8, mixed within 1e-6 relative (|dp| / max(|p|, 1)).

4,096 ragged double exponentials (m log-uniform in [200, 2e5]) in one
batched mixed launch (precision guard on, its default) with the autotuned
tile shapes (the batch benchmark's launch): every fit terminates by a
tolerance or at max_nfev; four fits re-run alone on views of the same device
buffers give bitwise the batch's results; on the first 24 fits, whole FP64
oracle fits and the per-fit criterion of oracle_checks: popt within 1e-6
where the oracle's popt is determined to that level, otherwise (standard
error above 10 %, rounding-sensitive or tolerance-limited oracle result) an
oracle cost at the GPU's popt no higher than the oracle's own by 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle_checks  # noqa: E402  (tests/ is on sys.path)
from oracle import reduce as red, trf
from paper_2208_12187_gb300 import build, gbfit, synth

pytestmark = pytest.mark.gpu
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)
CHUNK = 2_000_000


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


def oracle_sums(model, x, y, p):
    """(f, g, B) of the whole data set as sums over chunks of the oracle's definition."""
    f, g, B = 0.0, 0.0, 0.0
    for a in range(0, x.shape[0], CHUNK):
        xs = np.asarray(x[a:a + CHUNK], dtype=np.float64)
        ys = np.asarray(y[a:a + CHUNK], dtype=np.float64)
        fc, gc, Bc, _, _ = red.evaluate(model, xs[None, :], ys, np.ones(xs.shape[0]), p)
        f, g, B = f + fc, g + gc, B + Bc
    return f, g, B


@pytest.fixture(scope="module", params=[10_000_000, 50_000_000], ids=["1e7", "5e7"])
def sweep_problem(request):
    return synth.gauss1d(request.param, seed=0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sweep_full_size_sums_and_optimum(sweep_problem, precision):
    pr = sweep_problem if precision == "fp64" else sweep_problem.astype(np.float32)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    x = torch.as_tensor(pr.x).to(tdt).cuda()
    y = torch.as_tensor(pr.y).to(tdt).cuda()
    n = pr.n
    # fixed-p sums at p0
    f, g, B = oracle_sums(pr.model, pr.x, pr.y, pr.p0)
    Bp, gg, cost = gbfit.evaluate(pr.model, x, y, pr.p0, precision=precision)
    Bg = gbfit.unpack_upper(Bp, n)
    tol = 1e-10 if precision == "fp64" else 1e-5
    dscale = np.sqrt(np.outer(np.diag(B), np.diag(B)))
    assert np.max(np.abs(Bg - B) / dscale) <= tol
    assert np.max(np.abs(gg - g) / np.sqrt(np.diag(B) * 2 * f)) <= tol
    assert abs(cost - f) <= tol * f
    # the whole fit, against the stationary point one Gauss-Newton step away
    out = gbfit.curve_fit(pr.model, x, y, pr.p0, precision=precision, **TOL)
    assert out["status"] in (1, 2, 3, 4)
    f1, g1, B1 = oracle_sums(pr.model, pr.x, pr.y, out["popt"])
    p_star = out["popt"] - np.linalg.solve(B1, g1)
    assert relerr(out["popt"], p_star) <= (1e-8 if precision == "fp64" else 1e-6)
    assert out["cost"] == pytest.approx(f1, rel=1e-8 if precision == "fp64" else 1e-5)


def test_batch_full_size_sample_against_oracle():
    """The 4,096-fit double-exponential batch in its benchmarked launch
    (autotuned shapes, mixed precision with its precision guard): every fit
    ends on a tolerance or on max_nfev, fits re-run alone on views of the same
    buffers are bitwise equal, and on a sample of 24 fits every fit meets the
    oracle criterion of oracle_checks (popt within 1e-6 where the oracle's
    popt is determined to that level, else a cost no higher than the
    oracle's)."""
    bt = synth.dexp_batch(4096, seed=7, dtype=np.float32)
    saved = gbfit.tune_get()
    try:
        gbfit.autotune(bt.model, "mixed", m_max=200_000)
        x = torch.as_tensor(bt.x).cuda()
        y = torch.as_tensor(bt.y).cuda()
        out = gbfit.curve_fit_batch(bt.model, bt.offsets, x, y, bt.p0, lb=bt.lb, ub=bt.ub, precision="mixed", **TOL)
        st = out["status"]
        assert np.all(np.isin(st, (0, 1, 2, 3, 4)))
        assert np.all(out["nfev"][st == 0] >= 500)               # status 0 only at max_nfev (100 n)
        # alone, on views of the same buffers (same alignment), with the shape the batch gave the fit
        for k in (0, 5, 1000, 4095):
            a, b = int(bt.offsets[k]), int(bt.offsets[k + 1])
            tp, gt = gbfit.tune_shape(bt.model, "mixed", b - a)
            alone = gbfit.curve_fit(bt.model, x[a:b], y[a:b], bt.p0[k], lb=bt.lb[k], ub=bt.ub[k], precision="mixed",
                                    tile_points=tp, group_tiles=gt, **TOL)
            np.testing.assert_array_equal(out["popt"][k], alone["popt"])
            assert out["cost"][k] == alone["cost"] and out["nfev"][k] == alone["nfev"]
    finally:
        gbfit.tune_set(saved)
    for k in range(24):
        pr = bt.fit(k).astype(np.float64)
        ref = trf.curve_fit_problem(pr, **TOL)
        oracle_checks.check_mixed(pr, out["popt"][k], ref, TOL)
