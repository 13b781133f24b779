"""The mixed path's precision guard (gbfit_options.guard_cond / guard_floor).

FP32 evaluation limits a fit in two ways: the Gram formed from FP32 sums
squares the conditioning (steps of an ill-conditioned fit lose accuracy), and
FP32 rounding of the residuals moves the iteration's fixed point.  The guard
moves such a fit to FP64 passes: at once when the Gram's equilibrated
condition number exceeds guard_cond, or to finish when a tolerance is met
while the estimated rounding floor of popt exceeds guard_floor.  Checked here
through the C ABI: which fits it moves (the library's counters), that the
moved fits land where the FP64 iteration does, and that it stays idle on a
well-conditioned fit such as the 1024 x 1024 rotated 2D Gaussian.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle_checks
from oracle import trf
from paper_2208_12187_gb300 import build, gbfit, synth

pytestmark = pytest.mark.gpu
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)
OFF = dict(guard_cond=math.inf, guard_floor=math.inf)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


def _fit(pr, precision, **kw):
    dt = torch.float32 if precision == "mixed" else torch.float64
    x = None if pr.layout == synth.LAYOUT_GRID else torch.as_tensor(pr.x).to(dt).cuda()
    y = torch.as_tensor(pr.y).to(dt).cuda()
    s = None if pr.sigma is None else torch.as_tensor(pr.sigma).to(dt).cuda()
    return gbfit.curve_fit(pr.model, x, y, pr.p0, sigma=s, lb=pr.lb, ub=pr.ub, grid_wh=pr.grid_wh,
                           precision=precision, **kw)


def _counters(fn):
    gbfit.stats_reset()
    out = fn()
    ph = gbfit.stats()["phase_cycles"]
    return out, int(ph["n_eval64"]), int(ph["n_guard_escalated"]), int(ph["n_guard_finished"])


def test_ill_conditioned_fit_escalates_to_fp64():
    """Near-degenerate double exponential (t1 ~ t2): escalated at its first
    evaluation, it then runs the FP64 iteration from p0 (every evaluation
    after the FP32 one that measured the conditioning is FP64) and meets the
    oracle criterion."""
    pr = synth.dexp(20_000, seed=5, dtype=np.float32)
    out, n64, esc, fin = _counters(lambda: _fit(pr, "mixed", **TOL))
    assert esc == 1 and fin == 0 and n64 == out["nfev"] - 1
    ref = trf.curve_fit_problem(pr.astype(np.float64), **TOL)
    oracle_checks.check_mixed(pr.astype(np.float64), out["popt"], ref, TOL)
    # with the guard off every pass is FP32
    _, n64_off, esc_off, fin_off = _counters(lambda: _fit(pr, "mixed", **OFF, **TOL))
    assert n64_off == esc_off == fin_off == 0


def test_rounding_floor_triggers_fp64_finish():
    """A well-conditioned double exponential (equilibrated condition number
    ~1e2) whose estimated FP32 floor in popt (~5e-7) is above guard_floor:
    it converges in FP32, then finishes with FP64 passes and lands on the
    FP64 fixed point, within 2e-7 of the plain FP64 path's popt (the floor
    estimate with the guard off is what it removes)."""
    pr = synth.dexp(1500, seed=1, truth=[3.0, 1.0, 5.0, 8.0, 0.4], dtype=np.float32)
    pr64 = pr.astype(np.float64)
    out, n64, esc, fin = _counters(lambda: _fit(pr, "mixed", **TOL))
    assert esc == 0 and fin == 1 and n64 >= 1
    plain = _fit(pr64, "fp64", **TOL)
    assert oracle_checks.relerr(pr.model, out["popt"], plain["popt"]) <= 2e-7
    ref = trf.curve_fit_problem(pr64, **TOL)
    assert oracle_checks.relerr(pr.model, out["popt"], ref["popt"]) <= 2e-7
    off = _fit(pr, "mixed", **OFF, **TOL)
    assert oracle_checks.relerr(pr.model, off["popt"], plain["popt"]) <= 1e-5     # FP32 floor, not parity


def test_guard_idle_on_well_conditioned_2d_gaussian():
    """The 1024 x 1024 rotated 2D Gaussian (the headline workload): neither
    trigger fires, so every pass of the fit is FP32 and the guard costs
    nothing beyond its estimates inside the step."""
    pr = synth.gauss2d_grid(1024, seed=0, dtype=np.float32)
    out, n64, esc, fin = _counters(lambda: _fit(pr, "mixed", **TOL))
    assert n64 == esc == fin == 0
    off = _fit(pr, "mixed", **OFF, **TOL)
    np.testing.assert_array_equal(out["popt"], off["popt"])
    assert out["nfev"] == off["nfev"]


def test_guard_thresholds_are_honoured():
    """guard_cond above the fit's conditioning: no escalation; guard_floor
    above its floor estimate: no finish (the same fit as above)."""
    pr = synth.dexp(1500, seed=1, truth=[3.0, 1.0, 5.0, 8.0, 0.4], dtype=np.float32)
    _, n64, esc, fin = _counters(lambda: _fit(pr, "mixed", guard_cond=1e3, guard_floor=1e-5, **TOL))
    assert n64 == esc == fin == 0
    _, n64, esc, fin = _counters(lambda: _fit(pr, "mixed", guard_cond=10.0, guard_floor=math.inf, **TOL))
    assert esc == 1 and fin == 0 and n64 >= 1


def test_guarded_batch_fit_equals_alone():
    """Guard decisions depend on the fit's own sums only: a fit that the guard
    moves gives bitwise the same result alone and inside a batch."""
    bt = synth.dexp_batch(24, seed=21, m_lo=1000, m_hi=20_000, dtype=np.float32)
    x = torch.as_tensor(bt.x).cuda()
    y = torch.as_tensor(bt.y).cuda()
    gbfit.stats_reset()
    out = gbfit.curve_fit_batch(bt.model, bt.offsets, x, y, bt.p0, lb=bt.lb, ub=bt.ub, precision="mixed", **TOL)
    ph = gbfit.stats()["phase_cycles"]
    assert ph["n_guard_escalated"] + ph["n_guard_finished"] >= 1
    for k in range(bt.nfits):
        a, b = int(bt.offsets[k]), int(bt.offsets[k + 1])
        tp, gt = gbfit.tune_shape(bt.model, "mixed", b - a)
        alone = gbfit.curve_fit(bt.model, x[a:b], y[a:b], bt.p0[k], lb=bt.lb[k], ub=bt.ub[k], precision="mixed",
                                tile_points=tp, group_tiles=gt, **TOL)
        np.testing.assert_array_equal(out["popt"][k], alone["popt"])
        assert out["nfev"][k] == alone["nfev"]
