"""GPU: the direct evaluation form of the mixed path, and data checks in far tiles.

The mixed path evaluates a fit's first evaluation (and gbfit_evaluate) and
every trial whose predicted reduction is at least 1 % of f in the direct
form: model value and Jacobian row at the trial point alone, the actual
reduction of Eq. accuracy then being f - f' of two FP32-evaluated costs.
Trials closer to convergence keep the cancellation-free difference form.
Checked here against the FP64 oracle (tests/oracle_checks.py criteria:
popt within 1e-6 where the oracle's popt is determined to that level, else
no higher oracle cost), with the count of wide trials read from the
library's trace counters.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle_checks
from oracle import trf
from paper_2208_12187_gb300 import build, gbfit, synth

pytestmark = pytest.mark.gpu
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


def dev(a, dtype=torch.float32):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def far_start(pr, scale):
    """The same problem started further from the truth (p0 scaled per parameter)."""
    import dataclasses
    p0 = np.asarray(pr.truth, dtype=np.float64) * np.asarray(scale, dtype=np.float64)
    return dataclasses.replace(pr, p0=p0)


CASES = [
    ("gauss1d", lambda: far_start(synth.gauss1d(20_000, seed=3, dtype=np.float32), [1.3, 0.8, 1.25, 1.4])),
    ("gauss1d_sigma", lambda: far_start(synth.gauss1d(20_000, seed=4, with_sigma=True, dtype=np.float32),
                                        [0.7, 1.2, 0.8, 1.3])),
    ("dexp", lambda: far_start(synth.dexp(30_000, seed=7, truth=[4.0, 0.8, 6.0, 9.0, 0.5], dtype=np.float32),
                               [1.2, 0.8, 0.8, 1.2, 1.5])),
    ("gauss2d_grid", lambda: far_start(synth.gauss2d_grid(128, seed=6, dtype=np.float32),
                                       [1.2, 1.0, 1.0, 1.2, 0.85, 1.0, 1.1])),
]


@pytest.mark.parametrize("name,make", CASES)
def test_wide_trials_in_direct_form_match_oracle(name, make):
    pr = make()
    gbfit.stats_reset()
    x = None if pr.layout == synth.LAYOUT_GRID else dev(pr.x)
    out = gbfit.curve_fit(pr.model, x, dev(pr.y), pr.p0, sigma=dev(pr.sigma), lb=pr.lb, ub=pr.ub,
                          grid_wh=pr.grid_wh, precision="mixed", **TOL)
    n_wide = gbfit.stats()["phase_cycles"]["n_wide"]
    assert n_wide >= 1, "a fit started this far takes at least one wide trial"
    assert n_wide < out["nfev"]
    assert out["status"] in (1, 2, 3, 4)
    ref = trf.curve_fit_problem(pr, **TOL)
    oracle_checks.check_mixed(pr, out["popt"], ref, TOL)


def test_first_evaluation_direct_form_equals_fit_start():
    """gbfit_evaluate at p0 (direct form) and a fit stopped after its first
    evaluation (max_nfev = 1) report the same cost, bit for bit."""
    pr = synth.gauss2d_grid(200, seed=9, dtype=np.float32)
    B, g, cost = gbfit.evaluate(pr.model, None, dev(pr.y), pr.p0, sigma=dev(pr.sigma), grid_wh=pr.grid_wh,
                                precision="mixed")
    out = gbfit.curve_fit(pr.model, None, dev(pr.y), pr.p0, sigma=dev(pr.sigma), grid_wh=pr.grid_wh,
                          precision="mixed", max_nfev=1, **TOL)
    assert out["nfev"] == 1
    assert out["cost"] == cost


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_invalid_sigma_in_a_far_tile_rejected(precision):
    """The bad point sits in the last tile of a fit spread over every CTA, so
    that another CTA than the one that runs the fit's step raises the flag."""
    m = 3_000_000
    pr = synth.gauss1d(m, seed=12, with_sigma=True, dtype=np.float32)
    sig = pr.sigma.copy()
    sig[m - 7] = 0.0
    dt = torch.float32 if precision == "mixed" else torch.float64
    x, y, s = dev(pr.x, dt), dev(pr.y, dt), dev(sig, dt)
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.curve_fit(pr.model, x, y, pr.p0, sigma=s, precision=precision, **TOL)
    assert e.value.code == gbfit.E_INVALID_ARG
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.evaluate(pr.model, x, y, pr.p0, sigma=s, precision=precision)
    assert e.value.code == gbfit.E_INVALID_ARG
    # the same data with the point restored fits normally on the same context
    out = gbfit.curve_fit(pr.model, x, y, pr.p0, sigma=dev(pr.sigma, dt), precision=precision, **TOL)
    assert out["status"] in (1, 2, 3, 4)
