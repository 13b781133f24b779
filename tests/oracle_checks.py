"""Oracle-side criteria for comparing a mixed-precision fit with the FP64 oracle.

A fit's popt can be compared with the oracle's to 1e-6 (relative,
|dp| / max(|p|, 1)) only where the oracle's own popt is determined to that
level.  It is not determined (the fit is "ill-conditioned" here) when any of
these hold, all computed by the oracle alone:
  * some parameter's standard error (the oracle's pcov) exceeds 10 % of the
    parameter;
  * rounding-sensitive: the oracle's popt moves by more than 1e-7 when y is
    perturbed by 1e-12 relative (rounding-level changes at every evaluation
    decide where its iteration stops);
  * tolerance-limited: continuing the oracle from its own popt with
    tolerances 1e-15 moves popt by more than 1e-7 (the requested tolerances
    stop it before its optimum is resolved to 1e-6).
For such a fit the comparison is on the objective the paper minimises: the
oracle's FP64 cost (Eq. msqe) at the GPU's popt must not exceed the oracle's
own cost by more than 1e-9 relative.

The double exponential is symmetric under (a1, t1) <-> (a2, t2); popt is
compared with t1 <= t2 on both sides (the canonical form of reading c14).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import reduce as red, trf

MODEL_DEXP = 1


def canonical(model: int, p) -> np.ndarray:
    p = np.asarray(p, dtype=np.float64)
    if model == MODEL_DEXP and p[1] > p[3]:
        return p[[2, 3, 0, 1, 4]]
    return p


def relerr(model: int, a, b) -> float:
    a, b = canonical(model, a), canonical(model, b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


def oracle_cost(pr, p) -> float:
    """f = 1/2 sum r_i^2 at p by the oracle's FP64 reduction."""
    return float(red.evaluate(pr.model, pr.coords(), pr.y, red.weights(pr.sigma, pr.m), np.asarray(p))[0])


def determined(pr, ref, tol: dict) -> tuple[bool, str]:
    """Whether the oracle's popt (ref, from trf.curve_fit_problem(pr, **tol))
    is determined to 1e-6; the reason when it is not."""
    p = ref["popt"]
    se = np.sqrt(np.abs(np.diag(ref["pcov"])))
    if not np.all(np.isfinite(se)) or np.max(se / np.maximum(np.abs(p), 1e-300)) > 0.1:
        return False, "standard error above 10%"
    rng = np.random.default_rng(12345)
    yp = np.asarray(pr.y, dtype=np.float64) * (1.0 + 1e-12 * rng.standard_normal(pr.m))
    alt = trf.curve_fit_problem(dataclasses.replace(pr, y=yp), **tol)
    if relerr(pr.model, alt["popt"], p) > 1e-7:
        return False, "rounding-sensitive"
    tight = trf.curve_fit(pr.model, pr.coords(), pr.y, pr.sigma, p, pr.lb, pr.ub, ftol=1e-15, xtol=1e-15,
                          gtol=1e-15)
    if relerr(pr.model, tight["popt"], p) > 1e-7:
        return False, "tolerance-limited"
    return True, ""


def check_mixed(pr, popt, ref, tol: dict, rel: float = 1e-6, cost_rel: float = 1e-9) -> str:
    """Assert the mixed fit popt against the oracle's ref; returns the reason
    when the fit was judged by cost (empty when by popt)."""
    ok, why = determined(pr, ref, tol)
    if ok:
        e = relerr(pr.model, popt, ref["popt"])
        assert e <= rel, f"popt differs from the oracle by {e:.3e} (determined fit)"
        return ""
    f_gpu = oracle_cost(pr, popt)
    assert f_gpu <= ref["cost"] * (1.0 + cost_rel), \
        f"cost {f_gpu!r} above the oracle's {ref['cost']!r} by {(f_gpu - ref['cost']) / ref['cost']:.3e} ({why})"
    return why
