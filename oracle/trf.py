"""Trust-region-reflective least-squares fit, written out step by step (oracle).

Test infrastructure: see the package docstring.  FP64 NumPy throughout; slow
and plain on purpose.  Each function names the passage of the paper it
follows.  Where the paper is silent or garbled the reading taken is one of:

  R1  Algorithm 2 loops while |phi(alpha_q)| > sigma Delta (the printed test is
      inverted); sigma = 0.1; at most 10 passes.
  R2  Algorithm 1's step carries the minus sign of Eq. lm.
  R3  Algorithm 2 start: u0 = ||g_hat||/Delta, l0 = -phi(0)/phi'(0) when B_hat
      has full rank (else 0), alpha0 = the previous step's alpha (0 at first),
      safeguarded to max(0.001 u, sqrt(l u)) when outside [l0, u0].
  R4  Algorithm 2 order: trial alpha from Eq. alphaupdate at alpha_q, then l, u
      updated from alpha_q, then the trial kept only inside the updated [l, u].
  R5  Algorithm 3 as printed: gamma > 0.75 accept and double Delta;
      0.25 <= gamma <= 0.75 accept; else reject with Delta = ||p||/4.  A
      non-finite trial cost or a non-positive prediction rejects.
  R6  Delta0 = ||D x0|| (1 when zero).
  R7  D = diag(1/x_scale) (default I) or, for x_scale='jac', the running
      maximum of the Jacobian column norms (zeros read as 1).
  R8  Termination ('accuracy condition', unspecified): gtol ||v g||_inf < gtol
      before a trial; ftol accepted step with f - f_new < ftol f; xtol any
      trial with ||w|| < xtol (xtol + ||x||); max_nfev default 100 n.
  R9  Bounds by the Coleman-Li reflective method (named, not stated): see
      coleman_li and select_bounded_step.
  R10 Pseudo-inverse: lambda = s^2 <= lambda_max 8 n eps64 counts as zero.
  R11 sigma weights rows: J_ij / sigma_i, r_i / sigma_i (Eq. easy_jac, easy_res);
      a 2D sigma is the covariance matrix C = L L^T and the method runs on
      L^-1 r, L^-1 J (Eqs. covariance, slsq1, slsq2), pcov from those.
  R12 r = h - y (Eq. residual).
  R13 pcov = V diag(1/s^2) V^T of the unscaled J at the solution (R10 cutoff),
      times 2 f / (m - n) unless absolute_sigma.
  R14 Robust losses (named in Section 5, not stated): cost 1/2 C^2 sum rho(z),
      z = (r/C)^2; the method runs on rows rescaled to the loss's gradient and
      Gauss-Newton Hessian (see reduce.robust_rows); pcov from the rescaled J
      and the robust cost.

Outline of one fit (Algorithm 1, Section 2):
  x <- x0, Delta <- Delta0                                   R6
  evaluate r, J, f, g at x                                    Eqs. residual..gradient
  loop:
    gtol / max_nfev tests                                     R8
    scale: D, Coleman-Li v, dv, C                             Eq. hat, R9
    thin SVD of the scaled Jacobian, uf = U^T r               Appendix B
    trial step p_t = -B^-1 g (pseudo-inverse)                 Algorithm 1
    if ||p_t|| > Delta: alpha from Algorithm 2                Eqs. phi, alphaupdate
    bounded: choose among truncated / reflected / gradient    R9
    x_new, f(x_new), ratio gamma                              Eq. accuracy
    accept and new Delta by Algorithm 3                       R5
    ftol / xtol tests                                         R8
  pcov from the final Jacobian                                R13
"""
from __future__ import annotations

import math

import numpy as np

from . import reduce as _reduce

EPS = float(np.finfo(np.float64).eps)

# Algorithm 2's accuracy sigma (|phi| <= sigma Delta) and iteration cap (R1).
ALG2_SIGMA = 0.1
ALG2_MAX_ITERS = 10

STATUS_NUMERICAL = -1
STATUS_MAX_NFEV = 0
STATUS_GTOL = 1
STATUS_FTOL = 2
STATUS_XTOL = 3
STATUS_FTOL_XTOL = 4


def rank_cut(n: int) -> float:
    """Relative cutoff on lambda = s^2 below which a direction counts as null.

    R10: the paper gives no pseudo-inverse rule.  lambda_i <=
    lambda_max * 8 n eps64 is treated as zero.  The threshold is stated on the
    squared singular values so that a method working from J^T J (whose
    eigenvalues carry absolute error of order eps ||J^T J||) and one working
    from the SVD of J apply the same rule.
    """
    return 8.0 * n * EPS


# ------------------------------------------------------------------ scaling
def coleman_li(x, g, lb, ub):
    """Coleman-Li scaling vector v and its derivative dv (R9).

    v_i = u_i - x_i (dv = -1) if g_i < 0 and u_i finite;
    v_i = x_i - l_i (dv = +1) if g_i > 0 and l_i finite;
    v_i = 1 (dv = 0) otherwise.
    """
    n = x.shape[0]
    v = np.ones(n)
    dv = np.zeros(n)
    up = (g < 0) & np.isfinite(ub)
    lo = (g > 0) & np.isfinite(lb)
    v[up] = ub[up] - x[up]
    dv[up] = -1.0
    v[lo] = x[lo] - lb[lo]
    dv[lo] = 1.0
    return v, dv


def jac_scale_inv(J, prev=None):
    """Column norms of J for x_scale='jac' (R7): max with previous, 0 -> 1."""
    c = np.sqrt(np.sum(J * J, axis=0))
    if prev is not None:
        c = np.maximum(c, prev)
    c[c == 0] = 1.0
    return c


# ------------------------------------------------------------------ subproblem
def scaled_svd(J, r, d, C):
    """Thin SVD of the scaled (augmented) Jacobian (Appendix B).

    J_hat = J diag(d); when C (Coleman-Li diagonal) is given the matrix is
    augmented with rows diag(sqrt(C)) whose residual entries are zero.
    Returns lam = s^2 (after the rank cutoff), V, and gV = Sigma U^T r, which
    equals V^T g_hat (so that p(alpha) = -V (Sigma^2 + alpha)^-1 gV,
    Eq. reducedlm with the sign of Eq. lm).
    """
    n = J.shape[1]
    Jh = J * d[None, :]
    ra = r
    if C is not None:
        Jh = np.vstack([Jh, np.diag(np.sqrt(C))])
        ra = np.concatenate([r, np.zeros(n)])
    U, s, Vt = np.linalg.svd(Jh, full_matrices=False)
    uf = U.T @ ra
    lam = s * s
    lmax = lam.max() if lam.size else 0.0
    keep = lam > lmax * rank_cut(n) if lmax > 0 else np.zeros(n, dtype=bool)
    gV = np.where(keep, s * uf, 0.0)
    lam = np.where(keep, lam, 0.0)
    return lam, Vt.T, gV, bool(keep.all())


def _ratio(num, den):
    """num/den where num != 0, else 0 (null directions contribute nothing)."""
    out = np.zeros_like(num)
    nz = num != 0
    out[nz] = num[nz] / den[nz]
    return out


def phi_and_derivative(alpha, lam, gV, Delta):
    """phi(alpha) = ||(B + alpha I)^-1 g|| - Delta and phi'(alpha) (Eq. phi).

    With B = V diag(lam) V^T:  ||p||^2 = sum gV^2/(lam+alpha)^2 and
    d||p||/dalpha = -sum gV^2/(lam+alpha)^3 / ||p||.
    """
    den = lam + alpha
    q = _ratio(gV, den)
    pn = math.sqrt(float(q @ q))
    phi = pn - Delta
    dphi = -float(np.sum(_ratio(gV * gV, den ** 3))) / pn
    return phi, dphi


def lm_parameter(lam, gV, ghat_norm, Delta, alpha0, full_rank):
    """Levenberg-Marquardt parameter alpha by Algorithm 2.

    Readings of the printed algorithm (R1, R3, R4):
      * the loop runs while |phi(alpha_q)| > sigma Delta (the printed '<=' is
        inverted), sigma = 0.1, at most 10 iterations;
      * u_0 = ||g_hat|| / Delta; l_0 = -phi(0)/phi'(0) when B_hat has full
        rank, else 0; alpha_0 is the previous step's alpha, replaced by
        max(0.001 u, sqrt(l u)) when it lies outside [l_0, u_0];
      * each pass computes the Newton-type trial alpha_t (Eq. alphaupdate) and
        updates l and u from the current alpha_q, then keeps alpha_t only if
        it lies in the updated [l, u], else takes max(0.001 u, sqrt(l u)).
    """
    u = ghat_norm / Delta
    if full_rank:
        phi0, dphi0 = phi_and_derivative(0.0, lam, gV, Delta)
        l = -phi0 / dphi0
    else:
        l = 0.0
    alpha = alpha0
    if not (l <= alpha <= u):
        alpha = max(0.001 * u, math.sqrt(l * u))
    for _ in range(ALG2_MAX_ITERS):
        phi, dphi = phi_and_derivative(alpha, lam, gV, Delta)
        if abs(phi) <= ALG2_SIGMA * Delta:
            break
        alpha_t = alpha - ((phi + Delta) / Delta) * (phi / dphi)
        l = max(l, alpha - phi / dphi)
        if phi < 0:
            u = alpha
        if l <= alpha_t <= u:
            alpha = alpha_t
        else:
            alpha = max(0.001 * u, math.sqrt(l * u))
    return alpha


def tr_solve(lam, V, gV, ghat_norm, Delta, alpha_prev, full_rank):
    """Algorithm 1's step in scaled space: trial p_t, else Algorithm 2.

    p_t = -B_hat^+ g_hat (pseudo-inverse); if ||p_t|| <= Delta it is taken
    with alpha = 0, otherwise p = -(B_hat + alpha I)^-1 g_hat (R2:
    the sign of Eq. lm) with alpha from lm_parameter.
    """
    pt = -V @ _ratio(gV, lam)
    if np.linalg.norm(pt) <= Delta:
        return pt, 0.0
    alpha = lm_parameter(lam, gV, ghat_norm, Delta, alpha_prev, full_rank)
    return -V @ _ratio(gV, lam + alpha), alpha


def tr_radius_update(gamma, Delta, pnorm):
    """Algorithm 3 (R5: the paper's thresholds, not SciPy's).

    gamma > 0.75: accept, Delta <- 2 Delta; 0.25 <= gamma <= 0.75: accept,
    Delta kept; otherwise (including NaN) reject, Delta <- 0.25 ||p||.
    """
    if gamma > 0.75:
        return True, 2.0 * Delta
    if 0.25 <= gamma <= 0.75:
        return True, Delta
    return False, 0.25 * pnorm


# ------------------------------------------------------------------ bounds
def step_to_bound(x, s, lb, ub):
    """Largest t >= 0 with lb <= x + t s <= ub, and the components that bind."""
    t = np.full(x.shape[0], np.inf)
    pos = s > 0
    neg = s < 0
    t[pos] = (ub[pos] - x[pos]) / s[pos]
    t[neg] = (lb[neg] - x[neg]) / s[neg]
    tmin = float(np.min(t)) if t.size else np.inf
    return max(tmin, 0.0), (t == tmin) & np.isfinite(t)


def tr_intersect(s0, r, Delta):
    """Positive root t of ||s0 + t r|| = Delta (s0 inside the region)."""
    a = float(r @ r)
    b = 2.0 * float(s0 @ r)
    c = float(s0 @ s0) - Delta * Delta
    disc = math.sqrt(max(b * b - 4.0 * a * c, 0.0))
    if b <= 0:
        return (-b + disc) / (2.0 * a)
    return (2.0 * c) / (-b - disc)


def quad_value(Jh, gh, C, s):
    """Scaled quadratic model q(s) = g_hat.s + 1/2 (||J_hat s||^2 + sum C s^2) (Eq. hat)."""
    Js = Jh @ s
    val = float(gh @ s) + 0.5 * float(Js @ Js)
    if C is not None:
        val += 0.5 * float(np.sum(C * s * s))
    return val


def minimize_on_segment(Jh, gh, C, s0, r, t_lo, t_hi):
    """Minimise t -> q(s0 + t r) on [t_lo, t_hi]; returns (t, value)."""
    Jr = Jh @ r
    curv = float(Jr @ Jr) + (float(np.sum(C * r * r)) if C is not None else 0.0)
    slope = float(gh @ r) + float((Jh @ s0) @ Jr) + (float(np.sum(C * s0 * r)) if C is not None else 0.0)
    cands = [t_lo, t_hi]
    if curv > 0:
        ts = -slope / curv
        if t_lo < ts < t_hi:
            cands.append(ts)
    best_t, best_v = None, np.inf
    for t in cands:
        v = quad_value(Jh, gh, C, s0 + t * r)
        if v < best_v:
            best_t, best_v = t, v
    return best_t, best_v


def select_bounded_step(x, lb, ub, d, Jh, gh, C, s_tr, Delta, theta):
    """Coleman-Li reflective step selection (R9; parity unpinned).

    Section 2 cites the Coleman-Li method for bounds without stating it.  The
    candidates, all in scaled space (unscaled step = d * s):
      A  the trust-region step truncated at the first bound it crosses and
         stepped back by theta;
      B  from that bound point, the direction with the crossing components
         reflected, minimised along the segment that stays inside both the box
         (stepped back by theta) and the trust region, starting at
         (1 - theta) of the segment;
      C  the scaled anti-gradient -g_hat, limited by the region and the box
         (stepped back by theta), minimised along its segment.
    If the full step stays within the box it is taken as is.  Otherwise the
    candidate with the lowest model value wins (ties: A, then B, then C).
    Returns (s_hat, model value, kind) with kind in 'full', 'A', 'B', 'C'.
    """
    s_full = d * s_tr
    if np.all(x + s_full >= lb) and np.all(x + s_full <= ub):
        return s_tr, quad_value(Jh, gh, C, s_tr), "full"
    tau, hits = step_to_bound(x, s_full, lb, ub)
    # A: truncated
    sA = theta * tau * s_tr
    best_s, best_v, kind = sA, quad_value(Jh, gh, C, sA), "A"
    # B: reflected
    sb = tau * s_tr
    rh = s_tr.copy()
    rh[hits] = -rh[hits]
    xb = x + d * sb
    t_box, _ = step_to_bound(xb, d * rh, lb, ub)
    t_tr = tr_intersect(sb, rh, Delta)
    t_max = min(t_box, t_tr)
    if t_max > 0:
        t_lo = (1.0 - theta) * t_max
        t_hi = theta * t_box if t_box <= t_tr else t_tr
        if t_lo <= t_hi:
            tB, vB = minimize_on_segment(Jh, gh, C, sb, rh, t_lo, t_hi)
            if vB < best_v:
                best_s, best_v, kind = sb + tB * rh, vB, "B"
    # C: scaled anti-gradient
    ag = -gh
    agn = float(np.linalg.norm(ag))
    if agn > 0:
        t_tr = Delta / agn
        t_box, _ = step_to_bound(x, d * ag, lb, ub)
        t_hi = theta * t_box if t_box < t_tr else t_tr
        tC, vC = minimize_on_segment(Jh, gh, C, np.zeros_like(ag), ag, 0.0, t_hi)
        if vC < best_v:
            best_s, best_v, kind = tC * ag, vC, "C"
    return best_s, best_v, kind


def make_strictly_feasible(x, lb, ub):
    """Move components on or beyond a bound one ulp inside it."""
    x = x.copy()
    lo = x <= lb
    hi = x >= ub
    x[lo] = np.nextafter(lb[lo], np.inf)
    x[hi] = np.nextafter(ub[hi], -np.inf)
    return x


# ------------------------------------------------------------------ the fit
def covariance(J, cost, m, n, absolute_sigma):
    """pcov (R13): V diag(1/s^2) V^T of the unscaled J at the solution,
    null directions (rank_cut) dropped, times 2 cost / (m - n) unless
    absolute_sigma; all +inf when m <= n."""
    if m <= n:
        return np.full((n, n), np.inf)
    _, s, Vt = np.linalg.svd(J, full_matrices=False)
    lam = s * s
    keep = lam > lam.max() * rank_cut(n) if lam.max() > 0 else np.zeros(n, bool)
    inv = np.where(keep, 1.0 / np.where(keep, lam, 1.0), 0.0)
    pcov = (Vt.T * inv[None, :]) @ Vt
    if not absolute_sigma:
        pcov = pcov * (2.0 * cost / (m - n))
    return pcov


def curve_fit(model, X, y, sigma=None, p0=None, lb=None, ub=None, ftol=1e-8, xtol=1e-8,
              gtol=1e-8, max_nfev=None, x_scale=1.0, absolute_sigma=False, record=False,
              loss="linear", f_scale=1.0):
    """Fit model `model` to (X, y) with per-point sigma (or, 2D, the
    covariance matrix of y) by the TRF method.

    Returns a dict: popt, pcov, cost, nfev, njev, status and (if record) the
    per-trial history used by the invariant tests.

    Termination (R8; the paper's 'accuracy condition' is unspecified):
      gtol  ||v * g||_inf < gtol, tested before each trial (status 1);
      ftol  an accepted step with f - f_new < ftol f (status 2);
      xtol  any trial step with ||w|| < xtol (xtol + ||x||) (status 3);
      both ftol and xtol on the same step: status 4;
      nfev >= max_nfev (default 100 n): status 0;
      non-finite cost or Jacobian at x0: status -1.
    A non-finite cost at a trial point rejects the step (Delta <- 0.25 ||p||).
    """
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[None, :]
    y = np.asarray(y, dtype=np.float64)
    m = y.shape[0]
    x = np.array(p0, dtype=np.float64)
    n = x.shape[0]
    lb = np.full(n, -np.inf) if lb is None else np.asarray(lb, dtype=np.float64)
    ub = np.full(n, np.inf) if ub is None else np.asarray(ub, dtype=np.float64)
    if np.any(lb >= ub):
        raise ValueError("lb must be < ub")
    if np.any(x <= lb) or np.any(x >= ub):
        raise ValueError("p0 is not strictly inside the bounds")
    if max_nfev is None:
        max_nfev = 100 * n
    bounded = bool(np.any(np.isfinite(lb)) or np.any(np.isfinite(ub)))
    w = _reduce.weights(sigma, m)
    jac_scale = isinstance(x_scale, str) and x_scale == "jac"

    if loss not in _reduce.LOSSES:
        raise ValueError(f"unknown loss {loss!r}")
    if not f_scale > 0:
        raise ValueError("f_scale must be > 0")
    f, g, _, r, J = _reduce.evaluate(model, X, y, w, x, loss, f_scale)
    nfev, njev = 1, 1
    hist = []
    out = dict(nfev=nfev, njev=njev)
    if not (np.isfinite(f) and np.all(np.isfinite(J))):
        return dict(popt=x, pcov=np.full((n, n), np.inf), cost=f, nfev=1, njev=1,
                    status=STATUS_NUMERICAL, history=hist)

    if jac_scale:
        scale_inv = jac_scale_inv(J)
        sx = 1.0 / scale_inv
    else:
        scale_inv = None
        sx = np.broadcast_to(np.asarray(x_scale, dtype=np.float64), (n,)).copy()
    v, dv = coleman_li(x, g, lb, ub)
    Delta = float(np.linalg.norm(x / (np.sqrt(v) * sx)))   # R6: ||D x0||
    if Delta == 0.0:
        Delta = 1.0
    alpha = 0.0
    status = None
    while True:
        gnorm = float(np.max(np.abs(v * g)))
        if gnorm < gtol:
            status = STATUS_GTOL
            break
        if nfev >= max_nfev:
            status = STATUS_MAX_NFEV
            break
        d = np.sqrt(v) * sx
        gh = d * g
        C = g * dv * sx * sx if bounded else None
        lam, V, gV, full_rank = scaled_svd(J, r, d, C)
        Jh = J * d[None, :]
        theta = max(0.995, 1.0 - gnorm)

        s_tr, alpha = tr_solve(lam, V, gV, float(np.linalg.norm(gh)), Delta, alpha, full_rank)
        if bounded:
            s_h, qval, kind = select_bounded_step(x, lb, ub, d, Jh, gh, C, s_tr, Delta, theta)
        else:
            s_h, qval, kind = s_tr, quad_value(Jh, gh, None, s_tr), "full"
        predicted = -qval
        step = d * s_h
        x_new = x + step
        if bounded:
            x_new = make_strictly_feasible(x_new, lb, ub)
        f_new, g_new, _, r_new, J_new = _reduce.evaluate(model, X, y, w, x_new, loss, f_scale)
        nfev += 1
        actual = f - f_new
        s_norm = float(np.linalg.norm(s_h))
        if np.isfinite(f_new) and predicted > 0:
            gamma = actual / predicted
        else:
            gamma = -np.inf
        accepted, Delta_new = tr_radius_update(gamma, Delta, s_norm)
        step_norm = float(np.linalg.norm(step))
        ftol_ok = accepted and actual < ftol * f
        xtol_ok = step_norm < xtol * (xtol + float(np.linalg.norm(x)))
        if record:
            hist.append(dict(x=x.copy(), x_new=x_new.copy(), f=f, f_new=f_new,
                             predicted=predicted, gamma=gamma, accepted=accepted,
                             Delta=Delta, Delta_new=Delta_new, alpha=alpha,
                             s_norm=s_norm, step=step.copy(), g=g.copy(), v=v.copy(),
                             kind=kind))
        if accepted:
            x, f, g, r, J = x_new, f_new, g_new, r_new, J_new
            njev += 1
            if jac_scale:
                scale_inv = jac_scale_inv(J, scale_inv)
                sx = 1.0 / scale_inv
            v, dv = coleman_li(x, g, lb, ub)
        Delta = Delta_new
        if ftol_ok and xtol_ok:
            status = STATUS_FTOL_XTOL
        elif ftol_ok:
            status = STATUS_FTOL
        elif xtol_ok:
            status = STATUS_XTOL
        if status is not None:
            break

    pcov = covariance(J, f, m, n, absolute_sigma)
    out = dict(popt=x, pcov=pcov, cost=f, nfev=nfev, njev=njev, status=status, history=hist,
               g=g, v=v)
    return out


def curve_fit_problem(pr, **kw):
    """curve_fit on a synth.Problem-like object (coords(), y, sigma, p0, lb, ub)."""
    return curve_fit(pr.model, pr.coords(), pr.y, pr.sigma, pr.p0, pr.lb, pr.ub, **kw)
