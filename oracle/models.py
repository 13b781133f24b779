"""Model functions h(x; p) and analytic partials dh/dp (oracle, FP64, NumPy).

Test infrastructure: see the package docstring.

The paper obtains the Jacobian (Section 2, Eq. jacobian) by automatic
differentiation; the library fixes a registry of models with analytic partials
instead (an explicit Jacobian is the alternative Appendix C describes).  These
are written out directly from each model's formula.  Pinned by central
differences in tests/test_oracle_models.py.

Each function takes X as float64 [xdims, m] and p as float64 [n] and returns
(h [m], dh [m, n]).
"""
from __future__ import annotations

import numpy as np

GAUSS1D, DEXP, GAUSS2D, POLY2 = 0, 1, 2, 3
N_PARAMS = {GAUSS1D: 4, DEXP: 5, GAUSS2D: 7, POLY2: 3}
X_DIMS = {GAUSS1D: 1, DEXP: 1, GAUSS2D: 2, POLY2: 1}
NAMES = {GAUSS1D: "gauss1d", DEXP: "dexp", GAUSS2D: "gauss2d", POLY2: "poly2"}


def gauss1d(X, p):
    """h = A exp(-(x-mu)^2/(2 s^2)) + c,  p = (A, mu, s, c)."""
    A, mu, s, c = p
    x = X[0]
    d = x - mu
    e = np.exp(-(d * d) / (2.0 * s * s))
    h = A * e + c
    J = np.empty((x.shape[0], 4))
    J[:, 0] = e
    J[:, 1] = A * e * d / (s * s)
    J[:, 2] = A * e * d * d / (s * s * s)
    J[:, 3] = 1.0
    return h, J


def dexp(X, p):
    """h = a1 exp(-x/t1) + a2 exp(-x/t2) + c,  p = (a1, t1, a2, t2, c)."""
    a1, t1, a2, t2, c = p
    x = X[0]
    e1 = np.exp(-x / t1)
    e2 = np.exp(-x / t2)
    h = a1 * e1 + a2 * e2 + c
    J = np.empty((x.shape[0], 5))
    J[:, 0] = e1
    J[:, 1] = a1 * e1 * x / (t1 * t1)
    J[:, 2] = e2
    J[:, 3] = a2 * e2 * x / (t2 * t2)
    J[:, 4] = 1.0
    return h, J


def gauss2d(X, p):
    """Rotated elliptical 2D Gaussian, p = (A, x0, y0, sx, sy, theta, c).

    u =  (X-x0) cos th + (Y-y0) sin th,  v = -(X-x0) sin th + (Y-y0) cos th,
    h = A exp(-u^2/(2 sx^2) - v^2/(2 sy^2)) + c.
    Partials follow from du/dx0 = -cos, dv/dx0 = sin, du/dy0 = -sin,
    dv/dy0 = -cos, du/dth = v, dv/dth = -u.
    """
    A, x0, y0, sx, sy, th, c = p
    dx = X[0] - x0
    dy = X[1] - y0
    ct, st = np.cos(th), np.sin(th)
    u = dx * ct + dy * st
    v = -dx * st + dy * ct
    isx2 = 1.0 / (sx * sx)
    isy2 = 1.0 / (sy * sy)
    E = np.exp(-0.5 * (u * u * isx2 + v * v * isy2))
    q = A * E
    h = q + c
    J = np.empty((dx.shape[0], 7))
    J[:, 0] = E
    J[:, 1] = q * (u * isx2 * ct - v * isy2 * st)
    J[:, 2] = q * (u * isx2 * st + v * isy2 * ct)
    J[:, 3] = q * u * u * isx2 / sx
    J[:, 4] = q * v * v * isy2 / sy
    J[:, 5] = q * u * v * (isy2 - isx2)
    J[:, 6] = 1.0
    return h, J


def poly2(X, p):
    """h = p0 + p1 x + p2 x^2 (linear in p)."""
    x = X[0]
    J = np.stack([np.ones_like(x), x, x * x], axis=1)
    return J @ np.asarray(p, dtype=np.float64), J


_FUNCS = {GAUSS1D: gauss1d, DEXP: dexp, GAUSS2D: gauss2d, POLY2: poly2}


def value_and_jac(model, X, p):
    """(h, dh/dp) at parameters p; FP64.

    model: a built-in model id, or a callable (X [xdims, m], p [n]) ->
    (h [m], dh/dp [m, n]) -- a user-defined model (the paper's user-written
    fit function, Section 2), whose partials the caller writes out."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[None, :]
    f = model if callable(model) else _FUNCS[model]
    h, J = f(X, np.asarray(p, dtype=np.float64))
    return np.asarray(h, dtype=np.float64), np.asarray(J, dtype=np.float64)
