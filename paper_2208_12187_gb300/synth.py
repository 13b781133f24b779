"""Seeded synthetic curve-fit problems shaped like the paper's workloads.

This module only *draws inputs*: coordinates, noisy observations, per-point
uncertainties, seed parameters and bounds.  It holds none of the fitting
method's arithmetic (no residuals, Jacobians, reductions or trust-region
steps).  To synthesise observations it needs the forward value of each model
at the true parameters; those few lines are written here on their own so that
neither the CUDA path nor the oracle is imported by the other through it.

The paper's own dataset (Section 4: rotated elliptical 2D Gaussians with
uniformly drawn parameters and fixed-sigma Gaussian noise, data lengths 1e4 to
8e6) is itself synthetic and its parameter ranges are not given; the problems
below stand in for it with stated, seeded recipes.

Model ids (shared vocabulary of the library, the oracle and this module):
  0  gauss1d : h = A exp(-(x-mu)^2 / (2 s^2)) + c            p = (A, mu, s, c)
  1  dexp    : h = a1 exp(-x/t1) + a2 exp(-x/t2) + c          p = (a1, t1, a2, t2, c)
  2  gauss2d : h = A exp(-u^2/(2 sx^2) - v^2/(2 sy^2)) + c
               u =  (X-x0) cos(th) + (Y-y0) sin(th)
               v = -(X-x0) sin(th) + (Y-y0) cos(th)            p = (A, x0, y0, sx, sy, th, c)
  3  poly2   : h = p0 + p1 x + p2 x^2   (linear in p; closed-form test model)
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

MODEL_GAUSS1D = 0
MODEL_DEXP = 1
MODEL_GAUSS2D = 2
MODEL_POLY2 = 3

N_PARAMS = {MODEL_GAUSS1D: 4, MODEL_DEXP: 5, MODEL_GAUSS2D: 7, MODEL_POLY2: 3}
X_DIMS = {MODEL_GAUSS1D: 1, MODEL_DEXP: 1, MODEL_GAUSS2D: 2, MODEL_POLY2: 1}

# x layouts (same numbering as the C ABI)
LAYOUT_VEC = 0    # x: [m]
LAYOUT_SOA2 = 1   # x: [2, m]  (X row then Y row)
LAYOUT_GRID = 2   # no x array: point i is pixel (X = i % W, Y = i // W)


@dataclasses.dataclass
class Problem:
    """One fit's inputs.  Arrays are host NumPy arrays."""
    model: int
    x: Optional[np.ndarray]          # None for LAYOUT_GRID
    layout: int
    grid_wh: Optional[tuple]         # (W, H) for LAYOUT_GRID
    y: np.ndarray
    sigma: Optional[np.ndarray]
    p0: np.ndarray
    lb: Optional[np.ndarray]
    ub: Optional[np.ndarray]
    truth: np.ndarray
    n_user: Optional[int] = None     # parameter count of a user-defined model family

    @property
    def m(self) -> int:
        return int(self.y.shape[0])

    @property
    def n(self) -> int:
        return self.n_user if self.n_user is not None else N_PARAMS[self.model]

    def coords(self) -> np.ndarray:
        """Explicit coordinates as float64 [xdims, m] (grid expanded)."""
        if self.layout == LAYOUT_GRID:
            W, H = self.grid_wh
            i = np.arange(W * H, dtype=np.int64)
            return np.stack([(i % W).astype(np.float64), (i // W).astype(np.float64)])
        x = np.asarray(self.x, dtype=np.float64)
        return x.reshape(1, -1) if x.ndim == 1 else x

    def astype(self, dtype) -> "Problem":
        """Same problem with data arrays cast to dtype (parameters, and a
        covariance-matrix sigma, stay float64)."""
        cast = lambda a: None if a is None else np.ascontiguousarray(a, dtype=dtype)
        sg = self.sigma if (self.sigma is not None and np.ndim(self.sigma) == 2) else cast(self.sigma)
        return dataclasses.replace(self, x=cast(self.x), y=cast(self.y), sigma=sg)


# ---------------------------------------------------------------- forward values
def _forward(model: int, X: np.ndarray, p: np.ndarray) -> np.ndarray:
    """Noise-free model value used only to synthesise observations (float64)."""
    if model == MODEL_GAUSS1D:
        A, mu, s, c = p
        return A * np.exp(-((X[0] - mu) ** 2) / (2.0 * s * s)) + c
    if model == MODEL_DEXP:
        a1, t1, a2, t2, c = p
        return a1 * np.exp(-X[0] / t1) + a2 * np.exp(-X[0] / t2) + c
    if model == MODEL_GAUSS2D:
        A, x0, y0, sx, sy, th, c = p
        dx, dy = X[0] - x0, X[1] - y0
        ct, st = math.cos(th), math.sin(th)
        u = dx * ct + dy * st
        v = -dx * st + dy * ct
        return A * np.exp(-0.5 * (u * u / (sx * sx) + v * v / (sy * sy))) + c
    if model == MODEL_POLY2:
        return p[0] + p[1] * X[0] + p[2] * X[0] ** 2
    raise ValueError(f"unknown model {model}")


def forward_values(model: int, X: np.ndarray, p) -> np.ndarray:
    """Public alias of the synthesis forward model (float64 [m])."""
    return _forward(model, np.asarray(X, dtype=np.float64).reshape(-1, np.shape(X)[-1]),
                    np.asarray(p, dtype=np.float64))


# ---------------------------------------------------------------- generators
def gauss1d(m: int = 10_000, seed: int = 0, noise: float = 0.1, with_sigma: bool = False,
            truth=(5.0, 0.3, 1.2, 0.5), dtype=np.float64, noise_free: bool = False) -> Problem:
    """1D Gaussian + offset: x ~ U[-10, 10], additive N(0, noise^2), p0 = truth*(1+U(-.2,.2))."""
    rng = np.random.default_rng(seed)
    truth = np.asarray(truth, dtype=np.float64)
    x = rng.uniform(-10.0, 10.0, size=m)
    y = _forward(MODEL_GAUSS1D, x[None, :], truth)
    e = rng.normal(0.0, noise, size=m)
    if not noise_free:
        y = y + e
    p0 = truth * (1.0 + rng.uniform(-0.2, 0.2, size=4))
    sigma = np.ones(m) if with_sigma else None
    return Problem(MODEL_GAUSS1D, x, LAYOUT_VEC, None, y, sigma, p0, None, None,
                   truth).astype(dtype)


def dexp_params(rng) -> np.ndarray:
    """Double-exponential truth: t1,t2 log-U[0.1,100]; a1,a2 U[1,10]; c U[0,1]."""
    t1, t2 = np.exp(rng.uniform(math.log(0.1), math.log(100.0), size=2))
    a1, a2 = rng.uniform(1.0, 10.0, size=2)
    c = rng.uniform(0.0, 1.0)
    return np.array([a1, t1, a2, t2, c])


def dexp(m: int, seed: int = 0, truth=None, dtype=np.float64, noise_free: bool = False,
         bounded: bool = True) -> Problem:
    """Double exponential: x ~ U[0, 5 max(t)], noise N(0, (0.01 (a1+a2+c))^2), t > 0 bounds."""
    rng = np.random.default_rng(seed)
    truth = dexp_params(rng) if truth is None else np.asarray(truth, dtype=np.float64)
    x = rng.uniform(0.0, 5.0 * max(truth[1], truth[3]), size=m)
    y = _forward(MODEL_DEXP, x[None, :], truth)
    e = rng.normal(0.0, 0.01 * (truth[0] + truth[2] + truth[4]), size=m)
    if not noise_free:
        y = y + e
    p0 = truth * (1.0 + rng.uniform(-0.2, 0.2, size=5))
    lb = ub = None
    if bounded:
        lb = np.array([-np.inf, 0.0, -np.inf, 0.0, -np.inf])
        ub = np.full(5, np.inf)
    return Problem(MODEL_DEXP, x, LAYOUT_VEC, None, y, None, p0, lb, ub, truth).astype(dtype)


def gauss2d_grid(W: int = 1024, H: Optional[int] = None, seed: int = 0, truth=None,
                 dtype=np.float32, layout: int = LAYOUT_GRID, poisson: bool = True,
                 bounded: bool = True) -> Problem:
    """Rotated 2D Gaussian on a W x H pixel grid with Poisson counts.

    Default truth for 1024 x 1024: A=980, c=20 (peak 1000 on background 20),
    x0=512.3, y0=498.7, sx=60, sy=35, theta=0.4.  Other sizes scale centre and
    widths with W.  sigma = sqrt(max(y, 1)).  Bounds: sx, sy in [0.5, 500],
    theta in [-pi/2, pi/2].  p0: A, c, sx, sy x (1+U(-.2,.2)); x0, y0 + U(-5,5);
    theta + U(-0.1, 0.1).
    """
    H = W if H is None else H
    rng = np.random.default_rng(seed)
    if truth is None:
        k = W / 1024.0
        truth = np.array([980.0, 512.3 * k, 498.7 * H / 1024.0, 60.0 * k, 35.0 * k, 0.4, 20.0])
    truth = np.asarray(truth, dtype=np.float64)
    i = np.arange(W * H, dtype=np.int64)
    X = np.stack([(i % W).astype(np.float64), (i // W).astype(np.float64)])
    mu = _forward(MODEL_GAUSS2D, X, truth)
    y = rng.poisson(mu).astype(np.float64) if poisson else mu
    sigma = np.sqrt(np.maximum(y, 1.0))
    p0 = truth.copy()
    for j in (0, 6, 3, 4):
        p0[j] *= 1.0 + rng.uniform(-0.2, 0.2)
    p0[1] += rng.uniform(-5.0, 5.0)
    p0[2] += rng.uniform(-5.0, 5.0)
    p0[5] += rng.uniform(-0.1, 0.1)
    lb = ub = None
    if bounded:
        lb = np.array([-np.inf, -np.inf, -np.inf, 0.5, 0.5, -math.pi / 2, -np.inf])
        ub = np.array([np.inf, np.inf, np.inf, 500.0, 500.0, math.pi / 2, np.inf])
        p0 = np.clip(p0, lb + 1e-6, ub - 1e-6)
    x = None if layout == LAYOUT_GRID else X
    return Problem(MODEL_GAUSS2D, x, layout, (W, H) if layout == LAYOUT_GRID else None,
                   y, sigma, p0, lb, ub, truth).astype(dtype)


def poly2(m: int = 1000, seed: int = 0, truth=(1.5, -0.7, 0.25), noise: float = 0.05,
          with_sigma: bool = True, dtype=np.float64) -> Problem:
    """Quadratic polynomial (linear least squares): x ~ U[-3, 3], sigma ~ U[0.5, 2]."""
    rng = np.random.default_rng(seed)
    truth = np.asarray(truth, dtype=np.float64)
    x = rng.uniform(-3.0, 3.0, size=m)
    sigma = rng.uniform(0.5, 2.0, size=m) if with_sigma else None
    y = _forward(MODEL_POLY2, x[None, :], truth)
    y = y + rng.normal(0.0, noise, size=m) * (sigma if sigma is not None else 1.0)
    p0 = truth + rng.uniform(-1.0, 1.0, size=3)
    return Problem(MODEL_POLY2, x, LAYOUT_VEC, None, y, sigma, p0, None, None, truth).astype(dtype)


# ---------------------------------------------------------------- batched fits
@dataclasses.dataclass
class Batch:
    """Many independent fits of one model, concatenated (segment offsets)."""
    model: int
    x: np.ndarray            # [total]  (1D models)
    y: np.ndarray            # [total]
    sigma: Optional[np.ndarray]
    offsets: np.ndarray      # int64 [nfits + 1]
    p0: np.ndarray           # [nfits, n]
    lb: Optional[np.ndarray] # [nfits, n]
    ub: Optional[np.ndarray]
    truth: np.ndarray        # [nfits, n]

    @property
    def nfits(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def fit(self, k: int) -> Problem:
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        sig = None if self.sigma is None else self.sigma[a:b]
        lb = None if self.lb is None else self.lb[k]
        ub = None if self.ub is None else self.ub[k]
        return Problem(self.model, self.x[a:b], LAYOUT_VEC, None, self.y[a:b], sig,
                       self.p0[k].copy(), lb, ub, self.truth[k])


# ---------------------------------------------------------------- user-defined model families
# Fit functions a user supplies as source text (the library compiles them at
# run time; the tests write each one a second time as NumPy for the oracle).
# Here only their forward values, to synthesise observations.  The returned
# Problem has model = -1 until the caller puts in the registered model id.
USER_FAMILIES = {
    # name: (n, x_dims, formula)
    "lorentz1d": (4, 1, "A / (1 + ((x - x0) / g)^2) + c;  p = (A, x0, g, c)"),
    "gauss2d_axis": (6, 2, "A exp(-(X-x0)^2/(2 sx^2) - (Y-y0)^2/(2 sy^2)) + c;  p = (A, x0, y0, sx, sy, c)"),
    "damped_sine": (5, 1, "A exp(-x / tau) sin(w x + phi) + c;  p = (A, tau, w, phi, c)"),
}


def _user_forward(family: str, X: np.ndarray, p: np.ndarray) -> np.ndarray:
    if family == "lorentz1d":
        A, x0, g, c = p
        u = (X[0] - x0) / g
        return A / (1.0 + u * u) + c
    if family == "gauss2d_axis":
        A, x0, y0, sx, sy, c = p
        return A * np.exp(-((X[0] - x0) ** 2) / (2 * sx * sx) - ((X[1] - y0) ** 2) / (2 * sy * sy)) + c
    if family == "damped_sine":
        A, tau, w, phi, c = p
        return A * np.exp(-X[0] / tau) * np.sin(w * X[0] + phi) + c
    raise ValueError(f"unknown family {family}")


def user_family(family: str, m: int = 5000, seed: int = 0, dtype=np.float64, layout: int = LAYOUT_VEC,
                with_sigma: bool = False) -> Problem:
    """Seeded problem of a user-defined model family.

    lorentz1d:    x ~ U[-10, 10], truth (4, 0.5, 1.5, 0.3), noise N(0, 0.05^2), p0 = truth (1 + U(-.2, .2))
    gauss2d_axis: W x W pixel grid (W = round(sqrt(m))), truth (50, 0.45 W, 0.55 W, 0.1 W, 0.07 W, 2),
                  noise N(0, 1), p0: A, sx, sy, c x (1 + U(-.2, .2)), centre + U(-1, 1);
                  bounds sx, sy in [0.5, W]
    damped_sine:  x ~ U[0, 10], truth (3, 4, 2.5, 0.4, 0.2), noise N(0, 0.05^2), p0 = truth (1 + U(-.05, .05))
    with_sigma: per-point sigma ~ U[0.5, 1.5] (noise scaled by it)."""
    rng = np.random.default_rng(seed)
    n, xd, _ = USER_FAMILIES[family]
    lb = ub = None
    grid = None
    if family == "lorentz1d":
        truth = np.array([4.0, 0.5, 1.5, 0.3])
        x = rng.uniform(-10.0, 10.0, size=m)
        X = x[None, :]
        noise = 0.05
        p0 = truth * (1.0 + rng.uniform(-0.2, 0.2, size=n))
    elif family == "gauss2d_axis":
        W = int(round(math.sqrt(m)))
        m = W * W
        truth = np.array([50.0, 0.45 * W, 0.55 * W, 0.1 * W, 0.07 * W, 2.0])
        i = np.arange(m, dtype=np.int64)
        X = np.stack([(i % W).astype(np.float64), (i // W).astype(np.float64)])
        x = None if layout == LAYOUT_GRID else X.copy()
        grid = (W, W) if layout == LAYOUT_GRID else None
        noise = 1.0
        p0 = truth.copy()
        for k in (0, 3, 4, 5):
            p0[k] *= 1.0 + rng.uniform(-0.2, 0.2)
        p0[1:3] += rng.uniform(-1.0, 1.0, size=2)
        lb = np.array([-np.inf, -np.inf, -np.inf, 0.5, 0.5, -np.inf])
        ub = np.array([np.inf, np.inf, np.inf, float(W), float(W), np.inf])
    elif family == "damped_sine":
        truth = np.array([3.0, 4.0, 2.5, 0.4, 0.2])
        x = rng.uniform(0.0, 10.0, size=m)
        X = x[None, :]
        noise = 0.05
        p0 = truth * (1.0 + rng.uniform(-0.05, 0.05, size=n))
    else:
        raise ValueError(f"unknown family {family}")
    sig = rng.uniform(0.5, 1.5, size=m) if with_sigma else None
    e = rng.normal(0.0, noise, size=m) * (sig if sig is not None else 1.0)
    y = _user_forward(family, X, truth) + e
    lay = layout if xd == 2 else LAYOUT_VEC
    return Problem(-1, x, lay, grid, y, sig, p0, lb, ub, truth, n_user=n).astype(dtype)


# ---------------------------------------------------------------- correlated errors
def ar1_covariance(m: int, rho: float, scale: float, seed: int = 0) -> np.ndarray:
    """C_ij = s_i s_j rho^|i-j|: stationary exponential correlation between
    neighbouring points (in index order) with per-point scales s ~ scale U[0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    s = scale * rng.uniform(0.5, 1.5, m)
    i = np.arange(m)
    return np.outer(s, s) * rho ** np.abs(i[:, None] - i[None, :]).astype(np.float64)


def with_covariance(pr: Problem, rho: float = 0.5, scale: float = 0.1, seed: int = 0) -> Problem:
    """The problem with its noise replaced by N(0, C) for C = ar1_covariance
    and sigma = C (the [m, m] covariance matrix, FP64)."""
    C = ar1_covariance(pr.m, rho, scale, seed)
    rng = np.random.default_rng(seed + 1)
    if pr.model >= 0:
        clean = _forward(pr.model, pr.coords(), pr.truth)
    else:
        raise ValueError("with_covariance takes built-in model problems")
    y = clean + np.linalg.cholesky(C) @ rng.normal(size=pr.m)
    return dataclasses.replace(pr, y=np.asarray(y, dtype=pr.y.dtype), sigma=C)


def log_uniform_int(rng, lo: float, hi: float, size) -> np.ndarray:
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


def dexp_batch(nfits: int = 4096, seed: int = 0, m_lo: int = 200, m_hi: int = 200_000,
               dtype=np.float32) -> Batch:
    """Ragged batch of double-exponential fits (m log-uniform in [m_lo, m_hi])."""
    rng = np.random.default_rng(seed)
    ms = log_uniform_int(rng, m_lo, m_hi, nfits)
    offsets = np.zeros(nfits + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(ms)
    xs, ys, p0s, truths = [], [], [], []
    for k in range(nfits):
        pr = dexp(int(ms[k]), seed=int(rng.integers(1 << 62)), dtype=np.float64)
        xs.append(pr.x); ys.append(pr.y); p0s.append(pr.p0); truths.append(pr.truth)
    lb = np.tile(np.array([-np.inf, 0.0, -np.inf, 0.0, -np.inf]), (nfits, 1))
    ub = np.full((nfits, 5), np.inf)
    return Batch(MODEL_DEXP, np.concatenate(xs).astype(dtype), np.concatenate(ys).astype(dtype),
                 None, offsets, np.array(p0s), lb, ub, np.array(truths))


# ---------------------------------------------------------------- serving stream
SERVE_MIX = ((MODEL_GAUSS1D, 0.4), (MODEL_DEXP, 0.4), (MODEL_GAUSS2D, 0.2))


class ServeStream:
    """Request stream of the serving workload.

    Each request draws its model 40% gauss1d / 40% dexp / 20% gauss2d and its
    size m log-uniform in [m_lo, m_hi].  So that a stream of tens of thousands
    of requests costs seconds to draw, the observations come from a few
    pre-drawn datasets per model (`n_data` variants, each its own seed):
      * 1D models: the first m points of a dataset of m_hi points (the points
        are i.i.d., so any prefix is a valid draw of the same recipe);
      * gauss2d: a W x W pixel grid, W taken from a sqrt(2) ladder between
        sqrt(m_lo) and sqrt(m_hi), the rung nearest sqrt(m) in log scale
        (so 2D sizes are discrete, within a factor 2^(1/4) of the draw);
        widths sx, sy = W U(0.05, 0.15), centre uniform in the central half,
        A = 980, c = 20, theta = 0.4 (the 1024^2 recipe otherwise).
    Arrival times are drawn separately (`arrivals`).
    """

    def __init__(self, n_requests: int, seed: int = 0, m_lo: float = 1e3, m_hi: float = 4e6, n_data: int = 4,
                 dtype=np.float32):
        rng = np.random.default_rng(seed)
        ids = [mdl for mdl, _ in SERVE_MIX]
        self.models = rng.choice(ids, p=[w for _, w in SERVE_MIX], size=n_requests)
        self.m = log_uniform_int(rng, m_lo, m_hi, n_requests)
        self.variant = rng.integers(0, n_data, size=n_requests)
        self.m_hi = int(m_hi)
        self.data = {}
        for v in range(n_data):
            self.data[(MODEL_GAUSS1D, v)] = gauss1d(self.m_hi, seed=1000 + v, dtype=dtype)
            self.data[(MODEL_DEXP, v)] = dexp(self.m_hi, seed=2000 + v, dtype=dtype)
        w_lo, w_hi = math.sqrt(m_lo), math.sqrt(m_hi)
        k = int(math.floor(2.0 * math.log2(w_hi / w_lo) + 1e-9))
        self.ladder = sorted({int(round(w_lo * 2.0 ** (i / 2.0))) for i in range(k + 1)} | {int(math.floor(w_hi))})
        for v in range(n_data):
            for W in self.ladder:
                r2 = np.random.default_rng(3000 + 97 * v + W)
                truth = [980.0, W * r2.uniform(0.25, 0.75), W * r2.uniform(0.25, 0.75),
                         W * r2.uniform(0.05, 0.15), W * r2.uniform(0.05, 0.15), 0.4, 20.0]
                self.data[(MODEL_GAUSS2D, v, W)] = gauss2d_grid(W, seed=3000 + 97 * v + W, truth=truth, dtype=dtype)
        for k2 in range(n_requests):
            if self.models[k2] == MODEL_GAUSS2D:
                lw = 0.5 * math.log(float(self.m[k2]))
                W = min(self.ladder, key=lambda w: abs(math.log(w) - lw))
                self.m[k2] = W * W

    def __len__(self) -> int:
        return int(self.models.shape[0])

    def request(self, k: int) -> Problem:
        mdl, v, m = int(self.models[k]), int(self.variant[k]), int(self.m[k])
        if mdl == MODEL_GAUSS2D:
            return self.data[(mdl, v, int(round(math.sqrt(m))))]
        pr = self.data[(mdl, v)]
        return Problem(mdl, pr.x[:m], LAYOUT_VEC, None, pr.y[:m], None if pr.sigma is None else pr.sigma[:m],
                       pr.p0, pr.lb, pr.ub, pr.truth)

    @staticmethod
    def arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
        """Open-loop Poisson arrival times (s) at `rate` requests/s; rate=inf: all at t=0."""
        if not np.isfinite(rate):
            return np.zeros(n)
        rng = np.random.default_rng(seed)
        return np.cumsum(rng.exponential(1.0 / rate, size=n))
