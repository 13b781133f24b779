"""Per-evaluation quantities of the least-squares problem (oracle, FP64).

Test infrastructure: see the package docstring.

Written from the definitions, with no blocking or reordering:
  r_i = w_i (h(x_i; p) - y_i)            Eq. residual, weighted per Eq. easy_res
  J   = diag(w) dh/dp                     Eq. jacobian, weighted per Eq. easy_jac
  f   = 1/2 r^T r                         Eq. msqe (Eq. explicit when weighted)
  g   = J^T r                             Eq. gradient
  B   = J^T J                             Eq. hessian, Gauss-Newton term
with w_i = 1 / sigma_i (Eq. easesig; w = 1 when no sigma is given).

Full covariance (Appendix C, Eq. covariance): a 2D sigma is the covariance
matrix C = L L^T (Cholesky); the weighted residual and Jacobian are the
solutions of L r~ = r and L J~ = J (Eqs. slsq1, slsq2), by forward
substitution (a library triangular solve).

Robust losses (Section 5 names "various loss functions" without stating
them; reading R14): the cost becomes f = 1/2 C^2 sum rho(z_i), z_i = (r_i/C)^2,
with f_scale C and one of the standard losses below.  Its gradient is
sum rho'(z_i) r_i J_i and its Gauss-Newton Hessian sum s_i J_i^T J_i with
s_i = rho'(z_i) + 2 z_i rho''(z_i); both are those of an ordinary least-squares
problem in the rescaled rows
  J~_i = sqrt(s_i) J_i,   r~_i = rho'(z_i) r_i / sqrt(s_i)
(s_i clipped below at eps64), which the trust-region method then uses as its
Jacobian and residual; the ratio's actual reduction uses the robust cost.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import models


class CovFactor:
    """Cholesky factor L of a covariance matrix C = L L^T (lower triangular)."""

    def __init__(self, C):
        C = np.asarray(C, dtype=np.float64)
        if C.ndim != 2 or C.shape[0] != C.shape[1]:
            raise ValueError("a covariance matrix must be square")
        self.L = np.linalg.cholesky(C)

    def solve(self, b):
        """L^-1 b (Eqs. slsq1, slsq2) for a vector or a matrix of columns."""
        return solve_triangular(self.L, b, lower=True)


def weights(sigma, m):
    """w = 1/sigma (Appendix C, diagonal L^-1); ones when sigma is None; a
    CovFactor when sigma is an [m, m] covariance matrix (Eq. covariance)."""
    if sigma is None:
        return np.ones(m)
    s = np.asarray(sigma, dtype=np.float64)
    if s.ndim == 2:
        if s.shape != (m, m):
            raise ValueError("covariance matrix must be [m, m]")
        return CovFactor(s)
    return 1.0 / s


def residual_and_jac(model, X, y, w, p):
    """Weighted residual vector r [m] and Jacobian J [m, n] at p."""
    h, dh = models.value_and_jac(model, X, p)
    r0 = h - np.asarray(y, dtype=np.float64)
    if isinstance(w, CovFactor):
        return w.solve(r0), w.solve(dh)
    r = w * r0
    J = w[:, None] * dh
    return r, J


LOSSES = ("linear", "soft_l1", "huber", "cauchy", "arctan")
EPS = float(np.finfo(np.float64).eps)


def loss_rho(loss, z):
    """rho(z), rho'(z), rho''(z) of a robust loss, elementwise (R14):
      linear   z
      soft_l1  2 (sqrt(1 + z) - 1)
      huber    z for z <= 1, 2 sqrt(z) - 1 beyond
      cauchy   ln(1 + z)
      arctan   arctan(z)"""
    z = np.asarray(z, dtype=np.float64)
    if loss == "linear":
        return z.copy(), np.ones_like(z), np.zeros_like(z)
    if loss == "soft_l1":
        t = 1.0 + z
        return 2.0 * z / (np.sqrt(t) + 1.0), t ** -0.5, -0.5 * t ** -1.5      # = 2 (sqrt(t) - 1)
    if loss == "huber":
        inner = z <= 1.0
        zs = np.where(inner, 1.0, z)
        return (np.where(inner, z, 2.0 * np.sqrt(zs) - 1.0), np.where(inner, 1.0, zs ** -0.5),
                np.where(inner, 0.0, -0.5 * zs ** -1.5))
    if loss == "cauchy":
        return np.log1p(z), 1.0 / (1.0 + z), -1.0 / (1.0 + z) ** 2
    if loss == "arctan":
        return np.arctan(z), 1.0 / (1.0 + z * z), -2.0 * z / (1.0 + z * z) ** 2
    raise ValueError(f"unknown loss {loss!r}")


def robust_rows(r, J, loss, f_scale):
    """(f, r~, J~) of R14 from the weighted residual r and Jacobian J."""
    if loss == "linear":
        return 0.5 * float(r @ r), r, J
    C = float(f_scale)
    z = (r / C) ** 2
    rho, rho1, rho2 = loss_rho(loss, z)
    s = np.maximum(rho1 + 2.0 * z * rho2, EPS)
    rs = np.sqrt(s)
    return 0.5 * C * C * float(np.sum(rho)), rho1 * r / rs, rs[:, None] * J


def evaluate(model, X, y, w, p, loss="linear", f_scale=1.0):
    """(f, g, B, r, J) at p: cost, gradient J^T r, Gram J^T J (with a robust
    loss: the robust cost and the rescaled r~, J~ of R14)."""
    r, J = residual_and_jac(model, X, y, w, p)
    f, r, J = robust_rows(r, J, loss, f_scale)
    g = J.T @ r
    B = J.T @ J
    return f, g, B, r, J


def packed_upper(B):
    """Upper triangle of symmetric B, row-major (B00 B01 .. B0n-1 B11 ..)."""
    n = B.shape[0]
    return np.concatenate([B[i, i:] for i in range(n)])
