"""Per-evaluation quantities of the least-squares problem (oracle, FP64).

Test infrastructure: see the package docstring.

Written from the definitions, with no blocking or reordering:
  r_i = w_i (h(x_i; p) - y_i)            Eq. residual, weighted per Eq. easy_res
  J   = diag(w) dh/dp                     Eq. jacobian, weighted per Eq. easy_jac
  f   = 1/2 r^T r                         Eq. msqe (Eq. explicit when weighted)
  g   = J^T r                             Eq. gradient
  B   = J^T J                             Eq. hessian, Gauss-Newton term
with w_i = 1 / sigma_i (Eq. easesig; w = 1 when no sigma is given).
"""
from __future__ import annotations

import numpy as np

from . import models


def weights(sigma, m):
    """w = 1/sigma (Appendix C, diagonal L^-1); ones when sigma is None."""
    if sigma is None:
        return np.ones(m)
    return 1.0 / np.asarray(sigma, dtype=np.float64)


def residual_and_jac(model, X, y, w, p):
    """Weighted residual vector r [m] and Jacobian J [m, n] at p."""
    h, dh = models.value_and_jac(model, X, p)
    r = w * (h - np.asarray(y, dtype=np.float64))
    J = w[:, None] * dh
    return r, J


def evaluate(model, X, y, w, p):
    """(f, g, B, r, J) at p: cost, gradient J^T r, Gram J^T J."""
    r, J = residual_and_jac(model, X, y, w, p)
    f = 0.5 * float(r @ r)
    g = J.T @ r
    B = J.T @ J
    return f, g, B, r, J


def packed_upper(B):
    """Upper triangle of symmetric B, row-major (B00 B01 .. B0n-1 B11 ..)."""
    n = B.shape[0]
    return np.concatenate([B[i, i:] for i in range(n)])
