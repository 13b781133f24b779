"""User-defined test models, each written twice: as the CUDA source a user
hands to the library (compiled at run time, differentiated by dual numbers)
and as NumPy for the oracle (partials written out, or by complex step).

The two texts share nothing but the formula; the oracle side is pinned on
the CPU (tests/test_oracle_user_models.py) before any GPU comparison.
"""
import numpy as np

# ---- Lorentzian peak + offset, p = (A, x0, g, c)
LORENTZ_SRC = r"""
template <class T, class S>
__device__ T model(const T* p, S x, S x2) {
    T u = (x - p[1]) / p[2];
    return p[0] / (1.0 + square(u)) + p[3];
}
"""


def lorentz_np(X, p):
    A, x0, g, c = p
    u = (X[0] - x0) / g
    q = 1.0 / (1.0 + u * u)
    h = A * q + c
    J = np.empty((X.shape[1], 4))
    J[:, 0] = q
    J[:, 1] = A * q * q * 2.0 * u / g          # d/dx0 of A / (1 + u^2), du/dx0 = -1/g
    J[:, 2] = A * q * q * 2.0 * u * u / g      # du/dg = -u/g
    J[:, 3] = 1.0
    return h, J


# ---- axis-aligned 2D Gaussian + offset, p = (A, x0, y0, sx, sy, c)
GAUSS2D_AXIS_SRC = r"""
template <class T, class S>
__device__ T gauss_axis(const T* p, S x, S y) {
    T dx = x - p[1], dy = y - p[2];
    T q = square(dx) / (2.0 * square(p[3])) + square(dy) / (2.0 * square(p[4]));
    return p[0] * exp(-q) + p[5];
}
"""


def gauss2d_axis_np(X, p):
    A, x0, y0, sx, sy, c = p
    dx, dy = X[0] - x0, X[1] - y0
    E = np.exp(-dx * dx / (2 * sx * sx) - dy * dy / (2 * sy * sy))
    h = A * E + c
    J = np.empty((X.shape[1], 6))
    J[:, 0] = E
    J[:, 1] = A * E * dx / (sx * sx)
    J[:, 2] = A * E * dy / (sy * sy)
    J[:, 3] = A * E * dx * dx / (sx ** 3)
    J[:, 4] = A * E * dy * dy / (sy ** 3)
    J[:, 5] = 1.0
    return h, J


# ---- the built-in 1D Gaussian written as a user model, p = (A, mu, s, c)
GAUSS1D_SRC = r"""
template <class T, class S>
__device__ T model(const T* p, S x, S x2) {
    T d = x - p[1];
    return p[0] * exp(-square(d) / (2.0 * square(p[2]))) + p[3];
}
"""

# ---- every operation of the dual-number types in one function (n = 8),
# compared at fixed parameters only
ZOO_SRC = r"""
template <class T, class S>
__device__ T model(const T* p, S x, S x2) {
    T a = p[0] * exp(-(p[1] * x));
    T b = sqrt(p[2] * p[2] + x * x);
    T c = log(p[3] + x * x);
    T d = 0.1 * pow(p[4] + x * x, 1.5);
    T e = sin(p[5] * x) * cos(p[6] * x);
    T f = tanh(p[7] * x);
    T g = atan(p[1] * x) / (1.0 + square(p[0]));
    T k = p[2] / (p[3] + x) - 1.0 / (p[4] + x);
    return a + b + c + d + e + f + g + k - 3.0 * (x - p[0]);
}
"""


def zoo_value(X, p):
    """Value only, written for real or complex p (complex-step partials)."""
    x = X[0]
    a = p[0] * np.exp(-(p[1] * x))
    b = np.sqrt(p[2] * p[2] + x * x)
    c = np.log(p[3] + x * x)
    d = 0.1 * np.power(p[4] + x * x, 1.5)
    e = np.sin(p[5] * x) * np.cos(p[6] * x)
    f = np.tanh(p[7] * x)
    g = np.arctan(p[1] * x) / (1.0 + p[0] * p[0])
    k = p[2] / (p[3] + x) - 1.0 / (p[4] + x)
    return a + b + c + d + e + f + g + k - 3.0 * (x - p[0])


def complex_step_jac(value, X, p, h=1e-30):
    """dh/dp by the complex step: Im h(p + i h e_j) / h (no subtraction, exact to rounding)."""
    p = np.asarray(p, dtype=np.float64)
    J = np.empty((X.shape[1], p.size))
    for j in range(p.size):
        pc = p.astype(np.complex128)
        pc[j] += 1j * h
        J[:, j] = np.imag(value(X, pc)) / h
    return J


def zoo_np(X, p):
    return np.real(zoo_value(X, np.asarray(p, dtype=np.float64))), complex_step_jac(zoo_value, X, p)


ZOO_P = np.array([0.7, 0.9, 1.3, 2.0, 1.1, 1.7, 0.6, 0.8])
