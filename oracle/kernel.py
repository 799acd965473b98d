"""The plain kernel matrix and the GP solve (test infrastructure; see the package header).

Kernel: Sec. 3, Eq. (nonstat2)
    K(x, y) = w(x) w(y) (2 pi [sigma^2(x) + sigma^2(y)])^(-d/2)
              phi(|x - y| / sqrt(sigma^2(x) + sigma^2(y))).

Scale mapping (a reading; the paper never writes it).  The paper's sigma(x) is a
horizontal scale and the vertical scale is absorbed into w(x) (Sec. 3, the
remark after Eq. (kappa)).  The usual non-stationary Matern of Paciorek with
vertical scale s(x) and isotropic length l(x),
    s(x) s(y) (l_x l_y)^(d/2) ((l_x^2 + l_y^2)/2)^(-d/2) phi(|x-y| / sqrt((l_x^2 + l_y^2)/2)),
equals Eq. (nonstat2) exactly when
    sigma(x) = l(x) / sqrt(2),   w(x) = s(x) (2 pi)^(d/4) l(x)^(d/2).

Solve: Sec. 1, Eq. (gprsolve): (K + eta^2 I) alpha = y, by Cholesky (the
definition of the solution) and by plain conjugate gradients (x0 = 0, stop on
the relative recurrence residual), the iteration the paper wraps around its
matvec (Sec. 6.2).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .matern import phi


def paper_fields(s, l, d: int):
    """(w, sigma) of Eq. (nonstat2) from vertical scale s and length l (reading above)."""
    s = np.asarray(s, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    sigma = l / np.sqrt(2.0)
    w = s * (2.0 * np.pi) ** (d / 4.0) * l ** (d / 2.0)
    return w, sigma


def paciorek_dense(X, s, l, nu):
    """The Paciorek form written directly in (s, l); used to pin the mapping."""
    X = np.asarray(X, dtype=np.float64)
    d = X.shape[1]
    r = np.sqrt(np.maximum(np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=2), 0.0))
    q = 0.5 * (l[:, None] ** 2 + l[None, :] ** 2)
    pref = s[:, None] * s[None, :] * (l[:, None] * l[None, :]) ** (d / 2.0) * q ** (-d / 2.0)
    return pref * phi(r / np.sqrt(q), nu)


def kernel_cross(X, wX, sX, Y, wY, sY, nu):
    """Matrix (K(x_i, y_j)) of Eq. (nonstat2) for two point sets."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    d = X.shape[1]
    diff = X[:, None, :] - Y[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    ss = sX[:, None] ** 2 + sY[None, :] ** 2
    return (wX[:, None] * wY[None, :]) * (2.0 * np.pi * ss) ** (-d / 2.0) * phi(r / np.sqrt(ss), nu)


def kernel_dense(X, w, sigma, nu):
    """K of Eq. (boldK) with entries Eq. (nonstat2)."""
    return kernel_cross(X, w, sigma, X, w, sigma, nu)


def solve_cholesky(K, eta2: float, y):
    """alpha = (K + eta^2 I)^(-1) y, Eq. (gprsolve), by LAPACK Cholesky."""
    A = K + eta2 * np.eye(K.shape[0])
    c = scipy.linalg.cho_factor(A, lower=True)
    return scipy.linalg.cho_solve(c, y)


def cg(apply_A, y, rtol: float, maxit: int):
    """Plain conjugate gradients for a symmetric positive definite operator.

    x0 = 0; stops when ||r_k|| / ||y|| <= rtol with r_k the recurrence residual.
    Returns (x, iterations, final recurrence relative residual).
    """
    y = np.asarray(y, dtype=np.float64)
    x = np.zeros_like(y)
    r = y.copy()
    p = r.copy()
    rr = float(r @ r)
    ny = np.sqrt(float(y @ y))
    if ny == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxit and np.sqrt(rr) / ny > rtol:
        Ap = apply_A(p)
        a = rr / float(p @ Ap)
        x += a * p
        r -= a * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) / ny
