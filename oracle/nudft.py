"""Non-uniform discrete Fourier transforms, by direct summation (test infrastructure).

App. D (rescaled by the grid spacing dw):
  type 1:  f[n]   = sum_j c_j exp(-2 pi i (n dw) . x_j),   n in {-M..M}^d
  type 2:  g_j    = sum_n f[n] exp(+2 pi i (n dw) . x_j)
The two are formal adjoints of each other.

The d-dimensional exponential is the product of one factor per coordinate, so
the sums are written with einsum over per-coordinate factor matrices
E_a[j, n_a] = exp(-2 pi i n_a dw x_{j,a}); einsum evaluates exactly the sum of the
definition.
"""
from __future__ import annotations

import string

import numpy as np


def _factors(X, M: int, dw: float, sign: float):
    X = np.asarray(X, dtype=np.float64)
    n = np.arange(-M, M + 1, dtype=np.float64)
    return [np.exp(sign * 2j * np.pi * dw * X[:, a, None] * n[None, :]) for a in range(X.shape[1])]


def type1(X, c, M: int, dw: float):
    """c: (N,) or (K, N) strengths -> f: (K, 2M+1, ..., 2M+1) (d axes)."""
    c = np.atleast_2d(np.asarray(c))
    d = X.shape[1]
    E = _factors(X, M, dw, -1.0)
    ax = string.ascii_lowercase[:d]
    spec = "kz," + ",".join("z" + a for a in ax) + "->k" + ax
    return np.einsum(spec, c, *E, optimize=True)


def type2(X, f, M: int, dw: float):
    """f: (K, 2M+1, ..., 2M+1) -> g: (K, N)."""
    d = X.shape[1]
    E = _factors(X, M, dw, +1.0)
    ax = string.ascii_lowercase[:d]
    spec = "k" + ax + "," + ",".join("z" + a for a in ax) + "->kz"
    return np.einsum(spec, f, *E, optimize=True)
