"""Chebyshev interpolation in the value of sigma (test infrastructure).

Sec. 3.3, Eq. (chebscheme): Chebyshev-Lobatto nodes on [sigma_min, sigma_max]
    sigma_k = (cos(pi k / N_sigma) + 1)/2 (sigma_max - sigma_min) + sigma_min,  k = 0..N_sigma,
and P_k the Lagrange polynomials of degree N_sigma with P_k(sigma_j) = delta_jk.

Eq. (Wk): w_k(x) = w(x) [2 pi sigma(x)^2]^(-d/2) P_k(sigma(x)).

The Lagrange basis is evaluated by the plain product formula
    P_k(s) = prod_{j != k} (s - sigma_j) / (sigma_k - sigma_j),
which is slow but obviously the definition.

Degenerate interval (sigma_min == sigma_max, i.e. kappa = 1): a reading -- one
node sigma_0 and P_0 == 1 (the stationary case, N_sigma = 0).
"""
from __future__ import annotations

import numpy as np


def nodes(sigma_min: float, sigma_max: float, n_sigma: int):
    if n_sigma == 0:
        return np.array([sigma_max], dtype=np.float64)
    k = np.arange(n_sigma + 1)
    return (np.cos(np.pi * k / n_sigma) + 1.0) / 2.0 * (sigma_max - sigma_min) + sigma_min


def lagrange(s, nd):
    """Matrix P[i, k] = P_k(s_i) by the product formula."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    n = nd.size
    P = np.ones((s.size, n))
    for k in range(n):
        for j in range(n):
            if j != k:
                P[:, k] *= (s - nd[j]) / (nd[k] - nd[j])
    return P


def w_k(w, sigma, nd, d: int):
    """Matrix W[i, k] = w_k(x_i) of Eq. (Wk)."""
    w = np.asarray(w, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    return (w * (2.0 * np.pi * sigma ** 2) ** (-d / 2.0))[:, None] * lagrange(sigma, nd)


def lebesgue_constant(nd, n_eval: int = 4001):
    """Definition lebesgue: sup over [sigma_min, sigma_max] of sum_k |P_k|."""
    s = np.linspace(nd.min(), nd.max(), n_eval)
    return float(np.max(np.sum(np.abs(lagrange(s, nd)), axis=1)))
