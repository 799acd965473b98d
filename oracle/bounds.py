"""Error quantities of Sec. 5, evaluated directly (test infrastructure).

Definition epcheb / Lemma interp: for all x,
    |exp(-x^2/(2 s^2)) - sum_k P_k(s) exp(-x^2/(2 s_k^2))| <= 2 (kappa-1) ((kappa-1)/(kappa+1))^Ns.
(The lemma's sum is printed from k = 1; the nodes of Eq. (chebscheme) run from
k = 0, which is the reading used here.)

Definition eptrap: e^(-alpha t_max) + e^(nu t_min) + e^(-(1-delta) pi^2 / dt).
"""
from __future__ import annotations

import numpy as np

from . import chebyshev


def eps_cheb(n_sigma: int, kappa: float) -> float:
    return 2.0 * (kappa - 1.0) * ((kappa - 1.0) / (kappa + 1.0)) ** n_sigma


def interp_error(sigma_min: float, sigma_max: float, n_sigma: int, n_x: int = 400, n_s: int = 400) -> float:
    """sup over x and s of the Gaussian-in-width interpolation error (Lemma interp)."""
    nd = chebyshev.nodes(sigma_min, sigma_max, n_sigma)
    s = np.linspace(sigma_min, sigma_max, n_s)
    x = np.linspace(0.0, 6.0 * sigma_max, n_x)
    P = chebyshev.lagrange(s, nd)                          # (ns, K)
    exact = np.exp(-(x[None, :] ** 2) / (2.0 * s[:, None] ** 2))
    approx = P @ np.exp(-(x[None, :] ** 2) / (2.0 * nd[:, None] ** 2))
    return float(np.max(np.abs(exact - approx)))


def eps_trap(nu: float, alpha: float, delta: float, t_min: float, t_max: float, n_t: int) -> float:
    dt = (t_max - t_min) / n_t
    return float(np.exp(-alpha * t_max) + np.exp(nu * t_min) + np.exp(-(1.0 - delta) * np.pi ** 2 / dt))

