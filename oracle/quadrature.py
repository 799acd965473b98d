"""Schoenberg representation and its trapezoid discretisation (test infrastructure).

Sec. 3.1, Eq. (schoenberg2): phi(r) = int exp(-r^2 / (2 chi(t)^2)) u(t) dt.
Matern choice, Eq. (maternpres) (derived in App. C):
    u(t)   = exp(nu t - e^t) / Gamma(nu),
    chi(t) = exp(t/2) / sqrt(nu).
Operator weight, Eq. (v): v(t) = chi(t)^(-d) u(t).

Sec. 3.2, Eq. (trapsum) and Eq. (dtscheme): t_j = t_min + j (t_max - t_min)/N_t,
j = 0..N_t, with weights v_j = v(t_j) dt, halved at j = 0 and j = N_t.

Squared exponential (end of Sec. 3.1 and Sec. 3.2): N_t = 0, t_0 = 0, v_0 = 1,
chi_0 = 1.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def u_matern(t, nu: float):
    t = np.asarray(t, dtype=np.float64)
    return np.exp(nu * t - np.exp(t) - special.gammaln(nu))


def chi_matern(t, nu: float):
    t = np.asarray(t, dtype=np.float64)
    return np.exp(0.5 * t) / np.sqrt(nu)


def trapezoid_table(nu, d: int, t_min: float, t_max: float, n_t: int):
    """(t_j, v_j, chi_j, tau_j) for j = 0..N_t.

    tau_j are the bare trapezoid weights (dt, halved at the ends), so that
    v_j = tau_j chi_j^(-d) u(t_j).  nu = inf gives the squared-exponential table.
    """
    if nu is None or np.isinf(nu):
        one = np.ones(1)
        return np.zeros(1), one.copy(), one.copy(), one.copy()
    if n_t < 1:
        raise ValueError("N_t >= 1 for the Matern family")
    t = t_min + (t_max - t_min) * np.arange(n_t + 1) / n_t
    dt = (t_max - t_min) / n_t
    tau = np.full(n_t + 1, dt)
    tau[0] *= 0.5
    tau[-1] *= 0.5
    chi = chi_matern(t, nu)
    v = tau * chi ** (-d) * u_matern(t, nu)
    return t, v, chi, tau


def phi_from_quadrature(r, nu, t_min, t_max, n_t):
    """sum_j tau_j u(t_j) exp(-r^2/(2 chi_j^2)): the discretised Eq. (schoenberg2)."""
    t, _, chi, tau = trapezoid_table(nu, 1, t_min, t_max, n_t)
    r = np.asarray(r, dtype=np.float64)
    w = tau * u_matern(t, nu) if not (nu is None or np.isinf(nu)) else np.ones(1)
    return np.sum(w[None, :] * np.exp(-(r[:, None] ** 2) / (2.0 * chi[None, :] ** 2)), axis=1)
