"""Radial functions (test infrastructure; see the package header).

phi_nu  -- Matern function, Sec. 2, Eq. (matern):
    phi_nu(r) = 1/(2^(nu-1) Gamma(nu)) |sqrt(2 nu) r|^nu K_nu(sqrt(2 nu) r),  phi_nu(0) = 1.
phi_se  -- squared exponential, Sec. 2, Eq. (squaredexp): phi(r) = exp(-r^2/2).

The half-integer closed forms (nu = 1/2, 3/2, 5/2) follow from K_{n+1/2} being
elementary (Sec. 2 mentions that half-integer nu give closed forms); they are
written out here and the Bessel form is used for every other nu.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def phi_matern_bessel(r, nu: float):
    """Eq. (matern) evaluated with scipy's modified Bessel function K_nu."""
    r = np.asarray(r, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * np.abs(r)
    out = np.ones_like(z)
    pos = z > 0
    zp = z[pos]
    # same expression in log space: K_nu(z) = kve(nu, z) e^-z avoids overflow of Gamma(nu), z^nu
    logpre = (1.0 - nu) * np.log(2.0) - special.gammaln(nu) + nu * np.log(zp) - zp
    out[pos] = np.exp(logpre) * special.kve(nu, zp)
    return out


def phi_matern_closed(r, nu: float):
    """Closed forms of Eq. (matern) for nu in {1/2, 3/2, 5/2}."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    if nu == 0.5:
        return np.exp(-r)
    if nu == 1.5:
        a = np.sqrt(3.0) * r
        return (1.0 + a) * np.exp(-a)
    if nu == 2.5:
        a = np.sqrt(5.0) * r
        return (1.0 + a + a * a / 3.0) * np.exp(-a)
    raise ValueError("no closed form for nu=%r" % nu)


def phi_matern(r, nu: float):
    if nu in (0.5, 1.5, 2.5):
        return phi_matern_closed(r, nu)
    return phi_matern_bessel(r, nu)


def phi_se(r):
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-0.5 * r * r)


def phi(r, nu):
    """nu = inf selects the squared exponential (the nu -> infinity limit, Sec. 2)."""
    if nu is None or np.isinf(nu):
        return phi_se(r)
    return phi_matern(r, nu)
