"""Exact near-field correction of K~ (an extension, not in the paper; test infrastructure).

Only tests/ use this module; the CUDA path never imports it.

Why: for small nu the Matern kernel has a cusp at r = 0 (nu = 1/2: phi(r) = exp(-r)), and
the Fourier modes {-M..M}^d that fit on a grid leave out the slowly decaying tail of its
transform, so K~ (Eq. Ktilde) falls short of K (Eq. nonstat2) over a neighbourhood of
the diagonal, not on it alone.  The extension adds the defect exactly for every pair of
distinct points closer than a radius r_c:

    K~nf = K~ + sum_{i != j, |x_i - x_j| < r_c} (K_ij - K~_ij) e_i e_j^T,

which with the diagonal correction of diagcorr.py (i = j) gives K itself within r_c.

K~_ij for one pair, from Eq. (Ktilde) with the Fourier multiplier of Lemma stage3warmup:
Pi F B_j* maps the point x to the grid vector Z_j(x)[n] = sum_k w_k(x) G^_{k,j}[n]
exp(2 pi i n dw . x), G^_{k,j}[n] = prod_a e_kj(n_a) with
    e_kj(m) = sqrt(2 pi) sigma_k chi_j exp(-2 pi^2 sigma_k^2 chi_j^2 dw^2 m^2),
so K~(x, y) = sum_j v~_j sum_{k,l} w_k(x) w_l(y) sum_n G^_kj[n] G^_lj[n] cos(2 pi n dw . (x - y)).
The grid is a product of symmetric ranges and the summand even in each n_a, so the
sum over n factors by dimension:

    K~(x, y) = sum_j v~_j sum_{k,l} w_k(x) w_l(y) prod_a t_klj(x_a - y_a),
    t_klj(rho) = sum_{|m| <= M} e_kj(m) e_lj(m) cos(2 pi m dw rho).
"""
from __future__ import annotations

import numpy as np

from . import chebyshev, diagcorr, kernel, ktilde


def t_factor(p: ktilde.Params, rho):
    """t_klj(rho) for all (k, l, j): array (C, C, J) + rho.shape."""
    _, v, chi, nd = p.tables()
    rho = np.asarray(rho, dtype=np.float64)
    m = np.arange(-p.M, p.M + 1, dtype=np.float64)
    s = nd[:, None] * chi[None, :]                                         # (C, J)
    e = np.sqrt(2.0 * np.pi) * s[..., None] * np.exp(-2.0 * np.pi ** 2 * (s[..., None] * p.dw * m) ** 2)  # (C, J, m)
    ee = e[:, None, :, :] * e[None, :, :, :]                               # (C, C, J, m)
    ph = np.cos(2.0 * np.pi * p.dw * m[:, None] * rho.reshape(1, -1))       # (m, R)
    out = np.einsum("kljm,mr->kljr", ee, ph, optimize=True)
    return out.reshape(out.shape[:3] + rho.shape)


def ktilde_pairs(Xa, wa, sa, Xb, wb, sb, p: ktilde.Params):
    """K~(x_a[q], x_b[q]) for the pairs q (rows of Xa and Xb), by the separable form."""
    Xa = np.asarray(Xa, dtype=np.float64)
    Xb = np.asarray(Xb, dtype=np.float64)
    _, v, _, nd = p.tables()
    vt = (p.dw ** p.d) * v
    Wa = chebyshev.w_k(wa, sa, nd, p.d)                                    # (Q, C)
    Wb = chebyshev.w_k(wb, sb, nd, p.d)
    prod = np.ones((nd.size, nd.size, v.size, Xa.shape[0]))
    for a in range(p.d):
        prod = prod * t_factor(p, Xa[:, a] - Xb[:, a])
    return np.einsum("j,qk,ql,kljq->q", vt, Wa, Wb, prod, optimize=True)


def pairs_within(X, r_c: float):
    """All (i, j), i != j, with |x_i - x_j| < r_c (brute force; small N only)."""
    X = np.asarray(X, dtype=np.float64)
    r = np.sqrt(np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=2))
    i, j = np.nonzero((r < r_c) & ~np.eye(X.shape[0], dtype=bool))
    return i, j


def correction(X, w, sigma, nu, p: ktilde.Params, r_c: float):
    """(i, j, K_ij - K~_ij) over the pairs closer than r_c."""
    X = np.asarray(X, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    i, j = pairs_within(X, r_c)
    if i.size == 0:
        return i, j, np.zeros(0)
    kij = np.array([kernel.kernel_cross(X[a:a + 1], w[a:a + 1], sigma[a:a + 1], X[b:b + 1], w[b:b + 1],
                                        sigma[b:b + 1], nu)[0, 0] for a, b in zip(i, j)])
    ktij = ktilde_pairs(X[i], w[i], sigma[i], X[j], w[j], sigma[j], p)
    return i, j, kij - ktij


def dense(X, w, sigma, nu, p: ktilde.Params, r_c: float, diag: bool = False):
    """K~nf densely (and with diag=True also the diagonal defect of diagcorr.py)."""
    Kt = ktilde.dense(X, w, sigma, p)
    i, j, dv = correction(X, w, sigma, nu, p, r_c)
    Kt[i, j] += dv
    if diag:
        Kt[np.diag_indices_from(Kt)] += diagcorr.defect(w, sigma, p)
    return Kt


def matvec(X, w, sigma, nu, alpha, p: ktilde.Params, r_c: float, diag: bool = False):
    """K~nf alpha: K~ alpha by the exact NUDFTs plus the sparse near-field defect."""
    alpha = np.asarray(alpha, dtype=np.float64)
    out = ktilde.matvec(X, w, sigma, alpha, p) if not diag else diagcorr.matvec(X, w, sigma, alpha, p)
    i, j, dv = correction(X, w, sigma, nu, p, r_c)
    if alpha.ndim == 1:
        np.add.at(out, i, dv * alpha[j])
    else:
        np.add.at(out, i, dv[:, None] * alpha[j])
    return out
