"""Exact diagonal correction of K~ (an extension, not in the paper; test infrastructure).

Only tests/, the package smoke check and the benchmark's CPU-baseline leg use this
module; the CUDA path never imports it.

Why: the error of K~ (Theorem main) is largest where the kernel is least smooth.  For
the Matern family with small nu, phi has a cusp at r = 0 (nu = 1/2: phi(r) = exp(-r)),
the Fourier modes {-M..M}^d that fit on a grid leave out the slowly decaying tail of
its transform (the I_2 term in the proof of Lemma stage3warmup), and K~ falls short
of K most at x = y.  The extension adds the defect of the diagonal exactly:

    K~c = K~ + diag(K_ii - K~_ii),

    K_ii  = w_i^2 (4 pi sigma_i^2)^(-d/2)                     Eq. (nonstat2) at x = y, phi(0) = 1
    K~_ii = sum_{k,l} w_k(x_i) w_l(x_i) S_kl,
    S_kl  = sum_{n in {-M..M}^d} A_kl[n]                     Eq. (Ktilde) at x = y: every
                                                             phase exp(2 pi i n dw (x - y)) is 1

with w_k(x) the Chebyshev weights of Eq. (Wk) and A[n] the tensor of Remark
rem:step3 (no NUFFT deconvolution: this is K~ itself).  K~c is symmetric, and where the
defect is non-negative (the usual case: truncating a positive spectrum lowers K~_ii)
K~c - K~ is positive semi-definite.  The off-diagonal entries are unchanged.
"""
from __future__ import annotations

import numpy as np

from . import chebyshev, ktilde


def s_matrix(p: ktilde.Params):
    """S = sum over the Fourier grid of A[n], shape (C, C)."""
    A = ktilde.a_tensor(p)
    return A.reshape(A.shape[0], A.shape[1], -1).sum(axis=2)


def ktilde_diag(w, sigma, p: ktilde.Params):
    """K~_ii for the points with fields (w, sigma)."""
    _, _, _, nd = p.tables()
    W = chebyshev.w_k(w, sigma, nd, p.d)
    return np.einsum("ik,kl,il->i", W, s_matrix(p), W)


def k_diag(w, sigma, d: int):
    """K_ii = w_i^2 (4 pi sigma_i^2)^(-d/2)."""
    w = np.asarray(w, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    return w ** 2 * (4.0 * np.pi * sigma ** 2) ** (-d / 2.0)


def defect(w, sigma, p: ktilde.Params):
    """K_ii - K~_ii."""
    return k_diag(w, sigma, p.d) - ktilde_diag(w, sigma, p)


def matvec(X, w, sigma, alpha, p: ktilde.Params):
    """K~c alpha = K~ alpha + (K_ii - K~_ii) alpha_i (K~ alpha by the exact NUDFTs)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    dv = defect(w, sigma, p)
    out = ktilde.matvec(X, w, sigma, alpha, p)
    return out + (dv[:, None] * alpha if alpha.ndim == 2 else dv * alpha)
