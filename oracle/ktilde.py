"""The approximate kernel K~ and its matvec, written from the paper (test infrastructure).

Sec. 3.5, Eq. (Ktilde):
    K~ = sum_j v~_j B_{t_j}^(Ns) F* Pi* Pi F B_{t_j}^(Ns)*,   v~_j = (dw)^d v_j,
with B_t^(Ns) = sum_k W_k G_{k,t} (Eq. BWG), Pi the restriction to the Fourier
grid n dw, n in {-M..M}^d (Sec. 3.4), F the unitary Fourier transform with
kernel exp(-2 pi i omega . x) (App. D).

Fourier multiplier of G_{k,t} (the Gaussian transform in the proof of Lemma
stage3warmup, Eq. (fhat)):
    G^_{k,j}[n] = (2 pi sigma_k^2 chi_j^2)^(d/2) exp(-2 pi^2 sigma_k^2 chi_j^2 dw^2 |n|^2).
Remark rem:step3: A_{k',k}[n] = sum_j v~_j G^_{k',j}[n] G^_{k,j}[n].

Matvec, Sec. 4.2 steps (1)-(5):
  (1) c_{k,i} = w_k(x_i) alpha_i                           (Eq. c)
  (2) b_k = type-1 NUDFT of c_k on the grid               (App. D)
  (3) a_{k'}[n] = sum_j v~_j G^_{k',j}[n] sum_k G^_{k,j}[n] b_k[n]
  (4) beta_k = type-2 NUDFT of a_k at the points
  (5) (K~ alpha)_i = sum_k w_k(x_i) beta_{k,i}   (real by Hermitian symmetry)

Closed form on an infinite grid (M -> infinity), from Poisson summation Eq. (PSF)
with the inverse transform Eq. (fanalytic), P = 1/dw:
    K~_inf(x, y) = sum_j v_j sum_{k,l} w_k(x) w_l(y)
                   (2 pi sigma_k^2 sigma_l^2 chi_j^2 / (sigma_k^2 + sigma_l^2))^(d/2)
                   sum_{m in Z^d} exp(-|x - y + m P|^2 / (2 (sigma_k^2 + sigma_l^2) chi_j^2)).
The finite grid differs from it by the tail I_2 of the same proof
(``grid_tail_bound``).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

from . import chebyshev, nudft, quadrature


@dataclass(frozen=True)
class Params:
    """The hyperparameters of Sec. 3.5 plus the fixed problem data (d, nu)."""
    d: int
    nu: float               # inf for the squared exponential
    t_min: float
    t_max: float
    n_t: int
    sigma_min: float
    sigma_max: float
    n_sigma: int
    M: int
    dw: float

    def tables(self):
        t, v, chi, _ = quadrature.trapezoid_table(self.nu, self.d, self.t_min, self.t_max, self.n_t)
        nd = chebyshev.nodes(self.sigma_min, self.sigma_max, self.n_sigma)
        return t, v, chi, nd


def mode_grid(M: int, d: int):
    """|n|^2 on {-M..M}^d as an array of shape (2M+1,)*d."""
    n = np.arange(-M, M + 1, dtype=np.float64)
    sq = np.zeros((2 * M + 1,) * d)
    for a in range(d):
        shape = [1] * d
        shape[a] = 2 * M + 1
        sq = sq + (n ** 2).reshape(shape)
    return sq


def ghat(p: Params):
    """G^[k, j, n...] on the grid, shape (Ns+1, Nt+1, (2M+1)^d axes)."""
    _, _, chi, nd = p.tables()
    s2 = (nd[:, None] ** 2) * (chi[None, :] ** 2)             # (K, J)
    n2 = mode_grid(p.M, p.d)
    pref = (2.0 * np.pi * s2) ** (p.d / 2.0)
    expo = -2.0 * np.pi ** 2 * (p.dw ** 2) * s2[(...,) + (None,) * p.d] * n2[None, None]
    return pref[(...,) + (None,) * p.d] * np.exp(expo)


def a_tensor(p: Params):
    """A[k', k, n...] of Remark rem:step3."""
    _, v, _, _ = p.tables()
    vt = (p.dw ** p.d) * v
    G = ghat(p)
    return np.einsum("j,aj...,bj...->ab...", vt, G, G, optimize=True)


def matvec(X, w, sigma, alpha, p: Params):
    """K~ alpha by steps (1)-(5) of Sec. 4.2 with exact NUDFT sums.

    alpha: (N,) or (N, R).  Returns the same shape, float64.
    """
    X = np.asarray(X, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    one = alpha.ndim == 1
    al = alpha[:, None] if one else alpha
    _, _, _, nd = p.tables()
    W = chebyshev.w_k(w, sigma, nd, p.d)                       # (N, K)
    A = a_tensor(p)                                            # (K, K, grid)
    out = np.zeros_like(al)
    for r in range(al.shape[1]):
        c = (W * al[:, r:r + 1]).T                             # step (1): (K, N)
        b = nudft.type1(X, c, p.M, p.dw)                        # step (2): (K, grid)
        a = np.einsum("ab...,b...->a...", A, b, optimize=True)  # step (3)
        beta = nudft.type2(X, a, p.M, p.dw)                     # step (4): (K, N)
        out[:, r] = np.real(np.sum(W.T * beta, axis=0))         # step (5)
    return out[:, 0] if one else out


def apply_cross(Xq, wq, sigq, X, w, sigma, alpha, p: Params):
    """(K~ alpha) evaluated at other points x_q: Eq. (postmean) with K~ in place of K.

    Steps (1)-(3) use the training points; steps (4)-(5) use the query points and
    their own Chebyshev weights w_k(x_q).
    """
    X = np.asarray(X, dtype=np.float64)
    Xq = np.asarray(Xq, dtype=np.float64)
    _, _, _, nd = p.tables()
    W = chebyshev.w_k(w, sigma, nd, p.d)
    Wq = chebyshev.w_k(wq, sigq, nd, p.d)
    A = a_tensor(p)
    c = (W * np.asarray(alpha, dtype=np.float64)[:, None]).T
    a = np.einsum("ab...,b...->a...", A, nudft.type1(X, c, p.M, p.dw), optimize=True)
    return np.real(np.sum(Wq.T * nudft.type2(Xq, a, p.M, p.dw), axis=0))


def matvec_imag_part(X, w, sigma, alpha, p: Params):
    """max |Im| of step (5) before the real part is taken (Hermitian check)."""
    _, _, _, nd = p.tables()
    W = chebyshev.w_k(w, sigma, nd, p.d)
    A = a_tensor(p)
    c = (W * np.asarray(alpha)[:, None]).T
    a = np.einsum("ab...,b...->a...", A, nudft.type1(X, c, p.M, p.dw), optimize=True)
    return float(np.max(np.abs(np.imag(np.sum(W.T * nudft.type2(X, a, p.M, p.dw), axis=0)))))


def dense(X, w, sigma, p: Params):
    """K~ at the points, Eq. (Ktilde) literally: sum_j v~_j (Pi F B_j*)^* (Pi F B_j*).

    Z_j[x, n] = conj((Pi F B_j^(Ns)*)[n, x]) = sum_k w_k(x) G^_{k,j}[n] exp(+2 pi i n dw . x),
    and K~ = sum_j v~_j Re(Z_j Z_j^H).  For small N only.
    """
    X = np.asarray(X, dtype=np.float64)
    N, d = X.shape
    _, v, _, nd = p.tables()
    vt = (p.dw ** d) * v
    W = chebyshev.w_k(w, sigma, nd, d)                         # (N, K)
    G = ghat(p).reshape(nd.size, v.size, -1)                   # (K, J, nmodes)
    n1 = np.arange(-p.M, p.M + 1, dtype=np.float64)
    ph = np.ones((N, 1), dtype=np.complex128)
    for a in range(d):
        fa = np.exp(2j * np.pi * p.dw * X[:, a, None] * n1[None, :])   # (N, 2M+1)
        ph = (ph[:, :, None] * fa[:, None, :]).reshape(N, -1)
    Kt = np.zeros((N, N))
    for j in range(v.size):
        Z = ph * (W @ G[:, j, :])                              # (N, nmodes)
        Kt += vt[j] * (Z.real @ Z.real.T + Z.imag @ Z.imag.T)
    return Kt


def dense_poisson(X, w, sigma, p: Params, Y=None, wY=None, sigmaY=None, images: int = 2):
    """K~ on an infinite grid (closed form above), rows at X, columns at Y."""
    X = np.asarray(X, dtype=np.float64)
    if Y is None:
        Y, wY, sigmaY = X, w, sigma
    d = X.shape[1]
    _, v, chi, nd = p.tables()
    WX = chebyshev.w_k(w, sigma, nd, d)
    WY = chebyshev.w_k(wY, sigmaY, nd, d)
    P = 1.0 / p.dw
    diff = X[:, None, :] - Y[None, :, :]
    shifts = [np.array(m, dtype=np.float64) for m in itertools.product(range(-images, images + 1), repeat=d)]
    r2 = [np.sum((diff + P * m) ** 2, axis=2) for m in shifts]
    out = np.zeros((X.shape[0], Y.shape[0]))
    for j in range(v.size):
        for k in range(nd.size):
            for l in range(nd.size):
                ss = (nd[k] ** 2 + nd[l] ** 2) * chi[j] ** 2
                pref = v[j] * (2.0 * np.pi * nd[k] ** 2 * nd[l] ** 2 * chi[j] ** 2
                               / (nd[k] ** 2 + nd[l] ** 2)) ** (d / 2.0)
                img = sum(np.exp(-q / (2.0 * ss)) for q in r2)
                out += pref * np.outer(WX[:, k], WY[:, l]) * img
    return out


def grid_tail_bound(w, sigma, p: Params):
    """Upper bound on max |K~ - K~_inf| from the modes outside {-M..M}^d.

    The dropped part of each (j, k, l) term is v~_j w_k(x) w_l(y) times the sum of
    |G^_k G^_l| over n outside the grid (the I_2 term of the proof of Lemma
    stage3warmup), summed here numerically with the exact Gaussian.
    """
    _, v, chi, nd = p.tables()
    d = p.d
    W = chebyshev.w_k(w, sigma, nd, d)
    wmax = np.max(np.abs(W), axis=0)
    tot = 0.0
    n = np.arange(0, 40 * p.M + 200, dtype=np.float64)
    for j in range(v.size):
        for k in range(nd.size):
            for l in range(nd.size):
                c = 2.0 * np.pi ** 2 * (nd[k] ** 2 + nd[l] ** 2) * chi[j] ** 2 * p.dw ** 2
                g1 = np.exp(-c * n ** 2)
                full = g1[0] + 2.0 * np.sum(g1[1:])
                inside = g1[0] + 2.0 * np.sum(g1[1:p.M + 1])
                tail = full ** d - inside ** d
                pref = (p.dw ** d) * v[j] * (2.0 * np.pi * nd[k] * nd[l] * chi[j] ** 2) ** d
                tot += abs(pref * tail) * wmax[k] * wmax[l]
    return tot
