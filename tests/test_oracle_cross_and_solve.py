"""Pins of the two oracle functions every posterior-mean and CG parity test rests on.

* ``ktilde.apply_cross``: K~ alpha evaluated at query points (Eq. postmean with the
  K~ of Eq. Ktilde).  Pinned against (a) the training-point matvec when the queries
  are the training points, (b) the literal cross block sum_j v~_j Re(Z_j(q) Z_j(x)^H)
  of Eq. (Ktilde), which never forms the tensor A nor runs a NUDFT, (c) the Poisson
  closed form on an infinite grid within the grid-tail bound, and (d) the plain
  kernel K(x_q, x_n) as the parameters refine (Theorem main).  Two planted mistakes
  (training weights in step (5), training points in the type-2 sum) must each be
  caught by these pins as they stand.
* ``kernel.solve_cholesky``: the solution of Eq. (gprsolve).  Pinned by its normwise
  backward error, by LAPACK's LU solve (a different factorisation), by a system
  built with a known solution, and by a planted mistake (eta^2 dropped).

No GPU.
"""
import numpy as np
import pytest
from scipy import special

import gpinputs
from oracle import chebyshev, kernel, ktilde


def _params(sig_all, d, nu=1.5, n_t=30, n_s=10, M=400, P=2.5, tail=1e-11):
    t_min = np.log(special.gammaincinv(nu, tail))
    t_max = np.log(special.gammainccinv(nu, tail))
    return ktilde.Params(d, nu, t_min, t_max, n_t, float(np.min(sig_all)), float(np.max(sig_all)), n_s, M, 1.0 / P)


def _queries_1d(n, seed):
    rng = np.random.default_rng(seed)
    xq = rng.random((n, 1))
    s, l = gpinputs.fields_1d(xq)
    return xq, s, l


def _literal_cross(Xq, wq, sq, X, w, s, p):
    """The (q, n) block of Eq. (Ktilde), written from its definition: with
    Z_j(x)[m] = sum_k w_k(x) G^_{k,j}[m] exp(+2 pi i m dw . x) over the grid m in
    {-M..M}^d, K~(x_q, x_n) = sum_j v~_j Re(Z_j(x_q) . conj(Z_j(x_n)))."""
    _, v, chi, nd = p.tables()
    d = X.shape[1]
    vt = (p.dw ** d) * v
    m1 = np.arange(-p.M, p.M + 1, dtype=np.float64)

    def Z(P_, w_, s_, j):
        Wk = chebyshev.w_k(w_, s_, nd, d)                                   # (n, K)
        out = np.zeros((P_.shape[0],) + (2 * p.M + 1,) * d, dtype=np.complex128)
        for k in range(nd.size):
            s2 = nd[k] ** 2 * chi[j] ** 2
            g = np.ones((P_.shape[0],) + (2 * p.M + 1,) * d, dtype=np.complex128)
            for a in range(d):
                shape = [P_.shape[0]] + [1] * d
                shape[1 + a] = 2 * p.M + 1
                fac = np.sqrt(2 * np.pi * s2) * np.exp(-2 * np.pi ** 2 * s2 * p.dw ** 2 * m1 ** 2) \
                    * np.exp(2j * np.pi * p.dw * P_[:, a, None] * m1[None, :])
                g = g * fac.reshape(shape)
            out += Wk[:, k].reshape((-1,) + (1,) * d) * g
        return out.reshape(P_.shape[0], -1)

    Kt = np.zeros((Xq.shape[0], X.shape[0]))
    for j in range(v.size):
        Kt += vt[j] * np.real(Z(Xq, wq, sq, j) @ np.conj(Z(X, w, s, j)).T)
    return Kt


# ------------------------------------------------------------ ktilde.apply_cross
def test_apply_cross_at_the_training_points_is_the_matvec():
    w = gpinputs.config_1d(60)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    p = _params(sig, 1)
    a = ktilde.apply_cross(w.points, wp, sig, w.points, wp, sig, w.alpha, p)
    b = ktilde.matvec(w.points, wp, sig, w.alpha, p)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


@pytest.mark.parametrize("d", [1, 2])
def test_apply_cross_equals_the_literal_cross_block(d):
    if d == 1:
        w = gpinputs.config_1d(50)
        xq, sq_s, lq = _queries_1d(23, seed=5)
        p_args = dict(M=300)
    else:
        w = gpinputs.config_2d(30, 1.5)
        rng = np.random.default_rng(6)
        xq = rng.random((17, 2))
        sq_s, lq = gpinputs.fields_2d(xq)
        p_args = dict(M=24, n_t=16, n_s=5, P=2.0)
    wp, sig = kernel.paper_fields(w.s, w.l, d)
    wq, sq = kernel.paper_fields(sq_s, lq, d)
    p = _params(np.r_[sig, sq], d, **p_args)
    got = ktilde.apply_cross(xq, wq, sq, w.points, wp, sig, w.alpha, p)
    Kt = _literal_cross(xq, wq, sq, w.points, wp, sig, p)
    ref = Kt @ w.alpha
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_literal_cross_block_with_itself_is_the_dense_ktilde():
    # the helper above, at x_q = x_n, is the literal dense form of the oracle (independent check
    # that the helper is the definition and not a retyping of apply_cross)
    w = gpinputs.config_1d(25)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    p = _params(sig, 1, M=200)
    assert np.max(np.abs(_literal_cross(w.points, wp, sig, w.points, wp, sig, p)
                         - ktilde.dense(w.points, wp, sig, p))) <= 1e-13 * np.max(np.abs(ktilde.dense(w.points, wp, sig, p)))


def test_apply_cross_within_the_grid_tail_of_the_poisson_form():
    w = gpinputs.config_1d(40)
    xq, sq_s, lq = _queries_1d(19, seed=7)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    wq, sq = kernel.paper_fields(sq_s, lq, 1)
    p = _params(np.r_[sig, sq], 1, M=300)
    got = ktilde.apply_cross(xq, wq, sq, w.points, wp, sig, w.alpha, p)
    Kp = ktilde.dense_poisson(xq, wq, sq, p, Y=w.points, wY=wp, sigmaY=sig)
    tail = ktilde.grid_tail_bound(np.r_[wp, wq], np.r_[sig, sq], p)
    assert np.max(np.abs(got - Kp @ w.alpha)) <= tail * np.sum(np.abs(w.alpha))
    # and the gap closes as the grid grows
    p2 = _params(np.r_[sig, sq], 1, M=2400)
    gap2 = np.max(np.abs(ktilde.apply_cross(xq, wq, sq, w.points, wp, sig, w.alpha, p2)
                         - ktilde.dense_poisson(xq, wq, sq, p2, Y=w.points, wY=wp, sigmaY=sig) @ w.alpha))
    assert gap2 < np.max(np.abs(got - Kp @ w.alpha)) / 20


def test_apply_cross_converges_to_the_kernel_at_the_queries():
    w = gpinputs.config_1d(40)
    xq, sq_s, lq = _queries_1d(21, seed=8)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    wq, sq = kernel.paper_fields(sq_s, lq, 1)
    ref = kernel.kernel_cross(xq, wq, sq, w.points, wp, sig, 1.5) @ w.alpha
    errs = []
    for (n_t, n_s, M) in [(20, 6, 300), (40, 10, 900), (80, 16, 2400)]:
        got = ktilde.apply_cross(xq, wq, sq, w.points, wp, sig, w.alpha,
                                 _params(np.r_[sig, sq], 1, n_t=n_t, n_s=n_s, M=M, P=3.0))
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-6


def _bad_apply_cross(which):
    """apply_cross with one planted mistake (a copy of the oracle's steps)."""
    from oracle import nudft

    def f(Xq, wq, sigq, X, w, sigma, alpha, p):
        X = np.asarray(X, dtype=np.float64)
        Xq = np.asarray(Xq, dtype=np.float64)
        _, _, _, nd = p.tables()
        W = chebyshev.w_k(w, sigma, nd, p.d)
        Wq = chebyshev.w_k(wq, sigq, nd, p.d)
        A = ktilde.a_tensor(p)
        c = (W * np.asarray(alpha, dtype=np.float64)[:, None]).T
        a = np.einsum("ab...,b...->a...", A, nudft.type1(X, c, p.M, p.dw), optimize=True)
        if which == "train_weights":
            # step (5) with the training points' w_k (same count of rows here)
            return np.real(np.sum(W[:Xq.shape[0]].T * nudft.type2(Xq, a, p.M, p.dw), axis=0))
        # the type-2 sum at the training points instead of the queries
        return np.real(np.sum(Wq.T * nudft.type2(X[:Xq.shape[0]], a, p.M, p.dw), axis=0))
    return f


@pytest.mark.parametrize("which", ["train_weights", "train_points"])
def test_planted_cross_mistakes_are_caught(monkeypatch, which):
    monkeypatch.setattr(ktilde, "apply_cross", _bad_apply_cross(which))
    with pytest.raises(AssertionError):
        test_apply_cross_equals_the_literal_cross_block(1)


# ------------------------------------------------------------ kernel.solve_cholesky
def test_solve_cholesky_backward_error_and_lu():
    w = gpinputs.config_1d(300)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    K = kernel.kernel_dense(w.points, wp, sig, 1.5)
    eta2 = 0.01
    A = K + eta2 * np.eye(300)
    for y in (w.y, np.c_[w.y, w.alpha]):
        x = kernel.solve_cholesky(K, eta2, y)
        r = A @ x - y
        # normwise backward error of a backward-stable factorisation
        be = np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(x) + np.linalg.norm(y))
        assert be <= 1e-14, be
        # LU (a different factorisation) agrees within the conditioning
        ref = np.linalg.solve(A, y)
        cond = np.linalg.cond(A)
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 50 * cond * np.finfo(float).eps


def test_solve_cholesky_recovers_a_known_solution():
    w = gpinputs.config_2d(200, 1.5)
    wp, sig = kernel.paper_fields(w.s, w.l, 2)
    K = kernel.kernel_dense(w.points, wp, sig, 2.5)
    eta2 = 0.05 ** 2
    x_true = np.random.default_rng(3).standard_normal(200)
    y = K @ x_true + eta2 * x_true
    x = kernel.solve_cholesky(K, eta2, y)
    cond = np.linalg.cond(K + eta2 * np.eye(200))
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) <= 50 * cond * np.finfo(float).eps


def test_planted_dropped_noise_term_is_caught(monkeypatch):
    import scipy.linalg
    monkeypatch.setattr(kernel, "solve_cholesky",
                        lambda K, eta2, y: scipy.linalg.cho_solve(scipy.linalg.cho_factor(K + 1e-9 * np.eye(K.shape[0]),
                                                                                          lower=True), y))
    with pytest.raises(AssertionError):
        test_solve_cholesky_backward_error_and_lu()
