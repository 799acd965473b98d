"""Pins of the oracle's exact sampled rows (oracle/rows.c, the direct sum of Eq.
(nonstat2)) on the CPU.

The rows oracle backs the large-N error figures, so it is pinned to things other than
itself:
  * constant fields reduce it to the stationary kernel s^2 phi(r / l), checked against
    the textbook exponential (nu = 1/2), the squared exponential, and the general
    Matern written with scipy's modified Bessel function K_nu (nu = 3/2, 5/2);
  * with varying fields it equals the dense Python oracle K alpha (itself pinned to the
    Paciorek form and the closed forms) in d = 1, 2, 3 and for several right-hand sides;
  * K is symmetric, and relabelling the points relabels the rows;
  * an unsupported nu is refused.
"""
import numpy as np
import pytest
import scipy.special

import gpinputs
from oracle import kernel as okern
from oracle import rows as orows


def matern_bessel(r, nu):
    """Eq. (matern) through scipy's K_nu, with phi(0) = 1."""
    r = np.asarray(r, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * r
    out = np.ones_like(z)
    nz = z > 0
    out[nz] = 2.0 ** (1.0 - nu) / scipy.special.gamma(nu) * z[nz] ** nu * scipy.special.kv(nu, z[nz])
    return out


def _stationary(d, nu, n=60, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    s0, l0 = 1.7, 0.13
    w, sig = okern.paper_fields(np.full(n, s0), np.full(n, l0), d)
    alpha = rng.standard_normal((n, 2))
    r = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=2)
    return X, w, sig, alpha, r, s0, l0


@pytest.mark.parametrize("d", [1, 2, 3])
def test_constant_fields_give_exponential_and_squared_exponential(d):
    X, w, sig, alpha, r, s0, l0 = _stationary(d, 0.5)
    idx = np.arange(0, X.shape[0], 3)
    got = orows.rows(X, w, sig, 0.5, alpha, idx)
    want = (s0 ** 2 * np.exp(-r / l0) @ alpha)[idx]
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())
    got = orows.rows(X, w, sig, np.inf, alpha, idx)
    want = (s0 ** 2 * np.exp(-0.5 * (r / l0) ** 2) @ alpha)[idx]
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("nu", [1.5, 2.5])
@pytest.mark.parametrize("d", [1, 3])
def test_constant_fields_give_bessel_matern(d, nu):
    X, w, sig, alpha, r, s0, l0 = _stationary(d, nu, seed=1)
    idx = np.arange(X.shape[0])
    got = orows.rows(X, w, sig, nu, alpha, idx)
    want = s0 ** 2 * matern_bessel(r / l0, nu) @ alpha
    assert np.allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("d,nu", [(1, 1.5), (2, 1.5), (2, 0.5), (3, 2.5)])
def test_varying_fields_equal_the_dense_oracle(d, nu):
    wk = {1: gpinputs.config_1d, 2: gpinputs.config_2d, 3: gpinputs.config_3d}[d](300)
    w, sig = okern.paper_fields(wk.s, wk.l, d)
    rng = np.random.default_rng(5)
    alpha = rng.standard_normal((300, 3))
    K = okern.kernel_dense(wk.points, w, sig, nu)
    idx = rng.choice(300, size=40, replace=False)
    got = orows.rows(wk.points, w, sig, nu, alpha, idx)
    want = (K @ alpha)[idx]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    # one right-hand side comes back as a vector
    one = orows.rows(wk.points, w, sig, nu, alpha[:, 1], idx)
    assert one.shape == (40,) and np.allclose(one, got[:, 1], rtol=0, atol=0)


def test_symmetry_and_relabelling():
    wk = gpinputs.config_2d(80)
    w, sig = okern.paper_fields(wk.s, wk.l, 2)
    n = 80
    # unit right-hand sides give columns of K: K[idx, j] for j < 16
    E = np.eye(n)[:, :16]
    Kblk = orows.rows(wk.points, w, sig, 1.5, E, np.arange(16))
    assert np.allclose(Kblk, Kblk.T, rtol=1e-14, atol=0)
    assert np.all(np.diag(Kblk) > 0) and np.all(np.abs(Kblk) <= np.sqrt(np.outer(np.diag(Kblk), np.diag(Kblk))) * (1 + 1e-14))
    perm = np.random.default_rng(2).permutation(n)
    alpha = np.random.default_rng(3).standard_normal(n)
    full = orows.rows(wk.points, w, sig, 1.5, alpha, np.arange(n))
    relab = orows.rows(wk.points[perm], w[perm], sig[perm], 1.5, alpha[perm], np.arange(n))
    assert np.allclose(relab, full[perm], rtol=1e-12, atol=1e-12 * np.abs(full).max())


def test_unsupported_nu_is_refused():
    X = np.zeros((4, 1))
    with pytest.raises(ValueError):
        orows.rows(X, np.ones(4), np.ones(4), 1.0, np.ones(4), np.arange(2))
