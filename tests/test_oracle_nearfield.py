"""Pins of the near-field correction oracle (oracle/nearfield.py), an extension for small nu.

  * K~_ij by the separable form (one factor t_klj per dimension) against Eq. (Ktilde)
    written literally (ktilde.dense, the sum over the whole grid of Z_j(x) conj(Z_j(y))),
    entry by entry, d = 1 and 2;
  * radius beyond the box: every off-diagonal entry is K's exactly, and with the diagonal
    correction the whole matrix is K;
  * radius zero: K~ itself; the pair list is symmetric and excludes i = j;
  * the sparse matvec equals the dense corrected matrix times alpha;
  * for nu = 1/2 on sparse points the corrected operator is closer to K than K~ and than
    K~ with the diagonal correction alone;
  * a planted mistake (sine instead of cosine in t_klj) is caught.
No GPU.
"""
import numpy as np
import pytest
from scipy import special

import gpinputs
from oracle import diagcorr, kernel, ktilde, nearfield


def _params(d, sig, nu, n_t, n_s, M, P=2.5):
    t_min = np.log(special.gammaincinv(nu, 1e-11))
    t_max = np.log(special.gammainccinv(nu, 1e-11))
    return ktilde.Params(d, nu, t_min, t_max, n_t, sig.min(), sig.max(), n_s, M, 1.0 / P)


def _case(d, n, nu):
    w = gpinputs.config_1d(n) if d == 1 else gpinputs.config_2d(n, nu)
    wp, sig = kernel.paper_fields(w.s, w.l, d)
    return w, wp, sig


@pytest.mark.parametrize("d", [1, 2])
def test_separable_pairs_equal_the_literal_ktilde(d):
    w, wp, sig = _case(d, 30 if d == 1 else 20, 1.5)
    p = _params(d, sig, 1.5, 16, 5, 150 if d == 1 else 30)
    Kt = ktilde.dense(w.points, wp, sig, p)
    n = w.N
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    got = nearfield.ktilde_pairs(w.points[i], wp[i], sig[i], w.points[j], wp[j], sig[j], p).reshape(n, n)
    assert np.max(np.abs(got - Kt)) <= 1e-13 * np.max(np.abs(Kt))


def test_radius_beyond_the_box_gives_k_and_zero_gives_ktilde():
    w, wp, sig = _case(2, 25, 0.5)
    p = _params(2, sig, 0.5, 16, 5, 30)
    K = kernel.kernel_dense(w.points, wp, sig, 0.5)
    Kt = ktilde.dense(w.points, wp, sig, p)
    big = nearfield.dense(w.points, wp, sig, 0.5, p, 10.0)
    off = ~np.eye(w.N, dtype=bool)
    assert np.max(np.abs(big[off] - K[off])) <= 1e-13 * np.max(K)
    assert np.max(np.abs(np.diag(big) - np.diag(Kt))) == 0.0
    full = nearfield.dense(w.points, wp, sig, 0.5, p, 10.0, diag=True)
    assert np.max(np.abs(full - K)) <= 1e-13 * np.max(K)
    assert np.array_equal(nearfield.dense(w.points, wp, sig, 0.5, p, 0.0), Kt)
    i, j = nearfield.pairs_within(w.points, 0.2)
    assert np.all(i != j)
    assert set(zip(i.tolist(), j.tolist())) == set(zip(j.tolist(), i.tolist()))


def test_sparse_matvec_equals_dense():
    w, wp, sig = _case(2, 40, 0.5)
    p = _params(2, sig, 0.5, 16, 5, 30)
    a = w.alpha
    for diag in (False, True):
        Kd = nearfield.dense(w.points, wp, sig, 0.5, p, 0.08, diag=diag)
        got = nearfield.matvec(w.points, wp, sig, 0.5, a, p, 0.08, diag=diag)
        assert np.linalg.norm(got - Kd @ a) <= 1e-12 * np.linalg.norm(Kd @ a)


def test_nu_half_closer_to_k_than_ktilde_and_the_diagonal_alone():
    w, wp, sig = _case(2, 300, 0.5)
    p = _params(2, sig, 0.5, 30, 6, 40)
    K = kernel.kernel_dense(w.points, wp, sig, 0.5)
    ref = K @ w.alpha
    e0 = np.linalg.norm(ktilde.matvec(w.points, wp, sig, w.alpha, p) - ref)
    e1 = np.linalg.norm(diagcorr.matvec(w.points, wp, sig, w.alpha, p) - ref)
    e2 = np.linalg.norm(nearfield.matvec(w.points, wp, sig, 0.5, w.alpha, p, 0.1, diag=True) - ref)
    assert e2 < 0.5 * e1 and e1 < e0, (e0, e1, e2)


def test_planted_sine_in_the_factor_is_caught(monkeypatch):
    # t_klj with sin(2 pi m dw rho) where the even sum over m needs cos
    def bad(p, rho):
        _, v, chi, nd = p.tables()
        rho = np.asarray(rho, dtype=np.float64)
        m = np.arange(-p.M, p.M + 1, dtype=np.float64)
        s = nd[:, None] * chi[None, :]
        e = np.sqrt(2.0 * np.pi) * s[..., None] * np.exp(-2.0 * np.pi ** 2 * (s[..., None] * p.dw * m) ** 2)
        ee = e[:, None, :, :] * e[None, :, :, :]
        ph = np.sin(2.0 * np.pi * p.dw * m[:, None] * rho.reshape(1, -1))
        out = np.einsum("kljm,mr->kljr", ee, ph, optimize=True)
        return out.reshape(out.shape[:3] + rho.shape)
    monkeypatch.setattr(nearfield, "t_factor", bad)
    with pytest.raises(AssertionError):
        test_separable_pairs_equal_the_literal_ktilde(1)
