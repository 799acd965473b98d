"""Pins of the diagonal-correction oracle (oracle/diagcorr.py), an extension for small nu.

  * K~_ii from S = sum_n A[n] against the diagonal of Eq. (Ktilde) written literally
    (ktilde.dense, which never forms A);
  * the squared-exponential, constant-scale case in closed form: one channel, one
    quadrature node, A[n] = dw^d (2 pi sigma^2)^d exp(-4 pi^2 sigma^2 dw^2 |n|^2), so
    K~_ii = w^2 (dw sum_{|m|<=M} exp(-4 pi^2 sigma^2 dw^2 m^2))^d, and as the grid
    refines it tends to the Gaussian integral w^2 (4 pi sigma^2)^(-d/2) = K_ii;
  * the corrected operator has K's diagonal exactly, keeps K~'s off-diagonal entries,
    and for nu = 1/2 is closer to K than K~ is;
  * a planted mistake (S summed over the half grid only) is caught.
No GPU.
"""
import numpy as np
from scipy import special

import gpinputs
from oracle import diagcorr, kernel, ktilde


def _matern_params(d, sig, X, nu, n_t, n_s, M, P=2.5):
    t_min = np.log(special.gammaincinv(nu, 1e-11))
    t_max = np.log(special.gammainccinv(nu, 1e-11))
    return ktilde.Params(d, nu, t_min, t_max, n_t, sig.min(), sig.max(), n_s, M, 1.0 / P)


def test_diag_from_s_matrix_equals_literal_ktilde_diagonal():
    for d, w in [(1, gpinputs.config_1d(40)), (2, gpinputs.config_2d(30))]:
        wp, sig = kernel.paper_fields(w.s, w.l, d)
        p = _matern_params(d, sig, w.points, 1.5, 20, 6, 200 if d == 1 else 40)
        lit = np.diag(ktilde.dense(w.points, wp, sig, p))
        got = diagcorr.ktilde_diag(wp, sig, p)
        assert np.max(np.abs(got - lit)) < 1e-12 * np.max(lit)


def test_se_constant_scale_closed_form_and_limit():
    s0, w0 = 0.05, 1.3
    for d in (1, 2, 3):
        for M, dw in [(20, 1.0), (60, 0.5)]:
            p = ktilde.Params(d, np.inf, 0.0, 0.0, 0, s0, s0, 0, M, dw)
            m = np.arange(-M, M + 1, dtype=np.float64)
            closed = w0 ** 2 * (dw * np.sum(np.exp(-4 * np.pi ** 2 * s0 ** 2 * dw ** 2 * m ** 2))) ** d
            got = diagcorr.ktilde_diag(np.array([w0]), np.array([s0]), p)[0]
            assert abs(got - closed) < 1e-13 * closed, (d, M, got, closed)
        # grid fine and wide enough: the Riemann sum is the Gaussian integral
        p = ktilde.Params(d, np.inf, 0.0, 0.0, 0, s0, s0, 0, 400, 0.2)
        got = diagcorr.ktilde_diag(np.array([w0]), np.array([s0]), p)[0]
        kii = diagcorr.k_diag(np.array([w0]), np.array([s0]), d)[0]
        assert abs(got - kii) < 1e-12 * kii


def test_corrected_operator_diagonal_and_off_diagonal():
    w = gpinputs.config_1d(50)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    p = _matern_params(1, sig, w.points, 0.5, 40, 10, 300)
    Kt = ktilde.dense(w.points, wp, sig, p)
    K = kernel.kernel_dense(w.points, wp, sig, 0.5)
    Kc = Kt + np.diag(diagcorr.defect(wp, sig, p))
    assert np.max(np.abs(np.diag(Kc) - np.diag(K))) < 1e-12 * np.max(np.diag(K))
    off = ~np.eye(len(K), dtype=bool)
    assert np.array_equal(Kc[off], Kt[off])
    mv = diagcorr.matvec(w.points, wp, sig, w.alpha, p)
    assert np.linalg.norm(mv - Kc @ w.alpha) < 1e-12 * np.linalg.norm(mv)
    two = diagcorr.matvec(w.points, wp, sig, np.column_stack([w.alpha, 2 * w.alpha]), p)
    assert np.linalg.norm(two[:, 1] - 2 * mv) < 1e-12 * np.linalg.norm(mv)


def test_correction_reduces_the_error_for_nu_half():
    """nu = 1/2 on a grid too coarse for its cusp: K~ undershoots the diagonal, the
    defect is positive, and the corrected matvec is closer to K alpha."""
    for d, w in [(1, gpinputs.config_1d(300)), (2, gpinputs.config_2d(200))]:
        wp, sig = kernel.paper_fields(w.s, w.l, d)
        p = _matern_params(d, sig, w.points, 0.5, 40, 8, 150 if d == 1 else 40)
        dv = diagcorr.defect(wp, sig, p)
        assert np.all(dv > 0)
        K = kernel.kernel_dense(w.points, wp, sig, 0.5)
        ref = K @ w.alpha
        e0 = np.linalg.norm(ktilde.matvec(w.points, wp, sig, w.alpha, p) - ref) / np.linalg.norm(ref)
        e1 = np.linalg.norm(diagcorr.matvec(w.points, wp, sig, w.alpha, p) - ref) / np.linalg.norm(ref)
        assert e1 < 0.8 * e0, (d, e0, e1)


def test_planted_half_grid_sum_is_caught(monkeypatch):
    w = gpinputs.config_1d(20)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    p = _matern_params(1, sig, w.points, 1.5, 20, 6, 200)
    lit = np.diag(ktilde.dense(w.points, wp, sig, p))

    def half(p_):
        A = ktilde.a_tensor(p_)
        return A[..., p_.M:].sum(axis=-1)          # only n >= 0

    monkeypatch.setattr(diagcorr, "s_matrix", half)
    assert np.max(np.abs(diagcorr.ktilde_diag(wp, sig, p) - lit)) > 1e-3 * np.max(lit)
