"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test ties one oracle function to a closed form, an independent library
routine, a quadrature of the defining integral, an invariant, or a number the
paper prints.  No GPU.
"""

import numpy as np
import pytest
from scipy import integrate, interpolate, special

import gpinputs
from oracle import bounds, chebyshev, kernel, ktilde, matern, nudft, quadrature


# ---------------------------------------------------------------- phi (Eq. matern)
@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_forms_match_bessel(nu):
    r = np.linspace(0.0, 12.0, 241)
    assert np.max(np.abs(matern.phi_matern_closed(r, nu) - matern.phi_matern_bessel(r, nu))) < 1e-14


def test_matern_bessel_against_sympy_high_precision():
    sympy = pytest.importorskip("sympy")
    for nu in (0.8, 1.5, 3.3):
        for r in (0.05, 0.7, 2.0, 5.0):
            z = sympy.sqrt(2 * sympy.Rational(str(nu))) * sympy.Float(r, 40)
            val = (2 ** (1 - sympy.Float(nu, 40)) / sympy.gamma(sympy.Float(nu, 40))) * z ** sympy.Float(nu, 40) \
                * sympy.besselk(sympy.Float(nu, 40), z)
            assert abs(float(val) - float(matern.phi_matern(np.array([r]), nu)[0])) < 1e-13


def test_matern_half_is_exponential_and_large_nu_tends_to_se():
    r = np.linspace(0, 6, 61)
    assert np.max(np.abs(matern.phi_matern_bessel(r, 0.5) - np.exp(-r))) < 1e-14
    # nu -> infinity limit is the squared exponential (Sec. 2)
    assert np.max(np.abs(matern.phi_matern_bessel(r, 120.0) - np.exp(-r * r / 2))) < 1e-2
    assert matern.phi_matern(np.array([0.0]), 1.5)[0] == 1.0


# --------------------------------------------------------- kernel (Eq. nonstat2)
def test_scale_mapping_equals_paciorek_form():
    for d, w in [(1, gpinputs.config_1d(50)), (2, gpinputs.config_2d(60)), (3, gpinputs.config_3d(40))]:
        wp, sig = kernel.paper_fields(w.s, w.l, d)
        K = kernel.kernel_dense(w.points, wp, sig, w.nu)
        Kp = kernel.paciorek_dense(w.points, w.s, w.l, w.nu)
        assert np.max(np.abs(K - Kp)) < 1e-14 * np.max(np.abs(Kp))
        assert np.allclose(np.diag(K), w.s ** 2, rtol=1e-14)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_stationary_special_case(nu):
    rng = np.random.default_rng(0)
    X = rng.random((40, 2))
    s0, l0 = 1.7, 0.21
    wp, sig = kernel.paper_fields(np.full(40, s0), np.full(40, l0), 2)
    K = kernel.kernel_dense(X, wp, sig, nu)
    r = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1))
    expect = s0 ** 2 * matern.phi_matern_closed(r / l0, nu)
    assert np.max(np.abs(K - expect)) < 1e-14 * s0 ** 2
    if nu == 0.5:
        assert np.max(np.abs(K - s0 ** 2 * np.exp(-r / l0))) < 1e-14 * s0 ** 2


def test_kernel_symmetric_positive_definite():
    w = gpinputs.config_2d(120)
    wp, sig = kernel.paper_fields(w.s, w.l, 2)
    for nu in (0.5, 1.5, 2.5, np.inf):
        K = kernel.kernel_dense(w.points, wp, sig, nu)
        assert np.array_equal(K, K.T)
        assert np.linalg.eigvalsh(K).min() > 0.0
        kernel.solve_cholesky(K, 0.0, np.ones(120))      # factorises


def test_cg_oracle_matches_cholesky():
    w = gpinputs.config_1d(200)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    K = kernel.kernel_dense(w.points, wp, sig, 1.5)
    A = K + 0.01 * np.eye(200)
    x, it, rr = kernel.cg(lambda v: A @ v, w.y, 1e-12, 5000)
    ref = np.linalg.solve(A, w.y)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9
    assert rr <= 1e-12 and 0 < it < 5000


# ------------------------------------------- Schoenberg (Eq. maternpres, App. C)
@pytest.mark.parametrize("nu", [0.5, 0.8, 1.5, 2.5])
def test_schoenberg_integral_reproduces_matern(nu):
    # the continuous integral of Eq. (schoenberg2), by adaptive quadrature
    for r in (0.0, 0.3, 1.0, 3.0):
        f = lambda t: quadrature.u_matern(t, nu) * np.exp(-r * r / (2 * quadrature.chi_matern(t, nu) ** 2))
        val, _ = integrate.quad(f, -60, 8, limit=400, epsabs=1e-14)
        assert abs(val - matern.phi_matern(np.array([r]), nu)[0]) < 1e-10


def test_u_is_a_probability_density_with_gamma_tails():
    nu = 1.5
    tot, _ = integrate.quad(lambda t: quadrature.u_matern(t, nu), -80, 10, limit=400)
    assert abs(tot - 1.0) < 1e-12
    # tail mass below t is the regularised lower incomplete gamma P(nu, e^t)
    for t0 in (-6.0, -2.0, 0.5):
        m, _ = integrate.quad(lambda t: quadrature.u_matern(t, nu), -80, t0, limit=400)
        assert abs(m - special.gammainc(nu, np.exp(t0))) < 1e-12


def test_trapezoid_converges_and_halves_end_weights():
    nu = 1.5
    t_min, t_max = np.log(special.gammaincinv(nu, 1e-13)), np.log(special.gammainccinv(nu, 1e-13))
    r = np.linspace(0, 10, 200)
    errs = [np.max(np.abs(quadrature.phi_from_quadrature(r, nu, t_min, t_max, n) - matern.phi_matern(r, nu)))
            for n in (20, 40, 80)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-11   # Lemma dt: exponential in 1/dt
    _, _, _, tau = quadrature.trapezoid_table(nu, 1, -2.0, 2.0, 4)
    assert np.allclose(tau, [0.5, 1, 1, 1, 0.5])


def test_trapezoid_error_follows_lemma_dt():
    # tails negligible: the error is the discretisation term of Definition eptrap,
    # e^{-(1 - delta) pi^2 / dt}; the integrand is analytic in the strip |Im t| < pi/2,
    # so no rule can beat e^{-pi^2 / dt}
    nu, delta = 1.5, 0.2
    t_min, t_max = np.log(special.gammaincinv(nu, 1e-16)), np.log(special.gammainccinv(nu, 1e-16))
    r = np.linspace(0, 10, 400)
    inv_dt, log_err = [], []
    for n in (8, 12, 16, 20, 24, 28, 32):
        err = np.max(np.abs(quadrature.phi_from_quadrature(r, nu, t_min, t_max, n) - matern.phi_matern(r, nu)))
        assert err <= 10 * bounds.eps_trap(nu, 10.0, delta, t_min, t_max, n), n
        inv_dt.append(n / (t_max - t_min))
        log_err.append(np.log(err))
    rate = -np.polyfit(inv_dt, log_err, 1)[0]
    assert (1 - delta) * np.pi ** 2 <= rate <= 1.05 * np.pi ** 2, rate


# ---------------------------------------------- Gaussian identities (App. B, App. E)
def test_gaussian_product_integral_appendix_b():
    a, b, x, y = 0.13, 0.21, 0.05, 0.31
    val, _ = integrate.quad(lambda z: np.exp(-(x - z) ** 2 / (2 * a * a)) * np.exp(-(y - z) ** 2 / (2 * b * b)),
                            -5, 5, epsabs=1e-15, limit=200)
    closed = np.sqrt(2 * np.pi * a * a * b * b / (a * a + b * b)) * np.exp(-(x - y) ** 2 / (2 * (a * a + b * b)))
    assert abs(val - closed) < 1e-13


def test_ghat_is_the_fourier_transform_of_the_gaussian():
    # G^ of the oracle (d=1, one node, one t) against quad of int exp(-x^2/(2 s^2)) e^{-2 pi i w x} dx
    p = ktilde.Params(1, np.inf, 0, 0, 0, 0.07, 0.07, 0, 6, 1.3)
    G = ktilde.ghat(p)[0, 0]
    s = 0.07
    for idx, n in enumerate(range(-6, 7)):
        om = n * 1.3
        val, _ = integrate.quad(lambda x: np.exp(-x * x / (2 * s * s)) * np.cos(2 * np.pi * om * x), -2, 2,
                                epsabs=1e-15, limit=200)
        assert abs(val - G[idx]) < 1e-13


# ------------------------------------------------- Chebyshev (Eq. chebscheme, Wk)
def test_chebyshev_nodes_and_lagrange_basis():
    nd = chebyshev.nodes(0.2, 0.5, 10)
    assert nd[0] == pytest.approx(0.5) and nd[-1] == pytest.approx(0.2)
    P = chebyshev.lagrange(nd, nd)
    assert np.allclose(P, np.eye(11), atol=1e-13)
    s = np.linspace(0.2, 0.5, 77)
    Ps = chebyshev.lagrange(s, nd)
    assert np.allclose(Ps.sum(1), 1.0, atol=1e-12)
    # against scipy's barycentric interpolator on the same nodes
    for k in range(11):
        e = np.zeros(11)
        e[k] = 1.0
        ref = interpolate.BarycentricInterpolator(nd, e)(s)
        assert np.max(np.abs(ref - Ps[:, k])) < 1e-11
    # exact on polynomials of degree <= N_sigma
    poly = lambda x: 3 * x ** 10 - x ** 3 + 2.0
    assert np.max(np.abs(Ps @ poly(nd) - poly(s))) < 1e-10


@pytest.mark.parametrize("kappa", [1.5, 2.0, 4.0])
def test_lemma_interp_bound_holds(kappa):
    for n in (4, 8, 12):
        err = bounds.interp_error(0.1, 0.1 * kappa, n, 300, 200)
        assert err <= bounds.eps_cheb(n, kappa)


def test_lebesgue_constant_logarithmic():
    for n in (4, 10, 20):
        lam = chebyshev.lebesgue_constant(chebyshev.nodes(1.0, 2.0, n))
        assert 1.0 <= lam <= 2.0 / np.pi * np.log(n + 1) + 1.0


def test_w_k_sums_to_the_multiplier():
    w = gpinputs.config_2d(50)
    wp, sig = kernel.paper_fields(w.s, w.l, 2)
    nd = chebyshev.nodes(sig.min(), sig.max(), 7)
    W = chebyshev.w_k(wp, sig, nd, 2)
    assert np.allclose(W.sum(1), wp * (2 * np.pi * sig ** 2) ** -1.0, rtol=1e-12)


# --------------------------------------------------------- NUDFT (App. D)
def test_nudft_brute_force_and_adjointness():
    rng = np.random.default_rng(1)
    X = rng.random((7, 2)) - 0.5
    c = rng.standard_normal(7)
    M, dw = 3, 0.4
    f = nudft.type1(X, c, M, dw)[0]
    for a in range(-M, M + 1):
        for b in range(-M, M + 1):
            ref = sum(c[j] * np.exp(-2j * np.pi * dw * (a * X[j, 0] + b * X[j, 1])) for j in range(7))
            assert abs(f[a + M, b + M] - ref) < 1e-13
    g = rng.standard_normal((2 * M + 1, 2 * M + 1)) + 1j * rng.standard_normal((2 * M + 1, 2 * M + 1))
    lhs = np.vdot(g, f)                                     # <g, T1 c>
    rhs = np.vdot(nudft.type2(X, g[None], M, dw)[0], c)     # <T2 g, c>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ------------------------------------------------- K~ (Eq. Ktilde, Sec. 4.2)
def _params_1d(sig, nu=1.5, n_t=40, n_s=14, M=1500, P=2.5):
    t_min = np.log(special.gammaincinv(nu, 1e-11))
    t_max = np.log(special.gammainccinv(nu, 1e-11))
    return ktilde.Params(1, nu, t_min, t_max, n_t, sig.min(), sig.max(), n_s, M, 1.0 / P)


def test_ktilde_steps_equal_literal_definition_and_are_psd():
    w = gpinputs.config_1d(70)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    p = _params_1d(sig, n_t=30, n_s=10, M=400)
    Kt = ktilde.dense(w.points, wp, sig, p)
    mv = ktilde.matvec(w.points, wp, sig, w.alpha, p)
    assert np.linalg.norm(mv - Kt @ w.alpha) < 1e-13 * np.linalg.norm(mv)
    assert np.max(np.abs(Kt - Kt.T)) < 1e-14 * np.max(Kt)
    assert np.linalg.eigvalsh(Kt).min() > -1e-13 * np.max(Kt)      # PSD by construction (Sec. 4)
    assert ktilde.matvec_imag_part(w.points, wp, sig, w.alpha, p) < 1e-13 * np.max(np.abs(mv))


def test_ktilde_matches_poisson_closed_form_within_tail():
    w = gpinputs.config_1d(30)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    p = _params_1d(sig, n_t=30, n_s=10, M=300)
    Kt = ktilde.dense(w.points, wp, sig, p)
    Kp = ktilde.dense_poisson(w.points, wp, sig, p)
    gap = np.max(np.abs(Kt - Kp))
    assert gap <= ktilde.grid_tail_bound(wp, sig, p)
    # and the gap closes as M grows
    p2 = _params_1d(sig, n_t=30, n_s=10, M=2400)
    assert np.max(np.abs(ktilde.dense(w.points, wp, sig, p2) - ktilde.dense_poisson(w.points, wp, sig, p2))) < gap / 20


def test_ktilde_2d_poisson_agreement():
    w = gpinputs.config_2d(25)
    wp, sig = kernel.paper_fields(w.s, w.l, 2)
    nu = 2.5
    t_min, t_max = np.log(special.gammaincinv(nu, 1e-9)), np.log(special.gammainccinv(nu, 1e-9))
    p = ktilde.Params(2, nu, t_min, t_max, 16, sig.min(), sig.max(), 5, 70, 1 / 2.0)
    Kt = ktilde.dense(w.points, wp, sig, p)
    Kp = ktilde.dense_poisson(w.points, wp, sig, p)
    assert np.max(np.abs(Kt - Kp)) <= ktilde.grid_tail_bound(wp, sig, p)


def test_ktilde_converges_to_k_theorem_main():
    w = gpinputs.config_1d(40)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    K = kernel.kernel_dense(w.points, wp, sig, 1.5)
    errs = []
    for (n_t, n_s, M) in [(20, 6, 300), (40, 10, 900), (80, 16, 2400)]:
        Kt = ktilde.dense(w.points, wp, sig, _params_1d(sig, n_t=n_t, n_s=n_s, M=M, P=3.0))
        errs.append(np.max(np.abs(K - Kt)) / np.max(K))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-6


def test_constant_scale_gives_stationary_ktilde():
    # kappa = 1: N_sigma = 0, one channel (the stationary EFGP case): K~ depends on x - y only
    X = np.array([[0.1], [0.3], [0.5], [0.7]])
    wp, sig = kernel.paper_fields(np.ones(4), np.full(4, 0.08), 1)
    p = ktilde.Params(1, 1.5, -9.0, 2.8, 40, sig[0], sig[0], 0, 600, 1 / 2.0)
    Kt = ktilde.dense(X, wp, sig, p)
    assert abs(Kt[0, 1] - Kt[1, 2]) < 1e-14 * Kt[0, 0] and abs(Kt[1, 2] - Kt[2, 3]) < 1e-14 * Kt[0, 0]
    assert abs(Kt[0, 2] - Kt[1, 3]) < 1e-14 * Kt[0, 0]


# ---------------------------------------- numbers the paper prints (tests/golden)
def test_paper_se_matvec_accuracy_1d():
    """Sec. 6.1: SE kernel, N_sigma = 26, M = 100, d = 1 keeps relative matvec error near 1e-7."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_experiments.json")))["se_1d"]
    rng = np.random.default_rng(0)
    n = 400                                                  # the error is independent of N (Sec. 6.1)
    X = rng.uniform(-1, 1, (n, 1))
    sig = (np.cos(np.pi * X[:, 0]) + 2.0) / 6.0
    wp = np.ones(n)
    eps = g["eps_nufft"]
    smin, smax = 1 / 6 - 0.01, 0.5 + 0.01
    dw = min(1 / 8, 0.25 / smax / np.sqrt(np.log(1 / eps)))
    p = ktilde.Params(1, np.inf, 0, 0, 0, smin, smax, g["n_sigma"], g["M"], dw)
    alpha = rng.standard_normal(n)
    K = kernel.kernel_dense(X, wp, sig, np.inf)
    e = np.linalg.norm(ktilde.matvec(X, wp, sig, alpha, p) - K @ alpha) / np.linalg.norm(K @ alpha)
    assert e < g["reported_rel_error"] * 10, e


def test_paper_se_solve_regime_matvec_error_2d():
    """Sec. 6.2 noisy regime: SE, d = 2, N_sigma = 15, M = 75 keep matvec errors below 1e-5."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_experiments.json")))["se_2d_solve"]
    rng = np.random.default_rng(2)
    n = 250
    X = rng.uniform(-1, 1, (n, 2))
    sig = (np.prod(np.cos(np.pi * X), axis=1) + 2.0) / 6.0
    wp = np.ones(n)
    eps = g["eps"]
    smin, smax = 1 / 6 - 0.01, 0.5 + 0.01
    dw = min(1 / 8, 0.25 / smax / np.sqrt(np.log(1 / eps)))
    p = ktilde.Params(2, np.inf, 0, 0, 0, smin, smax, g["n_sigma"], g["M"], dw)
    alpha = rng.standard_normal(n)
    K = kernel.kernel_dense(X, wp, sig, np.inf)
    e = np.linalg.norm(ktilde.matvec(X, wp, sig, alpha, p) - K @ alpha) / np.linalg.norm(K @ alpha)
    assert e < g["reported_max_rel_error"], e


# ----------------------------- planted mistakes: each pin above must catch one
def test_planted_sign_error_in_type2_is_caught(monkeypatch):
    orig = nudft._factors
    monkeypatch.setattr(nudft, "_factors", lambda X, M, dw, sign: orig(X, M, dw, -1.0))   # type 2 uses e^{-...}
    rng = np.random.default_rng(1)
    X = rng.random((7, 2)) - 0.5
    c = rng.standard_normal(7)
    f = nudft.type1(X, c, 3, 0.4)[0]
    g = rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7))
    assert abs(np.vdot(g, f) - np.vdot(nudft.type2(X, g[None], 3, 0.4)[0], c)) > 1e-3


def test_planted_missing_chi_power_is_caught(monkeypatch):
    # v_j = tau_j u_j (dropping chi^-d of Eq. (v)) breaks K~ -> K (Theorem main)
    orig = quadrature.trapezoid_table

    def bad(nu, d, t_min, t_max, n_t):
        t, v, chi, tau = orig(nu, d, t_min, t_max, n_t)
        return t, v * chi ** d, chi, tau
    monkeypatch.setattr(quadrature, "trapezoid_table", bad)
    w = gpinputs.config_1d(30)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    K = kernel.kernel_dense(w.points, wp, sig, 1.5)
    Kt = ktilde.dense(w.points, wp, sig, _params_1d(sig, n_t=40, n_s=12, M=1200, P=3.0))
    assert np.max(np.abs(K - Kt)) / np.max(K) > 1e-2


def test_planted_unhalved_trapezoid_end_is_caught(monkeypatch):
    orig = quadrature.trapezoid_table

    def bad(nu, d, t_min, t_max, n_t):
        t, v, chi, tau = orig(nu, d, t_min, t_max, n_t)
        v = v.copy()
        v[-1] *= 2.0
        return t, v, chi, tau
    monkeypatch.setattr(quadrature, "trapezoid_table", bad)
    w = gpinputs.config_1d(30)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    K = kernel.kernel_dense(w.points, wp, sig, 1.5)
    # t_max short enough that the last node carries visible weight
    p = ktilde.Params(1, 1.5, -12.0, 1.5, 40, sig.min(), sig.max(), 12, 1200, 1 / 3.0)
    Kt = ktilde.dense(w.points, wp, sig, p)
    assert np.max(np.abs(K - Kt)) / np.max(K) > 1e-3


def test_planted_wrong_ghat_exponent_is_caught(monkeypatch):
    orig = ktilde.ghat

    def bad(p):
        G = orig(p)
        return G ** 1.01
    monkeypatch.setattr(ktilde, "ghat", bad)
    w = gpinputs.config_1d(30)
    wp, sig = kernel.paper_fields(w.s, w.l, 1)
    p = _params_1d(sig, n_t=30, n_s=10, M=300)
    assert np.max(np.abs(ktilde.dense(w.points, wp, sig, p) - ktilde.dense_poisson(w.points, wp, sig, p))) > \
        10 * ktilde.grid_tail_bound(wp, sig, p)


# Each planted mistake below is caught by one of the pins above, which is called as it
# stands and must fail.
def test_planted_unscaled_sigma_mapping_is_caught(monkeypatch):
    # sigma = l instead of l / sqrt(2)
    monkeypatch.setattr(kernel, "paper_fields",
                        lambda s, l, d: (np.asarray(s) * (2 * np.pi) ** (d / 4) * np.asarray(l) ** (d / 2),
                                         np.asarray(l, dtype=np.float64)))
    with pytest.raises(AssertionError):
        test_scale_mapping_equals_paciorek_form()


def test_planted_wrong_kernel_argument_is_caught(monkeypatch):
    # phi(|x - y| / sqrt(sigma_x^2 + sigma_y^2)) evaluated at sqrt(2) times the argument
    orig = kernel.phi
    monkeypatch.setattr(kernel, "phi", lambda r, nu: orig(np.sqrt(2.0) * r, nu))
    with pytest.raises(AssertionError):
        test_stationary_special_case(1.5)


def test_planted_wrong_chi_is_caught(monkeypatch):
    # chi(t) = e^t / sqrt(nu) instead of e^{t/2} / sqrt(nu) (Eq. maternpres)
    monkeypatch.setattr(quadrature, "chi_matern", lambda t, nu: np.exp(np.asarray(t, dtype=np.float64)) / np.sqrt(nu))
    with pytest.raises(AssertionError):
        test_schoenberg_integral_reproduces_matern(1.5)


def test_planted_off_by_one_chebyshev_nodes_is_caught(monkeypatch):
    # cos(pi k / (N_sigma + 1)): the last node misses sigma_min
    def bad(smin, smax, n):
        k = np.arange(n + 1)
        return (np.cos(np.pi * k / (n + 1)) + 1.0) / 2.0 * (smax - smin) + smin
    monkeypatch.setattr(chebyshev, "nodes", bad)
    with pytest.raises(AssertionError):
        test_chebyshev_nodes_and_lagrange_basis()


def test_planted_reversed_channel_index_is_caught(monkeypatch):
    # w_k(x) paired with the node sigma_{N_sigma - k}: the channels no longer match G^_k
    orig = chebyshev.w_k
    monkeypatch.setattr(chebyshev, "w_k", lambda w, sigma, nd, d: orig(w, sigma, nd, d)[:, ::-1])
    with pytest.raises(AssertionError):
        test_ktilde_converges_to_k_theorem_main()


def test_planted_missing_grid_weight_is_caught(monkeypatch):
    # v~_j = v_j, dropping the (dw)^d of Eq. (Ktilde)
    orig = ktilde.a_tensor
    monkeypatch.setattr(ktilde, "a_tensor", lambda p: orig(p) / p.dw ** p.d)
    with pytest.raises(AssertionError):
        test_ktilde_steps_equal_literal_definition_and_are_psd()
