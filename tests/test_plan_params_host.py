"""Plan parameter selection on the host (gp_plan_params), no GPU: the fine-grid rules per
dimension, the 3-D grid cost model, the transform and step-3 predictions, the footprint
estimate and argument checks."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def abi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03608_gb300 import abi
    return abi


def smooth7(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def params(abi, d, N, eps, smin, smax, nu=1.5, precision=1, **kw):
    # smin, smax: the paper's sigma
    o = abi.default_opts(precision=precision, param_mode=abi.GP_PARAMS_PAPER, **kw)
    return abi.gp_plan_params(d, N, nu, eps, smin, smax, [0.0] * d, [1.0] * d, o)


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_grids_up_to_two_dimensions_are_powers_of_two(abi, d, eps):
    i = params(abi, d, 10_000, eps, 0.01, 0.02)
    nf, M = i["nf"], i["M"]
    assert nf & (nf - 1) == 0
    assert nf >= 1.25 * (2 * M + 1) and nf // 2 < 1.25 * (2 * M + 1) or i["kernel_width"] > 9
    if d == 2:
        assert i["transform"] == 3          # the transposed pruned transforms
    # the points sit inside the grid with the kernel's margin, no wrap-around
    P = 1.0 / i["dw"]
    assert 1.0 / P * nf + i["kernel_width"] + 4 <= nf


def test_three_dimensional_grid_model(abi):
    smin, smax = 0.05 / np.sqrt(2), 0.10 / np.sqrt(2)
    widths = []
    for N in (2_000, 200_000, 2_000_000):
        i = params(abi, 3, N, 1e-6, smin, smax, nu=2.5)
        nf = i["nf"]
        assert nf % 4 == 0 and smooth7(nf)                      # 16-byte TMA rows, cuFFT-friendly
        assert nf >= 1.25 * (2 * i["M"] + 1)
        widths.append(i["kernel_width"])
    # more points buy a finer grid and a narrower spreading kernel
    assert widths == sorted(widths, reverse=True)
    assert widths[-1] <= 9
    big = params(abi, 3, 2_000_000, 1e-6, smin, smax, nu=2.5)
    assert (big["nf"], big["kernel_width"], big["tile"]) == (864, 9, 8)


def test_three_dimensional_nf_override_and_stride_rule(abi):
    smin, smax = 0.05 / np.sqrt(2), 0.10 / np.sqrt(2)
    base = params(abi, 3, 10_000, 1e-4, smin, smax, nu=2.5)
    o = abi.default_opts(precision=abi.GP_FP32, nf=base["nf"] + 4, set=abi.GP_SET_NF, param_mode=abi.GP_PARAMS_PAPER)
    i = abi.gp_plan_params(3, 10_000, 2.5, 1e-4, smin, smax, [0, 0, 0], [1, 1, 1], o)
    assert i["nf"] == base["nf"] + 4
    o = abi.default_opts(precision=abi.GP_FP32, nf=base["nf"] + 2, set=abi.GP_SET_NF, param_mode=abi.GP_PARAMS_PAPER)
    with pytest.raises(abi.GPError) as e:
        abi.gp_plan_params(3, 10_000, 2.5, 1e-4, smin, smax, [0, 0, 0], [1, 1, 1], o)
    assert e.value.status == abi.GP_EINVAL and "16-byte" in str(e.value)


def test_accuracy_drives_the_mode_count_and_channels(abi):
    Ms = [params(abi, 2, 50_000, eps, 0.01, 0.02)["M"] for eps in (1e-3, 1e-4, 1e-5, 1e-6)]
    assert Ms == sorted(Ms) and Ms[0] < Ms[-1]
    # a wider scale range needs more Chebyshev channels (Lemma interp)
    narrow = params(abi, 2, 50_000, 1e-6, 0.01, 0.012)["n_sigma"]
    wide = params(abi, 2, 50_000, 1e-6, 0.01, 0.04)["n_sigma"]
    assert narrow < wide
    # constant scale: one channel (the stationary special case)
    assert params(abi, 2, 50_000, 1e-6, 0.015, 0.015)["n_sigma"] == 0
    # the squared exponential needs no quadrature in t
    assert params(abi, 1, 2000, 1e-6, 0.01, 0.02, family=abi.GP_SE)["n_t"] == 0


def test_transform_and_step3_predictions(abi):
    # 1-D in FP64: the pruned row transforms; in FP32: the full-grid cuFFT path
    assert params(abi, 1, 2000, 1e-6, 0.01, 0.04, precision=abi.GP_FP64)["transform"] == 2
    assert params(abi, 1, 2000, 1e-6, 0.01, 0.04, precision=abi.GP_FP32)["transform"] == 1
    smin, smax = 0.05 / np.sqrt(2), 0.10 / np.sqrt(2)
    full = params(abi, 3, 2_000_000, 1e-6, smin, smax, nu=2.5)
    assert full["step3"] == 1
    lean = params(abi, 3, 2_000_000, 1e-6, smin, smax, nu=2.5, step3=2)
    assert lean["step3"] == 2 and lean["bytes_resident"] < full["bytes_resident"]
    # auto: the tensor when it fits max_bytes, the lean form when only that fits
    mid = (lean["bytes_resident"] + full["bytes_resident"]) // 2
    assert params(abi, 3, 2_000_000, 1e-6, smin, smax, nu=2.5, max_bytes=mid)["step3"] == 2
    assert params(abi, 3, 2_000_000, 1e-6, smin, smax, nu=2.5, max_bytes=full["bytes_resident"])["step3"] == 1


def test_footprint_estimate_scales_with_right_hand_sides(abi):
    one = params(abi, 2, 100_000, 1e-5, 0.01, 0.02)["bytes_resident"]
    eight = params(abi, 2, 100_000, 1e-5, 0.01, 0.02, max_rhs=8)["bytes_resident"]
    assert 5 * one < eight < 8 * one        # grids and spectra per rhs, A' shared


def test_invalid_arguments(abi):
    o = abi.default_opts()
    for args in [(0, 10, 1.5, 1e-6, 0.01, 0.02), (2, 0, 1.5, 1e-6, 0.01, 0.02), (2, 10, -1.0, 1e-6, 0.01, 0.02),
                 (2, 10, 1.5, 0.5, 0.01, 0.02), (2, 10, 1.5, 1e-6, 0.02, 0.01), (2, 10, 1.5, 1e-6, 0.0, 0.02)]:
        with pytest.raises(abi.GPError) as e:
            abi.gp_plan_params(*args, [0, 0, 0], [1, 1, 1], o)
        assert e.value.status == abi.GP_EINVAL
    abi.gp_plan_params(2, 10, 1.5, 1e-3, 0.01, 0.02, [0, 0], [1, 1], o)   # clears the error message
    assert abi.LIB.gp_last_error() == b""


# The parameters chosen for eps against the oracle's K~ (Eq. Ktilde written out densely)
# and the dense K (Eq. nonstat2): Theorem main's entrywise error relative to
# sqrt(K_ii K_jj) must meet eps, and the choice should not overshoot it by much (each
# stage of the selector aims at a share of eps).
@pytest.mark.parametrize("d,nu,eps", [(1, 0.5, 1e-3), (1, 1.5, 1e-3), (1, 1.5, 1e-5), (1, 2.5, 1e-7), (1, None, 1e-5),
                                      (2, 1.5, 1e-2), (2, 2.5, 1e-3)])
def test_chosen_parameters_meet_eps_against_the_oracle(abi, d, nu, eps):
    import gpinputs
    from oracle import kernel as okern
    from oracle import ktilde
    w = gpinputs.config_1d(200) if d == 1 else gpinputs.config_2d(120)
    X = w.points
    wp, sig = okern.paper_fields(w.s, w.l, d)
    fam = abi.GP_SE if nu is None else abi.GP_MATERN
    o = abi.default_opts(precision=abi.GP_FP64, family=fam, param_mode=abi.GP_PARAMS_PAPER)
    i = abi.gp_plan_params(d, X.shape[0], 1.0 if nu is None else nu, eps, float(sig.min()), float(sig.max()),
                           [float(v) for v in X.min(0)], [float(v) for v in X.max(0)], o)
    nu_o = np.inf if nu is None else nu
    p = ktilde.Params(d, nu_o, i["t_min"], i["t_max"], i["n_t"], i["sigma_lo"], i["sigma_hi"], i["n_sigma"],
                      int(i["M"]), i["dw"])
    Kt = ktilde.dense(X, wp, sig, p)
    K = okern.kernel_dense(X, wp, sig, nu_o)
    dg = np.sqrt(np.diag(K))
    err = float(np.max(np.abs(K - Kt) / np.outer(dg, dg)))
    assert eps / 30 <= err <= eps, (err, {k: i[k] for k in ("n_t", "n_sigma", "M")})


# Stage 1 (Lemma dt) of the host selector against the oracle's quadrature: the tails sit
# where the regularised incomplete gamma puts eps/12 (scipy), the selector's estimate
# of the trapezoid error equals the oracle's sup |phi - sum_j tau_j u_j e^{-r^2/(2 chi_j^2)}|,
# it meets eps/4, and one node fewer would not.
@pytest.mark.parametrize("nu", [1.5, 2.5, 3.2])
@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_stage_one_quadrature_matches_the_oracle(abi, nu, eps):
    from scipy import special
    from oracle import matern, quadrature
    i = abi.gp_plan_params(1, 1000, nu, eps, 0.01, 0.02, [0.0], [1.0], abi.default_opts(param_mode=abi.GP_PARAMS_PAPER))
    assert special.gammainc(nu, np.exp(i["t_min"])) == pytest.approx(eps / 12, rel=1e-6)
    assert special.gammaincc(nu, np.exp(i["t_max"])) == pytest.approx(eps / 12, rel=1e-6)
    r = np.concatenate([np.linspace(0, 2, 4001), np.linspace(2, 60, 4001)])

    def sup_err(n_t):
        q = quadrature.phi_from_quadrature(r, nu, i["t_min"], i["t_max"], n_t)
        return float(np.max(np.abs(q - matern.phi_matern(r, nu))))

    e = sup_err(i["n_t"])
    assert e == pytest.approx(i["est_err_t"], rel=1e-2)
    assert e <= eps / 4
    assert sup_err(i["n_t"] - 1) > 0.98 * eps / 4


# Stage 3 (Lemma stage3) of the host selector, recomputed with the oracle's trapezoid
# table (tau_j, u(t_j), chi_j): the truncation estimate d sum_j tau_j u_j erfc(2 pi
# sigma_lo chi_j M dw) meets eps/4 and one mode fewer would not; the alias estimate
# d sum_j tau_j u_j exp(-(1/dw - L)^2 / (4 sigma_hi^2 chi_j^2)) meets eps/8, with L the
# widest side of the box.
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("nu,eps", [(1.5, 1e-4), (2.5, 1e-7)])
def test_stage_three_estimates_match_the_oracle_tables(abi, d, nu, eps):
    from scipy import special
    from oracle import quadrature
    lo, hi = [0.0] * d, [1.0, 0.8, 0.6][:d]
    i = abi.gp_plan_params(d, 10_000, nu, eps, 0.02, 0.05, lo, hi, abi.default_opts(param_mode=abi.GP_PARAMS_PAPER))
    t, _, chi, tau = quadrature.trapezoid_table(nu, d, i["t_min"], i["t_max"], i["n_t"])
    wu = tau * quadrature.u_matern(t, nu)

    def trunc(M):
        return d * float(np.sum(wu * special.erfc(2 * np.pi * i["sigma_lo"] * chi * M * i["dw"])))

    assert trunc(i["M"]) == pytest.approx(i["est_err_trunc"], rel=1e-6)
    assert trunc(i["M"]) <= eps / 4 < trunc(i["M"] - 1)
    L = max(i["box_hi"][a] - i["box_lo"][a] for a in range(d))
    gap = 1.0 / i["dw"] - L
    alias = d * float(np.sum(wu * np.exp(-gap ** 2 / (4 * i["sigma_hi"] ** 2 * chi ** 2))))
    assert alias == pytest.approx(i["est_err_alias"], rel=1e-6)
    assert alias <= eps / 8


# Stage 2 (Lemma sigma) of the host selector with the oracle's Chebyshev nodes and
# Lagrange basis (product formula; the library evaluates the barycentric form): the
# sup over sigma_x, sigma_y and rho of the interpolated normalised Gaussian product,
#   |sum_kl P_k(s_x) P_l(s_y) c_kl e^{-rho^2/(2 s_kl)} - c(s_x, s_y) e^{-rho^2/(2 (s_x^2 + s_y^2))}|
#   / (s_x s_y / 2)^{d/2},   c(a, b) = (a^2 b^2 / (a^2 + b^2))^{d/2},
# sampled on grids that contain the selector's (so it can only find more), bounds the
# selector's estimate from above, stays near eps/4 at the chosen N_sigma and exceeds
# eps/4 with one node fewer.
def _stage2_sup(d, lo, hi, n_sigma, ns=47, nr=95):
    from oracle import chebyshev
    nd = chebyshev.nodes(lo, hi, n_sigma)
    sv = lo + (hi - lo) * np.arange(ns) / (ns - 1)
    P = chebyshev.lagrange(sv, nd)                                    # (ns, C)
    a2, b2 = nd[:, None] ** 2, nd[None, :] ** 2
    ckl, skl = (a2 * b2 / (a2 + b2)) ** (d / 2), a2 + b2
    x2, y2 = sv[:, None] ** 2, sv[None, :] ** 2
    cxy, sxy = (x2 * y2 / (x2 + y2)) ** (d / 2), x2 + y2
    norm = (0.5 * sv[:, None] * sv[None, :]) ** (d / 2)
    worst = 0.0
    for rho in 12.0 * hi * np.arange(nr) / (nr - 1):
        approx = P @ (ckl * np.exp(-rho ** 2 / (2 * skl))) @ P.T
        exact = cxy * np.exp(-rho ** 2 / (2 * sxy))
        worst = max(worst, float(np.max(np.abs(approx - exact) / norm)))
    return worst


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("smin,smax,eps", [(0.02, 0.03, 1e-4), (0.02, 0.04, 1e-7), (0.01, 0.04, 1e-6)])
def test_stage_two_estimate_against_the_oracle_basis(abi, d, smin, smax, eps):
    i = abi.gp_plan_params(d, 10_000, 1.5, eps, smin, smax, [0.0] * d, [1.0] * d,
                           abi.default_opts(param_mode=abi.GP_PARAMS_PAPER))
    n, lo, hi = i["n_sigma"], i["sigma_lo"], i["sigma_hi"]
    sup = _stage2_sup(d, lo, hi, n)
    assert sup >= i["est_err_sigma"] * (1 - 1e-9)
    assert i["est_err_sigma"] <= eps / 4 and sup <= 1.5 * eps / 4
    assert _stage2_sup(d, lo, hi, n - 1) > eps / 4


def test_scale_range_is_taken_in_the_plans_parametrisation(abi):
    # GP_PARAMS_SCALES (default): the range of the length l; the library maps it to the
    # paper's sigma = l / sqrt(2), the same plan as passing sigma with GP_PARAMS_PAPER
    lmin, lmax = 0.02, 0.04
    a = abi.gp_plan_params(2, 100_000, 1.5, 1e-5, lmin, lmax, [0, 0], [1, 1], abi.default_opts(precision=abi.GP_FP32))
    b = abi.gp_plan_params(2, 100_000, 1.5, 1e-5, lmin / np.sqrt(2), lmax / np.sqrt(2), [0, 0], [1, 1],
                           abi.default_opts(precision=abi.GP_FP32, param_mode=abi.GP_PARAMS_PAPER))
    for k in ("n_t", "n_sigma", "M", "nf", "kernel_width", "tile", "bytes_resident"):
        assert a[k] == b[k], k
    assert a["sigma_lo"] == pytest.approx(b["sigma_lo"], rel=1e-15)
    assert a["sigma_hi"] == pytest.approx(b["sigma_hi"], rel=1e-15)


def test_rhs_block_keeps_one_block_of_grids(abi):
    # grids, spectra and transform buffers for rhs_block right-hand sides, vectors for max_rhs
    base = params(abi, 2, 100_000, 1e-5, 0.01, 0.02, max_rhs=1)
    full = params(abi, 2, 100_000, 1e-5, 0.01, 0.02, max_rhs=64)
    blocked = params(abi, 2, 100_000, 1e-5, 0.01, 0.02, max_rhs=64, rhs_block=8)
    assert blocked["rhs_block"] == 8 and full["rhs_block"] == 64 and base["rhs_block"] == 1
    per_rhs_grids = (full["bytes_resident"] - base["bytes_resident"]) / 63.0
    assert blocked["bytes_resident"] < full["bytes_resident"] - 50 * per_rhs_grids
    eight = params(abi, 2, 100_000, 1e-5, 0.01, 0.02, max_rhs=8)
    # the same grids as max_rhs = 8, plus 56 more columns of the nine work vectors
    assert blocked["bytes_resident"] - eight["bytes_resident"] == 100_000 * 56 * 8 * 9
    # a block at least max_rhs is no block
    assert params(abi, 2, 100_000, 1e-5, 0.01, 0.02, max_rhs=4, rhs_block=9)["rhs_block"] == 4


@pytest.mark.parametrize("nf", [864, 1024])
def test_full_grid_footprint_counts_the_cufft_work_area(abi, nf):
    """3-D full-grid plans: cuFFT's transforms need a work area as large as the half
    spectrum when nf is not a power of two.  The forward one works in the interpolation
    grid and the inverse, with the memory-lean step 3, in the spreading grid, so the
    footprint adds a spectrum only for the stored-A' plan at nf = 864; each grid buffer
    holds max(nf^3, 2 S) reals either way."""
    N, rs = 200_000, 4
    full = params(abi, 3, N, 1e-5, 0.03, 0.06, nu=2.5, step3=1, nf=nf, set=abi.GP_SET_NF)
    lean = params(abi, 3, N, 1e-5, 0.03, 0.06, nu=2.5, step3=2, nf=nf, set=abi.GP_SET_NF)
    assert full["nf"] == lean["nf"] == nf and full["step3"] == 1 and lean["step3"] == 2
    C, M, J = full["n_sigma"] + 1, full["M"], full["n_t"] + 1
    S = nf * nf * (nf // 2 + 1)
    a_bytes = C * (C + 1) // 2 * (2 * M + 1) ** 2 * (M + 1) * rs
    lean_bytes = J * (M + 1) * (-(-C // (16 // rs)) * (16 // rs)) * rs
    work = C * S * 2 * rs if nf & (nf - 1) else 0
    assert full["bytes_resident"] - lean["bytes_resident"] == a_bytes - lean_bytes + work
    # the grid padding: two buffers of C max(nf^3, 2 S) reals against C nf^3 each
    plain = params(abi, 3, N, 1e-5, 0.03, 0.06, nu=2.5, step3=2, nf=nf, set=abi.GP_SET_NF, max_rhs=2)
    assert plain["bytes_resident"] - lean["bytes_resident"] >= 2 * C * max(nf ** 3, 2 * S) * rs
