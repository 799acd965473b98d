"""The exact diagonal correction (gp_plan_opts.diag_correct = 1), an extension for small
nu: out_i += (K_ii - K~_ii) alpha_i on top of the paper's K~ alpha.

Parity targets (relative l2, through the C ABI):
  * the oracle's corrected matvec (oracle/diagcorr.py) with the same hyperparameters:
    FP64 <= 1e-9 with a tight NUFFT tolerance, FP32 <= 1e-4;
  * the added term alone: corrected minus uncorrected GPU matvec equals the oracle's
    defect times alpha (FP64 <= 1e-9 of that term);
  * the CG solution of (K~c + eta^2 I) alpha = y against a Cholesky solve of the dense
    corrected matrix, <= 1e-6.
The gain it exists for: with nu = 1/2 the corrected matvec is closer to K alpha.
"""
import numpy as np
import pytest
import torch

import gpinputs
from oracle import diagcorr, kernel as okern, ktilde

from test_gpu_matvec import explicit_params, plan_kwargs, rel, rel_l2, small_case

pytestmark = pytest.mark.gpu

CASES = [
    # d, N, nu, n_t, n_sigma, M
    (1, 700, 0.5, 30, 10, 300),
    (2, 500, 0.5, 24, 6, 36),
    (2, 500, 1.5, 16, 6, 36),
    (3, 300, 2.5, 12, 5, 10),
]


@pytest.mark.parametrize("d,n,nu,n_t,n_sigma,M", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_corrected_matvec_vs_oracle(gpn, d, n, nu, n_t, n_sigma, M, precision):
    w = small_case(d, n, 0)
    X = w.points
    wp, sig = okern.paper_fields(w.s, w.l, d)
    p = explicit_params(d, nu, sig, X, n_t=n_t, n_sigma=n_sigma, M=M)
    prec = gpn.GP_FP64 if precision == "fp64" else gpn.GP_FP32
    tol = 1e-11 if precision == "fp64" else 1e-6
    kw = dict(nu=nu, eps=1e-6, precision=prec, nufft_tol=tol, **plan_kwargs(p))
    plan = gpn.Plan(X, w.s, w.l, diag_correct=1, **kw)
    assert plan.info["diag_correct"] == 1
    alpha = gpinputs.random_alpha(n, 1, seed=19)
    ref = diagcorr.matvec(X, wp, sig, alpha, p)
    got = plan.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy()
    assert rel(got, ref) <= (1e-9 if precision == "fp64" else 1e-4)
    if precision == "fp64":
        plain = gpn.Plan(X, w.s, w.l, **kw)
        assert plain.info["diag_correct"] == 0
        term = diagcorr.defect(wp, sig, p) * alpha
        diff = got - plain.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy()
        assert rel(diff, term) <= 1e-9


def test_corrected_solve_vs_cholesky(gpn):
    w = gpinputs.config_1d(400)
    X = w.points
    wp, sig = okern.paper_fields(w.s, w.l, 1)
    p = explicit_params(1, 0.5, sig, X, n_t=30, n_sigma=10, M=300)
    plan = gpn.Plan(X, w.s, w.l, nu=0.5, eps=1e-6, precision=gpn.GP_FP64, nufft_tol=1e-12, diag_correct=1,
                    **plan_kwargs(p))
    Kc = ktilde.dense(X, wp, sig, p) + np.diag(diagcorr.defect(wp, sig, p))
    eta2 = w.eta ** 2
    ref = okern.solve_cholesky(Kc, eta2, w.y)
    x, info = plan.solve(w.y, eta2=eta2, rtol=1e-12, maxit=20000)
    assert info["status"] == 0
    assert rel(x, ref) <= 1e-6


def test_correction_brings_nu_half_closer_to_k(gpn):
    """2-D, nu = 1/2 on a grid far too coarse for its cusp (plans from eps need 1.6e4
    cells per dimension already at eps = 1e-2): the diagonal defect is a large part of
    the error at this density, and removing it lowers the error against K."""
    w = gpinputs.config_2d(1500, 0.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    K = okern.kernel_dense(w.points, wp, sig, 0.5)
    ref = K @ w.alpha
    p = explicit_params(2, 0.5, sig, w.points, n_t=40, n_sigma=8, M=60)
    kw = dict(nu=0.5, eps=1e-6, precision=gpn.GP_FP64, **plan_kwargs(p))
    plain = gpn.Plan(w.points, w.s, w.l, **kw)
    corr = gpn.Plan(w.points, w.s, w.l, diag_correct=1, **kw)
    e0 = rel_l2(plain.matvec(w.alpha), ref)
    e1 = rel_l2(corr.matvec(w.alpha), ref)
    assert e1 < 0.8 * e0, (e0, e1)


def test_refined_solve_needs_matching_correction(gpn):
    w = gpinputs.config_1d(300)
    lo = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP32, diag_correct=1)
    hi_ok = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP64, **lo.matched_opts())
    assert hi_ok.info["diag_correct"] == 1
    x, info = hi_ok.solve_refined(lo, w.y, eta2=w.eta ** 2, rtol=1e-10)
    assert info["status"] == 0
    opts = lo.matched_opts()
    opts.pop("diag_correct")
    hi_bad = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP64, **opts)
    with pytest.raises(gpn.GPError) as e:
        hi_bad.solve_refined(lo, w.y, eta2=w.eta ** 2, rtol=1e-10)
    assert e.value.status == -1


def test_posterior_mean_is_not_corrected(gpn):
    w = gpinputs.config_1d(300)
    plain = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP64)
    corr = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP64, diag_correct=1,
                    **plain.matched_opts())
    rng = np.random.default_rng(3)
    xq = w.points[rng.choice(300, 40, replace=False)]           # queries at training points too
    sq, lq = gpinputs.fields_1d(xq)
    a = gpinputs.random_alpha(300, 1, seed=21)
    assert rel(corr.posterior_mean(a, xq, sq, lq), plain.posterior_mean(a, xq, sq, lq)) <= 1e-14
