"""Parity of the CUDA CG solve and posterior mean with the oracle.

* CG on (K~ + eta^2 I) vs Cholesky of the oracle's dense K~ (same hyperparameters,
  Eq. Ktilde literally): relative error <= 1e-6.
* CG with the plan's own eps vs Cholesky of the dense K (Eq. nonstat2): the
  paper's approximation error amplified by the conditioning; checked <= 1e-5 at
  eps = 1e-9 on the 1-D workload (cond(K + eta^2 I) ~ 5e4).
* Mixed precision (FP32 inner CG, FP64 refinement) vs the FP64 CG solution:
  <= 1e-6.
* Posterior mean (Eq. postmean) at query points vs the oracle's K~ applied at
  those points.
"""
import numpy as np
import pytest
import torch

import gpinputs
from oracle import kernel as okern
from oracle import ktilde

from test_gpu_matvec import explicit_params, plan_kwargs, rel

pytestmark = pytest.mark.gpu


def test_repeated_matvecs_are_independent(gpn):
    """Skipped (empty) spreading tiles must stay zero between calls."""
    w = gpinputs.config_2d(600, 1.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 1.5, sig, w.points, n_t=12, n_sigma=5, M=30)
    for prec, tol in ((gpn.GP_FP64, 1e-9), (gpn.GP_FP32, 1e-4)):
        plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=prec,
                        nufft_tol=1e-11 if prec == gpn.GP_FP64 else 1e-6, **plan_kwargs(p))
        a1 = gpinputs.random_alpha(600, 1, seed=21)
        a2 = gpinputs.random_alpha(600, 1, seed=22)
        plan.matvec(a1)
        got = plan.matvec(a2)
        assert rel(got, ktilde.matvec(w.points, wp, sig, a2, p)) <= tol


def test_cg_matches_cholesky_of_dense_ktilde(gpn):
    w = gpinputs.config_1d(300)
    wp, sig = okern.paper_fields(w.s, w.l, 1)
    p = explicit_params(1, 1.5, sig, w.points, n_t=24, n_sigma=10, M=300)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, nufft_tol=1e-11, **plan_kwargs(p))
    Kt = ktilde.dense(w.points, wp, sig, p)
    ref = okern.solve_cholesky(Kt, w.eta ** 2, w.y)
    x, info = plan.solve(torch.from_numpy(w.y).cuda(), eta2=w.eta ** 2, rtol=1e-12, maxit=5000)
    assert info["status"] == 0
    assert rel(x.cpu().numpy(), ref) <= 1e-6


def test_cg_config1_vs_cholesky_of_K(gpn):
    """d=1, N=2000, nu=3/2, eta=0.1: CG to 1e-10 against dense FP64 Cholesky of K."""
    w = gpinputs.config_1d()
    wp, sig = okern.paper_fields(w.s, w.l, 1)
    K = okern.kernel_dense(w.points, wp, sig, w.nu)
    ref = okern.solve_cholesky(K, w.eta ** 2, w.y)
    plan = gpn.Plan(w.points, w.s, w.l, nu=w.nu, eps=1e-9)
    x, info = plan.solve(w.y, eta2=w.eta ** 2, rtol=1e-10, maxit=5000)
    assert info["status"] == 0
    assert rel(x, ref) <= 1e-5, (rel(x, ref), info)
    # true residual with the oracle's K
    res = (K + w.eta ** 2 * np.eye(w.N)) @ x - w.y
    assert np.linalg.norm(res) / np.linalg.norm(w.y) <= 1e-7


def test_multi_rhs_solve_equals_single(gpn):
    w = gpinputs.config_1d(500)
    Y = gpinputs.random_alpha(500, 3, seed=30)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, max_rhs=3)
    X, info = plan.solve(Y, eta2=0.01, rtol=1e-10)
    for r in range(3):
        xr, _ = plan.solve(Y[:, r].copy(), eta2=0.01, rtol=1e-10)
        assert rel(X[:, r], xr) <= 1e-9


def test_refined_mixed_precision_solve(gpn):
    w = gpinputs.config_1d(2000)
    hi = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP64)
    lo = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP32, **hi.matched_opts())
    y = torch.from_numpy(w.y).cuda()
    x64, i64 = hi.solve(y, eta2=w.eta ** 2, rtol=1e-10)
    xmp, imp = hi.solve_refined(lo, y, eta2=w.eta ** 2, rtol=1e-10, inner_rtol=1e-4)
    assert imp["status"] == 0 and imp["relres"][0] <= 1e-10
    assert rel(xmp.cpu().numpy(), x64.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("d", [1, 2])
def test_posterior_mean_matches_oracle(gpn, d):
    w = gpinputs.config_1d(400) if d == 1 else gpinputs.config_2d(500, 1.5)
    wp, sig = okern.paper_fields(w.s, w.l, d)
    if d == 1:
        p = explicit_params(1, 1.5, sig, w.points, n_t=24, n_sigma=10, M=300)
    else:
        p = explicit_params(2, 1.5, sig, w.points, n_t=12, n_sigma=5, M=30)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, nufft_tol=1e-11, **plan_kwargs(p))
    # queries inside the plan box, with scale fields inside [sigma_lo, sigma_hi]
    rng = np.random.default_rng(9)
    lo = np.array(plan.info["box_lo"][:d])
    hi = np.array(plan.info["box_hi"][:d])
    xq = lo + (hi - lo) * rng.random((200, d))
    fields = gpinputs.fields_1d if d == 1 else gpinputs.fields_2d
    sq, lq = fields(xq)
    lq = np.clip(lq, np.sqrt(2) * p.sigma_min, np.sqrt(2) * p.sigma_max)
    wq, sigq = okern.paper_fields(sq, lq, d)
    alpha = gpinputs.random_alpha(w.N, 1, seed=12)
    mu = plan.posterior_mean(alpha, xq, sq, lq)
    ref = ktilde.apply_cross(xq, wq, sigq, w.points, wp, sig, alpha, p)
    assert rel(mu, ref) <= 1e-9


def test_posterior_mean_rejects_queries_outside_box(gpn):
    w = gpinputs.config_1d(300)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-5)
    xq = np.array([[plan.info["box_hi"][0] + 0.1]])
    with pytest.raises(gpn.GPError) as e:
        plan.posterior_mean(w.alpha, xq, np.ones(1), np.full(1, 0.05))
    assert e.value.status == -1
