"""Parity of the float-float plans (GP_DF64) with the oracle and with the float64 plans.

GP_DF64 runs spreading, the transposed pruned transforms (the library's own row and
column kernels), step 3 and interpolation in float-float arithmetic (two float32 words
a value, about 48 significant bits) on the FP32 pipe.  It is held to the float64 bars:
  * matvec vs the oracle's K~ (exact NUDFT sums, Eq. Ktilde with the same explicit
    hyperparameters), NUFFT tolerance 1e-11: <= 1e-9;
  * matvec vs a GP_FP64 plan on the same parameters: <= 1e-11 (both are float64-grade;
    what differs is rounding and the ES kernel evaluated to the same double);
  * CG vs Cholesky of the dense K~ <= 1e-6; the refined solve (FP32 inner CG, GP_DF64
    residuals) vs GP_FP64 CG <= 1e-6; posterior mean vs the oracle's apply_cross <= 1e-9.
Each bar holds for the relative l2 error and the largest error relative to the largest
entry (``rel``).  Configurations the float-float kernels do not cover are refused with
GP_EUNSUPPORTED.
"""
import numpy as np
import pytest
import torch

import gpinputs
from oracle import kernel as okern
from oracle import ktilde

from test_gpu_matvec import explicit_params, plan_kwargs, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,n_t,n_sigma,M,tile", [(500, 16, 6, 36, None), (900, 20, 8, 60, None),
                                                  (700, 12, 4, 120, 16)])
def test_df64_matvec_vs_exact_nudft(gpn, n, n_t, n_sigma, M, tile):
    """Several grid sizes (nf 128 to 512: column kernels of 2^7 to 2^9 points), tiles and
    ragged last tiles."""
    w = gpinputs.config_2d(n, 1.5)
    X = w.points
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 1.5, sig, X, n_t=n_t, n_sigma=n_sigma, M=M)
    kw = dict(tile=tile) if tile else {}
    plan = gpn.Plan(X, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_DF64, nufft_tol=1e-11, **kw,
                    **plan_kwargs(p))
    assert plan.info["precision"] == gpn.GP_DF64 and plan.info["transform"] == 3
    for seed in (11, 12):
        alpha = gpinputs.random_alpha(n, 1, seed=seed)
        ref = ktilde.matvec(X, wp, sig, alpha, p)
        got = plan.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy()
        e = rel(got, ref)
        assert e <= 1e-9, (seed, e)


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_df64_matches_fp64_plan(gpn, eps):
    """The plan's own parameters from eps (at 1e-6 the benchmark's grid, nf = 8192, and its
    2^13-point column kernel); the same parameters on a GP_FP64 plan."""
    w = gpinputs.config_2d(20_000, 1.5)
    dd_plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=eps, precision=gpn.GP_DF64, max_rhs=2)
    f64 = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=eps, precision=gpn.GP_FP64, max_rhs=2,
                   **dd_plan.matched_opts())
    assert dd_plan.info["nf"] == f64.info["nf"] and dd_plan.info["M"] == f64.info["M"]
    A = gpinputs.random_alpha(w.N, 2, seed=13)
    got = dd_plan.matvec(torch.from_numpy(A).cuda()).cpu().numpy()
    ref = f64.matvec(torch.from_numpy(A).cuda()).cpu().numpy()
    for r in range(2):
        assert rel(got[:, r], ref[:, r]) <= 1e-11, r
        # multi-RHS = columns
        col = dd_plan.matvec(torch.from_numpy(A[:, r].copy()).cuda()).cpu().numpy()
        assert rel(got[:, r], col) <= 1e-13


def test_df64_shift_and_repeated_calls(gpn):
    w = gpinputs.config_2d(600, 1.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 1.5, sig, w.points, n_t=12, n_sigma=5, M=30)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_DF64, nufft_tol=1e-11,
                    **plan_kwargs(p))
    a1 = gpinputs.random_alpha(600, 1, seed=21)
    a2 = gpinputs.random_alpha(600, 1, seed=22)
    plan.matvec(a1)
    got = plan.matvec(a2, shift=0.37)
    assert rel(got, ktilde.matvec(w.points, wp, sig, a2, p) + 0.37 * a2) <= 1e-9


def test_df64_cg_matches_cholesky_of_dense_ktilde(gpn):
    w = gpinputs.config_2d(400, 1.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 1.5, sig, w.points, n_t=16, n_sigma=6, M=36)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_DF64, nufft_tol=1e-11,
                    **plan_kwargs(p))
    Kt = ktilde.dense(w.points, wp, sig, p)
    ref = okern.solve_cholesky(Kt, w.eta ** 2, w.y)
    x, info = plan.solve(torch.from_numpy(w.y).cuda(), eta2=w.eta ** 2, rtol=1e-12, maxit=20000)
    assert info["status"] == 0
    assert rel(x.cpu().numpy(), ref) <= 1e-6


def test_df64_refined_solve_matches_fp64_cg(gpn):
    """FP32 inner CG with float-float residuals reaches the GP_FP64 CG solution."""
    w = gpinputs.config_2d(3000, 1.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 1.5, sig, w.points, n_t=16, n_sigma=6, M=60)
    lo = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP32, **plan_kwargs(p))
    hi = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_DF64, **lo.matched_opts())
    f64 = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP64, **lo.matched_opts())
    eta2 = w.eta ** 2
    x64, info64 = f64.solve(w.y, eta2=eta2, rtol=1e-10, maxit=50000)
    assert info64["status"] == 0
    xr, info = hi.solve_refined(lo, w.y, eta2=eta2, rtol=1e-10)
    assert info["status"] == 0
    assert rel(xr, x64) <= 1e-6


def test_df64_posterior_mean(gpn):
    w = gpinputs.config_2d(400, 1.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 1.5, sig, w.points, n_t=16, n_sigma=6, M=36)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_DF64, nufft_tol=1e-11,
                    **plan_kwargs(p))
    info = plan.info
    rng = np.random.default_rng(9)
    lo, hi = np.array(info["box_lo"][:2]), np.array(info["box_hi"][:2])
    xq = lo + (hi - lo) * rng.random((150, 2))
    sq, lq = gpinputs.fields_2d(xq)
    lq = np.clip(lq, np.sqrt(2) * info["sigma_lo"], np.sqrt(2) * info["sigma_hi"])
    wq, sgq = okern.paper_fields(sq, lq, 2)
    a = gpinputs.random_alpha(400, 1, seed=31)
    ref = ktilde.apply_cross(xq, wq, sgq, w.points, wp, sig, a, p)
    assert rel(plan.posterior_mean(a, xq, sq, lq), ref) <= 1e-9


@pytest.mark.parametrize("kw", [dict(d=1), dict(d=3), dict(step3=2), dict(transform=1)])
def test_df64_refuses_what_it_does_not_cover(gpn, kw):
    kw = dict(kw)
    d = kw.pop("d", 2)
    w = {1: gpinputs.config_1d(300), 2: gpinputs.config_2d(300, 1.5), 3: gpinputs.config_3d(300)}[d]
    with pytest.raises(gpn.GPError) as e:
        gpn.Plan(w.points, w.s, w.l, nu=w.nu, eps=1e-4, precision=gpn.GP_DF64, **kw)
    assert e.value.status == gpn.abi.GP_EUNSUPPORTED
