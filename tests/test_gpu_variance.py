"""Posterior variance at the training points (gp_posterior_variance) vs the oracle.

The oracle forms the dense K~ of Eq. (Ktilde) with the plan's hyperparameters and
evaluates the same probe estimator eta^2 - eta^4 (sum z x) / (sum z^2) with Cholesky
solves (oracle/variance.py).  Same probes on both sides, so the only difference is
the CG tolerance and rounding: FP64 <= 1e-8 relative l2, FP32 matvec <= 1e-4.
"""
import numpy as np
import pytest
import torch

import gpinputs
from oracle import kernel as okern
from oracle import ktilde
from oracle import variance

from test_gpu_matvec import explicit_params, plan_kwargs, rel, rel_l2

pytestmark = pytest.mark.gpu


def probes(n, R, seed):
    return np.where(np.random.default_rng(seed).random((n, R)) < 0.5, -1.0, 1.0)


@pytest.mark.parametrize("max_rhs", [1, 4])
def test_variance_d1_fp64_matches_oracle_estimator(gpn, max_rhs):
    w = gpinputs.config_1d(300)
    wp, sig = okern.paper_fields(w.s, w.l, 1)
    p = explicit_params(1, 1.5, sig, w.points, n_t=24, n_sigma=10, M=300)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, nufft_tol=1e-11, max_rhs=max_rhs, **plan_kwargs(p))
    eta2 = w.eta ** 2
    Z = probes(300, 10, seed=21)
    Kt = ktilde.dense(w.points, wp, sig, p)
    ref = variance.variance_probes(Kt, eta2, Z)
    var, info = plan.posterior_variance(Z, eta2, rtol=1e-13, maxit=20000)
    assert info["status"] == 0
    assert len(info["iters"]) == 10
    assert rel(var, ref) <= 1e-8, rel(var, ref)
    # a posterior variance: between 0 and the prior variance s^2, here with a margin for the
    # probe estimator's own scatter
    assert np.all(var > -0.5 * eta2)


def test_variance_d2_fp32_device_probes(gpn):
    w = gpinputs.config_2d(500, 1.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 1.5, sig, w.points, n_t=16, n_sigma=6, M=36)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP32, max_rhs=3, **plan_kwargs(p))
    eta2 = w.eta ** 2
    Z = probes(500, 7, seed=22)
    ref = variance.variance_probes(ktilde.dense(w.points, wp, sig, p), eta2, Z)
    var, info = plan.posterior_variance(torch.from_numpy(Z).cuda(), eta2, rtol=1e-10, maxit=20000)
    assert rel(var.cpu().numpy(), ref) <= 1e-4


def test_variance_many_probes_in_chunks(gpn):
    """512 probes solved 64 at a time: equal to the oracle's estimator with the same
    probes, and within the estimator's own scatter of the exact diagonal (the oracle's
    estimate with these probes is 5.5 % from it; the bound is 10 %)."""
    w = gpinputs.config_1d(200)
    wp, sig = okern.paper_fields(w.s, w.l, 1)
    p = explicit_params(1, 1.5, sig, w.points, n_t=24, n_sigma=10, M=300)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, nufft_tol=1e-11, max_rhs=64, **plan_kwargs(p))
    eta2 = 0.1
    Z = probes(200, 512, seed=23)
    Kt = ktilde.dense(w.points, wp, sig, p)
    ref = variance.variance_probes(Kt, eta2, Z)
    var, info = plan.posterior_variance(Z, eta2, rtol=1e-13, maxit=20000)
    assert rel(var, ref) <= 1e-8, rel(var, ref)
    # the estimator's scatter is per entry, so this bound is on the l2 norm only
    assert rel_l2(var, variance.variance_exact(Kt, eta2)) <= 0.10
