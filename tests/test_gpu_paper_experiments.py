"""Reruns of the paper's matvec experiments (Sec. 6.1, 6.2) on the GPU path.

Setup as in Sec. 6: x ~ U[-1,1]^d, w = 1, sigma(x) = (prod cos(pi x_i) + 2)/6 passed in
the paper's own (w, sigma) parametrisation; sigma_min = 1/6 - 0.01, sigma_max = 1/2 +
0.01; eps_NUFFT = 1e-6 with NUFFTs at eps_NUFFT/10; dw = min{1/8, rho_max^{-1}
log^{-1/2}(1/eps_NUFFT)/4}; for the Matern kernel t_min = (1 + log eps)/nu and
t_max = log(-2 log eps).  The error is the relative 2-norm error of K~ alpha against
the exact K alpha (Eq. nonstat2) on 400 sampled rows (the oracle's direct sum).

Printed values checked: the SE kernel in 1-D with N_sigma = 26, M = 100 reaches
roughly 1e-7, independently of N (Sec. 6.1); in 2-D with N_sigma = 15, M = 75 the
matvec error is never above 1e-5 (Sec. 6.2).  The Matern ablation (Fig. matvec1d,
whose values are lost) is checked for its claim, that each of N_t, N_sigma and M lowers
the error until another parameter limits it, and at its reference point against the
oracle's K~ (exact NUDFT with the same parameters).
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import gpinputs
from oracle import kernel as okern
from oracle import ktilde

pytestmark = pytest.mark.gpu

EPS = 1e-6
SIG_LO, SIG_HI = 1.0 / 6.0 - 0.01, 0.5 + 0.01
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_experiments.json")))


def paper_dw(nu):
    chi_max = 1.0 if nu is None else math.exp(math.log(-2.0 * math.log(EPS)) / 2.0) / math.sqrt(nu)
    return min(1.0 / 8.0, 0.25 / (SIG_HI * chi_max) / math.sqrt(math.log(1.0 / EPS)))


def run(gpn, d, n, nu, n_sigma, M, n_t=None, seed=0, rows=400, vs_ktilde=False):
    """Relative error of the GPU matvec vs exact K on sampled rows; nu=None is the SE kernel.
    With vs_ktilde, also the error vs the oracle's K~ (exact NUDFT, same parameters)."""
    x, w, sig = gpinputs.paper_setup(n, d, seed)
    kw = dict(n_sigma=n_sigma, sigma_lo=SIG_LO, sigma_hi=SIG_HI, M=M, dw=paper_dw(nu), nufft_tol=EPS / 10,
              box_lo=[-1.0] * d, box_hi=[1.0] * d)
    if nu is None:
        plan = gpn.Plan(x, w, sig, nu=1.0, eps=EPS, family=gpn.GP_SE, param_mode=gpn.GP_PARAMS_PAPER, **kw)
    else:
        kw.update(n_t=n_t, t_min=(1.0 + math.log(EPS)) / nu, t_max=math.log(-2.0 * math.log(EPS)))
        plan = gpn.Plan(x, w, sig, nu=nu, eps=EPS, param_mode=gpn.GP_PARAMS_PAPER, **kw)
    alpha = gpinputs.random_alpha(n, 1, seed=seed + 1)
    got = plan.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy()
    plan.close()
    idx = np.random.default_rng(seed + 2).choice(n, size=min(rows, n), replace=False)
    ref = okern.kernel_cross(x[idx], w[idx], sig[idx], x, w, sig, np.inf if nu is None else nu) @ alpha
    e = float(np.linalg.norm(got[idx] - ref) / np.linalg.norm(ref))
    if not vs_ktilde:
        return e
    p = ktilde.Params(d, np.inf if nu is None else nu, kw.get("t_min", 0.0), kw.get("t_max", 0.0), n_t or 0,
                      SIG_LO, SIG_HI, n_sigma, M, kw["dw"])
    rt = ktilde.apply_cross(x[idx], w[idx], sig[idx], x, w, sig, alpha, p)
    return e, float(np.linalg.norm(got[idx] - rt) / np.linalg.norm(rt))


def test_e4_se_1d_reaches_the_printed_accuracy(gpn):
    g = GOLDEN["se_1d"]
    e = run(gpn, 1, 10_000, None, g["n_sigma"], g["M"])
    assert e <= 2 * g["reported_rel_error"], e


def test_e5_se_1d_accuracy_independent_of_n(gpn):
    g = GOLDEN["se_1d"]
    errs = [run(gpn, 1, n, None, g["n_sigma"], g["M"], seed=s) for s, n in enumerate((1_000, 10_000, 100_000))]
    assert max(errs) <= 2 * g["reported_rel_error"], errs
    assert max(errs) <= 5 * min(errs), errs


def test_e6_se_2d_noisy_regime_bound(gpn):
    g = GOLDEN["se_2d_solve"]
    e = run(gpn, 2, 10_000, None, g["n_sigma"], g["M"])
    assert e <= g["reported_max_rel_error"], e


def test_e1_matern_1d_ablation_lowers_the_error(gpn):
    """At the figure's reference point (N_t = 20, N_sigma = 20, M = 400) the GPU matches the
    oracle's K~ to the NUFFT tolerance; its error vs K (measured 5e-5; the printed value
    is lost) comes from the approximation, and each coarser parameter raises it."""
    g = GOLDEN["matern_1d"]
    base = dict(n_t=g["n_t"], n_sigma=g["n_sigma"], M=g["M"])
    ref, impl = run(gpn, 1, 10_000, g["nu"], vs_ktilde=True, **base)
    assert impl <= 1e-6, impl
    # coarser values of each parameter, the others at their reference values
    for key, coarse in (("n_t", 6), ("n_sigma", 4), ("M", 60)):
        e = run(gpn, 1, 10_000, g["nu"], **dict(base, **{key: coarse}))
        assert e > 3 * ref, (key, e, ref)
    assert ref <= 1e-4, ref
