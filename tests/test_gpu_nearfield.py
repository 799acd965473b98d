"""The near-field correction (gp_plan_opts.near_radius, an extension for small nu) against
the oracle (oracle/nearfield.py) and against K.

  * parity: with explicit hyperparameters, the GPU matvec with the pairs closer than the
    radius corrected equals the oracle's K~ + sum (K_ij - K~_ij) e_i e_j^T (exact NUDFTs
    plus the separable pair form) within the float64 bar 1e-9 (FP32: 1e-4), with and without
    the diagonal correction; CG on it matches Cholesky of the oracle's dense matrix (1e-6);
  * accuracy: on the 2-D workload's recipe at nu = 1/2 and N = 2e4, with a grid too small
    for the spectrum (M = 40), the error against 512 exact rows of K alpha falls from K~ to
    the diagonal correction and to below half of that with the near field (r_c = 0.04);
  * refusal: a smoothness without a closed form.
Each bar holds for the relative l2 error and the largest error (``rel``).
"""
import numpy as np
import pytest
import torch

import gpinputs
from oracle import kernel as okern
from oracle import nearfield
from oracle import rows as orows

from test_gpu_matvec import explicit_params, plan_kwargs, rel, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("diag", [0, 1])
def test_near_field_matvec_vs_oracle(gpn, precision, diag):
    w = gpinputs.config_2d(400, 0.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 0.5, sig, w.points, n_t=20, n_sigma=5, M=40)
    prec = gpn.GP_FP64 if precision == "fp64" else gpn.GP_FP32
    tol = 1e-11 if precision == "fp64" else 1e-6
    plan = gpn.Plan(w.points, w.s, w.l, nu=0.5, eps=1e-6, precision=prec, nufft_tol=tol, near_radius=0.06,
                    diag_correct=diag, **plan_kwargs(p))
    assert plan.info["near_pairs"] == len(nearfield.pairs_within(w.points, 0.06)[0]) > 0
    for seed in (3, 4):
        a = gpinputs.random_alpha(w.N, 1, seed=seed)
        ref = nearfield.matvec(w.points, wp, sig, 0.5, a, p, 0.06, diag=bool(diag))
        got = plan.matvec(torch.from_numpy(a).cuda()).cpu().numpy()
        assert rel(got, ref) <= (1e-9 if precision == "fp64" else 1e-4), (seed, rel(got, ref))


def test_near_field_cg_vs_cholesky(gpn):
    w = gpinputs.config_2d(300, 0.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 0.5, sig, w.points, n_t=20, n_sigma=5, M=40)
    plan = gpn.Plan(w.points, w.s, w.l, nu=0.5, eps=1e-6, nufft_tol=1e-11, near_radius=0.06, diag_correct=1,
                    **plan_kwargs(p))
    Kc = nearfield.dense(w.points, wp, sig, 0.5, p, 0.06, diag=True)
    ref = okern.solve_cholesky(Kc, w.eta ** 2, w.y)
    x, info = plan.solve(w.y, eta2=w.eta ** 2, rtol=1e-12, maxit=20000)
    assert info["status"] == 0
    assert rel(x, ref) <= 1e-6


def test_near_field_brings_nu_half_closer_to_k(gpn):
    # a grid short of nu = 1/2's slowly decaying spectrum (M = 40): the defect K - K~ sits
    # on and near the diagonal, where the two corrections take it out
    w = gpinputs.config_2d(20_000, 0.5)
    wp, sig = okern.paper_fields(w.s, w.l, 2)
    p = explicit_params(2, 0.5, sig, w.points, n_t=30, n_sigma=6, M=40)
    idx = np.random.default_rng(5).choice(w.N, size=512, replace=False)
    ref = orows.rows(w.points, wp, sig, 0.5, w.alpha, idx)
    errs = {}
    for name, kw in (("plain", {}), ("diag", {"diag_correct": 1}), ("near", {"diag_correct": 1, "near_radius": 0.04})):
        plan = gpn.Plan(w.points, w.s, w.l, nu=0.5, eps=1e-6, precision=gpn.GP_FP64, nufft_tol=1e-10,
                        **plan_kwargs(p), **kw)
        got = plan.matvec(torch.from_numpy(w.alpha).cuda()).cpu().numpy()
        errs[name] = rel_l2(got[idx], ref)
        plan.close()
    assert errs["near"] < 0.5 * errs["diag"] and errs["diag"] < errs["plain"], errs


def test_near_field_needs_a_closed_form(gpn):
    w = gpinputs.config_2d(200, 1.5)
    with pytest.raises(gpn.GPError) as e:
        gpn.Plan(w.points, w.s, w.l, nu=1.3, eps=1e-3, near_radius=0.05)
    assert e.value.status == gpn.abi.GP_EUNSUPPORTED
