"""The memory-lean step 3 (gp_plan_opts.step3 = 2): a_k = sum_j v~_j G^_kj sum_l G^_lj b_l
formed per frequency from the separable per-dimension factors of G^ instead of the
stored tensor A[n] of Remark rem:step3.

Parity targets:
  * the oracle's exact-NUDFT K~ alpha with the same hyperparameters (FP64 <= 1e-9 with a
    tight NUFFT tolerance, FP32 <= 1e-4), for every spectrum layout: full-grid half
    spectra (d = 1, 2, 3) and the transposed pruned transforms (d = 2), with channel
    counts on the exact-C and on the runtime-C kernel variants;
  * the tensor path on the same plan parameters: the two evaluate the same sums in
    another order (FP64 <= 1e-12, FP32 <= 2e-6 relative l2), on repeated calls with new
    inputs (the spectrum outside the mode box must be zero on every call) and with
    several right-hand sides.
"""
import numpy as np
import pytest
import torch

import gpinputs
from oracle import kernel as okern
from oracle import ktilde

from test_gpu_matvec import explicit_params, plan_kwargs, rel, small_case

pytestmark = pytest.mark.gpu

CASES = [
    # d, N, nu, n_t, n_sigma, M, transform
    (1, 700, 1.5, 24, 10, 300, 1),
    (2, 500, 1.5, 16, 6, 36, 1),
    (2, 500, 1.5, 16, 6, 36, 3),
    (2, 400, 1.5, 10, 19, 24, 3),    # C = 20: runtime-C variant of the transposed kernel
    (2, 400, 1.5, 10, 19, 24, 1),    # C = 20: widest channel bucket of the full-grid kernel
    (3, 300, 2.5, 12, 5, 10, 1),
]


@pytest.mark.parametrize("d,n,nu,n_t,n_sigma,M,transform", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lean_matvec_vs_exact_nudft(gpn, d, n, nu, n_t, n_sigma, M, transform, precision):
    w = small_case(d, n, 0)
    X = w.points
    wp, sig = okern.paper_fields(w.s, w.l, d)
    p = explicit_params(d, nu, sig, X, n_t=n_t, n_sigma=n_sigma, M=M)
    prec = gpn.GP_FP64 if precision == "fp64" else gpn.GP_FP32
    tol = 1e-11 if precision == "fp64" else 1e-6
    plan = gpn.Plan(X, w.s, w.l, nu=nu, eps=1e-6, precision=prec, nufft_tol=tol, transform=transform, step3=2,
                    **plan_kwargs(p))
    assert plan.info["step3"] == 2
    assert plan.info["transform"] == transform
    alpha = gpinputs.random_alpha(n, 1, seed=17)
    ref = ktilde.matvec(X, wp, sig, alpha, p)
    got = plan.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy()
    e = rel(got, ref)
    assert e <= (1e-9 if precision == "fp64" else 1e-4), e


@pytest.mark.parametrize("d,transform", [(2, 3), (2, 1), (3, 1), (1, 1)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lean_matches_tensor_path(gpn, d, transform, precision):
    n = {1: 1500, 2: 3000, 3: 2000}[d]
    w = small_case(d, n, 0)
    prec = gpn.GP_FP64 if precision == "fp64" else gpn.GP_FP32
    eps = 1e-5 if d < 3 else 1e-4
    R = 3
    tensor = gpn.Plan(w.points, w.s, w.l, nu=w.nu, eps=eps, precision=prec, transform=transform, step3=1, max_rhs=R)
    lean = gpn.Plan(w.points, w.s, w.l, nu=w.nu, eps=eps, precision=prec, transform=transform, step3=2, max_rhs=R,
                    **tensor.matched_opts())
    assert tensor.info["step3"] == 1 and lean.info["step3"] == 2
    if d >= 2:   # in 1-D the tensor has C(C+1)/2 (M+1) entries, fewer than the factors
        assert lean.info["bytes_resident"] < tensor.info["bytes_resident"]
    tol = 1e-12 if precision == "fp64" else 2e-6
    for seed in (41, 42):
        a = torch.from_numpy(gpinputs.random_alpha(w.N, 1, seed=seed)).cuda()
        e = rel(lean.matvec(a).cpu().numpy(), tensor.matvec(a).cpu().numpy())
        assert e <= tol, (seed, e)
    A = torch.from_numpy(gpinputs.random_alpha(w.N, R, seed=43)).cuda()
    e = rel(lean.matvec(A).cpu().numpy(), tensor.matvec(A).cpu().numpy())
    assert e <= tol, e


def test_lean_auto_choice_under_max_bytes(gpn):
    """step3 = 0 keeps the tensor when it fits max_bytes and falls back to the lean form
    when only the lean plan fits."""
    w = gpinputs.config_2d(3000, 1.5)
    kw = dict(nu=1.5, eps=1e-5, precision=gpn.GP_FP32)
    tensor = gpn.Plan(w.points, w.s, w.l, step3=1, **kw)
    lean = gpn.Plan(w.points, w.s, w.l, step3=2, **kw)
    b1, b2 = tensor.info["bytes_resident"], lean.info["bytes_resident"]
    assert b2 < b1
    roomy = gpn.Plan(w.points, w.s, w.l, step3=0, max_bytes=int(b1 * 1.02) + (1 << 20), **kw)
    assert roomy.info["step3"] == 1
    tight = gpn.Plan(w.points, w.s, w.l, step3=0, max_bytes=int(b2 * 1.02) + (1 << 20), **kw)
    assert tight.info["step3"] == 2
    assert tight.info["bytes_resident"] == b2
    a = torch.from_numpy(gpinputs.random_alpha(w.N, 1, seed=44)).cuda()
    assert rel(tight.matvec(a).cpu().numpy(), tensor.matvec(a).cpu().numpy()) <= 2e-6


def test_lean_rejected_with_pruned_row_transforms(gpn):
    w = gpinputs.config_1d(300)
    with pytest.raises(gpn.GPError) as e:
        gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, transform=2, step3=2)
    assert e.value.status == -8


def test_lean_cg_solve_matches_tensor_solve(gpn):
    w = gpinputs.config_2d(2000, 1.5)
    kw = dict(nu=1.5, eps=1e-5, precision=gpn.GP_FP64)
    tensor = gpn.Plan(w.points, w.s, w.l, step3=1, **kw)
    lean = gpn.Plan(w.points, w.s, w.l, step3=2, **tensor.matched_opts(), **kw)
    y = torch.from_numpy(np.ascontiguousarray(w.y)).cuda()
    x1, i1 = tensor.solve(y, eta2=w.eta ** 2, rtol=1e-10)
    x2, i2 = lean.solve(y, eta2=w.eta ** 2, rtol=1e-10)
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-8
