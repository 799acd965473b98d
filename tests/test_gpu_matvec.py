"""Parity of the CUDA matvec (steps (1)-(5) of Sec. 4.2) with the oracle.

Two oracle targets:
  * O-K~: the exact-NUDFT evaluation of K~ alpha with the same hyperparameters
    (passed explicitly to both sides), which isolates the implementation;
  * O-K: the dense kernel of Eq. (nonstat2), which measures the method's accuracy
    with the plan's own parameter choice from eps.
Tolerances (relative l2): FP64 path <= 1e-6 vs either target, FP32 spread path
<= 1e-4; with a tight NUFFT tolerance the FP64 path matches O-K~ to 1e-9.
"""
import numpy as np
import pytest
import torch

import gpinputs
from oracle import kernel as okern
from oracle import ktilde

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    """max |a - b| / max |b|: an error at a few entries (a wrong tile or bin) shows here
    even when it barely moves the l2 norm."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel(a, b):
    """The larger of the relative l2 error and the max-elementwise error relative to
    max |b|, so that every bar a test states holds for both."""
    return max(rel_l2(a, b), rel_max(a, b))


def explicit_params(d, nu, sig, X, n_t=24, n_sigma=8, M=40, pad=1.5, se=False):
    smin, smax = float(sig.min()), float(sig.max())
    L = float(np.max(X.max(0) - X.min(0)))
    if se:
        p = ktilde.Params(d, np.inf, 0.0, 0.0, 0, smin, smax, n_sigma, M, 1.0 / (pad * L))
    else:
        t_min = (1.0 + np.log(1e-6)) / nu
        t_max = np.log(-2.0 * np.log(1e-6))
        p = ktilde.Params(d, nu, t_min, t_max, n_t, smin, smax, n_sigma, M, 1.0 / (pad * L))
    return p


def plan_kwargs(p, se=False):
    kw = dict(n_sigma=p.n_sigma, sigma_lo=p.sigma_min, sigma_hi=p.sigma_max, M=p.M, dw=p.dw)
    if not se:
        kw.update(n_t=p.n_t, t_min=p.t_min, t_max=p.t_max)
    return kw


def small_case(d, n, seed):
    if d == 1:
        w = gpinputs.config_1d(n)
    elif d == 2:
        w = gpinputs.config_2d(n, 1.5)
    else:
        w = gpinputs.config_3d(n)
    return w


CASES = [
    # d, N, nu, n_t, n_sigma, M
    (1, 700, 1.5, 24, 10, 300),
    (1, 600, 1.5, 20, 14, 200),     # 15 channels: the short-spectrum step-3 kernel (transform 1)
    (2, 500, 1.5, 16, 6, 36),
    (3, 300, 2.5, 12, 5, 10),
]


@pytest.mark.parametrize("d,n,nu,n_t,n_sigma,M", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("transform", [1, 2, 3])
def test_matvec_vs_exact_nudft(gpn, d, n, nu, n_t, n_sigma, M, precision, transform):
    """transform 1: full-grid cuFFT R2C/C2R; 2: pruned row transforms (d <= 2);
    3: pruned transposed transforms (d = 2)."""
    if transform == 2 and d == 3:
        pytest.skip("pruned row transforms cover d <= 2")
    if transform == 3 and d != 2:
        pytest.skip("transposed transforms cover d = 2")
    w = small_case(d, n, 0)
    X = w.points
    wp, sig = okern.paper_fields(w.s, w.l, d)
    p = explicit_params(d, nu, sig, X, n_t=n_t, n_sigma=n_sigma, M=M)
    prec = gpn.GP_FP64 if precision == "fp64" else gpn.GP_FP32
    tol = 1e-11 if precision == "fp64" else 1e-6
    plan = gpn.Plan(X, w.s, w.l, nu=nu, eps=1e-6, precision=prec, nufft_tol=tol, transform=transform,
                    **plan_kwargs(p))
    assert plan.info["transform"] == transform
    alpha = gpinputs.random_alpha(n, 1, seed=11)
    ref = ktilde.matvec(X, wp, sig, alpha, p)
    got = plan.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy()
    e = rel(got, ref)
    assert e <= (1e-9 if precision == "fp64" else 1e-4), e


def test_matvec_host_pointers_match_device(gpn):
    w = gpinputs.config_1d(400)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6)
    a = gpinputs.random_alpha(400, 1, seed=3)
    host = plan.matvec(a)                                     # numpy: staged through device memory
    dev = plan.matvec(torch.from_numpy(a).cuda()).cpu().numpy()
    assert rel(host, dev) < 1e-14


@pytest.mark.parametrize("transform", [1, 2, 3])
def test_matvec_multi_rhs_equals_columns(gpn, transform):
    w = gpinputs.config_2d(800, 1.5)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-4, max_rhs=3, transform=transform)
    A = gpinputs.random_alpha(800, 3, seed=4)
    full = plan.matvec(torch.from_numpy(A).cuda()).cpu().numpy()
    for r in range(3):
        col = plan.matvec(torch.from_numpy(A[:, r].copy()).cuda()).cpu().numpy()
        assert rel(full[:, r], col) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("transform", [2, 3])
def test_pruned_transforms_match_full_grid(gpn, precision, transform):
    """The pruned row/column transforms compute the same K~ alpha as the full 2-D cuFFT path,
    on repeated calls with different inputs (zero regions must stay zero)."""
    w = gpinputs.config_2d(3000, 1.5)
    prec = gpn.GP_FP64 if precision == "fp64" else gpn.GP_FP32
    full = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-5, precision=prec, transform=1)
    pruned = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-5, precision=prec, transform=transform,
                      **full.matched_opts())
    for seed in (31, 32, 33):
        a = torch.from_numpy(gpinputs.random_alpha(w.N, 1, seed=seed)).cuda()
        e = rel(pruned.matvec(a).cpu().numpy(), full.matvec(a).cpu().numpy())
        assert e <= (1e-12 if precision == "fp64" else 2e-6), (seed, e)


@pytest.mark.parametrize("nf", [512, 8192])
def test_row_kernels_at_forced_grid_sizes(gpn, nf):
    """FP32 transposed transforms at grid sizes the plans from eps do not pick here:
    nf = 512 against the exact NUDFT, nf = 8192 (the benchmark's row length) against the
    full-grid cuFFT path on the same parameters."""
    w = gpinputs.config_2d(500 if nf == 512 else 3000, 1.5)
    X = w.points
    if nf == 512:
        wp, sig = okern.paper_fields(w.s, w.l, 2)
        p = explicit_params(2, 1.5, sig, X, n_t=16, n_sigma=6, M=36)
        plan = gpn.Plan(X, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP32, nufft_tol=1e-6, transform=3, nf=nf,
                        **plan_kwargs(p))
        assert plan.info["nf"] == nf and plan.info["transform"] == 3
        alpha = gpinputs.random_alpha(w.N, 1, seed=61)
        e = rel(plan.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy(), ktilde.matvec(X, wp, sig, alpha, p))
        assert e <= 1e-4, e
    else:
        full = gpn.Plan(X, w.s, w.l, nu=1.5, eps=1e-5, precision=gpn.GP_FP32, transform=1, nf=nf)
        pruned = gpn.Plan(X, w.s, w.l, nu=1.5, eps=1e-5, precision=gpn.GP_FP32, transform=3, nf=nf,
                          **full.matched_opts())
        assert pruned.info["nf"] == nf
        for seed in (62, 63):
            a = torch.from_numpy(gpinputs.random_alpha(w.N, 1, seed=seed)).cuda()
            e = rel(pruned.matvec(a).cpu().numpy(), full.matvec(a).cpu().numpy())
            assert e <= 2e-6, (seed, e)


def test_shift_adds_eta2_alpha(gpn):
    w = gpinputs.config_1d(300)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6)
    a = gpinputs.random_alpha(300, 1, seed=5)
    base = plan.matvec(a)
    shifted = plan.matvec(a, shift=0.37)
    assert rel(shifted, base + 0.37 * a) < 1e-13


def test_config1_matvec_vs_dense_K(gpn):
    """d=1, N=2000, nu=3/2, eps=1e-6, plan parameters chosen from eps: <= 1e-6 vs K."""
    w = gpinputs.config_1d()
    wp, sig = okern.paper_fields(w.s, w.l, 1)
    K = okern.kernel_dense(w.points, wp, sig, w.nu)
    plan = gpn.Plan(w.points, w.s, w.l, nu=w.nu, eps=w.eps)
    got = plan.matvec(w.alpha)
    e = rel(got, K @ w.alpha)
    assert e <= 1e-6, e
    # FP32 spread path
    p32 = gpn.Plan(w.points, w.s, w.l, nu=w.nu, eps=w.eps, precision=gpn.GP_FP32)
    e32 = rel(p32.matvec(w.alpha), K @ w.alpha)
    assert e32 <= 1e-4, e32


def test_3d_many_channels_spreads_in_chunks(gpn):
    """d=3 with 25 channels and a wide FP64 kernel: no tile holds every channel in
    shared memory, so the spreading runs in channel chunks; parity vs the exact NUDFT."""
    w = gpinputs.config_3d(200)
    X = w.points
    wp, sig = okern.paper_fields(w.s, w.l, 3)
    p = explicit_params(3, 2.5, sig, X, n_t=10, n_sigma=24, M=8)
    plan = gpn.Plan(X, w.s, w.l, nu=2.5, eps=1e-6, precision=gpn.GP_FP64, nufft_tol=1e-11, **plan_kwargs(p))
    C = p.n_sigma + 1
    W = plan.info["kernel_width"]
    assert plan.info["tile"] ** 3 * C * 8 > 160 * 1024, (plan.info["tile"], W)   # a full tile cannot fit
    alpha = gpinputs.random_alpha(200, 1, seed=13)
    ref = ktilde.matvec(X, wp, sig, alpha, p)
    got = plan.matvec(torch.from_numpy(alpha).cuda()).cpu().numpy()
    assert rel(got, ref) <= 1e-9
