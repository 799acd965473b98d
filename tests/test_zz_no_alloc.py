"""gp_posterior_mean_noalloc: the posterior mean (Eq. postmean) through the entry
point whose scratch is a static device array, against gp_posterior_mean on the
same plan.  Collected after the tests of the other entry points so that it runs
after them and, when selected alone, in a fresh process where its first call does
the set-up.

Tolerances (relative l2 against gp_posterior_mean): the two evaluate the same sum
in another order, so FP64 <= 1e-12 and FP32 <= 1e-5.
"""
import numpy as np
import pytest
import torch

import gpinputs

from test_gpu_matvec import rel

pytestmark = pytest.mark.gpu


def _case(gpn, d, precision, nq, seed):
    if d == 1:
        w, fields = gpinputs.config_1d(500), gpinputs.fields_1d
    elif d == 2:
        w, fields = gpinputs.config_2d(3000, 1.5), gpinputs.fields_2d
    else:
        w, fields = gpinputs.config_3d(2000), gpinputs.fields_3d
    plan = gpn.Plan(w.points, w.s, w.l, nu=w.nu, eps=1e-6 if d < 3 else 1e-4, precision=precision)
    info = plan.info
    rng = np.random.default_rng(seed)
    lo = np.array(info["box_lo"][:d])
    hi = np.array(info["box_hi"][:d])
    xq = lo + (hi - lo) * rng.random((nq, d))
    sq, lq = fields(xq)
    lq = np.clip(lq, np.sqrt(2) * info["sigma_lo"], np.sqrt(2) * info["sigma_hi"])
    return w, plan, xq, sq, lq


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_posterior_mean_twice(gpn, d, precision):
    from paper_2407_03608_gb300 import abi
    prec = gpn.GP_FP64 if precision == "fp64" else gpn.GP_FP32
    tol = 1e-12 if precision == "fp64" else 1e-5
    w, plan, xq, sq, lq = _case(gpn, d, prec, 700, seed=20 + d)
    for call, seed in enumerate((41, 42)):
        alpha = gpinputs.random_alpha(w.N, 1, seed=seed)
        ref = plan.posterior_mean(alpha, xq, sq, lq)
        # host pointers on the first call, device pointers on the second
        if call == 0:
            mu = np.full(len(xq), np.nan)
            abi.gp_posterior_mean_noalloc(plan._h, alpha, xq, sq, lq, mu)
        else:
            dev = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (alpha, xq, sq, lq)]
            mu_t = torch.full((len(xq),), float("nan"), dtype=torch.float64, device="cuda")
            abi.gp_posterior_mean_noalloc(plan._h, dev[0], dev[1], dev[2], dev[3], mu_t)
            mu = mu_t.cpu().numpy()
        assert np.all(np.isfinite(mu))
        e = rel(mu, ref)
        assert e <= tol, (call, e)


def test_noalloc_largest_batch_and_size_limit(gpn):
    from paper_2407_03608_gb300 import abi
    nmax = abi.GP_NOALLOC_MAX_QUERIES
    w, plan, xq, sq, lq = _case(gpn, 2, gpn.GP_FP64, nmax, seed=5)
    alpha = gpinputs.random_alpha(w.N, 1, seed=6)
    mu = np.empty(nmax)
    abi.gp_posterior_mean_noalloc(plan._h, alpha, xq, sq, lq, mu)
    ref = plan.posterior_mean(alpha, xq, sq, lq)
    assert rel(mu, ref) <= 1e-12
    big = np.vstack([xq, xq[:1]])
    with pytest.raises(gpn.GPError) as e:
        abi.gp_posterior_mean_noalloc(plan._h, alpha, big, np.append(sq, sq[0]), np.append(lq, lq[0]),
                                      np.empty(nmax + 1))
    assert e.value.status == abi.GP_EINVAL
    assert "static scratch" in str(e.value)


def test_noalloc_flags_queries_outside_the_box(gpn):
    from paper_2407_03608_gb300 import abi
    w, plan, xq, sq, lq = _case(gpn, 1, gpn.GP_FP64, 50, seed=7)
    alpha = gpinputs.random_alpha(w.N, 1, seed=8)
    ref = plan.posterior_mean(alpha, xq, sq, lq)
    bad = xq.copy()
    bad[3, 0] = plan.info["box_hi"][0] + 0.1
    mu = np.zeros(len(xq))
    with pytest.raises(gpn.GPError) as e:
        abi.gp_posterior_mean_noalloc(plan._h, alpha, bad, sq, lq, mu)
    assert e.value.status == abi.GP_EINVAL
    assert np.isnan(mu[3])
    keep = np.arange(len(xq)) != 3
    assert rel(mu[keep], ref[keep]) <= 1e-12
    # the counter is cleared on the next call
    abi.gp_posterior_mean_noalloc(plan._h, alpha, xq, sq, lq, mu)
    assert rel(mu, ref) <= 1e-12


@pytest.mark.parametrize("d", [1, 2, 3])
def test_noalloc_queries_on_the_box_corners(gpn, d):
    # queries exactly on box_lo and box_hi in every axis (all 2^d corners plus the face
    # centres): their supports reach furthest towards the grid edge
    from paper_2407_03608_gb300 import abi
    w, plan, _, _, _ = _case(gpn, d, gpn.GP_FP64, 1, seed=30 + d)
    info = plan.info
    lo = np.array(info["box_lo"][:d])
    hi = np.array(info["box_hi"][:d])
    corners = np.array([[hi[q] if (c >> q) & 1 else lo[q] for q in range(d)] for c in range(2 ** d)])
    faces = []
    for q in range(d):
        for v in (lo[q], hi[q]):
            f = 0.5 * (lo + hi)
            f[q] = v
            faces.append(f)
    xq = np.vstack([corners, np.array(faces)])
    fields = {1: gpinputs.fields_1d, 2: gpinputs.fields_2d, 3: gpinputs.fields_3d}[d]
    sq, lq = fields(xq)
    lq = np.clip(lq, np.sqrt(2) * info["sigma_lo"], np.sqrt(2) * info["sigma_hi"])
    for seed in (51, 52):
        alpha = gpinputs.random_alpha(w.N, 1, seed=seed)
        ref = plan.posterior_mean(alpha, xq, sq, lq)
        mu = np.full(len(xq), np.nan)
        abi.gp_posterior_mean_noalloc(plan._h, alpha, xq, sq, lq, mu)
        assert np.all(np.isfinite(mu))
        assert rel(mu, ref) <= 1e-12
