"""The plan-time tile autotuner (gp_plan_opts.autotune): it times matvecs of plans with
the heuristic tile and its neighbours in gp_tile_candidates and keeps the fastest.  The
kept plan computes the same K~ alpha as a plan built with that tile directly (bit for
bit) and as the heuristic's plan (FP32 <= 1e-6: another tile sums in another order)."""
import numpy as np
import pytest
import torch

import gpinputs

from test_gpu_matvec import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d", [2, 3])
def test_autotuned_plan_matches_fixed_tile_plans(gpn, d):
    from paper_2407_03608_gb300 import abi
    w = gpinputs.config_2d(20000, 1.5) if d == 2 else gpinputs.config_3d(20000)
    eps = 1e-5 if d == 2 else 1e-4
    kw = dict(nu=w.nu, eps=eps, precision=gpn.GP_FP32)
    base = gpn.Plan(w.points, w.s, w.l, **kw)
    assert base.info["tuned"] == 0
    tuned = gpn.Plan(w.points, w.s, w.l, autotune=3, **kw)
    i = tuned.info
    cands = abi.gp_tile_candidates(d, i["n_sigma"] + 1, gpn.GP_FP32, i["kernel_width"])
    assert i["tile"] in cands
    assert 1 <= i["tuned"] <= 4 and i["tuned"] == min(4, len(cands))
    assert i["tune_ms"] > 0
    fixed = gpn.Plan(w.points, w.s, w.l, tile=i["tile"], **kw)
    a = torch.from_numpy(gpinputs.random_alpha(w.N, 1, seed=51)).cuda()
    out = tuned.matvec(a).cpu().numpy()
    assert np.array_equal(out, fixed.matvec(a).cpu().numpy())
    assert rel(out, base.matvec(a).cpu().numpy()) <= 1e-6


def test_autotune_is_ignored_with_a_fixed_tile(gpn):
    w = gpinputs.config_2d(5000, 1.5)
    p = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-5, precision=gpn.GP_FP32, tile=16, autotune=4)
    assert p.info["tuned"] == 0 and p.info["tile"] == 16
