"""The library's phase timing (gp_profile_*): the split of each transform phase into the
library's own row kernels and cuFFT's part, for the three transform forms."""
import numpy as np
import pytest
import torch

import gpinputs

pytestmark = pytest.mark.gpu


def _profile(gpn, plan, n, matvecs=4):
    a = torch.from_numpy(gpinputs.random_alpha(n, 1, seed=4)).cuda()
    plan.matvec(a)
    gpn.gp_profile_enable(plan.handle, True)
    for _ in range(matvecs):
        plan.matvec(a)
    phases, count = gpn.gp_profile_read(plan.handle)
    rows = gpn.gp_profile_read_rows(plan.handle)
    gpn.gp_profile_enable(plan.handle, False)
    assert count == matvecs
    assert all(ms > 0 for ms in phases)
    return phases, rows


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_transposed_transforms_split_rows_from_columns(gpn, precision):
    w = gpinputs.config_2d(20_000)
    prec = gpn.GP_FP32 if precision == "fp32" else gpn.GP_FP64
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-4, precision=prec, transform=3)
    assert plan.info["transform"] == 3
    phases, rows = _profile(gpn, plan, 20_000)
    # both halves take time: the rows are ours, the columns cuFFT's
    assert 0 < rows[0] < phases[1] and 0 < rows[1] < phases[3]


def test_row_transforms_without_cufft_take_the_whole_phase(gpn):
    w = gpinputs.config_1d(2000)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-6, precision=gpn.GP_FP64, transform=2)
    assert plan.info["transform"] == 2
    phases, rows = _profile(gpn, plan, 2000)
    assert np.isclose(rows[0], phases[1], rtol=0.05, atol=0.003)
    assert np.isclose(rows[1], phases[3], rtol=0.05, atol=0.003)


def test_cufft_only_transforms_report_no_rows(gpn):
    w = gpinputs.config_3d(20_000)
    plan = gpn.Plan(w.points, w.s, w.l, nu=2.5, eps=1e-3, precision=gpn.GP_FP32)
    assert plan.info["transform"] == 1
    phases, rows = _profile(gpn, plan, 20_000)
    assert rows[0] < 0.05 * phases[1] + 0.003 and rows[1] < 0.05 * phases[3] + 0.003
    # profiling off again: the counters stay where they were
    plan.matvec(torch.zeros(20_000, dtype=torch.float64, device="cuda"))
    assert gpn.gp_profile_read(plan.handle)[1] == 4
