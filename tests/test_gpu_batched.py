"""Many right-hand sides per CG iteration through a plan that holds grids for only a block
of them (rhs_block): every column of the blocked matvec and of the blocked CG solve equals
the same column computed alone.  The columns share each matvec call and each CG
iteration (Sec. 4.2 steps (1)-(5) run block after block on the stream; the CG
reductions cover all columns at once)."""
import numpy as np
import pytest
import torch

import gpinputs

from test_gpu_matvec import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32", "df64"])
def test_blocked_matvec_columns_equal_single_columns(gpn, precision):
    prec = {"fp64": gpn.GP_FP64, "fp32": gpn.GP_FP32, "df64": gpn.GP_DF64}[precision]
    w = gpinputs.config_2d(2000, 1.5)
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-4, precision=prec, max_rhs=7, rhs_block=3)
    one = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-4, precision=prec, **plan.matched_opts())
    assert plan.info["rhs_block"] == 3 and plan.info["max_rhs"] == 7
    A = gpinputs.random_alpha(w.N, 7, seed=41)
    full = plan.matvec(torch.from_numpy(A).cuda(), shift=0.01).cpu().numpy()
    for r in range(7):
        col = one.matvec(torch.from_numpy(A[:, r].copy()).cuda(), shift=0.01).cpu().numpy()
        assert rel(full[:, r], col) <= 1e-12, r


def test_blocked_cg_columns_equal_single_solves(gpn):
    """8 noisy right-hand sides and 8 +-1 probes (the batched workload's mix, at a small
    size) in one solve, blocks of 4: each column within 1e-8 of its own solve."""
    w = gpinputs.config_2d(3000, 1.5)
    rng = np.random.default_rng(10)
    Y = np.column_stack([w.y + 0.05 * rng.standard_normal(w.N) for _ in range(8)] +
                        [rng.choice([-1.0, 1.0], w.N) for _ in range(8)])
    plan = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-4, precision=gpn.GP_FP64, max_rhs=16, rhs_block=4)
    one = gpn.Plan(w.points, w.s, w.l, nu=1.5, eps=1e-4, precision=gpn.GP_FP64, **plan.matched_opts())
    eta2 = w.eta ** 2
    X, info = plan.solve(torch.from_numpy(Y).cuda(), eta2=eta2, rtol=1e-11, maxit=20000)
    assert info["status"] == 0
    X = X.cpu().numpy()
    for r in range(16):
        x1, i1 = one.solve(Y[:, r].copy(), eta2=eta2, rtol=1e-11, maxit=20000)
        assert i1["status"] == 0
        assert rel(X[:, r], x1) <= 1e-8, r
