"""GB300 (sm_103a) NUFFT-based matvec and CG solve for non-stationary Matern GPs.

Implements the hot path of Kielstra & Lindsey (arXiv 2407.03608): the matvec with
the approximate kernel K~ (Eq. Ktilde) by the five steps of Sec. 4.2, conjugate
gradients for (K + eta^2 I) alpha = y (Eq. gprsolve) and the posterior mean
(Eq. postmean).  The compute lives in ``libgpnufft.so`` (CUDA, C ABI in
``include/gpnufft.h``); this package only marshals arguments.

    import paper_2407_03608_gb300 as gpn
    plan = gpn.Plan(points, s, l, nu=1.5, eps=1e-6)      # (N, d) points, vertical/length scales
    out = plan.matvec(alpha)                             # (K~ + shift I) alpha
    alpha, info = plan.solve(y, eta2=0.01, rtol=1e-8)
"""
from __future__ import annotations

import numpy as np

from . import abi
from .abi import (GP_DF64, GP_FP32, GP_FP64, GP_MATERN, GP_PARAMS_PAPER, GP_PARAMS_SCALES, GP_SE, GPError,  # noqa: F401
                  gp_cg_solve, gp_cg_solve_refined, gp_destroy, gp_matvec, gp_plan, gp_profile_enable, gp_profile_read,
                  gp_profile_read_rows,
                  gp_plan_info_get, gp_posterior_mean, gp_posterior_variance, gp_version)

__all__ = ["Plan", "GPError", "gp_plan", "gp_matvec", "gp_cg_solve", "gp_cg_solve_refined", "gp_posterior_mean",
           "gp_posterior_variance",
           "gp_profile_enable", "gp_profile_read", "gp_profile_read_rows",
           "gp_plan_info_get", "gp_destroy", "gp_version", "GP_FP32", "GP_FP64", "GP_DF64", "GP_MATERN", "GP_SE",
           "GP_PARAMS_SCALES", "GP_PARAMS_PAPER"]


def _torch():
    import torch
    return torch


def _like(x, shape):
    """A float64 output of the given shape on the same side (device/host) as x."""
    try:
        torch = _torch()
        if isinstance(x, torch.Tensor):
            return torch.empty(shape, dtype=torch.float64, device=x.device)
    except ImportError:  # pragma: no cover
        pass
    return np.empty(shape, dtype=np.float64)


def _as_cols(a):
    """(flat column-major buffer, R, was_1d) for an (N,) or (N, R) input."""
    try:
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.dim() == 1:
                return a.contiguous().to(torch.float64), 1, True
            return a.t().contiguous().to(torch.float64), a.shape[1], False  # (R, N) row-major = col-major
    except ImportError:  # pragma: no cover
        pass
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return np.ascontiguousarray(a), 1, True
    return np.ascontiguousarray(a.T), a.shape[1], False


def _from_cols(buf, R, was_1d):
    if was_1d:
        return buf
    return buf.t() if hasattr(buf, "t") and not isinstance(buf, np.ndarray) else buf.T


class Plan:
    """Plan for K~ on fixed points and scale fields (owns device memory)."""

    def __init__(self, points, field_a, field_b, nu: float = 1.5, eps: float = 1e-6, *, precision=GP_FP64,
                 family=GP_MATERN, param_mode=GP_PARAMS_SCALES, max_rhs: int = 1, stream=None, **overrides):
        opts = abi.default_opts(precision=precision, family=family, param_mode=param_mode, max_rhs=max_rhs)
        setbits = 0
        keymap = {"n_t": abi.GP_SET_NT, "t_min": abi.GP_SET_NT, "t_max": abi.GP_SET_NT,
                  "n_sigma": abi.GP_SET_NSIGMA, "sigma_lo": abi.GP_SET_SIGMA_RANGE, "sigma_hi": abi.GP_SET_SIGMA_RANGE,
                  "M": abi.GP_SET_M, "dw": abi.GP_SET_DW, "nufft_tol": abi.GP_SET_NUFFT,
                  "upsampfac": abi.GP_SET_NUFFT, "box_lo": abi.GP_SET_BOX, "box_hi": abi.GP_SET_BOX,
                  "nf": abi.GP_SET_NF, "tile": abi.GP_SET_TILE, "max_bytes": 0, "transform": 0, "step3": 0, "diag_correct": 0,
                  "autotune": 0, "rhs_block": 0, "near_radius": 0}
        for k, v in overrides.items():
            if k not in keymap:
                raise TypeError("unknown plan option %r" % k)
            setbits |= keymap[k]
            if k in ("box_lo", "box_hi"):
                arr = getattr(opts, k)
                for i, x in enumerate(v):
                    arr[i] = float(x)
            else:
                setattr(opts, k, v)
        opts.set = setbits
        pts = points
        if hasattr(pts, "ndim") and pts.ndim == 1:
            pts = pts.reshape(-1, 1)
        self._h = gp_plan(pts, field_a, field_b, nu, eps, opts, stream)
        self.info = gp_plan_info_get(self._h)
        self.N = self.info["N"]
        self.d = self.info["d"]
        self.max_rhs = max_rhs

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            gp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def matvec(self, alpha, shift: float = 0.0, out=None, stream=None):
        buf, R, one = _as_cols(alpha)
        res = out if out is not None else _like(buf, tuple(buf.shape))
        gp_matvec(self._h, buf, res, R, shift, stream)
        return _from_cols(res, R, one)

    def solve(self, y, eta2: float, rtol: float = 1e-8, maxit: int = 10000, stream=None):
        buf, R, one = _as_cols(y)
        res = _like(buf, tuple(buf.shape))
        st, iters, rel = gp_cg_solve(self._h, buf, res, R, eta2, rtol, maxit, stream)
        return _from_cols(res, R, one), {"status": st, "iters": iters, "relres": rel}

    def solve_refined(self, lo: "Plan", y, eta2: float, rtol: float = 1e-8, inner_rtol: float = 1e-4,
                      outer_max: int = 10, maxit: int = 10000, stream=None):
        """Mixed precision: inner CG on plan ``lo`` (FP32), residuals on this plan (FP64)."""
        buf, R, one = _as_cols(y)
        res = _like(buf, tuple(buf.shape))
        st, iters, rel = gp_cg_solve_refined(lo._h, self._h, buf, res, R, eta2, rtol, inner_rtol, outer_max,
                                             maxit, stream)
        return _from_cols(res, R, one), {"status": st, "iters": iters, "relres": rel}

    def posterior_mean(self, alpha, xq, field_aq, field_bq, stream=None):
        if hasattr(xq, "ndim") and xq.ndim == 1:
            xq = xq.reshape(-1, 1)
        mu = _like(alpha, (xq.shape[0],))
        gp_posterior_mean(self._h, alpha, xq, field_aq, field_bq, mu, stream)
        return mu

    def posterior_variance(self, probes, eta2: float, rtol: float = 1e-8, maxit: int = 10000, stream=None):
        """Posterior variance at the training points from (N, R) probe vectors (entries +-1):
        eta2 - eta2^2 diag((K~ + eta2 I)^{-1}), the diagonal estimated from the probes."""
        buf, R, one = _as_cols(probes)
        var = _like(buf, (int(self.info["N"]),))
        st, iters = gp_posterior_variance(self._h, buf, R, eta2, rtol, maxit, var, stream)
        return var, {"status": st, "iters": iters}

    def matched_opts(self):
        """Overrides that rebuild exactly this plan's K~ (for a second precision)."""
        i = self.info
        o = {"n_sigma": i["n_sigma"], "sigma_lo": i["sigma_lo"], "sigma_hi": i["sigma_hi"], "M": i["M"],
             "dw": i["dw"], "box_lo": i["box_lo"], "box_hi": i["box_hi"]}
        if i["family"] == GP_MATERN:
            o.update(n_t=i["n_t"], t_min=i["t_min"], t_max=i["t_max"])
        if i["diag_correct"]:
            o["diag_correct"] = 1
        if i["near_radius"] > 0:
            o["near_radius"] = i["near_radius"]
        return o
