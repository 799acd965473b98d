"""ctypes binding of include/gpnufft.h (argument marshalling only).

Every function here forwards to the C ABI of ``libgpnufft.so``; all arithmetic
runs in the library's CUDA kernels.  The library is loaded from the package's
``_build`` directory and there is no fallback: if it cannot be loaded, importing
this module raises.

Arrays may be float64 CUDA torch tensors (used in place, stream ordered on the
current torch stream) or float64 NumPy arrays / CPU tensors (the library stages
them through device memory and synchronises before returning).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgpnufft.so")

GP_OK, GP_EINVAL, GP_ENOMEM, GP_ECUDA, GP_ECUFFT, GP_ENOTCONV, GP_EBREAKDOWN, GP_ETIMEOUT, GP_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
GP_FP64, GP_FP32, GP_DF64 = 0, 1, 2
GP_NOALLOC_MAX_QUERIES = 32768
GP_MATERN, GP_SE = 0, 1
GP_PARAMS_SCALES, GP_PARAMS_PAPER = 0, 1
GP_SET_NT, GP_SET_NSIGMA, GP_SET_SIGMA_RANGE, GP_SET_M, GP_SET_DW, GP_SET_NUFFT, GP_SET_BOX, GP_SET_NF, GP_SET_TILE = \
    (1 << i for i in range(9))

STATUS_NAMES = {0: "GP_OK", -1: "GP_EINVAL", -2: "GP_ENOMEM", -3: "GP_ECUDA", -4: "GP_ECUFFT", -5: "GP_ENOTCONV",
                -6: "GP_EBREAKDOWN", -7: "GP_ETIMEOUT", -8: "GP_EUNSUPPORTED"}

#: every symbol include/gpnufft.h declares
EXPORTED = ["gp_plan_opts_default", "gp_plan", "gp_matvec", "gp_cg_solve", "gp_cg_solve_refined",
            "gp_posterior_mean", "gp_posterior_mean_noalloc", "gp_posterior_variance", "gp_profile_enable",
            "gp_profile_read", "gp_profile_read_rows", "gp_plan_info_get", "gp_destroy", "gp_last_error",
            "gp_version", "gp_tile_candidates", "gp_plan_params"]


class gp_plan_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("family", ctypes.c_int), ("param_mode", ctypes.c_int),
                ("set", ctypes.c_uint),
                ("n_t", ctypes.c_int), ("t_min", ctypes.c_double), ("t_max", ctypes.c_double),
                ("n_sigma", ctypes.c_int), ("sigma_lo", ctypes.c_double), ("sigma_hi", ctypes.c_double),
                ("M", ctypes.c_longlong), ("dw", ctypes.c_double),
                ("nufft_tol", ctypes.c_double), ("upsampfac", ctypes.c_double),
                ("box_lo", ctypes.c_double * 3), ("box_hi", ctypes.c_double * 3),
                ("nf", ctypes.c_longlong), ("tile", ctypes.c_int), ("transform", ctypes.c_int),
                ("max_rhs", ctypes.c_int), ("max_bytes", ctypes.c_longlong), ("step3", ctypes.c_int),
                ("diag_correct", ctypes.c_int), ("autotune", ctypes.c_int), ("rhs_block", ctypes.c_int),
                ("near_radius", ctypes.c_double)]


class gp_plan_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("N", ctypes.c_longlong), ("family", ctypes.c_int), ("precision", ctypes.c_int),
                ("nu", ctypes.c_double), ("eps", ctypes.c_double),
                ("n_t", ctypes.c_int), ("t_min", ctypes.c_double), ("t_max", ctypes.c_double),
                ("n_sigma", ctypes.c_int), ("sigma_lo", ctypes.c_double), ("sigma_hi", ctypes.c_double),
                ("M", ctypes.c_longlong), ("dw", ctypes.c_double), ("nf", ctypes.c_longlong),
                ("kernel_width", ctypes.c_int), ("kernel_beta", ctypes.c_double),
                ("upsampfac", ctypes.c_double), ("nufft_tol", ctypes.c_double), ("tile", ctypes.c_int),
                ("transform", ctypes.c_int),
                ("box_lo", ctypes.c_double * 3), ("box_hi", ctypes.c_double * 3),
                ("est_err_t", ctypes.c_double), ("est_err_sigma", ctypes.c_double),
                ("est_err_trunc", ctypes.c_double), ("est_err_alias", ctypes.c_double),
                ("bytes_resident", ctypes.c_longlong), ("max_rhs", ctypes.c_int), ("step3", ctypes.c_int),
                ("diag_correct", ctypes.c_int), ("tuned", ctypes.c_int), ("tune_ms", ctypes.c_double),
                ("rhs_block", ctypes.c_int), ("near_radius", ctypes.c_double), ("near_pairs", ctypes.c_longlong)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgpnufft.so is not built (expected at %s); run __graft_entry__.build() or "
                          "python -m paper_2407_03608_gb300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    lib.gp_plan_opts_default.argtypes = [ctypes.POINTER(gp_plan_opts)]
    lib.gp_plan_opts_default.restype = None
    lib.gp_plan.argtypes = [ctypes.POINTER(vp), dp, ctypes.c_longlong, ctypes.c_int, dp, dp, ctypes.c_double,
                            ctypes.c_double, ctypes.POINTER(gp_plan_opts), vp]
    lib.gp_plan.restype = ctypes.c_int
    lib.gp_matvec.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.c_double, vp]
    lib.gp_matvec.restype = ctypes.c_int
    lib.gp_cg_solve.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ip, dp, vp]
    lib.gp_cg_solve.restype = ctypes.c_int
    lib.gp_cg_solve_refined.argtypes = [vp, vp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, dp, vp]
    lib.gp_cg_solve_refined.restype = ctypes.c_int
    lib.gp_posterior_mean.argtypes = [vp, dp, dp, ctypes.c_longlong, dp, dp, dp, vp]
    lib.gp_posterior_mean.restype = ctypes.c_int
    lib.gp_posterior_variance.argtypes = [vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp,
                                          ip, vp]
    lib.gp_posterior_variance.restype = ctypes.c_int
    lib.gp_posterior_mean_noalloc.argtypes = [vp, dp, dp, ctypes.c_longlong, dp, dp, dp, vp]
    lib.gp_posterior_mean_noalloc.restype = ctypes.c_int
    lib.gp_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.gp_profile_enable.restype = ctypes.c_int
    lib.gp_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.gp_profile_read.restype = ctypes.c_int
    lib.gp_profile_read_rows.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.gp_profile_read_rows.restype = ctypes.c_int
    lib.gp_plan_info_get.argtypes = [vp, ctypes.POINTER(gp_plan_info)]
    lib.gp_plan_info_get.restype = ctypes.c_int
    lib.gp_destroy.argtypes = [vp]
    lib.gp_destroy.restype = None
    lib.gp_last_error.argtypes = []
    lib.gp_last_error.restype = ctypes.c_char_p
    lib.gp_version.argtypes = []
    lib.gp_version.restype = ctypes.c_char_p
    lib.gp_tile_candidates.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.gp_tile_candidates.restype = ctypes.c_int
    lib.gp_plan_params.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(gp_plan_opts),
                                   ctypes.POINTER(gp_plan_info)]
    lib.gp_plan_params.restype = ctypes.c_int
    return lib


LIB = _load()


class GPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


def check(status: int, allow=()):
    if status != GP_OK and status not in allow:
        raise GPError(status, LIB.gp_last_error().decode())
    return status


def _torch():
    try:
        import torch  # noqa: F401
        return torch
    except ImportError:  # pragma: no cover
        return None


def ptr_of(a):
    """(address, keepalive) of a float64 contiguous array or tensor."""
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        if a.dtype != t.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr.ctypes.data, arr


def current_stream():
    t = _torch()
    if t is not None and t.cuda.is_available():
        return t.cuda.current_stream().cuda_stream
    return None


def default_opts(**kw) -> gp_plan_opts:
    o = gp_plan_opts()
    LIB.gp_plan_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("box_lo", "box_hi"):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(o, k, v)
    return o


# ---- the C entry points, same names ------------------------------------------

def gp_plan(points, field_a, field_b, nu: float, eps: float, opts: gp_plan_opts = None, stream=None):
    xp, xk = ptr_of(points)
    shape = tuple(points.shape)
    n = shape[0]
    d = 1 if len(shape) == 1 else shape[1]
    ap, ak = ptr_of(field_a)
    bp, bk = ptr_of(field_b)
    h = ctypes.c_void_p()
    check(LIB.gp_plan(ctypes.byref(h), xp, n, d, ap, bp, float(nu), float(eps),
                      ctypes.byref(opts) if opts is not None else None,
                      stream if stream is not None else current_stream()))
    return h


def gp_matvec(plan, alpha, out, R: int, shift: float = 0.0, stream=None):
    ap, ak = ptr_of(alpha)
    op, ok = ptr_of(out)
    if not _is_writable_target(out, ok):
        raise TypeError("out must be a contiguous float64 array or tensor")
    return check(LIB.gp_matvec(plan, ap, op, int(R), float(shift),
                               stream if stream is not None else current_stream()))


def gp_cg_solve(plan, y, alpha, R: int, eta2: float, rtol: float, maxit: int, stream=None):
    yp, yk = ptr_of(y)
    xp, xk = ptr_of(alpha)
    iters = (ctypes.c_int * R)()
    rel = (ctypes.c_double * R)()
    st = check(LIB.gp_cg_solve(plan, yp, xp, int(R), float(eta2), float(rtol), int(maxit), iters, rel,
                               stream if stream is not None else current_stream()),
               allow=(GP_ENOTCONV,))
    return st, list(iters), list(rel)


def gp_cg_solve_refined(plan_lo, plan_hi, y, alpha, R: int, eta2: float, rtol: float, inner_rtol: float,
                        outer_max: int, maxit: int, stream=None):
    yp, yk = ptr_of(y)
    xp, xk = ptr_of(alpha)
    iters = (ctypes.c_int * R)()
    rel = (ctypes.c_double * R)()
    st = check(LIB.gp_cg_solve_refined(plan_lo, plan_hi, yp, xp, int(R), float(eta2), float(rtol),
                                       float(inner_rtol), int(outer_max), int(maxit), iters, rel,
                                       stream if stream is not None else current_stream()),
               allow=(GP_ENOTCONV,))
    return st, list(iters), list(rel)


def gp_posterior_mean(plan, alpha, xq, field_aq, field_bq, mu, stream=None):
    ap, ak = ptr_of(alpha)
    qp, qk = ptr_of(xq)
    fa, fak = ptr_of(field_aq)
    fb, fbk = ptr_of(field_bq)
    mp, mk = ptr_of(mu)
    return check(LIB.gp_posterior_mean(plan, ap, qp, int(xq.shape[0]), fa, fb, mp,
                                       stream if stream is not None else current_stream()))


def gp_posterior_variance(plan, probes, R: int, eta2: float, rtol: float, maxit: int, var, stream=None):
    pp, pk = ptr_of(probes)
    vp_, vk = ptr_of(var)
    iters = (ctypes.c_int * R)()
    st = check(LIB.gp_posterior_variance(plan, pp, int(R), float(eta2), float(rtol), int(maxit), vp_, iters,
                                         stream if stream is not None else current_stream()),
               allow=(GP_ENOTCONV,))
    return st, list(iters)


def gp_posterior_mean_noalloc(plan, alpha, xq, field_aq, field_bq, mu, stream=None):
    """Posterior mean through the entry point that allocates no device memory (at most
    GP_NOALLOC_MAX_QUERIES queries); mu must be preallocated by the caller."""
    ap, ak = ptr_of(alpha)
    qp, qk = ptr_of(xq)
    fa, fak = ptr_of(field_aq)
    fb, fbk = ptr_of(field_bq)
    mp, mk = ptr_of(mu)
    return check(LIB.gp_posterior_mean_noalloc(plan, ap, qp, int(xq.shape[0]), fa, fb, mp,
                                               stream if stream is not None else current_stream()))


def gp_profile_enable(plan, on: bool):
    return check(LIB.gp_profile_enable(plan, 1 if on else 0))


def gp_profile_read(plan):
    """(average ms per launch of [spread, fft_fwd, diag, fft_inv, interp], matvecs recorded)."""
    ms = (ctypes.c_double * 5)()
    cnt = ctypes.c_longlong()
    check(LIB.gp_profile_read(plan, ms, ctypes.byref(cnt)))
    return list(ms), cnt.value


def gp_profile_read_rows(plan):
    """Average ms per matvec of the library's own row kernels in [fft_fwd, fft_inv]."""
    ms = (ctypes.c_double * 2)()
    check(LIB.gp_profile_read_rows(plan, ms))
    return list(ms)


def gp_plan_info_get(plan) -> dict:
    info = gp_plan_info()
    check(LIB.gp_plan_info_get(plan, ctypes.byref(info)))
    return info.as_dict()


def gp_destroy(plan):
    LIB.gp_destroy(plan)


def gp_version() -> str:
    return LIB.gp_version().decode()


def gp_plan_params(d: int, N: int, nu: float, eps: float, scale_min: float, scale_max: float, box_lo, box_hi,
                   opts: gp_plan_opts = None) -> dict:
    """The plan gp_plan would build for data with these ranges, and its footprint (no GPU).
    scale_min/scale_max: range of the second field in opts.param_mode (l, or the paper's sigma)."""
    lo = (ctypes.c_double * 3)(*[float(v) for v in box_lo] + [0.0] * (3 - len(box_lo)))
    hi = (ctypes.c_double * 3)(*[float(v) for v in box_hi] + [0.0] * (3 - len(box_hi)))
    info = gp_plan_info()
    check(LIB.gp_plan_params(int(d), int(N), float(nu), float(eps), float(scale_min), float(scale_max), lo, hi,
                             ctypes.byref(opts) if opts is not None else None, ctypes.byref(info)))
    return info.as_dict()


def gp_tile_candidates(d: int, n_channels: int, precision: int, width: int) -> list:
    """The autotuner's search space: tile edges the kernels accept, largest first (no GPU)."""
    buf = (ctypes.c_int * 32)()
    n = LIB.gp_tile_candidates(d, n_channels, precision, width, buf, 32)
    check(min(n, 0))
    return [buf[i] for i in range(min(n, 32))]


def _is_writable_target(orig, keep):
    # numpy outputs must be the caller's own array (not a converted copy)
    if isinstance(orig, np.ndarray):
        return keep is orig
    return True
