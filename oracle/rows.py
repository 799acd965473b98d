"""Exact sampled rows of K alpha for large N (test infrastructure; see the package header).

Thin ctypes wrapper around ``rows.c`` (direct sum of Eq. (nonstat2)).  The
shared object is compiled from source by ``build()`` with gcc and OpenMP.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_rows.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "rows.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.oracle_rows.restype = ctypes.c_int
        lib.oracle_rows.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        _lib = lib
    return _lib


def rows(X, w, sigma, nu, alpha, row_idx):
    """out[q, r] = (K alpha[:, r])_{row_idx[q]} exactly (nu=inf: squared exponential)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, d = X.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    one = alpha.ndim == 1
    A = np.asfortranarray(alpha[:, None] if one else alpha)
    R = A.shape[1]
    if R > 64:
        raise ValueError("at most 64 right-hand sides")
    idx = np.ascontiguousarray(row_idx, dtype=np.int64)
    out = np.zeros((idx.size, R), order="F")
    nu_c = -1.0 if (nu is None or np.isinf(nu)) else float(nu)
    rc = lib.oracle_rows(X.ctypes.data, w.ctypes.data, sigma.ctypes.data, N, d, nu_c, A.ctypes.data, R,
                         idx.ctypes.data, idx.size, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_rows: unsupported nu=%r or shape" % nu)
    return out[:, 0] if one else out


def threads_used() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
