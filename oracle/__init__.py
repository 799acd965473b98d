"""CPU oracle for the non-stationary Matern GP matvec and solve (TEST INFRASTRUCTURE).

This package is test infrastructure, not part of the library.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg and reference arm of
``bench.py`` may import or run it.  The CUDA library never calls it, and it shares no code,
table or constant with the CUDA library: both sides take their inputs from the
seeded generators in ``gpinputs`` and nothing else.

Everything is plain float64 NumPy/SciPy (plus one small C direct sum for
sampled rows at large N).  Each function cites the equation or section of
Kielstra & Lindsey, "Gaussian process regression with log-linear scaling for
common non-stationary kernels" (arXiv 2407.03608) that it writes out.

Two targets are provided:

* O-K  (the plain definition): the kernel matrix K of Eq. (nonstat2) formed
  densely, multiplied directly and factored by Cholesky; and, for large N,
  exact rows of K alpha by direct summation (``rows``).
* O-K~ (what the fast method computes exactly): the approximate kernel
  K~ of Eq. (Ktilde) applied through steps (1)-(5) of Sec. 4.2 with
  brute-force (non-uniform DFT) sums, and the same K~ in closed form by
  Poisson summation (Eq. (PSF) with Eq. (fanalytic)).

Modules:
  matern      phi_nu (Eq. matern), squared exponential (Eq. squaredexp)
  kernel      scale mapping, dense K (Eq. nonstat2), Cholesky solve, plain CG
  quadrature  Schoenberg representation (Eq. maternpres) and trapezoid rule (Eq. trapsum)
  chebyshev   Chebyshev-Lobatto nodes (Eq. chebscheme), Lagrange basis, w_k (Eq. Wk)
  ktilde      Fourier tables, tensor A (Remark rem:step3), exact K~ matvec, Poisson K~
  nudft       type-1 / type-2 non-uniform DFTs (App. D)
  rows        exact sampled rows of K alpha (C, OpenMP) for large N
  bounds      the error quantities of Sec. 5 (Definition eptrap; Lemma interp)
  diagcorr    the exact diagonal K~_ii and the diagonal-corrected matvec (an extension)
  nearfield   K~ for single pairs (separable form) and the near-field-corrected matvec (an extension)
  variance    posterior variance at the training points and its probe estimator (an extension)
"""
from . import matern, kernel, quadrature, chebyshev, nudft, ktilde, bounds, rows  # noqa: F401
