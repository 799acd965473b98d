"""Oracle: posterior variance of the latent function at the training points.

Test infrastructure only (used by tests/, never by the library).

The posterior covariance of Eq. (postcov) at the training points is
    V = K - K (K + eta^2 I)^{-1} K,
and since K and (K + eta^2 I)^{-1} commute,
    V = eta^2 K (K + eta^2 I)^{-1} = eta^2 (I - eta^2 (K + eta^2 I)^{-1}),
so its diagonal is eta^2 - eta^4 diag((K + eta^2 I)^{-1}).  The diagonal of the
inverse is estimated from R probe vectors z_r with entries +-1 (a Hutchinson-type
estimator; an extension, the paper gives no estimator):
    d_i ~ (sum_r z_ri x_ri) / (sum_r z_ri^2),   x_r = (K + eta^2 I)^{-1} z_r,
which for +-1 probes is the mean of z_ri x_ri over r.  Everything is float64 with
dense linear algebra (Cholesky), for small N.
"""
import numpy as np
import scipy.linalg as sla


def variance_direct(K, eta2):
    """diag(K - K (K + eta^2 I)^{-1} K), formed literally."""
    n = K.shape[0]
    S = K + eta2 * np.eye(n)
    return np.diag(K - K @ np.linalg.solve(S, K)).copy()


def variance_exact(K, eta2):
    """eta^2 - eta^4 diag((K + eta^2 I)^{-1}) by Cholesky."""
    n = K.shape[0]
    c = sla.cho_factor(K + eta2 * np.eye(n), lower=True)
    inv_diag = np.diag(sla.cho_solve(c, np.eye(n)))
    return eta2 - eta2 * eta2 * inv_diag


def variance_probes(K, eta2, Z):
    """The probe estimate: eta^2 - eta^4 (sum_r z_r * x_r) / (sum_r z_r^2), x_r = (K + eta^2 I)^{-1} z_r.

    Z: (N, R) probe matrix.
    """
    n = K.shape[0]
    c = sla.cho_factor(K + eta2 * np.eye(n), lower=True)
    X = sla.cho_solve(c, Z)
    d = np.sum(Z * X, axis=1) / np.sum(Z * Z, axis=1)
    return eta2 - eta2 * eta2 * d


def all_sign_probes(n):
    """Every +-1 vector of length n as columns (2^n of them): the probe average is then
    exactly the diagonal, because sum over all sign patterns of z_i z_j is 0 for i != j."""
    k = np.arange(2 ** n)
    return np.array([1.0 - 2.0 * ((k >> i) & 1) for i in range(n)])
