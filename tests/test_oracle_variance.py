"""Pins of the posterior-variance oracle (oracle/variance.py), on the CPU.

* the identity K - K (K + eta^2 I)^{-1} K = eta^2 (I - eta^2 (K + eta^2 I)^{-1}) on the
  diagonal, against the literal formula;
* the probe estimator over every +-1 sign pattern equals the exact diagonal;
* with a single probe the estimate is eta^2 - eta^4 z*x, checked by hand;
* the variance lies in [0, K_ii] (a posterior variance never exceeds the prior one).
"""
import numpy as np

import gpinputs
from oracle import kernel as okern
from oracle import variance


def small_K(n=40, seed=0):
    w = gpinputs.config_1d(n)
    wp, sig = okern.paper_fields(w.s, w.l, 1)
    return okern.kernel_dense(w.points, wp, sig, 1.5), w


def test_identity_matches_literal_formula():
    K, _ = small_K()
    for eta2 in (1e-2, 0.3):
        a = variance.variance_direct(K, eta2)
        b = variance.variance_exact(K, eta2)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a)) + 1e-14


def test_all_sign_probes_give_the_exact_diagonal():
    K, _ = small_K(10)
    Z = variance.all_sign_probes(10)
    assert Z.shape == (10, 1024)
    est = variance.variance_probes(K, 0.05, Z)
    ex = variance.variance_exact(K, 0.05)
    assert np.max(np.abs(est - ex)) <= 1e-12


def test_single_probe_by_hand():
    K, _ = small_K(12)
    eta2 = 0.1
    z = np.where(np.arange(12) % 3 == 0, 1.0, -1.0)
    x = np.linalg.solve(K + eta2 * np.eye(12), z)
    est = variance.variance_probes(K, eta2, z[:, None])
    assert np.allclose(est, eta2 - eta2 ** 2 * z * x, rtol=0, atol=1e-14)


def test_variance_between_zero_and_prior():
    K, _ = small_K(60)
    v = variance.variance_exact(K, 0.01)
    assert np.all(v >= -1e-12)
    assert np.all(v <= np.diag(K) + 1e-12)
