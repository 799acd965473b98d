"""Seeded synthetic workloads for the non-stationary Matern GP matvec and solve.

This module only draws inputs: point clouds, the two spatially varying scale
fields sampled at the points, right-hand sides and test vectors.  It holds none
of the method's arithmetic, so the CPU oracle and the CUDA path can both take
their inputs from here without sharing any computation.

Every generator is seeded (NumPy PCG64) and returns float64 NumPy arrays:

* ``points`` (N, d), row-major,
* ``s``  (N,)  vertical scale s(x_i)  (standard deviation of the prior),
* ``l``  (N,)  horizontal scale l(x_i) (Matern length),
* ``y``  (N,) or (N, R), ``alpha`` (N,) test vector.

The shapes follow the synthetic workloads of the paper's experiments
(Sec. 6: points drawn independently, smooth scale fields, y drawn from a
simple distribution) at the sizes of the five benchmark workloads.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    name: str
    points: np.ndarray          # (N, d)
    s: np.ndarray               # (N,)
    l: np.ndarray               # (N,)
    nu: float
    eta: float
    y: np.ndarray               # (N,) or (N, R)
    alpha: np.ndarray           # (N,)
    eps: float = 1e-6
    extra: Dict[str, object] = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.points.shape[0]

    @property
    def d(self) -> int:
        return self.points.shape[1]


# --------------------------------------------------------------------------
# field definitions (workload recipes, evaluated at the sampled points)
# --------------------------------------------------------------------------

def fields_1d(x: np.ndarray):
    """s(x)=1+0.5 sin(2 pi x), l(x)=0.05+0.03 cos(2 pi x) on [0,1]."""
    x = x[:, 0]
    return 1.0 + 0.5 * np.sin(2 * np.pi * x), 0.05 + 0.03 * np.cos(2 * np.pi * x)


def fields_2d(x: np.ndarray):
    """s=1+0.3 x, l=0.02+0.02 (1+sin(2 pi x) cos(2 pi y))/2 on the unit square."""
    a, b = x[:, 0], x[:, 1]
    s = 1.0 + 0.3 * a
    l = 0.02 + 0.02 * (1.0 + np.sin(2 * np.pi * a) * np.cos(2 * np.pi * b)) / 2.0
    return s, l


def fields_3d(x: np.ndarray):
    """s=exp(-|x-0.5|^2), l=0.05+0.05 |x|^2/3 in the unit cube."""
    s = np.exp(-np.sum((x - 0.5) ** 2, axis=1))
    l = 0.05 + 0.05 * np.sum(x ** 2, axis=1) / 3.0
    return s, l


# --------------------------------------------------------------------------
# point clouds
# --------------------------------------------------------------------------

def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    return _rng(seed).random((n, d))


def clustered_points_2d(n: int, seed: int, n_clusters: int = 8, std: float = 0.03) -> np.ndarray:
    """Half uniform on the unit square, half from seeded Gaussian clusters.

    Cluster centres are uniform on [0.1, 0.9]^2; cluster points are not clipped.
    """
    g = _rng(seed)
    n_uni = n // 2
    n_cl = n - n_uni
    uni = g.random((n_uni, 2))
    centres = 0.1 + 0.8 * g.random((n_clusters, 2))
    sizes = np.full(n_clusters, n_cl // n_clusters)
    sizes[: n_cl - sizes.sum()] += 1
    parts = [uni]
    for c, m in zip(centres, sizes):
        parts.append(c + std * g.standard_normal((m, 2)))
    return np.concatenate(parts, axis=0)


# --------------------------------------------------------------------------
# the benchmark workloads (full size) and their scaled-down test variants
# --------------------------------------------------------------------------

def config_1d(n: int = 2000) -> Workload:
    """d=1, N=2000 uniform on [0,1], nu=3/2, eta=0.1, eps=1e-6."""
    x = uniform_points(n, 1, seed=0)
    s, l = fields_1d(x)
    y = np.sin(12.0 * x[:, 0]) + 0.1 * _rng(1).standard_normal(n)
    alpha = _rng(2).standard_normal(n)
    return Workload("d1_N%d_matern32" % n, x, s, l, 1.5, 0.1, y, alpha, 1e-6)


def config_2d(n: int = 1_000_000, nu: float = 1.5) -> Workload:
    """d=2, N=1e6: 50% uniform + 50% in 8 Gaussian clusters (std 0.03), eta=0.05."""
    x = clustered_points_2d(n, seed=3)
    s, l = fields_2d(x)
    eta = 0.05
    y = np.sin(6 * np.pi * x[:, 0]) * np.cos(4 * np.pi * x[:, 1]) + eta * _rng(4).standard_normal(n)
    alpha = _rng(5).standard_normal(n)
    return Workload("d2_N%d_clustered_matern%d2" % (n, int(round(2 * nu))), x, s, l, nu, eta, y, alpha, 1e-6)


def config_3d(n: int = 2_000_000) -> Workload:
    """d=3, N=2e6 uniform in the unit cube, nu=5/2, eta=0.1, eps=1e-6."""
    x = uniform_points(n, 3, seed=6)
    s, l = fields_3d(x)
    y = _rng(7).random(n)
    alpha = _rng(8).standard_normal(n)
    return Workload("d3_N%d_matern52" % n, x, s, l, 2.5, 0.1, y, alpha, 1e-6)


def batched_rhs(n: int, noisy_fn, n_noisy: int = 8, n_probe: int = 56) -> np.ndarray:
    """(N, n_noisy + n_probe): noisy observation vectors then Rademacher probes."""
    cols = [noisy_fn(_rng(10 + r)) for r in range(n_noisy)]
    probes = _rng(18).integers(0, 2, size=(n, n_probe)).astype(np.float64) * 2.0 - 1.0
    return np.concatenate([np.stack(cols, axis=1), probes], axis=1)


def config_2d_batched(n: int = 1_000_000) -> Workload:
    w = config_2d(n, 1.5)
    x = w.points
    base = np.sin(6 * np.pi * x[:, 0]) * np.cos(4 * np.pi * x[:, 1])
    y = batched_rhs(n, lambda g: base + w.eta * g.standard_normal(n))
    return Workload("d2_N%d_clustered_matern32_R64" % n, x, w.s, w.l, 1.5, w.eta, y, w.alpha, 1e-6)


def random_alpha(n: int, r: int, seed: int) -> np.ndarray:
    a = _rng(seed).standard_normal((n, r))
    return a[:, 0].copy() if r == 1 else a


# --------------------------------------------------------------------------
# serving stream: GP solve requests of uneven size, dimension and smoothness
# --------------------------------------------------------------------------

@dataclass
class Request:
    rid: int
    arrival_s: float
    points: np.ndarray
    s: np.ndarray
    l: np.ndarray
    nu: float
    eta: float
    y: np.ndarray          # (N,) or (N, R)
    model: int = -1        # requests with the same model share points, fields and nu (-1: its own)


def _trig_series(x: np.ndarray, g: np.random.Generator, degree: int = 3) -> np.ndarray:
    """Random smooth function of degree <= 3 per axis, normalised to [-1, 1] on the points."""
    n, d = x.shape
    f = np.zeros(n)
    for _ in range(4):
        k = g.integers(0, degree + 1, size=d)
        ph = g.random(d) * 2 * np.pi
        amp = g.standard_normal()
        f += amp * np.prod(np.cos(2 * np.pi * k[None, :] * x + ph[None, :]), axis=1)
    m = np.max(np.abs(f))
    return f / m if m > 0 else f


def _serving_model(g: np.random.Generator, n_min: int, n_max: int, dims, nus):
    n = int(round(np.exp(g.uniform(np.log(n_min), np.log(n_max)))))
    d = int(g.choice(dims))
    nu = float(g.choice(nus))
    x = g.random((n, d))
    l0 = 0.08 * (n / 1000.0) ** (-1.0 / d)
    l0 = max(l0, {1: 0.004, 2: 0.02, 3: 0.05}[d])
    l = l0 * (1.0 + 0.4 * _trig_series(x, g))
    s = 1.0 + 0.3 * _trig_series(x, g)
    return x, s, l, nu


def serving_stream(n_requests: int = 2000, rate_hz: float = 50.0, n_min: int = 1000,
                   n_max: int = 1_000_000, seed: int = 100, max_rhs: int = 16,
                   dims=(1, 2, 3), nus=(0.5, 1.5, 2.5), n_models: int = 0) -> List[Request]:
    """Poisson arrivals; N log-uniform in [n_min, n_max]; seeded smooth fields.

    l(x) = l0 (1 + 0.4 g1(x)), s(x) = 1 + 0.3 g2(x) with g1, g2 random trigonometric
    series normalised to [-1, 1]; l0 shrinks like (N/1000)^(-1/d) so that each row
    of K keeps a bounded number of significant entries (the narrow scaling regime).
    R in 1..max_rhs right-hand sides, uniform on [0, 1] (as in Sec. 6.2).

    n_models = 0: every request is a model of its own.  n_models > 0: the models
    (points, fields, nu) are drawn first, and each request solves new right-hand sides
    on one of them, model k with probability proportional to 1 / (k + 1) (a few popular
    models, a long tail), so that a server can keep the plans of the popular ones.
    """
    g = _rng(seed)
    t = 0.0
    out = []
    models = [_serving_model(g, n_min, n_max, dims, nus) for _ in range(n_models)]
    if n_models:
        pop = 1.0 / np.arange(1, n_models + 1)
        pop /= pop.sum()
    for rid in range(n_requests):
        t += g.exponential(1.0 / rate_hz)
        if n_models:
            m = int(g.choice(n_models, p=pop))
            x, s, l, nu = models[m]
        else:
            m = -1
            x, s, l, nu = _serving_model(g, n_min, n_max, dims, nus)
        n = x.shape[0]
        r = int(g.integers(1, max_rhs + 1))
        y = g.random((n, r)) if r > 1 else g.random(n)
        out.append(Request(rid, t, x, s, l, nu, 0.1, y, m))
    return out


def paper_setup(n: int, d: int, seed: int = 0):
    """The setup of the paper's experiments (Sec. 6): x ~ U[-1, 1]^d, w(x) = 1 and
    sigma(x) = (prod_i cos(pi x_i) + 2) / 6, in the paper's own (w, sigma) fields."""
    x = _rng(seed).uniform(-1.0, 1.0, (n, d))
    sigma = (np.prod(np.cos(np.pi * x), axis=1) + 2.0) / 6.0
    return x, np.ones(n), sigma
