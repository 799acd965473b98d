"""The synthetic input recipe (gpinputs): sizes, ranges and structure of each workload
as the documented recipe states them, and determinism under the fixed seeds.  No GPU."""
import numpy as np

import gpinputs


def test_one_dimensional_workload():
    w = gpinputs.config_1d(2000)
    assert w.points.shape == (2000, 1) and w.nu == 1.5 and w.eta == 0.1 and w.eps == 1e-6
    x = w.points[:, 0]
    assert np.all((x >= 0) & (x < 1))
    assert 0.02 <= w.l.min() and w.l.max() <= 0.08 and w.l.max() / w.l.min() > 3.5
    assert 0.5 <= w.s.min() and w.s.max() <= 1.5
    # y = sin 12x + N(0, 0.1^2)
    resid = w.y - np.sin(12 * x)
    assert abs(resid.std() - 0.1) < 0.01 and abs(resid.mean()) < 0.01


def test_two_dimensional_clustered_workload():
    n = 40_000
    w = gpinputs.config_2d(n)
    assert w.points.shape == (n, 2) and w.eta == 0.05
    uni, cl = w.points[: n // 2], w.points[n // 2:]
    assert np.all((uni >= 0) & (uni < 1))
    # eight clusters of equal size with standard deviation 0.03 around centres in [0.1, 0.9]^2
    parts = np.split(cl, 8)
    for p in parts:
        c = p.mean(axis=0)
        assert np.all((c > 0.09) & (c < 0.91))
        assert np.allclose(p.std(axis=0), 0.03, rtol=0.1)
    assert 0.02 <= w.l.min() and w.l.max() <= 0.04
    assert np.allclose(w.s, 1 + 0.3 * w.points[:, 0])


def test_three_dimensional_workload():
    w = gpinputs.config_3d(20_000)
    assert w.points.shape == (20_000, 3) and w.nu == 2.5
    assert np.all((w.points >= 0) & (w.points < 1))
    assert 0.05 <= w.l.min() and w.l.max() <= 0.10
    assert np.exp(-0.75) <= w.s.min() and w.s.max() <= 1.0
    assert np.all((w.y >= 0) & (w.y < 1))


def test_batched_right_hand_sides():
    w = gpinputs.config_2d_batched(5000)
    assert w.y.shape == (5000, 64)
    probes = w.y[:, 8:]
    assert set(np.unique(probes)) == {-1.0, 1.0}
    assert abs(probes.mean()) < 0.02
    # the eight noisy vectors share the noiseless field and differ by noise of std eta
    d = w.y[:, 0] - w.y[:, 1]
    assert abs(d.std() - np.sqrt(2) * w.eta) < 0.01


def test_serving_stream():
    reqs = gpinputs.serving_stream(60, n_min=1000, n_max=20_000, seed=5)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    for r in reqs:
        n, d = r.points.shape
        assert 1000 <= n <= 20_000 and d in (1, 2, 3) and r.nu in (0.5, 1.5, 2.5)
        assert r.l.min() > 0 and r.l.max() / r.l.min() <= 1.4 / 0.6 + 1e-12
        assert 0.7 - 1e-12 <= r.s.min() and r.s.max() <= 1.3 + 1e-12
        rhs = 1 if r.y.ndim == 1 else r.y.shape[1]
        assert 1 <= rhs <= 16


def test_paper_setup():
    x, w, sigma = gpinputs.paper_setup(3000, 2, seed=1)
    assert np.all((x >= -1) & (x <= 1)) and np.all(w == 1)
    assert 1 / 6 - 1e-12 <= sigma.min() and sigma.max() <= 0.5 + 1e-12


def test_seeds_make_the_inputs_reproducible():
    a, b = gpinputs.config_2d(3000), gpinputs.config_2d(3000)
    assert np.array_equal(a.points, b.points) and np.array_equal(a.y, b.y) and np.array_equal(a.alpha, b.alpha)
    r1 = gpinputs.serving_stream(5, n_max=5000, seed=9)
    r2 = gpinputs.serving_stream(5, n_max=5000, seed=9)
    assert all(np.array_equal(p.points, q.points) and p.arrival_s == q.arrival_s for p, q in zip(r1, r2))
    assert not np.array_equal(gpinputs.random_alpha(100, 1, 1), gpinputs.random_alpha(100, 1, 2))
