"""Host logic of the request loop (no GPU): the replayed FIFO clock and the admission
by predicted footprint."""
import numpy as np
import pytest

import gpinputs
from paper_2407_03608_gb300.serving import EPS_LADDER, predicted_eps, replay_latency


def test_idle_server_latency_is_service_time():
    # arrivals far apart relative to service: nobody waits
    arr = np.array([0.0, 10.0, 20.0, 30.0])
    svc = np.array([0.1, 0.2, 0.1, 0.3])
    lat, rate = replay_latency(arr, svc, load=0.01)
    assert np.allclose(lat, svc)
    assert np.isclose(rate, 0.01 / svc.mean())


def test_fifo_queueing_matches_hand_computation():
    # evenly spaced arrivals at the offered rate: inter-arrival 1/rate
    arr = np.arange(4, dtype=float)
    svc = np.array([1.5, 0.5, 0.5, 0.5])          # mean 0.75
    lat, rate = replay_latency(arr, svc, load=1.0)  # rate 4/3: arrivals 0, .75, 1.5, 2.25
    a = np.arange(4) * 0.75
    finish = [1.5, 2.0, 2.5, 3.0]
    assert np.allclose(lat, np.array(finish) - a)


def test_higher_load_never_lowers_latency():
    rng = np.random.default_rng(1)
    arr = np.cumsum(rng.exponential(1.0, 200))
    svc = rng.uniform(0.2, 1.0, 200)
    l1, _ = replay_latency(arr, svc, 0.5)
    l2, _ = replay_latency(arr, svc, 0.9)
    assert np.percentile(l2, 99) >= np.percentile(l1, 99) - 1e-12
    assert np.all(l1 >= svc - 1e-12)


@pytest.fixture(scope="module")
def abi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03608_gb300 import abi
    return abi


def test_admission_takes_the_finest_eps_that_fits(abi):
    # d <= 2 and N <= 5e4, as in the bench's served sample (the stream's 3-D requests have
    # length scales so short that even eps = 1e-4 needs terabytes)
    reqs = gpinputs.serving_stream(6, n_min=1000, n_max=50_000, dims=(1, 2), nus=(1.5,), max_rhs=2)
    for req in reqs:
        roomy = predicted_eps(abi, req, 10 ** 13, 1e-6)
        assert roomy == 1e-6
        # the predicted level coarsens as the budget shrinks, and never gets finer
        levels = [predicted_eps(abi, req, b, 1e-6) for b in (10 ** 13, 10 ** 10, 10 ** 9, 10 ** 8, 10 ** 7)]
        seen = [EPS_LADDER.index(e) if e is not None else len(EPS_LADDER) for e in levels]
        assert seen == sorted(seen)
        assert predicted_eps(abi, req, 1, 1e-6) is None
        # a coarser target is never refined
        assert predicted_eps(abi, req, 10 ** 13, 1e-4) == 1e-4


def test_short_length_scales_are_admitted_coarser(abi):
    # a 3-D request of the stream under the 120 GB budget: only a coarse level fits
    req = gpinputs.serving_stream(8, n_min=1000, n_max=50_000, dims=(3,), nus=(1.5,), max_rhs=1)[0]
    eps = predicted_eps(abi, req, 120 * 10 ** 9, 1e-6)
    assert eps is not None and eps >= 1e-4
