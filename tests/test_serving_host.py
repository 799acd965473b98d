"""Host logic of the request loop (no GPU): the replayed FIFO clock."""
import numpy as np

from paper_2407_03608_gb300.serving import replay_latency


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
