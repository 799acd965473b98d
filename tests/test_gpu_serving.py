"""Continuous batching in the serving loop (Server.serve_concurrent): several requests in
flight on their own streams give each request the result it gets alone, within the
solve tolerance; the memory gate keeps requests out while the budget is taken."""
import numpy as np
import pytest

import gpinputs
from paper_2407_03608_gb300.serving import Server, predicted_footprint

pytestmark = pytest.mark.gpu


def _requests(n):
    return gpinputs.serving_stream(n, n_min=1000, n_max=6000, dims=(1, 2), nus=(1.5, 2.5), max_rhs=2, seed=7)


def test_results_alone_and_in_the_mix(gpn):
    reqs = _requests(5)
    srv = Server(hbm_budget=120e9, eps_target=1e-5, rtol=1e-10)
    alone, info1 = srv.serve_concurrent(reqs, slots=1)
    assert info1["max_inflight"] == 1
    mixed, info3 = srv.serve_concurrent(reqs, slots=3)
    assert info3["max_inflight"] >= 2
    for (a1, r1, _, _), (a3, r3, _, _) in zip(alone, mixed):
        assert r1.eps == r3.eps and r1.relres <= 1e-10 and r3.relres <= 1e-10
        e = np.linalg.norm(a3 - a1) / np.linalg.norm(a1)
        assert e <= 1e-8, (r1.rid, e)


def test_memory_gate_serialises_what_does_not_fit_together(gpn):
    req = _requests(1)[0]
    srv = Server(hbm_budget=120e9, eps_target=1e-5)
    need = predicted_footprint(gpn.abi, req, 1e-5)
    srv.budget = int(1.5 * need)          # one request fits, two do not
    res, info = srv.serve_concurrent([req, req, req], slots=3)
    assert info["max_inflight"] == 1
    for a, rec, _, _ in res[1:]:
        assert np.linalg.norm(a - res[0][0]) <= 1e-8 * np.linalg.norm(res[0][0])


def test_cached_plans_give_the_uncached_results(gpn):
    """Requests on a few models: with the plans kept resident (PlanCache) every request gets
    the solution it gets with plans built for it alone, alone and with three in flight; the
    repeated models hit the cache."""
    reqs = gpinputs.serving_stream(8, n_min=1000, n_max=6000, dims=(1, 2), nus=(1.5, 2.5), max_rhs=3, seed=8,
                                   n_models=3)
    assert len({r.model for r in reqs}) < len(reqs)
    plain = Server(hbm_budget=120e9, eps_target=1e-5, rtol=1e-10)
    cached = Server(hbm_budget=120e9, eps_target=1e-5, rtol=1e-10, cache_plans=True, max_rhs=3, rhs_block=2)
    ref = [plain.serve_one(r, keep_alpha=True)[0] for r in reqs]
    one = [cached.serve_one(r, keep_alpha=True) for r in reqs]
    assert sum(rec.cache_hit for _, rec in one) == len(reqs) - len({r.model for r in reqs})
    mixed, info = cached.serve_concurrent(reqs, slots=3)
    for i, r in enumerate(reqs):
        for a in (one[i][0], mixed[i][0]):
            e = np.linalg.norm(a - ref[i]) / np.linalg.norm(ref[i])
            assert e <= 1e-8, (r.rid, e)
    assert cached.cache.stats()["hits"] >= len(reqs)
    cached.cache.clear()


def test_served_solution_matches_the_plain_fp64_solve(gpn):
    reqs = gpinputs.serving_stream(3, n_min=1000, n_max=4000, dims=(1, 2), nus=(1.5,), max_rhs=2, seed=9,
                                   n_models=2)
    srv = Server(hbm_budget=120e9, eps_target=1e-6, rtol=1e-10, cache_plans=True, max_rhs=2)
    for r in reqs:
        alpha, rec = srv.serve_one(r, keep_alpha=True)
        assert srv.check_vs_fp64(r, alpha) <= 1e-6
    srv.cache.clear()
