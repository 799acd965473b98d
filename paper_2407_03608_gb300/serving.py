"""Request loop for GP solves of uneven size, dimension and hyperparameters.

Each request is a GP regression problem (points, scale fields s and l, smoothness nu,
noise eta, right-hand sides y).  The server takes the requests in arrival order on one
GPU and, for each one:

1. admits it by device-memory footprint: the plan is built at the target eps when its
   resident bytes fit the HBM budget, else at the next coarser eps (1e-5, 1e-4, ...),
   and the eps used is recorded;
2. builds the plans (FP32 for the inner CG, FP64 for the residuals of the iterative
   refinement; both hold the sorted points, Chebyshev weights, A' and grids resident
   on the device for the whole solve);
3. solves (K~ + eta^2 I) alpha = y for all right-hand sides at once with
   ``gp_cg_solve_refined`` and copies alpha back to the host;
4. frees the plans.

Two ways of serving share those steps:

* ``Server.serve``: one request at a time.  Latency is finish - arrival on a replayed
  clock: a request starts when it has arrived and the previous one has finished, and its
  service time is the measured wall time of steps 1-4 (host-synchronised).  The arrival
  times are rescaled so that the offered load is a chosen fraction of the measured
  capacity, which gives p50/p99 latency at that load without idling the GPU.
* ``Server.serve_concurrent`` / ``serve_batched``: continuous batching.  Up to ``slots``
  requests are in flight, each on a CUDA stream and host thread of its own, so their
  kernels overlap on the device; a request is admitted in arrival order as soon as a slot
  is free and its predicted footprint fits beside the requests in flight.  Latency is
  measured on the wall clock against arrivals rescaled to the chosen load.
"""
from __future__ import annotations

import argparse
import json
import sys
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

EPS_LADDER = (1e-6, 1e-5, 1e-4, 1e-3, 1e-2)


@dataclass
class Served:
    rid: int
    n: int
    d: int
    nu: float
    r: int
    eps: float
    service_s: float
    plan_s: float
    solve_s: float
    iters: int
    relres: float
    bytes_resident: int
    cache_hit: bool = False
    rejected: bool = False     # no eps level of the ladder fits the budget (nothing solved)


def _rhs(req) -> int:
    y = np.asarray(req.y)
    return 1 if y.ndim == 1 else int(y.shape[1])


def predicted_footprint(abi, req, eps: float, max_rhs: Optional[int] = None, rhs_block: int = 0) -> int:
    """Device bytes of the request's FP64 and FP32 plans at `eps`, predicted on the host
    (gp_plan_params, no allocation); max_rhs (default: the request's R) and rhs_block as
    the plans will be built."""
    x = np.asarray(req.points, dtype=np.float64)
    N, d = x.shape
    l = np.asarray(req.l, dtype=np.float64)                      # the plan's fields are (s, l)
    lo, hi = x.min(axis=0), x.max(axis=0)
    total = 0
    for prec in (abi.GP_FP64, abi.GP_FP32):
        info = abi.gp_plan_params(d, N, req.nu, eps, float(l.min()), float(l.max()), lo, hi,
                                  abi.default_opts(precision=prec, max_rhs=max_rhs or _rhs(req),
                                                   rhs_block=rhs_block))
        total += int(info["bytes_resident"])
    return total


def predicted_eps(abi, req, budget: int, eps_target: float, max_rhs: Optional[int] = None,
                  rhs_block: int = 0) -> Optional[float]:
    """The finest eps of the ladder (from eps_target) at which the request's FP64 and FP32
    plans together are predicted to fit `budget` bytes.  None when even the coarsest level
    does not fit.  A level whose parameters are out of reach (gp_plan_params reports
    GP_ENOMEM or GP_EUNSUPPORTED, as for nu = 1/2 at tight eps) does not fit."""
    for eps in [e for e in EPS_LADDER if e >= eps_target * (1 - 1e-12)]:
        try:
            need = predicted_footprint(abi, req, eps, max_rhs, rhs_block)
        except abi.GPError as e:
            if e.status in (abi.GP_ENOMEM, abi.GP_EUNSUPPORTED):
                continue
            raise
        if need <= budget:
            return eps
    return None


def _plan_fitting(gpn, req, budget: int, eps_target: float, precision, extra: Optional[dict] = None):
    """The plan at the finest eps of the ladder (from eps_target) whose footprint fits."""
    last = None
    for eps in [e for e in EPS_LADDER if e >= eps_target * (1 - 1e-12)]:
        try:
            kw = dict(extra or {})
            mr = kw.pop("max_rhs_override", _rhs(req))
            return gpn.Plan(req.points, req.s, req.l, nu=req.nu, eps=eps, precision=precision,
                            max_rhs=mr, max_bytes=int(budget), **kw), eps
        except gpn.GPError as e:
            if e.status != gpn.abi.GP_ENOMEM:
                raise
            last = e
    raise last


class PlanCache:
    """Resident plans of the models served so far: the FP64 and FP32 plans of a model (its
    sorted points, Chebyshev weights, A' and grids) stay on the device between the requests
    that use it, keyed by (model, eps), within `budget` bytes.  Idle entries are evicted
    least recently used first when a new one needs room; an entry in use is never evicted.
    One request uses an entry at a time (a plan's calls must not overlap): a second
    request for the same model waits for it."""

    class Entry:
        def __init__(self):
            self.plans = None          # (hi, lo, eps)
            self.bytes = 0
            self.users = 0
            self.ready = threading.Event()
            self.use = threading.Lock()
            self.error = None

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.lock = threading.Lock()
        self.entries: "OrderedDict[tuple, PlanCache.Entry]" = OrderedDict()
        self.bytes = 0
        self.hits = 0
        self.misses = 0
        self.evictions = 0

    def _evict_for(self, need: int):
        # caller holds self.lock
        for key in list(self.entries.keys()):
            if self.bytes + need <= self.budget:
                break
            e = self.entries[key]
            if e.users == 0 and e.ready.is_set():
                del self.entries[key]
                self.bytes -= e.bytes
                self.evictions += 1
                if e.plans is not None:
                    hi, lo, _ = e.plans
                    lo.close()
                    hi.close()

    def acquire(self, key, predicted: int, build):
        """The entry for `key`, built by build() -> (hi, lo, eps) on a miss, locked for the
        caller's exclusive use; returns (entry, hit).  Release with release()."""
        with self.lock:
            e = self.entries.get(key)
            hit = e is not None
            if hit:
                self.entries.move_to_end(key)
                self.hits += 1
            else:
                self.misses += 1
                e = PlanCache.Entry()
                self.entries[key] = e
                self._evict_for(predicted)
            e.users += 1
        if not hit:
            try:
                hi, lo, eps = build()
                e.plans = (hi, lo, eps)
                e.bytes = int(hi.info["bytes_resident"] + lo.info["bytes_resident"])
                with self.lock:
                    self.bytes += e.bytes
            except BaseException as err:
                e.error = err
                with self.lock:
                    self.entries.pop(key, None)
                    e.users -= 1
                e.ready.set()
                raise
            e.ready.set()
        else:
            e.ready.wait()
            if e.error is not None:
                with self.lock:
                    e.users -= 1
                raise e.error
        e.use.acquire()
        return e, hit

    def release(self, e):
        e.use.release()
        with self.lock:
            e.users -= 1
            self._evict_for(0)

    def clear(self):
        with self.lock:
            for e in self.entries.values():
                if e.plans is not None:
                    hi, lo, _ = e.plans
                    lo.close()
                    hi.close()
            self.entries.clear()
            self.bytes = 0

    def stats(self) -> dict:
        return {"hits": self.hits, "misses": self.misses, "evictions": self.evictions,
                "resident_bytes": self.bytes, "entries": len(self.entries)}


class Server:
    """Serves requests on the current CUDA device, one after another (``serve``) or
    several in flight on their own streams (``serve_concurrent``, ``serve_batched``).
    With ``cache_plans`` the FP64/FP32 plans of each model stay resident between the
    requests on that model (``PlanCache``, within the HBM budget); without it every
    request builds its plans and frees them."""

    def __init__(self, hbm_budget: float = 120e9, eps_target: float = 1e-6, rtol: float = 1e-8,
                 inner_rtol: float = 1e-4, maxit: int = 20000, outer_max: int = 20, cache_plans: bool = False,
                 max_rhs: int = 16, rhs_block: int = 1):
        import paper_2407_03608_gb300 as gpn
        self.gpn = gpn
        self.budget = int(hbm_budget)
        self.eps_target = eps_target
        self.rtol = rtol
        self.inner_rtol = inner_rtol
        self.maxit = maxit
        self.outer_max = outer_max
        # cached plans take any request on their model: max_rhs columns through grids held for
        # rhs_block of them (one by default: the columns share every CG iteration, and a
        # three-dimensional grid set can take tens of GB)
        self.cache = PlanCache(self.budget) if cache_plans else None
        self.max_rhs = max_rhs
        self.rhs_block = rhs_block
        self.progress = False          # serve(): one JSON line per served request on stderr

    def _build_pair(self, req, stream_handle=None):
        """The FP64 (residual) and FP32 (inner CG) plans of a request at the finest eps that
        fits, sized for any request on the same model when plans are cached."""
        gpn = self.gpn
        extra = {} if stream_handle is None else {"stream": stream_handle}
        if self.cache is not None:
            extra.update(max_rhs_override=self.max_rhs, rhs_block=min(self.rhs_block, self.max_rhs))
        start = predicted_eps(gpn.abi, req, self.budget, self.eps_target, *self._sizes(req)) or EPS_LADDER[-1]
        hi, eps = _plan_fitting(gpn, req, self.budget // 2, max(start, self.eps_target), gpn.GP_FP64, extra=extra)
        try:
            kw = dict(extra)
            mr = kw.pop("max_rhs_override", _rhs(req))
            lo = gpn.Plan(req.points, req.s, req.l, nu=req.nu, eps=eps, precision=gpn.GP_FP32, max_rhs=mr,
                          **kw, **hi.matched_opts())
        except BaseException:
            hi.close()
            raise
        return hi, lo, eps

    def _rejected(self, req, seconds):
        return Served(req.rid, req.points.shape[0], req.points.shape[1], req.nu, _rhs(req), None, seconds, seconds,
                      0.0, 0, 0.0, 0, False, True)

    def _sizes(self, req):
        """(max_rhs, rhs_block) the request's plans are built with."""
        if self.cache is None:
            return _rhs(req), 0
        return self.max_rhs, min(self.rhs_block, self.max_rhs)

    def _plans(self, req, stream_handle=None):
        """(hi, lo, eps, release, hit): the request's plans, from the cache when it has them."""
        if self.cache is None:
            hi, lo, eps = self._build_pair(req, stream_handle)

            def release():
                lo.close()
                hi.close()
            return hi, lo, eps, release, False
        key = (req.model if req.model >= 0 else -1 - req.rid, self.eps_target)
        eps0 = predicted_eps(self.gpn.abi, req, self.budget, self.eps_target, *self._sizes(req))
        need = self.budget if eps0 is None else predicted_footprint(self.gpn.abi, req, eps0, *self._sizes(req))
        entry, hit = self.cache.acquire(key, need, lambda: self._build_pair(req, stream_handle))
        hi, lo, eps = entry.plans
        return hi, lo, eps, (lambda: self.cache.release(entry)), hit

    def serve_one(self, req, keep_alpha: bool = False):
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # admission by the host-side footprint prediction; building at that level can still
        # run out of memory, so the ladder continues from there (or the model's plans are
        # already resident)
        try:
            hi, lo, eps, release, hit = self._plans(req)
        except self.gpn.GPError as e:
            if e.status not in (self.gpn.abi.GP_ENOMEM, self.gpn.abi.GP_EUNSUPPORTED):
                raise
            rec = self._rejected(req, time.perf_counter() - t0)
            return (None, rec) if keep_alpha else rec
        try:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            y = np.asarray(req.y, dtype=np.float64)
            alpha, info = hi.solve_refined(lo, y, req.eta ** 2, rtol=self.rtol, inner_rtol=self.inner_rtol,
                                           outer_max=self.outer_max, maxit=self.maxit)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            iters = int(np.max(info["iters"]))
            relres = float(np.max(info["relres"]))
            nbytes = int(hi.info["bytes_resident"] + lo.info["bytes_resident"])
        finally:
            release()
        rec = Served(req.rid, req.points.shape[0], req.points.shape[1], req.nu, _rhs(req), eps, t2 - t0, t1 - t0,
                     t2 - t1, iters, relres, nbytes, hit)
        return (np.asarray(alpha), rec) if keep_alpha else rec

    def solve_on(self, req, stream):
        """One request on `stream`, from the calling host thread, with no device-wide
        synchronisation (other requests may run on other streams meanwhile): the FP64 and
        FP32 plans at the admitted eps, then the refined solve.  Returns (alpha, Served)."""
        sh = stream.cuda_stream
        t0 = time.perf_counter()
        try:
            hi, lo, eps, release, hit = self._plans(req, sh)
        except self.gpn.GPError as e:
            if e.status not in (self.gpn.abi.GP_ENOMEM, self.gpn.abi.GP_EUNSUPPORTED):
                raise
            return None, self._rejected(req, time.perf_counter() - t0)
        try:
            stream.synchronize()
            t1 = time.perf_counter()
            y = np.asarray(req.y, dtype=np.float64)
            alpha, info = hi.solve_refined(lo, y, req.eta ** 2, rtol=self.rtol, inner_rtol=self.inner_rtol,
                                           outer_max=self.outer_max, maxit=self.maxit, stream=sh)
            stream.synchronize()
            t2 = time.perf_counter()
            nbytes = int(hi.info["bytes_resident"] + lo.info["bytes_resident"])
        finally:
            release()
        rec = Served(req.rid, req.points.shape[0], req.points.shape[1], req.nu, _rhs(req), eps, t2 - t0, t1 - t0,
                     t2 - t1, int(np.max(info["iters"])), float(np.max(info["relres"])), nbytes, hit)
        return np.asarray(alpha), rec

    def serve_concurrent(self, requests, slots: int = 3, arrivals=None):
        """Continuous batching.  Up to `slots` requests are in flight, each on a CUDA stream
        of its own driven by a host thread of its own, so their kernels overlap on the
        device.  A request starts, in arrival order, once it has arrived (`arrivals`:
        seconds from the start; default all at once), a slot is free, and its predicted
        footprint fits the HBM budget beside the requests in flight (one request is always
        admitted).  Returns (results, info): results[i] = (alpha, Served, start_s, end_s) on
        the wall clock of this call; info holds the makespan and the most requests seen in
        flight at once."""
        import torch
        arr = np.zeros(len(requests)) if arrivals is None else np.asarray(arrivals, dtype=np.float64)
        need = []
        for req in requests:
            eps = predicted_eps(self.gpn.abi, req, self.budget, self.eps_target, *self._sizes(req))
            # a request that fits no level is admitted alone (it holds the whole budget)
            need.append(self.budget if eps is None else predicted_footprint(self.gpn.abi, req, eps,
                                                                            *self._sizes(req)))
        device = torch.cuda.current_device()

        def make_stream():
            torch.cuda.set_device(device)
            return torch.cuda.Stream()

        done, info = run_slots(arr, need, self.budget, slots, lambda i, stream: self.solve_on(requests[i], stream),
                               make_stream)
        return [(alpha, rec, begin, end) for (alpha, rec), begin, end in done], info

    def serve_batched(self, requests, load: float = 0.8, slots: int = 3) -> dict:
        """Continuous batching measured on the wall clock: capacity from all requests at once
        (requests per second of makespan), then the stream's Poisson arrivals rescaled to
        `load` times that capacity, with latency = finish - arrival of each request."""
        _, first = self.serve_concurrent(requests, slots=slots)
        capacity = len(requests) / first["makespan_s"]
        arr = np.array([r.arrival_s for r in requests], dtype=np.float64)
        span = arr[-1] - arr[0] if len(arr) > 1 else 0.0
        rate0 = (len(arr) - 1) / span if span > 0 else 1.0
        rate = load * capacity
        rel = (arr - arr[0]) * (rate0 / rate)
        res, info = self.serve_concurrent(requests, slots=slots, arrivals=rel)
        keep = [i for i, r in enumerate(res) if not r[1].rejected]
        lat = np.array([res[i][3] - rel[i] for i in keep])
        service = np.array([res[i][3] - res[i][2] for i in keep])
        rejected = len(res) - len(keep)
        res = [res[i] for i in keep]
        return {
            "slots": slots,
            "requests": len(res),
            "load": load,
            "offered_rate_per_s": rate,
            "capacity_solves_per_s": capacity,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "service_p50_s": float(np.percentile(service, 50)),
            "service_p99_s": float(np.percentile(service, 99)),
            "max_in_flight": int(info["max_inflight"]),
            "rejected": rejected,
            "max_relres": float(max(r[1].relres for r in res)),
            "cache_hit_rate": float(np.mean([r[1].cache_hit for r in res])),
        }

    def check_vs_fp64(self, req, alpha, columns: int = 2, rtol: float = 1e-10) -> float:
        """Largest relative error of served columns against the plain float64 GPU path on
        the same plan parameters: plain CG (no refinement, one right-hand side at a time)
        with the request's FP64 plan, to `rtol`.  Uses the cached plan when there is one."""
        hi, lo, eps, release, _ = self._plans(req)
        try:
            y = np.asarray(req.y, dtype=np.float64).reshape(req.points.shape[0], -1)
            a = np.asarray(alpha, dtype=np.float64).reshape(y.shape)
            worst = 0.0
            for r in range(min(columns, y.shape[1])):
                x, info = hi.solve(y[:, r].copy(), req.eta ** 2, rtol=rtol, maxit=10 * self.maxit)
                x = np.asarray(x)
                worst = max(worst, float(np.linalg.norm(a[:, r] - x) / np.linalg.norm(x)))
        finally:
            release()
        return worst

    def serve(self, requests, load: float = 0.8, check_every: int = 0) -> dict:
        """Serve all requests; latency statistics at `load` times the measured capacity.
        check_every = k > 0: every k-th request's solution is also compared with the plain
        float64 GPU solve (check_vs_fp64; outside the measured service time)."""
        done: List[Served] = []
        errs = []
        for i, r in enumerate(requests):
            alpha, rec = self.serve_one(r, keep_alpha=True)
            done.append(rec)
            if check_every and i % check_every == 0 and not rec.rejected:
                errs.append(self.check_vs_fp64(r, alpha))
            if self.progress:
                print(json.dumps(dict(rec.__dict__, err_vs_fp64=errs[-1] if check_every and i % check_every == 0
                                      and not rec.rejected else None)), file=sys.stderr, flush=True)
        rejected = [s for s in done if s.rejected]
        done = [s for s in done if not s.rejected]
        requests = [r for r in requests if r.rid not in {s.rid for s in rejected}]
        service = np.array([s.service_s for s in done])
        arrivals = np.array([r.arrival_s for r in requests])
        lat, rate = replay_latency(arrivals, service, load)
        return {
            "requests": len(done),
            "load": load,
            "offered_rate_per_s": rate,
            "capacity_solves_per_s": 1.0 / float(np.mean(service)),
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "service_p50_s": float(np.percentile(service, 50)),
            "service_p99_s": float(np.percentile(service, 99)),
            "plan_share": float(np.sum([s.plan_s for s in done]) / np.sum(service)),
            "eps_used": {str(e): int(sum(1 for s in done if s.eps == e)) for e in sorted({s.eps for s in done})},
            "max_relres": float(max(s.relres for s in done)),
            "max_iters": int(max(s.iters for s in done)),
            "points_total": int(sum(s.n * s.r for s in done)),
            "rejected": len(rejected),
            "cache": self.cache.stats() if self.cache is not None else None,
            "cache_hit_rate": float(np.mean([s.cache_hit for s in done])),
            "checked_vs_fp64": len(errs),
            "max_rel_err_vs_fp64_gpu": float(max(errs)) if errs else None,
            "records": [s.__dict__ for s in done],
        }


def run_slots(arrivals, need, budget: int, slots: int, run, make_ctx=lambda: None):
    """The scheduler of continuous batching, on the host.  Job i becomes eligible at
    ``arrivals[i]`` seconds after the start; jobs start in arrival order (ties in index
    order) on ``slots`` worker threads, each of which calls ``make_ctx()`` once (a CUDA
    stream, say) and then ``run(i, ctx)`` for the jobs it takes.  Job i holds ``need[i]``
    bytes of ``budget`` while it runs; the head of the queue waits until it fits beside
    the jobs in flight, except that a job is always admitted when nothing is in flight.
    Returns (results, info): results[i] = (run's value, start_s, end_s) on the clock of
    this call, info = {"makespan_s", "max_inflight"}.  The first exception raised by a
    job stops further admissions and is re-raised once the running jobs have ended."""
    n = len(need)
    arr = np.asarray(arrivals, dtype=np.float64)
    order = [int(i) for i in np.argsort(arr, kind="stable")]
    cond = threading.Condition()
    st = {"next": 0, "bytes": 0, "inflight": 0, "max_inflight": 0}
    results = [None] * n
    errors = []
    t_start = time.perf_counter()

    def worker():
        ctx = make_ctx()
        while True:
            with cond:
                while True:
                    if st["next"] >= n or errors:
                        return
                    i = order[st["next"]]
                    wait = arr[i] - (time.perf_counter() - t_start)
                    fits = st["inflight"] == 0 or st["bytes"] + need[i] <= budget
                    if wait <= 0 and fits:
                        st["next"] += 1
                        st["bytes"] += need[i]
                        st["inflight"] += 1
                        st["max_inflight"] = max(st["max_inflight"], st["inflight"])
                        break
                    cond.wait(timeout=min(max(wait, 1e-3), 0.05) if wait > 0 else 0.05)
            begin = time.perf_counter() - t_start
            try:
                value = run(i, ctx)
                results[i] = (value, begin, time.perf_counter() - t_start)
            except BaseException as e:   # re-raised by the caller after the join
                errors.append(e)
            finally:
                with cond:
                    st["bytes"] -= need[i]
                    st["inflight"] -= 1
                    cond.notify_all()

    threads = [threading.Thread(target=worker, daemon=True) for _ in range(max(1, slots))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return results, {"makespan_s": time.perf_counter() - t_start, "max_inflight": st["max_inflight"]}


def replay_latency(arrivals, service, load: float):
    """Latency (finish - arrival) of FIFO service on one server when the arrival times
    are rescaled to an offered rate of load / mean(service).  Returns (latency, rate)."""
    arrivals = np.asarray(arrivals, dtype=np.float64)
    service = np.asarray(service, dtype=np.float64)
    span = arrivals[-1] - arrivals[0] if len(arrivals) > 1 else 0.0
    rate0 = (len(arrivals) - 1) / span if span > 0 else 1.0
    rate = load / float(np.mean(service))
    arr = (arrivals - arrivals[0]) * (rate0 / rate)
    finish = np.empty_like(arr)
    free_at = -np.inf
    for i, (a, s) in enumerate(zip(arr, service)):
        start = max(a, free_at)
        free_at = start + s
        finish[i] = free_at
    return finish - arr, rate


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--n-min", type=float, default=1e3)
    ap.add_argument("--n-max", type=float, default=1e6)
    ap.add_argument("--max-rhs", type=int, default=16)
    ap.add_argument("--dims", default="1,2,3")
    ap.add_argument("--nus", default="0.5,1.5,2.5")
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--slots", type=int, default=0,
                    help="requests in flight at once (continuous batching); 0 serves one at a time")
    ap.add_argument("--records", action="store_true", help="include per-request records")
    ap.add_argument("--models", type=int, default=0,
                    help="requests draw from this many models (points, fields, nu); 0: each its own")
    ap.add_argument("--cache", action="store_true", help="keep each model's plans resident (PlanCache)")
    ap.add_argument("--check-every", type=int, default=0,
                    help="compare every k-th served solution with the plain float64 GPU solve")
    ap.add_argument("--progress", action="store_true", help="one JSON line per served request on stderr")
    args = ap.parse_args()
    import gpinputs
    reqs = gpinputs.serving_stream(args.requests, n_min=int(args.n_min), n_max=int(args.n_max), seed=args.seed,
                                   max_rhs=args.max_rhs, dims=tuple(int(v) for v in args.dims.split(",")),
                                   nus=tuple(float(v) for v in args.nus.split(",")), n_models=args.models)
    srv = Server(hbm_budget=args.budget_gb * 1e9, eps_target=args.eps, cache_plans=args.cache,
                 max_rhs=args.max_rhs)
    srv.progress = args.progress
    if args.slots > 0:
        out = srv.serve_batched(reqs, load=args.load, slots=args.slots)
    else:
        out = srv.serve(reqs, load=args.load, check_every=args.check_every)
        if not args.records:
            out.pop("records")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
