"""Continuous-batching server for independent USP-ESBGK solves.

Requests arrive over time (a Poisson stream for the benchmark).  The server
keeps one batch resident on the GPU and, between batched steps:

* admits every waiting request whose arrival time has passed, in arrival
  order, while the batch's HBM budget and slot count allow (usp_batch_admit
  returns CAPACITY otherwise and the request waits);
* advances all resident solves together with usp_batch_step (a captured CUDA
  graph), by at most `chunk` steps and never past the closest completion;
* retires every solve that reached its step count: fields (the Eq. 34
  averages) are read back, the handle is released, and the time from arrival
  to result is recorded.

New solves are created and initialised on their own streams while the batch
stream keeps running, so admission work overlaps the resident solves' steps.
The backend is injected (`make_sim`, `make_batch`) so that the scheduling
logic can be exercised without a GPU.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field


@dataclass(order=True)
class Request:
    arrival: float
    rid: int = field(compare=True)   # ties in arrival keep submission order
    workload: dict = field(compare=False)
    steps: int = field(compare=False)
    # filled by the server
    admitted: float = field(default=-1.0, compare=False)
    done: float = field(default=-1.0, compare=False)
    particles: int = field(default=0, compare=False)
    result: object = field(default=None, compare=False, repr=False)


@dataclass
class Resident:
    req: Request
    sim: object
    remaining: int


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


class Server:
    """One GPU, one resident batch, continuous admission and retirement."""

    def __init__(self, make_sim, make_batch, hbm_budget, max_sims=256, chunk=8, clock=time.perf_counter,
                 keep_results=True):
        self.make_sim = make_sim
        self.batch = make_batch(hbm_budget, max_sims)
        self.chunk = chunk
        self.clock = clock
        self.keep_results = keep_results
        self.waiting: list[Request] = []
        self.resident: list[Resident] = []
        self.finished: list[Request] = []
        self.pending_sim = None          # a created solve that did not fit yet
        self.steps_done = 0.0
        self.updates = 0.0

    def submit(self, req: Request):
        heapq.heappush(self.waiting, req)

    # -- admission ----------------------------------------------------------
    def _admit(self, now):
        while self.waiting and self.waiting[0].arrival <= now:
            req = self.waiting[0]
            sim = self.pending_sim
            if sim is None:
                sim = self.make_sim(req.workload)
                req.particles = sim.info()["n_particles"]
            rc = self.batch.admit(sim)
            if rc != 0:
                self.pending_sim = sim   # keep it ready for the next chance
                return
            self.pending_sim = None
            heapq.heappop(self.waiting)
            req.admitted = self.clock()
            self.resident.append(Resident(req, sim, req.steps))

    # -- retirement -----------------------------------------------------------
    def _retire(self):
        keep = []
        for r in self.resident:
            if r.remaining > 0:
                keep.append(r)
                continue
            self.batch.retire(r.sim)
            fields = r.sim.sample(averaged=True)
            r.req.done = self.clock()
            if self.keep_results:
                r.req.result = {"fields": fields, "sim": r.sim}
            else:
                r.sim.close()
            self.finished.append(r.req)
        self.resident = keep

    def run(self, idle_sleep=1e-4):
        """Serve until every submitted request is finished."""
        t_first = None
        while self.waiting or self.resident:
            now = self.clock()
            self._admit(now)
            if not self.resident:
                if self.waiting:
                    time.sleep(min(idle_sleep, max(0.0, self.waiting[0].arrival - now)))
                continue
            if t_first is None:
                t_first = now
            k = min(self.chunk, min(r.remaining for r in self.resident))
            self.batch.step(k)
            for r in self.resident:
                r.remaining -= k
                self.updates += k * r.req.particles
            self.steps_done += k
            if any(r.remaining == 0 for r in self.resident):
                self._retire()
        return self.report(t_first)

    def report(self, t_first=None):
        lat = [r.done - r.arrival for r in self.finished]
        span = (max(r.done for r in self.finished) - min(r.arrival for r in self.finished)) if self.finished else 0.0
        return {"requests": len(self.finished), "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
                "mean_s": sum(lat) / len(lat) if lat else float("nan"), "makespan_s": span,
                "particle_updates": self.updates,
                "aggregate_updates_per_s": self.updates / span if span > 0 else float("nan")}


def poisson_arrivals(n, rate, seed=0, t0=0.0):
    """Arrival times of a Poisson process with the given rate (1/s)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return t0 + np.cumsum(rng.exponential(1.0 / rate, n))


def gpu_backend(pipeline="fused", precision="fp32"):
    """(make_sim, make_batch) on the CUDA library."""
    from . import usp as U
    from . import workloads as W

    def make_sim(w):
        w = W.with_precision(w, precision)
        w["params"]["pipeline"] = pipeline
        return U.Simulation(w).init_particles()

    def make_batch(budget, max_sims):
        return U.Batch(hbm_budget=budget, max_sims=max_sims)

    return make_sim, make_batch


def serve_requests(workloads, rate, hbm_budget, pipeline="fused", precision="fp32", chunk=8, seed=0,
                   keep_results=False):
    """Run a request stream (list of workload dicts with a 'steps' entry)
    arriving as a Poisson process of `rate` per second; returns the report
    and the finished requests."""
    make_sim, make_batch = gpu_backend(pipeline, precision)
    srv = Server(make_sim, make_batch, hbm_budget, max_sims=max(1, len(workloads)), chunk=chunk,
                 keep_results=keep_results)
    t0 = time.perf_counter()
    for i, (w, t) in enumerate(zip(workloads, poisson_arrivals(len(workloads), rate, seed, t0))):
        srv.submit(Request(float(t), i, w, int(w["steps"])))
    rep = srv.run()
    return rep, srv.finished
