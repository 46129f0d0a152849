"""Continuous-batching serving loop for relax-to-equilibrium requests.

Requests (a case: lattice, parameters, initial density, tolerance, step
budget) arrive over time.  The loop admits waiting requests into the
resident batch in arrival order whenever a case slot, arena range and tile
room are free, advances every resident running case together one persistent
launch at a time, and retires each case as soon as it stops (converged,
budget reached or unstable), which frees its memory for the next admission.
Requests that arrive while others are on the device therefore share launches
with them.  Latency is completion time minus arrival time.  A request that
the batch refuses while it holds no case can never fit (it is larger than
the whole arena or tile table): it is rejected instead of blocking the queue.

The batch object is injected (``paper_2012_11075_gb300.wblbe.Batch`` on the
GPU); the loop itself is host logic and is tested on the CPU with a fake.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


REJECTED = -2                   # Request.state of a request that can never fit
# Request.state after completion: the batch's case states
CONVERGED, BUDGET, UNSTABLE = 1, 2, 3
OUTCOMES = {CONVERGED: "converged", BUDGET: "budget", UNSTABLE: "unstable"}


@dataclass
class Request:
    rid: int
    arrival: float              # seconds since the start of the run
    params: object              # wblbe.Params
    rho: object                 # [ny][nx] float64, or a callable building it
    umax_tol: float
    max_steps: int
    admitted: float = math.nan
    finished: float = math.nan
    state: int = -1
    steps: int = 0
    case_id: int = -1


@dataclass
class ServeReport:
    completed: list = field(default_factory=list)
    rejected: list = field(default_factory=list)
    offered: int = 0
    admitted: int = 0
    backlog: int = 0
    running_at_end: int = 0
    elapsed: float = 0.0
    node_steps: float = 0.0
    launches: int = 0

    def latencies(self, state=None):
        """Completion minus arrival of the completed requests (of one outcome
        state, or all)."""
        return np.array([r.finished - r.arrival for r in self.completed
                         if state is None or r.state == state])

    def summary(self) -> dict:
        """Counts, throughput and latency percentiles.  Latency is reported
        for all completed requests and separately per outcome: converged
        (max|u| below the tolerance), budget (step budget reached) and
        unstable (a non-finite value); the converged requests' step counts
        to the tolerance are given too."""
        def pct(a, q):
            return float(np.percentile(a, q)) if len(a) else None

        lat = self.latencies()
        states = collections.Counter(r.state for r in self.completed)
        out = {
            "offered": self.offered,
            "admitted": self.admitted,
            "completed": len(self.completed),
            "rejected": len(self.rejected),
            "backlog_at_end": self.backlog,
            "running_at_end": self.running_at_end,
            "elapsed_s": self.elapsed,
            "completed_per_s": len(self.completed) / self.elapsed if self.elapsed > 0 else 0.0,
            "p50_latency_s": pct(lat, 50),
            "p99_latency_s": pct(lat, 99),
            "mlups": self.node_steps / self.elapsed / 1e6 if self.elapsed > 0 else 0.0,
            "launches": self.launches,
            "states": {str(k): v for k, v in sorted(states.items())},
        }
        for state, name in OUTCOMES.items():
            a = self.latencies(state)
            out[f"{name}_count"] = int(len(a))
            out[f"{name}_p50_latency_s"] = pct(a, 50)
            out[f"{name}_p99_latency_s"] = pct(a, 99)
        steps = np.array([r.steps for r in self.completed if r.state == CONVERGED])
        out["converged_p50_steps"] = pct(steps, 50)
        out["converged_p99_steps"] = pct(steps, 99)
        return out


class Server:
    """Admission, advance and retirement around one batch."""

    def __init__(self, batch, clock=time.perf_counter, on_finish=None):
        self.batch = batch
        self.clock = clock
        self.on_finish = on_finish             # called (request, batch) before retirement
        self.t0 = clock()
        self.queue = collections.deque()       # waiting requests, arrival order
        self.resident = {}                     # case_id -> Request
        self.report = ServeReport()

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request):
        self.queue.append(req)
        self.report.offered += 1

    def admit_waiting(self):
        """Admit from the head of the queue until the batch refuses."""
        while self.queue:
            req = self.queue[0]
            if callable(req.rho):
                req.rho = req.rho()            # built when it is first offered
            cid = self.batch.admit(req.params, req.rho, req.umax_tol, req.max_steps)
            if cid is None:
                if self.resident:
                    break                      # full: keep it queued
                # refused by an empty batch: it will never fit
                self.queue.popleft()
                req.state = REJECTED
                req.finished = self.now()
                self.report.rejected.append(req)
                continue
            self.queue.popleft()
            req.case_id = cid
            req.admitted = self.now()
            self.resident[cid] = req
            self.report.admitted += 1

    def step(self):
        """One launch for every resident running case, then retire finished."""
        running = [r for r in self.resident.values() if r.state == -1]
        if not running:
            return
        cfg = self.batch.get_config()
        self.batch.advance(1)
        self.report.launches += 1
        self.report.node_steps += cfg[2] * sum(r.params.nx * r.params.ny for r in running)
        t = self.now()
        for cid in self.batch.poll():
            req = self.resident.pop(cid)
            info = self.batch.info(cid)
            req.state = info["state"]
            req.steps = info["steps"]
            req.finished = t
            if self.on_finish is not None:
                self.on_finish(req, self.batch)
            self.batch.retire(cid)
            self.report.completed.append(req)

    def run(self, requests, duration: float, drain: bool = False, stop_after=None,
            time_cap=None):
        """Serve ``requests`` (sorted by arrival) in real time until
        ``duration`` seconds (and, with ``drain``, until all finished), or
        until ``stop_after`` requests have completed, or ``time_cap`` seconds
        have passed, whichever comes first."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        while True:
            if stop_after is not None and len(self.report.completed) >= stop_after:
                break
            if time_cap is not None and self.now() >= time_cap:
                break
            t = self.now()
            while pending and pending[0].arrival <= t:
                self.submit(pending.popleft())
            self.admit_waiting()
            if self.resident:
                self.step()
            elif pending and not self.queue:
                # idle until the next arrival
                wait = pending[0].arrival - self.now()
                if wait > 0:
                    time.sleep(min(wait, 0.01))
            if t >= duration and (not drain or (not pending and not self.queue
                                                and not self.resident)):
                break
        self.report.elapsed = self.now()
        self.report.backlog = len(self.queue) + len(pending)
        self.report.running_at_end = len(self.resident)
        return self.report


def poisson_arrivals(rate: float, duration: float, seed: int):
    """Arrival times of a Poisson process of the given rate on [0, duration)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append(t)


def make_requests(rate: float, duration: float, seed: int, precision: int, scheme: int,
                  side_min=32, side_max=1024, umax_tol=None, max_steps=200000):
    """Relax-to-equilibrium requests of the serving workload: sides
    log-uniform in [side_min, side_max], flat slab or droplet, parameters as
    the batched case mix; tolerance 1e-6 (FP32) or 1e-10 (FP64)."""
    import functools

    from . import workloads as wl
    from .wblbe import FP64, Params
    times = poisson_arrivals(rate, duration, seed)
    specs = wl.batched_case_specs(count=len(times), seed=seed + 1, side_min=side_min,
                                  side_max=side_max)
    tol = umax_tol if umax_tol is not None else (1e-10 if precision == FP64 else 1e-6)
    reqs = []
    for k, (t, sp) in enumerate(zip(times, specs)):
        p = Params(sp["nx"], sp["ny"], sp["tau"], sp["kappa"], sp["beta"], sp["rho_l"],
                   sp["rho_g"], scheme=scheme, precision=precision)
        reqs.append(Request(k, t, p, functools.partial(wl.case_field, sp), tol, max_steps))
    return reqs
