"""Continuous-batching request loop over the batch ABI (dirac_batch_*).

Each request is one simulation (grid, metric, packet, step count). Requests that have
arrived are admitted as soon as their device footprint fits the budget -- also while
others are running -- and join the next tick of the shared batch; finished requests are
retired at once and their memory is freed for the next admissions. Latency is measured
from arrival to the moment the request's last step has completed on the device.

Admission policy: "fifo" admits arrived requests in arrival order; "sjf" admits the
arrived request with the least work (grid points x steps) first and keeps the points of
the active requests under a cap, so that under overload short requests finish early
instead of every request sharing the GPU until the end. Neither changes any result: each
request is stepped exactly as it would be alone.

A seeded subset of requests is checked after the run against the same simulation in
complex128 (the FP64 path), at full length and over a short horizon while the packet still
holds its norm, reported as rel-L2.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import (DIRAC_C64, DIRAC_C128, Simulation, dirac_batch_active, dirac_batch_create,
               dirac_batch_destroy, dirac_batch_poll, dirac_batch_release, dirac_batch_run,
               dirac_batch_submit, dirac_batch_synchronize, dirac_footprint_bytes)
from . import workloads as W


@dataclass(order=True)
class Request:
    arrival: float
    rid: int  # orders requests that arrive at the same time
    make: Callable[[], "W.Workload"] = field(compare=False)
    nx: int = field(compare=False)
    ny: int = field(compare=False)
    steps: int = field(compare=False)
    check: bool = field(compare=False, default=False)


@dataclass
class Result:
    rid: int
    nx: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    state: Optional[np.ndarray] = None
    workload: Optional["W.Workload"] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """One device-memory budget, one batch, requests admitted between ticks."""

    def __init__(self, budget_bytes: int, precision: int = DIRAC_C64, steps_per_tick: int = 32,
                 stream=None, keep_states: bool = False, policy: str = "fifo",
                 max_active_points: Optional[int] = None):
        if policy not in ("fifo", "sjf"):
            raise ValueError(f"unknown admission policy {policy!r}")
        self.policy = policy
        self.max_active_points = max_active_points
        self.active_points = 0
        self.ready: List = []  # sjf: arrived requests, a heap by (work, arrival)
        self.precision = precision
        self.budget = int(budget_bytes)
        self.used = 0
        self.batch = dirac_batch_create(self.budget, precision, steps_per_tick, stream)
        self.stream = stream
        self.keep_states = keep_states
        self.pending: List[Request] = []
        self.active = {}  # slot -> (request, sim, admitted time)
        self.results: List[Result] = []
        self.ticks = 0
        self.max_active = 0
        self.admitted_while_busy = 0  # admissions into a batch that already had work

    def close(self):
        for _, entry in list(self.active.items()):
            entry[1].close()
        self.active.clear()
        dirac_batch_destroy(self.batch)
        self.batch = None

    def submit(self, req: Request):
        heapq.heappush(self.pending, req)

    def _start(self, req: Request, need: int):
        w = req.make()
        sim = Simulation(w, precision=self.precision, stream=self.stream)
        sim.set_state(w.psi0)
        if self.active:
            self.admitted_while_busy += 1
        slot = dirac_batch_submit(self.batch, sim.ctx, req.steps, w.dt)
        self.used += need
        self.active_points += req.nx * req.ny
        self.active[slot] = (req, sim, time.perf_counter(), w)

    def _admit(self, now: float):
        if self.policy == "fifo":
            while self.pending and self.pending[0].arrival <= now:
                req = self.pending[0]
                need = dirac_footprint_bytes(req.nx, req.ny, self.precision)
                if self.used + need > self.budget:
                    break  # wait for memory; keep arrival order
                heapq.heappop(self.pending)
                self._start(req, need)
            return
        # sjf: the least work first, within the budget and the active-points cap (a request
        # always starts when nothing else runs)
        while self.pending and self.pending[0].arrival <= now:
            req = heapq.heappop(self.pending)
            heapq.heappush(self.ready, (req.nx * req.ny * req.steps, req.arrival, req.rid, req))
        while self.ready:
            req = self.ready[0][3]
            need = dirac_footprint_bytes(req.nx, req.ny, self.precision)
            if self.used + need > self.budget:
                break
            if (self.active and self.max_active_points is not None
                    and self.active_points + req.nx * req.ny > self.max_active_points):
                break
            heapq.heappop(self.ready)
            self._start(req, need)

    def _retire(self):
        for slot in list(self.active):
            if dirac_batch_poll(self.batch, slot):
                req, sim, admitted, w = self.active.pop(slot)
                done = time.perf_counter()
                dirac_batch_release(self.batch, slot)
                state = sim.get_state() if (self.keep_states or req.check) else None
                sim.close()
                self.used -= dirac_footprint_bytes(req.nx, req.ny, self.precision)
                self.active_points -= req.nx * req.ny
                self.results.append(Result(req.rid, req.nx, req.steps, req.arrival, admitted,
                                           done, state, w if req.check else None))

    def run(self, t0: Optional[float] = None, deadline: Optional[float] = None):
        """Serve until every submitted request has finished (arrival times are seconds
        after t0, default now)."""
        if t0 is None:
            t0 = time.perf_counter()
        for r in self.pending:
            r.arrival += t0
        heapq.heapify(self.pending)
        while self.pending or self.ready or self.active:
            now = time.perf_counter()
            if deadline is not None and now - t0 > deadline:
                raise TimeoutError("serving deadline exceeded")
            self._admit(now)
            self.max_active = max(self.max_active, len(self.active))
            if self.active:
                dirac_batch_run(self.batch, 1)
                self.ticks += 1
                self._retire()
            elif self.ready:  # nothing runs and the cheapest ready request does not fit
                raise ValueError(f"request {self.ready[0][2]} does not fit the budget")
            elif self.pending:
                time.sleep(max(0.0, min(0.01, self.pending[0].arrival - now)))
        dirac_batch_synchronize(self.batch)
        return self.results


def graphene_requests(rate=200.0, duration=60.0, seed=1914, sizes=W.SERVE_SIZES,
                      steps_range=(500, 5000), check_fraction=0.01):
    """The strained-graphene request stream: Poisson arrivals, grid from `sizes`,
    steps uniform in `steps_range`, seeded strain and packet per request."""
    reqs = []
    rng = np.random.default_rng(seed + 1)
    for rid, (t, n, steps, s) in enumerate(W.serve_requests(rate, duration, seed, sizes,
                                                            steps_range)):
        reqs.append(Request(t, rid, (lambda n=n, steps=steps, s=s: W.serve_instance(n, steps, s)),
                            n, n, steps, bool(rng.uniform() < check_fraction)))
    return reqs


def latency_summary(results: List[Result]):
    lat = np.array([r.latency for r in results]) * 1e3
    return {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "max_ms": float(lat.max())}


def fp64_check(results: List[Result], stream=None, short_steps: int = 200,
               reference: Optional[Callable] = None):
    """Each checked complex64 result against complex128 (the FP64 path).

    Full length: the served state against the same request run in complex128 -- rel-L2,
    the error relative to the initial norm, and the fraction of the norm the absorbing
    layer left. When the layer has removed nearly all of the wave packet (long requests),
    rel-L2 divides FP32 rounding of the absorbed part by a near-zero residual, so that
    figure is judged by its error against the initial norm.
    Short horizon: the same request over min(steps, short_steps) steps, while the packet
    still holds its norm, in complex64 (alone, which equals the served computation bit for
    bit) against `reference(workload, steps)` if given (e.g. the FP64 CPU oracle), else
    the complex128 path: rel-L2 and the kept norm."""
    out = []
    for r in results:
        if r.workload is None or r.state is None:
            continue
        w = r.workload
        with Simulation(w, precision=DIRAC_C128, stream=stream) as s:
            s.set_state(w.psi0)
            s.step(r.steps, w.dt)
            ref = s.get_state()
        n0 = float(np.linalg.norm(w.psi0))
        kept = float(np.linalg.norm(ref)) / n0
        err0 = float(np.linalg.norm(r.state - ref)) / n0
        k = min(r.steps, short_steps)
        with Simulation(w, precision=DIRAC_C64, stream=stream) as s:
            s.set_state(w.psi0)
            s.step(k, w.dt)
            got_k = s.get_state()
        ref_k, ref_kind = (reference(w, k), "oracle") if reference is not None else (None, None)
        if ref_k is None:
            with Simulation(w, precision=DIRAC_C128, stream=stream) as s:
                s.set_state(w.psi0)
                s.step(k, w.dt)
                ref_k, ref_kind = s.get_state(), "c128"
        out.append({"rid": r.rid, "n": r.nx, "steps": r.steps, "rel_l2": W.rel_l2(r.state, ref),
                    "err_vs_initial_norm": err0, "kept_norm": kept,
                    "short_steps": k, "short_rel_l2": W.rel_l2(got_k, ref_k),
                    "short_kept_norm": float(np.linalg.norm(ref_k)) / n0,
                    "short_reference": ref_kind})
    return out
