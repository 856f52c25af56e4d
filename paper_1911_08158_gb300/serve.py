"""Continuous-batching request loop over the C ABI.

Requests (a grid, a degree, a time step, a number of steps and a source)
arrive over time.  The loop admits them in arrival order while their device
footprint (ads_estimate_bytes) fits the HBM budget, keeps every admitted
simulation's state resident on the device, and advances all live
simulations together with ads_batch_step: scalar-wave simulations of one
precision and degree share one grouped launch per kernel and step,
elasticity steps on its own stream meanwhile.  Each call runs as many steps
as the live simulation closest to completion still needs (at most `chunk`),
so a finished simulation leaves, and its memory returns to the budget, at
the earliest step boundary; requests that arrived meanwhile join the next
call.  Latency is the time from a request's arrival to its result (the
final displacement) being on the host.

The loop itself is plain host logic; the simulation factory, the batch call
and the clock are injectable so it can be exercised without a GPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


def request_dofs(req) -> int:
    """Degrees of freedom of a request: prod(n_elem + p) times components."""
    comps = 3 if req.kind == "elastic" else 1
    return int(np.prod([n + req.p for n in req.n_elem])) * comps


def shard_requests(requests, rank: int, world: int):
    """Requests of one rank when a stream is served by `world` independent
    GPUs (whole simulations per GPU, no communication): greedy assignment in
    arrival order to the rank with the least DOF-steps so far.  Every rank
    computes the same assignment, so the shards are disjoint and cover the
    stream."""
    if world <= 1:
        return list(requests)
    load = [0] * world
    mine = []
    for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        k = min(range(world), key=lambda i: (load[i], i))
        load[k] += request_dofs(r) * int(r.steps)
        if k == rank:
            mine.append(r)
    return mine


def make_simulation(req, precision="fp32"):
    """Library simulation of a request: zero initial state, the request's
    Ricker x Gaussian source (vector direction for elasticity)."""
    from .ads import Simulation
    sim = Simulation(req.n_elem, req.p, req.tau, kind=req.kind, precision=precision)
    sim.set_source(dict(req.source))
    sim.set_gaussian_state(None, None)
    return sim


@dataclass
class Result:
    rid: int
    kind: str
    arrival: float
    admitted: float
    done: float
    dof_steps: int
    state: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Report:
    results: dict = field(default_factory=dict)
    rejected: list = field(default_factory=list)
    makespan: float = 0.0
    peak_bytes: int = 0
    batch_calls: int = 0
    max_live: int = 0

    def latencies(self, kind=None):
        return np.array([r.latency for r in self.results.values() if kind is None or r.kind == kind])

    def summary(self) -> dict:
        lat = self.latencies()
        dof_steps = sum(r.dof_steps for r in self.results.values())
        out = {
            "requests": len(self.results), "rejected": len(self.rejected),
            "makespan_s": self.makespan, "dof_steps": dof_steps,
            "dof_steps_per_s": dof_steps / self.makespan if self.makespan > 0 else 0.0,
            "peak_resident_bytes": self.peak_bytes, "batch_calls": self.batch_calls, "max_live": self.max_live,
        }
        if lat.size:
            out.update(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                       mean_s=float(lat.mean()))
        for kind in ("wave", "elastic"):
            lk = self.latencies(kind)
            if lk.size:
                out["p50_s_" + kind] = float(np.percentile(lk, 50))
                out["p99_s_" + kind] = float(np.percentile(lk, 99))
        return out


class Server:
    """budget_bytes: HBM budget for resident simulations.
    factory(req) -> simulation; batch(sims, k) advances them by k steps;
    estimate(req) -> device bytes; fetch(sim) -> result (syncs);
    close(sim) releases it.  Defaults use the CUDA library."""

    def __init__(self, budget_bytes, precision="fp32", chunk=16, keep_state=False, factory=None, batch=None,
                 estimate=None, fetch=None, close=None, clock=time.perf_counter, sleep=time.sleep):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.keep_state = keep_state
        self.precision = precision
        self.factory = factory or (lambda r: make_simulation(r, precision))
        if batch is None:
            from .ads import batch_step as batch
        self.batch = batch
        if estimate is None:
            from .ads import estimate_bytes

            def estimate(r):
                return estimate_bytes(r.n_elem, r.p, r.kind, precision)
        self.estimate = estimate
        self.fetch = fetch or (lambda sim: sim.get_state(fields=("u",))[0])
        self.close = close or (lambda sim: sim.close())
        self.clock, self.sleep = clock, sleep

    def run(self, requests) -> Report:
        rep = Report()
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        live = []   # [req, sim, steps_left, bytes, t_admit]
        resident = 0
        t0 = self.clock()
        now = lambda: self.clock() - t0   # noqa: E731
        while pending or live:
            t = now()
            # admission in arrival order while the head fits the budget
            while pending and pending[0].arrival <= t:
                r = pending[0]
                need = int(self.estimate(r))
                if need > self.budget:
                    rep.rejected.append(r.rid)
                    pending.popleft()
                    continue
                if resident + need > self.budget:
                    break
                pending.popleft()
                sim = self.factory(r)
                resident += need
                rep.peak_bytes = max(rep.peak_bytes, resident)
                live.append([r, sim, int(r.steps), need, now()])
            if not live:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival - now()))
                continue
            rep.max_live = max(rep.max_live, len(live))
            k = min(self.chunk, min(e[2] for e in live))
            self.batch([e[1] for e in live], k)
            rep.batch_calls += 1
            keep = []
            for e in live:
                e[2] -= k
                if e[2] > 0:
                    keep.append(e)
                    continue
                r, sim, _, need, t_adm = e
                state = self.fetch(sim)
                done = now()
                rep.results[r.rid] = Result(r.rid, r.kind, r.arrival, t_adm, done,
                                            request_dofs(r) * int(r.steps), state if self.keep_state else None)
                self.close(sim)
                resident -= need
            live = keep
        rep.makespan = now()
        return rep
