"""Serving crystal simulations: a request loop with continuous batching.

Jobs (a crystal, its trap and lasers, a step count) arrive over time.  The
server admits an arrived job as soon as its device memory fits the budget
(first fit in arrival order, so a large job waiting for room does not hold
back smaller ones behind it), keeps every admitted job's plan (octree,
expansions, work list) and state resident, and advances all admitted jobs
together through one ensemble graph per step, in chunks that end at the
nearest completion.  A finished job's state is copied to the host and its
memory returned; jobs that arrived meanwhile are admitted before the next
chunk.  Each job's result equals the job run alone, bit for bit: the kernels
are deterministic and the jobs share only the device.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import Ensemble, Plan, State, make_laser, make_trap, plan_footprint


@dataclass
class Job:
    """One simulation request (host arrays, SI units)."""
    id: int
    pos: np.ndarray
    vel: np.ndarray
    q: np.ndarray
    trap: dict
    beams: list
    seed: int
    dt: float
    n_steps: int
    arrival: float = 0.0          # s after the server starts
    gamma0: float | None = None
    # filled in by the server
    admitted: float = -1.0
    done: float = -1.0
    bytes: int = 0
    result: tuple | None = None
    remaining: int = field(default=0, repr=False)
    _plan: Plan | None = field(default=None, repr=False)
    _state: State | None = field(default=None, repr=False)

    @property
    def n(self) -> int:
        return len(self.q)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def first_fit(waiting, used, budget, slots):
    """Indices of the waiting jobs (arrival order) admitted under a memory
    budget and a slot count: each job is taken if it still fits."""
    take = []
    for i, (need, _) in enumerate(waiting):
        if slots <= 0:
            break
        if used + need <= budget:
            take.append(i)
            used += need
            slots -= 1
    return take


class Server:
    def __init__(self, hbm_budget: int, p: int = 12, precision: str = "bf16x3",
                 max_active: int = 64, chunk: int = 256, leaf_max: int = 32):
        self.budget = int(hbm_budget)
        self.p, self.precision = int(p), precision
        self.max_active, self.chunk, self.leaf_max = int(max_active), int(chunk), int(leaf_max)
        self.peak_bytes = 0
        self.recaptures = 0
        self.chunks = 0

    # device pages are granted in 2 MB units: a plan's some thirty buffers end
    # up to a few MB above their summed sizes (measured: +0.1 to +8 MB)
    PAGE_SLACK = 8 << 20

    def footprint(self, job: Job) -> int:
        plan_b, _ = plan_footprint(job.n, self.p, self.leaf_max, -1, self.precision)
        # plan workspace + state (7 FP64 arrays) + page rounding
        return plan_b + 56 * job.n + self.PAGE_SLACK

    def _admit(self, job: Job, now: float):
        job._plan = Plan(job.n, p=self.p, leaf_max=self.leaf_max, depth=-1,
                         precision=self.precision)
        job._state = State.from_numpy(job.pos, job.vel, job.q)
        job.remaining = int(job.n_steps)
        job.admitted = now

    def _finish(self, job: Job, now: float):
        st = job._state
        job.result = (st.pos().cpu().numpy(), st.vel().cpu().numpy(), st.t, st.step)
        job.done = now
        job._plan.close()
        job._plan = job._state = None

    def run(self, jobs, clock=time.perf_counter):
        """Serve jobs (their .arrival in s from now) to completion; returns them."""
        pending = sorted(jobs, key=lambda j: (j.arrival, j.id))
        for j in pending:
            j.bytes = self.footprint(j)
            if j.bytes > self.budget:
                raise ValueError(f"job {j.id} needs {j.bytes} B, more than the budget")
        _, op_bytes = plan_footprint(1, self.p, self.leaf_max, -1, self.precision)
        budget = self.budget - op_bytes           # the shared operators, held once
        active: list[Job] = []
        used = 0
        ens, ens_members = None, None
        t0 = clock()
        while pending or active:
            now = clock() - t0
            arrived = [j for j in pending if j.arrival <= now]
            take = first_fit([(j.bytes, j) for j in arrived], used, budget,
                             self.max_active - len(active))
            for i in take:
                j = arrived[i]
                self._admit(j, now)
                used += j.bytes
                active.append(j)
                pending.remove(j)
            self.peak_bytes = max(self.peak_bytes, used + (op_bytes if active else 0))
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - now)))
                continue
            ids = [j.id for j in active]
            if ids != ens_members:
                if ens is not None:
                    ens.close()
                ens = Ensemble([j._plan for j in active])
                ens_members = ids
                self.recaptures += 1
            k = min(self.chunk, min(j.remaining for j in active))
            ens.step([j._state for j in active], [make_trap(j.trap) for j in active],
                     [make_laser(j.beams, seed=j.seed, gamma0=j.gamma0) for j in active],
                     [j.dt for j in active], k)
            ens.sync()
            self.chunks += 1
            now = clock() - t0
            for j in list(active):
                j.remaining -= k
                if j.remaining == 0:
                    self._finish(j, now)
                    used -= j.bytes
                    active.remove(j)
        if ens is not None:
            ens.close()
        torch.cuda.synchronize()
        return jobs


def report(jobs, makespan: float) -> dict:
    lat = np.array([j.latency for j in jobs])
    work = float(sum(j.n * j.n_steps for j in jobs))
    return {"jobs": len(jobs), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "max_s": float(lat.max()),
            "ion_steps": work, "ion_steps_per_s": work / makespan, "makespan_s": makespan}
