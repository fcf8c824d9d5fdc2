"""Depth autotuner for plans of a given ion count, order and precision.

The octree depth sets the balance of the step: a deeper tree moves work from
the near field (pairs grow with the leaf occupancy) to the expansions (cells
grow eightfold per level).  For an ion-count band (powers of two) the tuner
times a few steps of a synthetic crystal of that size at the automatic depth
and its neighbours and keeps the fastest; results are cached per
(band, p, precision, batch).  batch = 1 times the crystal alone (latency);
batch > 1 times that many copies advanced together as an ensemble, the
throughput that a batched run of many crystals sees (it favours deeper
trees: their many small launches overlap across crystals).  The leaf size
follows from the depth.  Work items and tile shapes inside a step are sized
by the library itself from the tree it builds (the pair-packed M2L has no
run lengths to choose).
"""
from __future__ import annotations

import math

import torch

from . import Ensemble, Plan, State, make_trap

_cache: dict = {}


def band(n: int) -> int:
    return max(0, int(math.floor(math.log2(max(int(n), 1)))))


def _time_steps(plan, st, trap, dt, steps):
    plan.step(st, trap, None, dt, 2)                 # builds the step graph
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    plan.step_async(st, trap, None, dt, steps)
    b.record()
    torch.cuda.synchronize()
    plan.sync()
    return a.elapsed_time(b) / steps


def _time_batch(plans, states, trap, dt, steps):
    k = len(plans)
    ens = Ensemble(plans)
    ens.step(states, [trap] * k, None, [dt] * k, 2)  # builds the ensemble graph
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    ens.step(states, [trap] * k, None, [dt] * k, steps)
    b.record()
    torch.cuda.synchronize()
    ens.sync()
    ens.close()
    return a.elapsed_time(b) / steps


def tune_depth(n: int, p: int, precision: str, crystal, steps: int = 8, batch: int = 1) -> int:
    """Fastest octree depth for n ions.  crystal(n) -> (pos, vel, q, trap dict,
    dt) builds the synthetic crystal the band is timed on; batch > 1 times
    that many copies stepped together (ensemble throughput)."""
    key = (band(n), int(p), precision, int(batch))
    if key in _cache:
        return _cache[key]
    pos, vel, q, trap, dt = crystal(n)
    tr = make_trap(trap)
    probe = Plan(len(q), p=p, leaf_max=32, depth=-1, precision=precision)
    st = State.from_numpy(pos, vel, q)
    probe.step(st, tr, None, dt, 1)
    d0 = probe.last_depth
    probe.close()
    best, best_ms = d0, float("inf")
    for d in sorted({max(1, d0 - 1), d0, d0 + 1}):
        if batch > 1:
            plans = [Plan(len(q), p=p, leaf_max=32, depth=d, precision=precision)
                     for _ in range(batch)]
            sts = [State.from_numpy(pos, vel, q) for _ in range(batch)]
            ms = _time_batch(plans, sts, tr, dt, steps)
            for pl in plans:
                pl.close()
        else:
            plan = Plan(len(q), p=p, leaf_max=32, depth=d, precision=precision)
            st = State.from_numpy(pos, vel, q)
            ms = _time_steps(plan, st, tr, dt, steps)
            plan.close()
        if ms < best_ms:
            best, best_ms = d, ms
    _cache[key] = best
    return best
