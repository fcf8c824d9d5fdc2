#!/usr/bin/env python
"""Benchmark: ion-steps/s of the FMM + cyclotronic push on a 10,000-ion
spheroidal Penning-trap crystal (aspect 0.3, rigid-rotor density, laser
cooling on: two axial beams and one planar beam), dt = 1 ns, at the
expansion order whose relative RMS force error against the FP64 direct sum
is <= 1e-6 (p = 12; p = 10 stops at about 3e-6 on this crystal, set by the
FMM truncation itself, so its numbers are reported beside the headline).

One benchmark step is one time step of the whole path (drift + root cube,
octree, upward pass, M2L/L2L, L2P + P2P, kick with photon recoils + drift).
Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream, with a 512 MiB write between steps to flush the
129 MB L2 (the inputs are smaller than L2).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|tf32x3|bf16x3|fp64] [--p P] [--p10-steps K10]
                  [--forces N] [--config1-steps K1] [--sweep N1,N2,...]
                  [--ensemble-extra M] [--serve-extra J]

The default line also carries, as extra keys, the 1,000-ion FP64 run
(1,000 steps at p = 8, oracle timed in the same run: "config1") and the
single-evaluation sweep over ion counts, orders and precisions with errors
against the FP64 direct sum ("sweep"), a 256-crystal batched ensemble
(10 steps, "ensemble") and a 24-job serving run ("serving").  --forces N
times only single force
evaluations of the N-ion sweep sphere (--p, --precision) and prints their
line (the command the kernel profiles are taken with).

--impl reference times the FP64 CPU oracle (direct O(N^2) Coulomb sum and
the literal step) on the host cores, one oracle step per benchmark step.
Under torchrun each rank runs an independent replica (no collective on the
data path); the value is the whole job's ion-steps over the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "ion-steps/s (FMM+push), mixed vs FP64 at <=1e-6 force err; p50/p99 latency"
UNIT = "ion-steps/s"
def workload_name(p):
    return f"spheroid aspect 0.3, N=10000, cooling on, p={p}, leaf<=32, dt=1ns"


KERNEL_SOURCES = ("paper_2405_13973_gb300/csrc/m2l_tc.cu",)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernel source changed since the counters were taken."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for src in KERNEL_SOURCES:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    r = rec.get(kernel)
    if not r or r.get("source_sha256") != h.hexdigest():
        return None
    return r
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal per-GPU rates used where no measured peak exists (GB300, 152 SMs):
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # FP32 FMA lanes x 2 flop x max SM clock
FP64_TFLOPS = 1.25                                # nominal dense FP64
TF32_OVER_BF16 = 1.1 / 2.25                       # nominal dense TF32 / BF16 rate


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def launches_per_step(depth: int, precision: str, schedule: str = "tiles") -> int:
    tc = precision in ("tf32x3", "bf16x3")
    # drift + cube, keys, scatter, leaf gather, P2P, L2P, kick; the leaf and
    # cell scans: one launch together while both fit one block (depth <= 5),
    # else three each
    k = 7 + (1 if depth <= 5 else 6)
    if depth >= 2:
        if tc:
            m2m = max(depth - 3, 0)          # P2M covers the leaves and their parents
            k += 1 + 2 * m2m                 # P2M; M2M and its reduction per level
            if schedule == "pairs":          # counts, scans, pairs, M2L, pair reduction
                k += 5 + max(depth - 3, 0)   # (+ one memset node); L2L per level
            else:                            # plan, items, M2L, tile reduction; L2L per level
                k += 4 + max(depth - 3, 0)   # down to the leaves' parents
            k += 1 if precision == "bf16x3" else 0   # split of M into bf16 pieces
        else:
            k += 1 + (depth - 2)             # P2M, M2M per level
            k += depth - 1                   # M2L (+ folded L2L) per level
    return k


def replica_seeds(rank):
    """(crystal seed, photon-stream seed) of an independent replica: every
    rank simulates its own crystal and draws its own photons."""
    return 2 + rank, 1 + rank


def job_rate(local_ms, world, n, steps, dist=None, device="cpu"):
    """Slowest rank's timed milliseconds and the whole job's ion-steps/s
    (every rank advanced its own n ions by `steps` steps)."""
    t = float(local_ms)
    if dist is not None:
        import torch
        tt = torch.tensor([t], device=device, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, world * n * steps / (t * 1e-3)


def run_cpu_baseline(cr, budget_s=12.0, max_steps=30):
    import oracle
    pos, vel, q, tr = cr["pos"], cr["vel"], cr["q"], cr["trap"]
    beams = cr["beams"]
    t0 = time.perf_counter()
    steps = 0
    p, v = pos, vel
    while steps < max_steps and time.perf_counter() - t0 < budget_s:
        p, v = oracle.step(p, v, q, tr, cr["dt"], 1, t0=steps * cr["dt"], step0=steps,
                           beams=beams, gamma0=W.GAMMA0, seed=1, laser_on=True)
        steps += 1
    el = time.perf_counter() - t0
    n = len(q)
    return {"value": n * steps / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{steps} oracle steps of the full N={n} workload (direct O(N^2) FP64 sum, "
                      f"literal step), {el:.1f} s"}


def reference_arm(args, rank):
    if rank != 0:
        return 0
    import oracle
    cr = W.crystal_spheroid_10k()
    pos, vel, q, tr, beams = cr["pos"], cr["vel"], cr["q"], cr["trap"], cr["beams"]
    n = len(q)
    p, v = pos, vel
    for s in range(args.warmup):
        p, v = oracle.step(p, v, q, tr, cr["dt"], 1, t0=s * cr["dt"], step0=s, beams=beams,
                           gamma0=W.GAMMA0, seed=1, laser_on=True)
    t0 = time.perf_counter()
    for s in range(args.steps):
        k = args.warmup + s
        p, v = oracle.step(p, v, q, tr, cr["dt"], 1, t0=k * cr["dt"], step0=k, beams=beams,
                           gamma0=W.GAMMA0, seed=1, laser_on=True)
    el = time.perf_counter() - t0
    val = n * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args.p), "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} oracle steps of the full N={n} workload"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def ensemble_arm(args, rank):
    """Batched ensemble: every crystal its own plan (depth from the autotuner
    for its ion-count band), all advanced by one graph launch per step."""
    line = ensemble_measure(args.ensemble, args.p, args.precision, args.steps, args.warmup, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def ensemble_measure(members, p, precision, steps, warmup, rank=0):
    import torch
    import paper_2405_13973_gb300 as pt
    from paper_2405_13973_gb300 import autotune
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    crs = W.ensemble_crystals(members, seed=17 * rank)

    def crystal(n):
        c = W.ensemble_member(n, 0.3, seed=3, cooling=False)
        return c["pos"], c["vel"], c["q"], c["trap"], c["dt"]

    t_tune = time.perf_counter()
    # depths tuned for ensemble throughput (16 copies of a band's crystal
    # stepped together), not for one crystal's latency
    depths = [autotune.tune_depth(len(c["q"]), p, precision, crystal, batch=16) for c in crs]
    t_tune = time.perf_counter() - t_tune
    plans = [pt.Plan(len(c["q"]), p=p, leaf_max=32, depth=d, precision=precision)
             for c, d in zip(crs, depths)]
    states = [pt.State.from_numpy(c["pos"], c["vel"], c["q"]) for c in crs]
    traps = [pt.make_trap(c["trap"]) for c in crs]
    lasers = [pt.make_laser(c["beams"], seed=1 + k, gamma0=W.GAMMA0) for k, c in enumerate(crs)]
    dts = [c["dt"] for c in crs]
    ens = pt.Ensemble(plans)
    ens.step(states, traps, lasers, dts, warmup)
    ens.sync()
    ions = sum(len(c["q"]) for c in crs)
    flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush_buf.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.step(states, traps, lasers, dts, 1)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ens.sync()
    total = float(sum(ms))
    line = {"metric": "ion-steps/s (batched ensemble of independent crystals)",
            "value": ions * steps / (total * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": total / steps,
            "higher_is_better": True, "dtype": precision, "data": "synthetic",
            "config": {"workload": f"{members} crystals, N log-uniform [100, 20000], "
                                   f"aspect U[0.1, 1], cooling on, p={p}, dt=1ns",
                       "ions": ions, "depths": sorted(set(depths)),
                       "l2": "flushed between timed steps (512 MiB write)"},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "autotune_s": t_tune, "graph_launches_per_step": 1}
    ens.close()
    for pl in plans:
        pl.close()
    del flush_buf
    torch.cuda.empty_cache()
    return line


def serve_arm(args, rank):
    """Serving: jobs with Poisson arrivals (mean args.serve_rate per s), N
    log-uniform in [200, 50000], step counts log-uniform in args.serve_steps,
    random aspect and seeds, cooling on; admitted by device-memory budget,
    continuously batched.  Reports latency percentiles and throughput."""
    line = serve_measure(args.serve, args.serve_rate, args.serve_steps, args.serve_budget_gb,
                         args.p, args.precision, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serve_measure(m, rate, step_range, budget_gb, p, precision, rank=0):
    import torch
    from paper_2405_13973_gb300.serving import Job, Server, report
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rng = np.random.default_rng(101 + rank)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, m))
    ns = np.exp(rng.uniform(math.log(200), math.log(50000), m)).astype(int)
    lo, hi = step_range
    steps = np.exp(rng.uniform(math.log(lo), math.log(hi), m)).astype(int)
    aspects = rng.uniform(0.1, 1.0, m)
    jobs = []
    for k in range(m):
        c = W.ensemble_member(int(ns[k]), float(aspects[k]), seed=1000 + k)
        jobs.append(Job(k, c["pos"], c["vel"], c["q"], c["trap"], c["beams"], 77 + k, c["dt"],
                        int(steps[k]), arrival=float(arrivals[k]), gamma0=W.GAMMA0))
    srv = Server(int(budget_gb * 2**30), p=p, precision=precision,
                 chunk=256)
    t0 = time.perf_counter()
    srv.run(jobs)
    makespan = time.perf_counter() - t0
    rep = report(jobs, makespan)
    line = {"metric": "serving: job latency p50/p99 and aggregate ion-steps/s",
            "value": rep["ion_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "dtype": precision, "data": "synthetic",
            "config": {"workload": f"{m} jobs, Poisson arrivals {rate}/s, N log-uniform "
                                   f"[200, 50000], steps log-uniform [{lo:g}, {hi:g}], aspect "
                                   f"U[0.1, 1], cooling on, p={p}, dt=1ns",
                       "hbm_budget_gb": budget_gb},
            "latency_s": {"p50": rep["p50_s"], "p99": rep["p99_s"], "max": rep["max_s"]},
            "makespan_s": makespan, "ion_steps": rep["ion_steps"],
            "peak_admitted_gb": srv.peak_bytes / 2**30, "graph_recaptures": srv.recaptures,
            "chunks": srv.chunks}
    return line


def sweep_reference(pt, torch, w, n_sample=512):
    """FP64 reference field of a sweep sphere: the GPU direct sum (pinned to
    the oracle's to 1e-13) up to 1e5 ions, else the oracle's direct sum at a
    seeded sample of n_sample ions.  Returns (E_ref (n_s, 3), sample index or
    None, what)."""
    pos, q = w["pos"], w["q"]
    n = len(q)
    if n <= 100000:
        pd = torch.tensor(np.ascontiguousarray(pos.T), dtype=torch.float64, device="cuda")
        qd = torch.tensor(q, dtype=torch.float64, device="cuda")
        E, _ = pt.direct(pd, qd, want_phi=False)
        return E.cpu().numpy().T, None, "FP64 GPU direct sum, every ion"
    import oracle
    idx = np.sort(np.random.default_rng(7).choice(n, n_sample, replace=False))
    Eo, _ = oracle.coulomb_targets(pos, q, idx, want_phi=False)
    return Eo, idx, f"FP64 oracle direct sum at {n_sample} sampled ions"


def m2l_peak(precision, pk, pk_src):
    """Roof of the M2L kernel for a precision: (peak TFLOP/s of FP32-accurate
    (or FP64) products, bound, note)."""
    if precision == "tf32x3":
        return (pk["bf16_tflops"] * TF32_OVER_BF16 / 3.0, "tensor",
                f"TF32 rate / 3 (3 products per FP32-accurate product), from {pk_src} bf16 x "
                f"nominal ratio")
    if precision == "bf16x3":
        return (pk["bf16_tflops"] / 6.0, "tensor",
                f"{pk_src} bf16 rate / 6 (6 products per FP32-accurate product)")
    if precision == "fp32":
        return FP32_ALU_TFLOPS, "alu", "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
    return FP64_TFLOPS, "alu", "nominal dense FP64"


def force_eval_point(pt, torch, w, p, precision, steps, flush, ref=None, warmup=1, schedule=""):
    """Single force evaluations (config-3 sweep point): mean CUDA-event time
    of `steps` evaluations (L2 flushed before each) and the relative RMS force
    error against ref."""
    pos, q = w["pos"], w["q"]
    n = len(q)
    pd = torch.tensor(np.ascontiguousarray(pos.T), dtype=torch.float64, device="cuda")
    qd = torch.tensor(q, dtype=torch.float64, device="cuda")
    try:
        plan = pt.Plan(n, p=p, leaf_max=32, depth=-1, precision=precision)
        if schedule:
            plan.set_m2l_schedule(schedule)
    except pt.PenningError as exc:
        return {"status": str(exc)}
    E = torch.empty((3, n), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        plan.forces(pd, qd, E=E, want_phi=False)
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.forces(pd, qd, E=E, want_phi=False)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    out = {"ms": float(np.mean(ms)), "evals_per_s": 1e3 / float(np.mean(ms)),
           "ion_evals_per_s": n * 1e3 / float(np.mean(ms)), "depth": plan.last_depth}
    out["m2l_schedule"] = plan.m2l_schedule
    # the M2L kernel alone in one more, profiled evaluation: its rate in
    # 2 P^2 flop per (target, source) translation against its roof
    try:
        plan.profile(True)
        flush()
        plan.forces(pd, qd, E=E, want_phi=False)
        torch.cuda.synchronize()
        kms = plan.kernel_times()["m2l_kernel"]
        pairs = plan.stats()["m2l_pairs"]
        if kms > 0 and pairs > 0:
            pk, pk_src = peaks()
            peak, bound, _ = m2l_peak(precision, pk, pk_src)
            if plan.m2l_schedule == "rotation":
                # rotate to the z axis, translate along z, rotate back:
                # 2 sum_n (2n+1)^2 + sum_m (p+1-m)^2 (twice for m > 0) multiply-adds
                macs = (2 * sum((2 * k + 1) ** 2 for k in range(p + 1)) +
                        sum((p + 1 - m) ** 2 * (1 if m == 0 else 2) for m in range(p + 1)))
                work = "2 x rotation multiply-adds per translation"
            else:
                macs = (p + 1) ** 4
                work = "2 P^2 per translation"
            rate = 2.0 * macs * pairs / (kms * 1e-3) / 1e12
            out["m2l_kernel"] = {"ms": kms, "tflops": rate, "peak": peak, "frac": rate / peak,
                                 "bound": bound, "m2l_pairs": pairs, "work": work}
    except pt.PenningError:
        pass
    finally:
        plan.profile(False)
    if ref is not None:
        Er, idx, _ = ref
        e = E.cpu().numpy().T
        if idx is not None:
            e = e[idx]
        out["force_err"] = float(np.sqrt(((e - Er) ** 2).sum() / (Er ** 2).sum()))
    plan.close()
    return out


def sweep_arm(pt, torch, ns, ps, precisions, flush, steps=2):
    """Config-3 sweep: N uniform in a sphere at 2e14 m^-3 plus 1% jitter, one
    force evaluation per point, errors against sweep_reference."""
    res = {}
    for n in ns:
        w = W.sphere_sweep(n)
        ref = sweep_reference(pt, torch, w)
        row = {"reference": ref[2]}
        for p in ps:
            for prec in precisions:
                k = steps if n <= 100000 or prec != "fp64" else 1
                row[f"{prec}_p{p}"] = force_eval_point(pt, torch, w, p, prec, k, flush, ref)
        res[str(n)] = row
        torch.cuda.empty_cache()
    return res


def config1_arm(pt, torch, steps, flush, with_oracle=True):
    """Config 1: N = 1,000 uniform in a 100 um sphere, rotating 10 mK
    Maxwellian, FP64, p = 8, leaf <= 32, dt = 1 ns, cooling off; `steps`
    steps timed on the GPU (one replayed step graph per step) beside the same
    steps of the FP64 oracle on the host cores.  Checked: the initial force
    error against the oracle's direct sum and the energies of the two final
    states (Error_en, Eq. rms_en)."""
    import oracle
    cr = W.crystal_sphere_1k()
    pos, vel, q, tr = cr["pos"], cr["vel"], cr["q"], cr["trap"]
    n = len(q)
    plan = pt.Plan(n, p=8, leaf_max=32, depth=-1, precision="fp64")
    pd = torch.tensor(np.ascontiguousarray(pos.T), dtype=torch.float64, device="cuda")
    qd = torch.tensor(q, dtype=torch.float64, device="cuda")
    E, _ = plan.forces(pd, qd, want_phi=False)
    Eo, _ = oracle.coulomb_direct(pos, q, want_phi=False)
    ferr = float(np.sqrt(((E.cpu().numpy().T - Eo) ** 2).sum() / (Eo ** 2).sum()))
    st = pt.State.from_numpy(pos, vel, q)
    trap = pt.make_trap(tr)
    plan.step(st, trap, None, cr["dt"], 1)       # captures the step graph
    st = pt.State.from_numpy(pos, vel, q)
    flush()
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.step_async(st, trap, None, cr["dt"], steps)
    b.record(stream)
    b.synchronize()
    plan.sync()
    ms = a.elapsed_time(b)
    out = {"workload": f"sphere 100 um, N={n}, FP64, p=8, leaf<=32, dt=1ns, cooling off, "
                       f"{steps} steps", "value": n * steps / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms / steps, "force_err_vs_oracle": ferr, "depth": plan.last_depth}
    if with_oracle:
        t0 = time.perf_counter()
        po, vo = oracle.step(pos, vel, q, tr, cr["dt"], steps)
        el = time.perf_counter() - t0
        eg = pt.energy(st, trap)[3]
        eo = oracle.energy_rot(po, vo, q, tr, steps * cr["dt"])[3]
        out["oracle"] = {"value": n * steps / el, "unit": UNIT, "cores": oracle.num_threads(),
                         "seconds": el, "kind": "oracle (direct O(N^2) FP64 sum, literal step)"}
        out["error_en"] = abs(eg - eo) / abs(eo)
        out["max_pos_diff_m"] = float(np.abs(st.pos().cpu().numpy() - po).max())
    plan.close()
    return out


def forces_arm(args):
    """Only single force evaluations of the N-ion sweep sphere (one JSON line)."""
    import torch
    import paper_2405_13973_gb300 as pt
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        flush_buf.fill_(1.0)
    w = W.sphere_sweep(args.forces)
    ref = sweep_reference(pt, torch, w) if not args.no_ref else None
    r = force_eval_point(pt, torch, w, args.p, args.precision, args.steps, flush, ref,
                         warmup=args.warmup, schedule=args.schedule)
    line = {"metric": "single force evaluations/s (sweep sphere, 2e14 m^-3)",
            "value": r.get("evals_per_s"), "unit": "evaluations/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"sphere N={args.forces}, 2e14 m^-3 + 1% jitter, p={args.p}",
                       "l2": "flushed between timed evaluations (512 MiB write)"},
            "result": r, "reference": ref[2] if ref else None}
    print(json.dumps(line), flush=True)
    return 0


def timed_steps(pt, torch, plan, st, trap, laser, dt, K, flush, profile=True, kernels=False):
    """K single steps, each timed with CUDA events, L2 flushed in between."""
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    phases = []
    for k in range(K):
        flush()
        ev[k][0].record(stream)
        plan.step_async(st, trap, laser, dt, 1)
        ev[k][1].record(stream)
        if profile:
            ev[k][1].synchronize()
            ph = plan.phase_times()
            if kernels:
                ph.update(plan.kernel_times())
            phases.append(ph)
    torch.cuda.synchronize()
    plan.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, phases


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "tf32x3", "bf16x3", "fp64"])
    ap.add_argument("--p", type=int, default=12)
    ap.add_argument("--p10-steps", type=int, default=20)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", type=int, default=0,
                    help="serving measurement with this many Poisson-arriving jobs instead of the "
                         "single-crystal step")
    ap.add_argument("--serve-rate", type=float, default=50.0, help="mean arrivals per second")
    ap.add_argument("--serve-steps", type=float, nargs=2, default=[100.0, 10000.0],
                    help="job step counts, log-uniform in this range")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--ensemble", type=int, default=0,
                    help="batched-ensemble measurement with this many crystals instead of the "
                         "single-crystal step (N log-uniform in [100, 20000], aspect 0.1-1)")
    ap.add_argument("--no-mirror", action="store_true",
                    help="BF16x3 pair schedule without offset mirroring (offsets o and -o in "
                         "runs of their own)")
    ap.add_argument("--schedule", default="", choices=["", "tiles", "pairs", "rotation"],
                    help="M2L schedule (default: the library's for the plan)")
    ap.add_argument("--forces", type=int, default=0,
                    help="only single force evaluations of this many ions (sweep sphere)")
    ap.add_argument("--no-ref", action="store_true", help="--forces without the error reference")
    ap.add_argument("--config1-steps", type=int, default=1000,
                    help="steps of the 1,000-ion FP64 run carried by the default line (0: skip)")
    ap.add_argument("--ensemble-extra", type=int, default=256,
                    help="crystals of the ensemble run carried by the default line (0: skip)")
    ap.add_argument("--serve-extra", type=int, default=24,
                    help="jobs of the serving run carried by the default line (0: skip)")
    ap.add_argument("--sweep", default="10000,100000,1000000",
                    help="ion counts of the single-evaluation sweep in the default line ('' skips)")
    args = ap.parse_args()
    if args.forces > 0:
        return forces_arm(args)
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)
    if args.ensemble > 0:
        return ensemble_arm(args, rank)
    if args.serve > 0:
        return serve_arm(args, rank)

    import torch
    import paper_2405_13973_gb300 as pt

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    crystal_seed, photon_seed = replica_seeds(rank)
    cr = W.crystal_spheroid_10k(seed=crystal_seed)
    n = len(cr["q"])
    trap = pt.make_trap(cr["trap"])
    laser = pt.make_laser(cr["beams"], seed=photon_seed, gamma0=W.GAMMA0)
    dt = cr["dt"]
    flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        flush_buf.fill_(1.0)

    # force error of this precision at the initial state vs the FP64 GPU direct sum
    st0 = pt.State.from_numpy(cr["pos"], cr["vel"], cr["q"])
    pos0 = torch.stack([st0.x, st0.y, st0.z]).contiguous()
    Ed, _ = pt.direct(pos0, st0.q, want_phi=False)

    def force_err(plan):
        E, _ = plan.forces(pos0, st0.q, want_phi=False)
        return float(torch.sqrt(((E - Ed) ** 2).sum() / (Ed ** 2).sum()))

    def force_err_oracle(plan):
        """Err_F of the plan's field against the FP64 CPU oracle's direct sum."""
        import oracle
        Eo, _ = oracle.coulomb_direct(cr["pos"], cr["q"], want_phi=False)
        E, _ = plan.forces(pos0, st0.q, want_phi=False)
        e = E.cpu().numpy().T
        return float(np.sqrt(((e - Eo) ** 2).sum() / (Eo ** 2).sum()))

    plan = pt.Plan(n, p=args.p, leaf_max=32, depth=-1, precision=args.precision)
    if args.schedule and args.precision in ("tf32x3", "bf16x3"):
        plan.set_m2l_schedule(args.schedule)
    if args.no_mirror and args.precision == "bf16x3":
        plan.set_m2l_mirror(False)
    schedule = plan.m2l_schedule if args.precision in ("tf32x3", "bf16x3") else "cuda-core"
    ferr = force_err(plan)
    ferr_oracle = force_err_oracle(plan) if rank == 0 and not args.no_cpu else None
    st = pt.State.from_numpy(cr["pos"], cr["vel"], cr["q"])
    plan.profile(False)
    plan.step(st, trap, laser, dt, args.warmup)           # warm-up; chooses the depth
    depth = plan.last_depth
    stats = plan.stats()
    tc = plan.tc_stats()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall = time.perf_counter()
    ms, _ = timed_steps(pt, torch, plan, st, trap, laser, dt, args.steps, flush, profile=False)
    t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms, value = job_rate(sum(ms), world, n, args.steps, dist, "cuda")
    ms_per_step = total_ms / args.steps

    # phase breakdown: a second pass of K steps with event records between the
    # phases captured into the step graph (they cost the pass ~25 us a step,
    # so the headline above is timed without them)
    plan.profile(True)
    plan.step(st, trap, laser, dt, 1)                     # recaptures with the events
    ms_prof, phases = timed_steps(pt, torch, plan, st, trap, laser, dt, args.steps, flush,
                                  kernels=True)
    plan.profile(False)

    # phase breakdown and the roofline of the dominant kernel
    ph = {k: float(np.mean([p[k] for p in phases])) for k in phases[0]}
    kern = {k: ph.pop(k) for k in ("m2l_kernel", "p2p_kernel") if k in ph}
    P = (args.p + 1) ** 2
    m2l_flops = 2.0 * P * P * (stats["m2l_pairs"] + stats["l2l_shifts"])
    p2p_flops = 20.0 * stats["p2p_pairs"]
    pk, pk_src = peaks()
    dom = max(ph, key=ph.get)
    roof = {"kernel": dom, "phases_ms": ph, "kernels_ms": kern,
            "phases_pass_ms_per_step": float(np.mean(ms_prof))}
    if dom == "m2l":
        # the dominant kernel: the M2L launch alone (events right before and
        # after it, in the profiled pass); the phase (split, M2L, reduction,
        # L2L) beside it
        m2l_only = 2.0 * P * P * stats["m2l_pairs"]
        achieved = m2l_only / (kern["m2l_kernel"] * 1e-3) / 1e12
        roof["kernel"] = "M2L kernel (k_m2l_tc)" if args.precision in ("tf32x3", "bf16x3") \
            else "M2L kernels (k_m2l_simt, all levels)"
        roof["kernel_ms"] = kern["m2l_kernel"]
        roof["phase_achieved"] = m2l_flops / (ph["m2l"] * 1e-3) / 1e12
        peak, bound, note = m2l_peak(args.precision, pk, pk_src)
        roof.update(bound=bound, peak_note=note)
        roof.update(achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                    work=f"2 P^2 x {stats['m2l_pairs']} M2L translations per launch",
                    phase_frac=roof["phase_achieved"] / peak,
                    phase_work=f"2 P^2 x ({stats['m2l_pairs']} M2L + {stats['l2l_shifts']} L2L) "
                               f"flop")
        if tc["products"]:
            # what the tensor cores execute: 128-row products of the work list
            roof["tensor_work"] = dict(tc, row_fill=stats["m2l_pairs"] / (128.0 * tc["products"]))
    elif dom == "near_far":
        achieved = p2p_flops / (ph["near_far"] * 1e-3) / 1e12
        peak = FP32_ALU_TFLOPS if args.precision != "fp64" else FP64_TFLOPS
        roof.update(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                    frac=achieved / peak, work=f"20 flop x {stats['p2p_pairs']} P2P pairs")
    else:
        # HBM-bound phase: algorithmic bytes of the state pass (x, v read+write)
        byts = 96.0 * n
        achieved = byts / (ph[dom] * 1e-3) / 1e9
        roof.update(bound="hbm", achieved=achieved, peak=pk["hbm_gbs"], unit="GB/s",
                    frac=achieved / pk["hbm_gbs"], work="96 B per ion")
    mirrored = schedule == "pairs" and args.precision == "bf16x3" and not args.no_mirror
    tr = recorded_traffic(f"k_m2l_tc:{args.precision}:p{args.p}:{schedule}"
                          f"{':mirrored' if mirrored else ''}") if dom == "m2l" else None
    roof["traffic"] = tr["dram_bytes_per_launch"] if tr else None
    if tr:
        roof["traffic_note"] = tr["note"]
    roof["peak_source"] = pk_src

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "tf32x3": "tf32x3", "bf16x3": "bf16x3",
                                                             "fp64": "f64"}[args.precision],
           "data": "synthetic",
           "config": {"workload": workload_name(args.p), "precision": args.precision, "p": args.p,
                      "depth": depth, "n": n, "m2l_schedule": schedule,
                      "m2l_mirrored_offsets": mirrored,
                      "l2": "flushed between timed steps (512 MiB write)",
                      "parallelism": "replicas" if world > 1 else "single"},
           "force_err": ferr, "force_err_note": "relative RMS vs the FP64 GPU direct sum, initial state",
           "force_err_vs_oracle": ferr_oracle,
           "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                          "max": float(max(ms))},
           "stats": stats, "roofline": roof, "clocks": clk,
           "gpu_launches": launches_per_step(depth, args.precision, schedule) * args.steps,
           "wall_s_timed_region": t_wall}

    # the plain FP64 GPU path beside it (same workload, fewer steps)
    if rank == 0 and args.precision != "fp64" and args.fp64_steps > 0:
        plan64 = pt.Plan(n, p=args.p, leaf_max=32, depth=-1, precision="fp64")
        e64 = force_err(plan64)
        st64 = pt.State.from_numpy(cr["pos"], cr["vel"], cr["q"])
        plan64.step(st64, trap, laser, dt, 3)
        ms64, _ = timed_steps(pt, torch, plan64, st64, trap, laser, dt, args.fp64_steps, flush,
                              profile=False)
        out["fp64_path"] = {"value": n * args.fp64_steps / (sum(ms64) * 1e-3),
                            "ms_per_step": sum(ms64) / args.fp64_steps, "force_err": e64,
                            "depth": plan64.last_depth, "m2l_schedule": plan64.m2l_schedule}
        plan64.close()

    # order p = 10 beside the headline (both tensor-core operand formats)
    if rank == 0 and args.p10_steps > 0 and args.p != 10:
        p10 = {}
        for prec in ("bf16x3", "tf32x3"):
            pl = pt.Plan(n, p=10, leaf_max=32, depth=-1, precision=prec)
            e10 = force_err(pl)
            s10 = pt.State.from_numpy(cr["pos"], cr["vel"], cr["q"])
            pl.step(s10, trap, laser, dt, 3)
            m10, _ = timed_steps(pt, torch, pl, s10, trap, laser, dt, args.p10_steps, flush,
                                 profile=False)
            p10[prec] = {"value": n * args.p10_steps / (sum(m10) * 1e-3),
                         "ms_per_step": sum(m10) / args.p10_steps, "force_err": e10,
                         "depth": pl.last_depth}
            pl.close()
        out["p10"] = p10

    # config 1 (1,000 ions, FP64, p = 8) and the single-evaluation sweep
    if rank == 0 and args.config1_steps > 0:
        out["config1"] = config1_arm(pt, torch, args.config1_steps, flush,
                                     with_oracle=not args.no_cpu)
    if rank == 0 and args.sweep:
        ns = [int(float(x)) for x in args.sweep.split(",") if x]
        out["sweep"] = {"workload": "sphere at 2e14 m^-3 + 1% jitter, one force evaluation, "
                                    "leaf<=32, automatic depth",
                        "points": sweep_arm(pt, torch, ns, (4, 6, 8, 10, 12, 16),
                                            ("fp64", "fp32", "bf16x3"), flush)}

    # batched ensemble and serving, each a short run of its own measurement
    if rank == 0 and args.ensemble_extra > 0:
        out["ensemble"] = ensemble_measure(args.ensemble_extra, args.p, args.precision, 10, 3)
    if rank == 0 and args.serve_extra > 0:
        out["serving"] = serve_measure(args.serve_extra, 50.0, (100.0, 2000.0), 40.0, args.p,
                                       args.precision)

    # end to end through the public API: every step copies the state in from
    # pinned host memory, advances it (pt_step_async) and copies it back; the
    # six state arrays are rows of one buffer on each side, one copy each way
    if not args.no_e2e:
        host = torch.empty((6, n), dtype=torch.float64).pin_memory()
        host.copy_(torch.from_numpy(np.ascontiguousarray(
            np.concatenate([cr["pos"].T, cr["vel"].T]))))
        devbuf = torch.empty((6, n), dtype=torch.float64, device="cuda")
        ste = pt.State(*[devbuf[k] for k in range(6)],
                       torch.tensor(cr["q"], dtype=torch.float64, device="cuda"), 0.0, 0)
        devbuf.copy_(host)
        plan.step(ste, trap, laser, dt, 1)
        host.copy_(devbuf)
        torch.cuda.synchronize()
        el = 0.0
        for _ in range(args.steps):
            flush()                    # L2 flushed between steps, outside the timed span
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            devbuf.copy_(host, non_blocking=True)
            plan.step_async(ste, trap, laser, dt, 1)
            host.copy_(devbuf, non_blocking=True)
            torch.cuda.synchronize()
            el += time.perf_counter() - t0
        plan.sync()  # device errors latched by the steps
        if dist:
            tt = torch.tensor([el], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        out["e2e"] = {"value": world * n * args.steps / el, "unit": UNIT,
                      "h2d_bytes_per_step": 48 * n, "d2h_bytes_per_step": 48 * n,
                      "l2": "flushed between steps, outside the timed spans"}

    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = run_cpu_baseline(cr)
    plan.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
