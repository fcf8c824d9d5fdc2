"""The serving loop on the GPU: jobs arriving over time under a memory budget
that holds only some of them at once are admitted as room frees up, advance
together, and each ends exactly where the same job run alone ends."""
import numpy as np
import pytest
import torch

import paper_2405_13973_gb300 as pt
import workloads as W
from paper_2405_13973_gb300.serving import Job, Server, report

pytestmark = pytest.mark.gpu


def make_jobs():
    spec = [(400, 0.5, 40, 0.00), (1500, 0.3, 25, 0.00), (250, 1.0, 60, 0.01),
            (2500, 0.2, 30, 0.02), (800, 0.7, 20, 0.03), (300, 0.9, 35, 0.05)]
    jobs = []
    for k, (n, a, steps, t) in enumerate(spec):
        c = W.ensemble_member(n, a, seed=40 + k)
        jobs.append(Job(k, c["pos"], c["vel"], c["q"], c["trap"], c["beams"], 9 + k, c["dt"],
                        steps, arrival=t, gamma0=W.GAMMA0))
    return jobs


def alone(job, p, precision):
    plan = pt.Plan(job.n, p=p, depth=-1, precision=precision)
    st = pt.State.from_numpy(job.pos, job.vel, job.q)
    plan.step(st, pt.make_trap(job.trap), pt.make_laser(job.beams, seed=job.seed, gamma0=job.gamma0),
              job.dt, job.n_steps)
    out = (st.pos().cpu().numpy(), st.vel().cpu().numpy())
    plan.close()
    return out


@pytest.mark.parametrize("precision,p", [("fp64", 6), ("bf16x3", 8)])
def test_each_job_alone_equals_the_job_in_the_mix(precision, p):
    jobs = make_jobs()
    srv = Server(hbm_budget=0, p=p, precision=precision, chunk=16)
    need = [srv.footprint(j) for j in jobs]
    _, ops = pt.plan_footprint(1, p, precision=precision)
    srv.budget = ops + sorted(need)[-1] + sorted(need)[-2]   # room for about two jobs
    done = srv.run(jobs)
    assert all(j.result is not None and j.done >= j.admitted >= j.arrival for j in done)
    assert srv.peak_bytes <= srv.budget
    assert srv.recaptures >= 3        # the mix changed as jobs came and went
    for j in done:
        x, v = alone(j, p, precision)
        assert j.result[3] == j.n_steps
        assert np.array_equal(j.result[0], x) and np.array_equal(j.result[1], v)
    rep = report(done, max(j.done for j in done))
    assert rep["p99_s"] >= rep["p50_s"] > 0


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_footprint_matches_device_memory(precision):
    # a second plan of one kind (the operators already shared) takes the
    # reported workspace, up to the 2 MB page rounding of its buffers
    torch.cuda.synchronize()
    first = pt.Plan(20000, p=12, precision=precision)
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    second = pt.Plan(20000, p=12, precision=precision)
    torch.cuda.synchronize()
    delta = before - torch.cuda.mem_get_info()[0]
    need, _ = pt.plan_footprint(20000, 12, precision=precision)
    assert need - (4 << 20) <= delta <= need + Server.PAGE_SLACK
    first.close()
    second.close()
