"""Diagnostics and the damped step on the GPU against the oracle.

Temperatures: FP64 compensated sums on both sides (relative 1e-12).  Damped
steps at depth 1 (every pair in the near field, so the GPU field is the
direct sum up to rounding order) follow the oracle's damped step to 1e-9
over 40 steps; damping 0 leaves the step bit for bit unchanged.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2405_13973_gb300 as pt
import workloads as W

pytestmark = pytest.mark.gpu


def test_temperatures_match_the_oracle():
    tr = W.trap(beta=1.0)
    pos = W.sphere(2000, 100e-6, 6)
    vel = W.rotating_maxwellian(pos, tr["omega_r"], 7e-3, 7)
    st = pt.State.from_numpy(pos, vel, W.charges(2000))
    got = pt.temperatures(st, tr)
    want = oracle.temperatures(pos, vel, tr)
    assert all(math.isclose(a, b, rel_tol=1e-12) for a, b in zip(got, want))


def test_damped_steps_follow_the_oracle():
    cr = W.crystal_sphere_1k(seed=12)
    n = 300
    pos, vel, q, tr = cr["pos"][:n], cr["vel"][:n], cr["q"][:n], cr["trap"]
    plan = pt.Plan(n, p=4, depth=1, precision="fp64")
    plan.set_damping(1e6)
    st = pt.State.from_numpy(pos, vel, q)
    plan.step(st, tr, None, 1e-9, 40)
    po, vo = oracle.step(pos, vel, q, tr, 1e-9, 40, damping=1e6)
    x, v = st.pos().cpu().numpy(), st.vel().cpu().numpy()
    assert np.abs(x - po).max() < 1e-9 * np.abs(po).max()
    assert np.abs(v - vo).max() < 1e-9 * np.abs(vo).max()
    # damping off again: the plain step, bit for bit
    plan.set_damping(0.0)
    a = pt.State.from_numpy(pos, vel, q)
    plan.step(a, tr, None, 1e-9, 5)
    plain = pt.Plan(n, p=4, depth=1, precision="fp64")
    b = pt.State.from_numpy(pos, vel, q)
    plain.step(b, tr, None, 1e-9, 5)
    assert torch.equal(a.pos(), b.pos()) and torch.equal(a.vel(), b.vel())
    plan.close()
    plain.close()


def test_position_moments_and_rms():
    tr = W.trap(beta=1.0)
    pos = W.sphere(500, 80e-6, 9)
    vel = W.rotating_maxwellian(pos, tr["omega_r"], 5e-3, 10)
    q = W.charges(500)
    plan = pt.Plan(500, p=6, precision="fp64")
    st = pt.State.from_numpy(pos, vel, q)
    acc = torch.zeros((4, 500), dtype=torch.float64, device="cuda")
    snaps = []
    for _ in range(3):
        plan.step(st, tr, None, 1e-9, 7)
        pt.position_moments(st, tr, acc)
        c, s = math.cos(tr["omega_r"] * st.t), math.sin(tr["omega_r"] * st.t)
        p = st.pos().cpu().numpy()
        snaps.append(np.stack([c * p[:, 0] - s * p[:, 1], s * p[:, 0] + c * p[:, 1], p[:, 2]], 1))
    snaps = np.array(snaps)                          # (3, n, 3)
    a = acc.cpu().numpy()
    assert np.allclose(a[:3].T, snaps.sum(0), rtol=1e-13, atol=0)
    assert np.allclose(a[3], (snaps ** 2).sum((0, 2)), rtol=1e-13, atol=0)
    want = np.sqrt(((snaps - snaps.mean(0)) ** 2).sum(2).mean(0))
    got = pt.rms_displacement(acc, 3).cpu().numpy()
    assert np.allclose(got, want, rtol=1e-6, atol=1e-15)
    # the reference configuration's own potential temperature is zero
    assert pt.potential_temperature(st, tr, st) == 0.0
    plan.close()
