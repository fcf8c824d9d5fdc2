"""Pins of the oracle's push: gyration, external fields, single-ion trap
frequencies and rotating-frame energy conservation.

Independent references: the Lorentz force law (finite differences of U0), the
guiding-centre invariant, the paper's potentials phi_trap and phi_wall
differentiated numerically (Eqs. pot_trap, pot_wall), the closed-form
single-ion Penning frequencies (w_z, w_+, w_-) with the exact discrete
dispersion of a drift-kick-drift step, and conservation of the rotating-frame
energy (a time-independent Hamiltonian in that frame, Eq. rotation).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

WC = W.omega_c()


def test_u0_is_the_lorentz_force_clockwise_gyration():
    rng = np.random.default_rng(0)
    pos = rng.normal(size=(5, 3)) * 1e-5
    vel = rng.normal(size=(5, 3)) * 100.0
    h = 1e-12
    _, vp = oracle.u0(pos, vel, h, WC)
    _, vm = oracle.u0(pos, vel, -h, WC)
    dvdt = (vp - vm) / (2 * h)
    # dv/dt = (q/m) v x B with B = +B z:  (w_c v_y, -w_c v_x, 0)
    lorentz = np.stack([WC * vel[:, 1], -WC * vel[:, 0], np.zeros(5)], 1)
    assert np.allclose(dvdt, lorentz, rtol=1e-6, atol=1e-6 * np.abs(lorentz).max())


def test_u0_invariants_period_and_group_property():
    rng = np.random.default_rng(1)
    pos = rng.normal(size=(8, 3)) * 1e-5
    vel = rng.normal(size=(8, 3)) * 100.0
    gc0 = pos[:, :2] + np.stack([vel[:, 1], -vel[:, 0]], 1) / WC
    for h in (1e-10, 3.7e-9, 1e-7):
        p1, v1 = oracle.u0(pos, vel, h, WC)
        gc1 = p1[:, :2] + np.stack([v1[:, 1], -v1[:, 0]], 1) / WC
        assert np.allclose(gc1, gc0, rtol=0, atol=1e-14 * np.abs(pos).max() + 1e-18)
        assert np.allclose(np.hypot(v1[:, 0], v1[:, 1]), np.hypot(vel[:, 0], vel[:, 1]), rtol=1e-14)
        assert np.allclose(p1[:, 2], pos[:, 2] + vel[:, 2] * h, rtol=1e-15)
        assert np.array_equal(v1[:, 2], vel[:, 2])
    T = 2 * math.pi / WC
    pT, vT = oracle.u0(pos, vel, T, WC)
    assert np.allclose(pT[:, :2], pos[:, :2], atol=1e-13 * np.abs(pos).max())
    assert np.allclose(vT[:, :2], vel[:, :2], atol=1e-12 * np.abs(vel).max())
    pa, va = oracle.u0(*oracle.u0(pos, vel, 2e-9, WC), 3e-9, WC)
    pb, vb = oracle.u0(pos, vel, 5e-9, WC)
    assert np.allclose(pa, pb, rtol=1e-13, atol=1e-20) and np.allclose(va, vb, rtol=1e-12)


def _potential(trap, t, p):
    kz = trap["mass"] * trap["omega_z"] ** 2 / trap["charge"]
    x, y, z = p
    r2 = x * x + y * y
    phi_az = math.atan2(y, x)
    trap_pot = 0.25 * kz * (2 * z * z - x * x - y * y)                        # Eq. pot_trap
    wall = 0.25 * kz * trap["delta"] * r2 * math.cos(2 * (phi_az + trap["omega_r"] * t))  # Eq. pot_wall
    return trap_pot + wall


def test_external_field_is_minus_gradient_of_paper_potentials():
    tr = W.trap(beta=0.4, delta=0.05)
    rng = np.random.default_rng(2)
    pos = rng.normal(size=(6, 3)) * 40e-6
    for t in (0.0, 1.3e-7, 4.1e-6):
        E = oracle.external_field(pos, tr, t)
        h = 1e-10
        for i in range(6):
            for a in range(3):
                pp, pm = pos[i].copy(), pos[i].copy()
                pp[a] += h
                pm[a] -= h
                g = (_potential(tr, t, pp) - _potential(tr, t, pm)) / (2 * h)
                assert -g == pytest.approx(E[i, a], rel=1e-6, abs=1e-7 * np.abs(E[i]).max())


def _trajectory(pos, vel, trap, dt, n_chunks, chunk):
    q = np.full(len(pos), W.E_CHARGE)
    out = [pos.copy()]
    vout = [vel.copy()]
    t = 0.0
    for k in range(n_chunks):
        pos, vel = oracle.step(pos, vel, q, trap, dt, chunk, t0=t, step0=k * chunk)
        t += chunk * dt
        out.append(pos.copy())
        vout.append(vel.copy())
    return np.array(out), np.array(vout)


def test_axial_frequency_has_the_drift_kick_drift_dispersion():
    tr = W.trap(beta=1.0, delta=0.0)
    dt = 1e-9
    pos = np.array([[0.0, 0.0, 2e-6]])
    vel = np.zeros((1, 3))
    traj, _ = _trajectory(pos, vel, tr, dt, 3000, 1)
    z = traj[:, 0, 2]
    # z_{n+1} + z_{n-1} = 2 cos(w dt) z_n for any linear two-step oscillator;
    # a drift-kick-drift step with the trap force has cos(w dt) = 1 - (w_z dt)^2/2
    c = np.sum(z[1:-1] * (z[2:] + z[:-2])) / (2 * np.sum(z[1:-1] ** 2))
    assert c == pytest.approx(1 - 0.5 * (W.OMEGA_Z * dt) ** 2, rel=1e-13)
    w_num = math.acos(c) / dt
    assert w_num == pytest.approx(W.OMEGA_Z, rel=2e-5)
    assert not np.isclose(w_num, W.OMEGA_Z, rtol=1e-7)   # the splitting error is visible


def test_planar_frequencies_are_the_modified_cyclotron_and_magnetron():
    tr = W.trap(beta=1.0, delta=0.0)
    dt = 1e-9
    every = 20
    pos = np.array([[10e-6, 3e-6, 0.0]])
    vel = np.array([[5.0, -2.0, 0.0]])
    traj, _ = _trajectory(pos, vel, tr, dt, 600, every)
    w = traj[:, 0, 0] + 1j * traj[:, 0, 1]
    # the one-step map is complex-linear in (x+iy, vx+ivy): w_n = A l1^n + B l2^n.
    # Prony: w_{n+1} = a w_n + b w_{n-1}; the roots of l^2 - a l - b are l1, l2.
    M = np.stack([w[1:-1], w[:-2]], 1)
    a, b = np.linalg.lstsq(M, w[2:], rcond=None)[0]
    roots = np.roots([1, -a, -b])
    assert np.allclose(np.abs(roots), 1.0, atol=1e-9)          # no numerical damping
    freqs = sorted(-np.angle(roots) / (every * dt))            # clockwise -> positive
    root = math.sqrt(WC * WC - 2 * W.OMEGA_Z**2)
    wp, wm = 0.5 * (WC + root), 0.5 * (WC - root)
    assert freqs[1] == pytest.approx(wp, rel=2e-5)
    assert freqs[0] == pytest.approx(wm, rel=2e-5)
    assert freqs[0] / (2 * math.pi) == pytest.approx(167.7e3, rel=2e-3)


def _energy_series(pos, vel, trap, dt, n, every):
    q = np.full(len(pos), W.E_CHARGE)
    es = [oracle.energy_rot(pos, vel, q, trap, 0.0)[3]]
    t = 0.0
    for k in range(n // every):
        pos, vel = oracle.step(pos, vel, q, trap, dt, every, t0=t, step0=k * every)
        t += every * dt
        es.append(oracle.energy_rot(pos, vel, q, trap, t)[3])
    return np.array(es)


@pytest.mark.parametrize("delta", [0.0, 0.02])
def test_rotating_frame_energy_is_conserved_single_ion(delta):
    tr = W.trap(beta=0.5, delta=delta)
    pos = np.array([[25e-6, -8e-6, 6e-6]])
    vel = W.rotating_maxwellian(pos, tr["omega_r"], 10e-3, seed=3)
    e1 = _energy_series(pos, vel, tr, 1e-9, 4000, 10)
    e2 = _energy_series(pos, vel, tr, 0.5e-9, 8000, 20)
    scale = abs(e1[0])
    d1 = np.abs(e1 - e1[0]).max() / scale
    d2 = np.abs(e2 - e2[0]).max() / scale
    assert d1 < 1e-4, d1
    # a second-order splitting: halving dt cuts the excursion about four-fold
    assert 2.5 < d1 / d2 < 6.0, (d1, d2)


def test_rotating_frame_energy_is_conserved_with_coulomb():
    tr = W.trap(beta=1.0, delta=0.01)
    pos = W.sphere(40, 30e-6, seed=4)
    vel = W.rotating_maxwellian(pos, tr["omega_r"], 10e-3, seed=5)
    e = _energy_series(pos, vel, tr, 1e-9, 3000, 50)
    rel = np.abs(e - e[0]) / abs(e[0])
    assert rel.max() < 1e-4, rel.max()
    # no secular growth: the late excursion is not larger than the early one
    third = len(rel) // 3
    assert rel[-third:].max() < 3 * rel[:third].max() + 1e-9


def test_energy_parts_for_a_rigid_rotor_at_rest_in_the_rotating_frame():
    tr = W.trap(beta=0.7, delta=0.0)
    pos = np.array([[12e-6, 5e-6, -3e-6]])
    vel = np.array([[tr["omega_r"] * pos[0, 1], -tr["omega_r"] * pos[0, 0], 0.0]])
    ke, pe, ce, tot = oracle.energy_rot(pos, vel, [W.E_CHARGE], tr, 0.0)
    assert ke == pytest.approx(0.0, abs=1e-40)
    r2 = pos[0, 0] ** 2 + pos[0, 1] ** 2
    want = 0.5 * W.MASS * W.OMEGA_Z**2 * (tr["beta"] * r2 + pos[0, 2] ** 2)   # Eq. pe_rot
    assert pe == pytest.approx(want, rel=1e-12)
    assert ce == 0.0
