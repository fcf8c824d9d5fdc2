"""Pins of the oracle's diagnostics and damped step.

Temperatures (Eqs. temp_ax, temp_pl): zero for a rigid rotor, the sampling
temperature for a rotating Maxwellian (equipartition), and a hand-worked pair.
Damped step (artificial damping toward crystal equilibria, Sec. 6): no damping
reproduces the undamped step bit for bit; two ions relax to the closed-form
equilibrium of the rotating-frame potential (along its weakest axis, y_r for
delta > 0 at beta = 1), with the rotating-frame energy falling step by step.
"""
import math

import numpy as np

import oracle
import workloads as W

KB = 1.380649e-23


def test_rigid_rotor_has_zero_temperature():
    tr = W.trap(beta=1.0)
    rng = np.random.default_rng(0)
    pos = rng.normal(size=(500, 3)) * 30e-6
    vel = np.zeros_like(pos)
    vel[:, 0] = tr["omega_r"] * pos[:, 1]
    vel[:, 1] = -tr["omega_r"] * pos[:, 0]
    assert oracle.temperatures(pos, vel, tr) == (0.0, 0.0)


def test_rotating_maxwellian_equipartition():
    tr = W.trap(beta=1.0)
    pos = W.sphere(200000, 100e-6, 4)
    vel = W.rotating_maxwellian(pos, tr["omega_r"], 10e-3, 5)
    t_par, t_perp = oracle.temperatures(pos, vel, tr)
    # relative sampling spread sqrt(2/N) = 0.3 % and sqrt(1/N) = 0.2 %
    assert abs(t_par / 10e-3 - 1) < 0.015 and abs(t_perp / 10e-3 - 1) < 0.01


def test_hand_worked_pair():
    tr = W.trap(beta=1.0)
    m, wr = tr["mass"], tr["omega_r"]
    pos = np.array([[1e-6, 2e-6, 0.0], [0.0, -1e-6, 3e-6]])
    # rotating-frame velocities (1, 2, 3) and (-2, 0, 1) m/s on top of the rotor
    w = np.array([[1.0, 2.0, 3.0], [-2.0, 0.0, 1.0]])
    vel = w.copy()
    vel[:, 0] += wr * pos[:, 1]
    vel[:, 1] -= wr * pos[:, 0]
    t_par, t_perp = oracle.temperatures(pos, vel, tr)
    assert math.isclose(t_par, m * (9 + 1) / (2 * KB), rel_tol=1e-12)
    assert math.isclose(t_perp, m * (1 + 4 + 4 + 0) / (4 * KB), rel_tol=1e-12)


def test_zero_damping_is_the_undamped_step():
    cr = W.crystal_sphere_1k(seed=8)
    pos, vel, q, tr = cr["pos"][:200], cr["vel"][:200], cr["q"][:200], cr["trap"]
    a = oracle.step(pos, vel, q, tr, 1e-9, 5)
    b = oracle.step(pos, vel, q, tr, 1e-9, 5, damping=0.0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_damped_pair_relaxes_to_the_closed_form_equilibrium():
    tr = W.trap(beta=1.0)
    m, q, wz, wr, dl = tr["mass"], tr["charge"], tr["omega_z"], tr["omega_r"], tr["delta"]
    ke = 1.0 / (4.0 * math.pi * W.EPS0)
    # rotating-frame potential m wz^2/2 [(beta + dl/2) x_r^2 + (beta - dl/2) y_r^2 + z^2]:
    # weakest along y_r; balance m wz^2 C_y d/2 = ke q^2 / d^2
    d = (2.0 * ke * q * q / (m * wz * wz * (1.0 - dl / 2))) ** (1.0 / 3.0)
    pos = np.array([[0.3e-6, 0.4 * d, 0.2e-6], [-0.2e-6, -0.6 * d, -0.1e-6]])
    vel = W.rotating_maxwellian(pos, wr, 1e-3, 3)
    qs = np.array([q, q])
    gamma, dt, t = 1e6, W.DT, 0.0
    energies = []
    p, v = pos, vel
    for _ in range(30):
        p, v = oracle.step(p, v, qs, tr, dt, 10000, t0=t, damping=gamma)
        t += 10000 * dt
        energies.append(oracle.energy_rot(p, v, qs, tr, t)[3])
    e = np.array(energies)
    assert np.all(np.diff(e) <= 1e-12 * abs(e[-1]))          # energy falls (to rounding)
    c, s = math.cos(wr * t), math.sin(wr * t)
    xr = c * p[:, 0] - s * p[:, 1]
    yr = s * p[:, 0] + c * p[:, 1]
    # the discrete fixed point sits O(gamma dt) = 1e-3 away from the continuous one
    assert abs((yr[0] - yr[1]) / d - 1.0) < 5e-4
    assert np.all(np.abs(xr) < 1e-3 * d) and np.all(np.abs(p[:, 2]) < 1e-6 * d)
    assert oracle.temperatures(p, v, tr)[1] < 1e-6
