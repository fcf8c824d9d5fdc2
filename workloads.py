"""Seeded synthetic inputs and trap/beam presets for the Penning-trap workloads.

This module only builds inputs: ion positions, charges, velocities and the
trap and laser parameters of the paper's synthetic workloads (ions placed
uniformly in a sphere or spheroid, Sec. 3 and Sec. 5).  It holds none of the
method's arithmetic (no field, push, tree or random-kick code) and is the one
module that both the oracle side (tests, CPU baseline) and the CUDA side
(tests, bench) draw inputs from.

Readings of the paper used here (the paper does not state these values):
  * mass 9 u, charge +e, B = 4.46 T, omega_z = 2 pi 1.58 MHz, dt = 1 ns;
  * rotating-wall strength delta = 0.01;
  * beams: two uniform axial beams along +-z with S0 = 5e-3 and detuning
    -gamma0/2 (Fig. 1 caption, Sec. 5); one planar beam along +x centred at
    y = d = 5 um with w_y = 2.48 um, w_z = 1 mm and detuning +2 pi 13.6 MHz
    (Sec. 5), saturation S0 = 9e-3 so that its peak rate is 1e6 /s (the
    paper's run uses S0 = 0.5: ``paper_beams``);
  * gamma0 = 2 pi 18 MHz (Eq. scattering_rate), wavelength 313 nm.
"""
from __future__ import annotations

import math

import numpy as np

AMU = 1.66053906660e-27
E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12
K_B = 1.380649e-23
TWO_PI = 2.0 * math.pi

MASS = 9.0 * AMU
B_FIELD = 4.46
OMEGA_Z = TWO_PI * 1.58e6
DELTA_WALL = 0.01
DT = 1e-9
GAMMA0 = TWO_PI * 18e6
K_313 = TWO_PI / 313e-9


def omega_c(B=B_FIELD, q=E_CHARGE, m=MASS):
    return q * B / m


def omega_r_for_beta(beta, B=B_FIELD, wz=OMEGA_Z, q=E_CHARGE, m=MASS):
    """Lower root of w_r (w_c - w_r) = (beta + 1/2) w_z^2 (Eq. beta)."""
    wc = omega_c(B, q, m)
    disc = wc * wc - 4.0 * (beta + 0.5) * wz * wz
    if disc < 0:
        raise ValueError("no confined rotation frequency for this beta")
    return 0.5 * (wc - math.sqrt(disc))


def axial_depolarization(aspect):
    """N_z of a uniform spheroid with a_z / a_r = aspect (Sec. 4 shape law)."""
    a = float(aspect)
    if abs(a - 1.0) < 1e-12:
        return 1.0 / 3.0
    if a < 1.0:
        e = math.sqrt(1.0 - a * a)
        return (1.0 - a * math.asin(e) / e) / (e * e)
    e = math.sqrt(1.0 - 1.0 / (a * a))
    return (1.0 - e * e) / (e * e) * (math.atanh(e) / e - 1.0)


def beta_for_aspect(aspect):
    """beta = (1 - N_z) / (2 N_z) for a uniform spheroid (delta = 0)."""
    nz = axial_depolarization(aspect)
    return (1.0 - nz) / (2.0 * nz)


def rigid_rotor_density(omega_r, B=B_FIELD, q=E_CHARGE, m=MASS):
    """n0 = 2 eps0 m w_r (w_c - w_r) / q^2."""
    wc = omega_c(B, q, m)
    return 2.0 * EPS0 * m * omega_r * (wc - omega_r) / (q * q)


def trap(beta=1.0, aspect=None, delta=DELTA_WALL, B=B_FIELD, wz=OMEGA_Z, m=MASS, q=E_CHARGE):
    if aspect is not None:
        beta = beta_for_aspect(aspect)
    return {"B": B, "omega_z": wz, "omega_r": omega_r_for_beta(beta, B, wz, q, m), "delta": delta,
            "mass": m, "charge": q, "beta": beta}


def axial_beams(s0=5e-3):
    return [
        {"s0": s0, "detuning": -0.5 * GAMMA0, "k": (0.0, 0.0, K_313), "uniform": True},
        {"s0": s0, "detuning": -0.5 * GAMMA0, "k": (0.0, 0.0, -K_313), "uniform": True},
    ]


def planar_beam(s0=9e-3, detuning=TWO_PI * 13.6e6, waist_y=2.48e-6, waist_z=1e-3, offset_d=5e-6):
    return {"s0": s0, "detuning": detuning, "k": (K_313, 0.0, 0.0), "uniform": False,
            "waist_y": waist_y, "waist_z": waist_z, "offset_d": offset_d}


def cooling_beams(planar_s0=9e-3):
    return axial_beams() + [planar_beam(s0=planar_s0)]


def paper_beams():
    return cooling_beams(planar_s0=0.5)


# ---- positions and velocities ---------------------------------------------------
def _unit_ball(rng, n):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return v * rng.random(n)[:, None] ** (1.0 / 3.0)


def sphere(n, radius, seed):
    rng = np.random.default_rng(seed)
    return _unit_ball(rng, n) * radius


def spheroid(n, a_r, a_z, seed):
    rng = np.random.default_rng(seed)
    return _unit_ball(rng, n) * np.array([a_r, a_r, a_z])


def rotating_maxwellian(pos, omega_r, temperature, seed, m=MASS):
    """v = (w_r y, -w_r x, 0) + N(0, k_B T / m) per component (clockwise rotor)."""
    rng = np.random.default_rng(seed)
    sig = math.sqrt(K_B * temperature / m)
    v = rng.normal(size=pos.shape) * sig
    v[:, 0] += omega_r * pos[:, 1]
    v[:, 1] -= omega_r * pos[:, 0]
    return v


def lattice_sphere(n, density, jitter, seed):
    """The n sites of a simple-cubic lattice (spacing density^(-1/3)) nearest
    the origin, each displaced by Gaussian jitter of `jitter` x spacing: a
    start without close pairs."""
    a = density ** (-1.0 / 3.0)
    m = int(math.ceil((3.0 * n / (4.0 * math.pi)) ** (1.0 / 3.0))) + 2
    g = np.arange(-m, m + 1, dtype=np.float64)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r = np.linalg.norm(pts, axis=1) + 1e-9 * (pts @ np.array([1.0, 1e-3, 1e-6]))
    pts = pts[np.argsort(r, kind="stable")[:n]]
    rng = np.random.default_rng(seed)
    return (pts + rng.normal(size=pts.shape) * jitter) * a


def charges(n, q=E_CHARGE):
    return np.full(n, q, dtype=np.float64)


# ---- the workloads --------------------------------------------------------------
def crystal_sphere_1k(seed=1):
    """N = 1,000 uniform in a 100 um sphere, 10 mK rotating Maxwellian, beta = 1."""
    tr = trap(beta=1.0)
    pos = sphere(1000, 100e-6, seed)
    vel = rotating_maxwellian(pos, tr["omega_r"], 10e-3, seed + 1000)
    return {"name": "sphere_N1000", "pos": pos, "vel": vel, "q": charges(1000), "trap": tr,
            "beams": [], "laser": False, "p": 8, "leaf": 32, "dt": DT, "n_steps": 1000}


def crystal_lattice_1k(seed=5, n=1000, temperature=10e-3):
    """N = 1,000 on a jittered cubic lattice at the beta = 1 rigid-rotor density,
    rigid rotation plus a 10 mK Maxwellian: no close pairs."""
    tr = trap(beta=1.0)
    n0 = rigid_rotor_density(tr["omega_r"])
    pos = lattice_sphere(n, n0, 0.05, seed)
    vel = rotating_maxwellian(pos, tr["omega_r"], temperature, seed + 1000)
    return {"name": f"lattice_N{n}", "pos": pos, "vel": vel, "q": charges(n), "trap": tr,
            "beams": [], "laser": False, "p": 10, "leaf": 32, "dt": DT, "n_steps": 1000}


def crystal_spheroid_10k(seed=2, n=10000, aspect=0.3):
    """N = 10,000 uniform at the rigid-rotor density in an aspect-0.3 spheroid, cooling on."""
    tr = trap(aspect=aspect)
    n0 = rigid_rotor_density(tr["omega_r"])
    a_r = (3.0 * n / (4.0 * math.pi * n0 * aspect)) ** (1.0 / 3.0)
    pos = spheroid(n, a_r, aspect * a_r, seed)
    vel = rotating_maxwellian(pos, tr["omega_r"], 10e-3, seed + 1000)
    return {"name": f"spheroid{aspect}_N{n}", "pos": pos, "vel": vel, "q": charges(n), "trap": tr,
            "beams": cooling_beams(), "laser": True, "p": 10, "leaf": 32, "dt": DT,
            "n_steps": 10000, "a_r": a_r, "a_z": aspect * a_r, "n0": n0}


def sphere_sweep(n, seed=3, density=2e14):
    """N uniform in a sphere at 2e14 m^-3 plus Gaussian jitter of 1% of a_ws."""
    rng = np.random.default_rng(seed)
    radius = (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    a_ws = (3.0 / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    pos = _unit_ball(rng, n) * radius + rng.normal(size=(n, 3)) * 0.01 * a_ws
    return {"name": f"sphere_sweep_N{n}", "pos": pos, "q": charges(n), "radius": radius}


def ensemble_member(n, aspect, seed, temperature=10e-3, cooling=True):
    """One crystal of a batched ensemble: n ions uniform at the rigid-rotor
    density in a spheroid of the given aspect (the rotation frequency follows
    from the shape law), rotating Maxwellian, the cooling beams."""
    tr = trap(aspect=aspect)
    n0 = rigid_rotor_density(tr["omega_r"])
    a_r = (3.0 * n / (4.0 * math.pi * n0 * aspect)) ** (1.0 / 3.0)
    pos = spheroid(n, a_r, aspect * a_r, seed)
    vel = rotating_maxwellian(pos, tr["omega_r"], temperature, seed + 1000)
    return {"name": f"member{seed}_N{n}_a{aspect:.2f}", "pos": pos, "vel": vel, "q": charges(n),
            "trap": tr, "beams": cooling_beams() if cooling else [], "laser": cooling, "dt": DT,
            "aspect": aspect}


def ensemble_crystals(n_members=256, n_lo=100, n_hi=20000, seed=0):
    """Batched ensemble: n_members crystals, N log-uniform in [n_lo, n_hi],
    aspect uniform in [0.1, 1.0], seeds seed + k, cooling on."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_members)).astype(int)
    aspects = rng.uniform(0.1, 1.0, n_members)
    return [ensemble_member(int(n), float(a), seed + 7 * k) for k, (n, a) in enumerate(zip(ns, aspects))]
