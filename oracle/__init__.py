"""Plain FP64 CPU oracle for the Penning-trap FMM step (arXiv:2405.13973).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``; never by the product
library.  The arithmetic lives in ``penning_oracle.c`` (each function cites the
paper passage it follows); this module compiles it with gcc on first use and
wraps it with ctypes.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "penning_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64
_U32P = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_U32P, _U32P, _U32P]
            L.orc_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_u01.restype = ctypes.c_double
            L.orc_exp.argtypes = [ctypes.c_double]
            L.orc_exp.restype = ctypes.c_double
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_coulomb_direct.argtypes = [_I64, _D, _D, _D, _D, _D, _D, _D, _D]
            L.orc_coulomb_near.argtypes = [_I64, _D, _D, _D, _D, ctypes.c_int, _D, _D, _D, _D]
            L.orc_coulomb_targets.argtypes = [_I64, _D, _D, _D, _D, _I64,
                                              ctypes.POINTER(ctypes.c_int64), _D, _D, _D, _D]
            L.orc_root_cube.argtypes = [_I64, _D, _D, _D, _D, _D]
            L.orc_leaf_keys.argtypes = [_I64, _D, _D, _D, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_uint64), _D, _D]
            L.orc_external_field.argtypes = [_I64, _D, ctypes.c_double, _D, _D, _D, _D, _D, _D]
            L.orc_u0.argtypes = [_I64, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D, _D, _D]
            L.orc_saturation.argtypes = [_D, ctypes.c_double, ctypes.c_double]
            L.orc_saturation.restype = ctypes.c_double
            L.orc_scatter_rate.argtypes = [_D, ctypes.c_double] + [ctypes.c_double] * 5
            L.orc_scatter_rate.restype = ctypes.c_double
            L.orc_poisson.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_poisson.restype = ctypes.c_int
            L.orc_laser_kick.argtypes = [_I64, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_uint64, _I64, ctypes.c_double,
                                         _D, _D, _D, _D, _D, _D,
                                         ctypes.POINTER(ctypes.c_int32), _D, _D, _D]
            L.orc_step.argtypes = [_I64, _D, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, _I64, _I64]
            L.orc_step_damped.argtypes = L.orc_step.argtypes + [ctypes.c_double]
            L.orc_temperatures.argtypes = [_I64, _D, _D, _D, _D, _D, _D, _D]
            L.orc_energy_rot.argtypes = [_I64, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_double, _D]
            L.orc_mh_scans.argtypes = [_I64, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                       _I64, _I64, _D]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---- random numbers ---------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u01(a: int, b: int) -> float:
    return float(lib().orc_u01(a, b))


def exp(x: float) -> float:
    return float(lib().orc_exp(float(x)))


def poisson(lam: float, u: float) -> int:
    return int(lib().orc_poisson(float(lam), float(u)))


# ---- Coulomb ----------------------------------------------------------------
def coulomb_direct(pos, q, want_phi=True):
    """E (n,3) in V/m and phi (n,) in V of every ion from all others (SI)."""
    pos = _f64(pos)
    x, y, z = (_f64(pos[:, a]) for a in range(3))
    q = _f64(q)
    n = len(q)
    E = [np.empty(n) for _ in range(3)]
    phi = np.empty(n) if want_phi else None
    lib().orc_coulomb_direct(n, _p(x), _p(y), _p(z), _p(q), _p(E[0]), _p(E[1]), _p(E[2]),
                             _p(phi) if want_phi else None)
    return np.stack(E, 1), phi


def coulomb_targets(pos, q, idx, want_phi=True):
    """E (m,3) and phi (m,) at the ions idx from all other ions (SI)."""
    pos = _f64(pos)
    x, y, z = (_f64(pos[:, a]) for a in range(3))
    q = _f64(q)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = len(idx)
    E = [np.empty(m) for _ in range(3)]
    phi = np.empty(m) if want_phi else None
    lib().orc_coulomb_targets(len(q), _p(x), _p(y), _p(z), _p(q), m,
                              idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              _p(E[0]), _p(E[1]), _p(E[2]), _p(phi) if want_phi else None)
    return np.stack(E, 1), phi


def coulomb_near(pos, q, depth):
    pos = _f64(pos)
    x, y, z = (_f64(pos[:, a]) for a in range(3))
    q = _f64(q)
    n = len(q)
    E = [np.empty(n) for _ in range(3)]
    phi = np.empty(n)
    lib().orc_coulomb_near(n, _p(x), _p(y), _p(z), _p(q), int(depth), _p(E[0]), _p(E[1]),
                           _p(E[2]), _p(phi))
    return np.stack(E, 1), phi


def root_cube(pos):
    pos = _f64(pos)
    x, y, z = (_f64(pos[:, a]) for a in range(3))
    lo = np.empty(3)
    side = np.empty(1)
    lib().orc_root_cube(len(x), _p(x), _p(y), _p(z), _p(lo), _p(side))
    return lo, float(side[0])


def leaf_keys(pos, depth):
    pos = _f64(pos)
    x, y, z = (_f64(pos[:, a]) for a in range(3))
    n = len(x)
    key = np.empty(n, np.uint64)
    lo = np.empty(3)
    side = np.empty(1)
    lib().orc_leaf_keys(n, _p(x), _p(y), _p(z), int(depth),
                        key.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _p(lo), _p(side))
    return key, lo, float(side[0])


# ---- trap, push, lasers -----------------------------------------------------
def trap_array(trap) -> np.ndarray:
    """double[6] = {B, omega_z, omega_r, delta, m, q} from a mapping."""
    return np.array([trap["B"], trap["omega_z"], trap["omega_r"], trap["delta"], trap["mass"],
                     trap["charge"]], dtype=np.float64)


def beams_array(beams) -> np.ndarray:
    """double[9 * n_beams] = {S0, Delta, kx, ky, kz, w_y, w_z, d, uniform} per beam."""
    rows = [[b["s0"], b["detuning"], b["k"][0], b["k"][1], b["k"][2], b.get("waist_y", 1.0),
             b.get("waist_z", 1.0), b.get("offset_d", 0.0), 1.0 if b.get("uniform", False) else 0.0]
            for b in beams]
    return np.ascontiguousarray(np.array(rows, dtype=np.float64).reshape(-1))


def external_field(pos, trap, t):
    pos = _f64(pos)
    x, y, z = (_f64(pos[:, a]) for a in range(3))
    n = len(x)
    E = [np.empty(n) for _ in range(3)]
    tr = trap_array(trap)
    lib().orc_external_field(n, _p(tr), float(t), _p(x), _p(y), _p(z), _p(E[0]), _p(E[1]),
                             _p(E[2]))
    return np.stack(E, 1)


def u0(pos, vel, h, wc):
    st = [_f64(pos[:, a]).copy() for a in range(3)] + [_f64(vel[:, a]).copy() for a in range(3)]
    lib().orc_u0(len(st[0]), float(h), float(wc), *[_p(a) for a in st])
    return np.stack(st[:3], 1), np.stack(st[3:], 1)


def saturation(beam, y, z):
    b = beams_array([beam])
    return float(lib().orc_saturation(_p(b), float(y), float(z)))


def scatter_rate(beam, gamma0, y, z, v):
    b = beams_array([beam])
    return float(lib().orc_scatter_rate(_p(b), float(gamma0), float(y), float(z), float(v[0]),
                                        float(v[1]), float(v[2])))


def laser_kick(pos, vel, beams, gamma0, mass, seed, step, dt):
    """Photon counts (n, n_beams) and recoil dv (n, 3) at the midpoint state."""
    pos = _f64(pos)
    vel = _f64(vel)
    n = len(pos)
    b = beams_array(beams)
    nb = len(beams)
    cols = [_f64(pos[:, a]) for a in range(3)] + [_f64(vel[:, a]) for a in range(3)]
    counts = np.zeros((n, max(nb, 1)), np.int32)
    dv = [np.empty(n) for _ in range(3)]
    lib().orc_laser_kick(n, _p(b), nb, float(gamma0), float(mass), int(seed) & (2**64 - 1),
                         int(step), float(dt), *[_p(c) for c in cols],
                         counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         _p(dv[0]), _p(dv[1]), _p(dv[2]))
    return counts[:, :nb], np.stack(dv, 1)


def step(pos, vel, q, trap, dt, n_steps, t0=0.0, step0=0, beams=(), gamma0=0.0, seed=0,
         laser_on=False, damping=None):
    """Advance (pos, vel) by n_steps literal cyclotronic steps; returns copies.
    damping (1/s): rotating-frame velocities scaled by exp(-damping dt) after
    every kick (None: the undamped step)."""
    st = [_f64(pos[:, a]).copy() for a in range(3)] + [_f64(vel[:, a]).copy() for a in range(3)]
    q = _f64(q)
    tr = trap_array(trap)
    b = beams_array(beams) if len(beams) else np.zeros(9)
    args = (len(q), *[_p(a) for a in st], _p(q), _p(tr), _p(b), len(beams), float(gamma0),
            int(seed) & (2**64 - 1), 1 if laser_on else 0, float(dt), float(t0), int(step0),
            int(n_steps))
    if damping is None:
        lib().orc_step(*args)
    else:
        lib().orc_step_damped(*args, float(damping))
    return np.stack(st[:3], 1), np.stack(st[3:], 1)


def temperatures(pos, vel, trap):
    """(T_par, T_perp) in K of the rotating-frame motion."""
    x, y = _f64(pos[:, 0]), _f64(pos[:, 1])
    vx, vy, vz = (_f64(vel[:, a]) for a in range(3))
    out = np.empty(2)
    lib().orc_temperatures(len(x), _p(x), _p(y), _p(vx), _p(vy), _p(vz), _p(trap_array(trap)),
                           _p(out))
    return float(out[0]), float(out[1])


def energy_rot(pos, vel, q, trap, t):
    """Rotating-frame energy parts {kinetic, external, Coulomb, total} (J)."""
    cols = [_f64(pos[:, a]) for a in range(3)] + [_f64(vel[:, a]) for a in range(3)]
    q = _f64(q)
    tr = trap_array(trap)
    out = np.empty(4)
    lib().orc_energy_rot(len(q), *[_p(c) for c in cols], _p(q), _p(tr), float(t), _p(out))
    return out


def mh_scans(pos, q, trap, temp, dx, seed, scan0, n_scans, wall_cs):
    """Metropolis-Hastings potential-energy scans (returns new positions,
    accepted moves, sum of the accepted energy changes in J).  wall_cs =
    (cos w_r t, sin w_r t) of the state's time."""
    x, y, z = (np.ascontiguousarray(pos[:, a], dtype=np.float64).copy() for a in range(3))
    q = _f64(q)
    out = np.empty(2)
    lib().orc_mh_scans(len(q), _p(x), _p(y), _p(z), _p(q), _p(trap_array(trap)),
                       float(wall_cs[0]), float(wall_cs[1]), float(temp), float(dx),
                       int(seed) & (2**64 - 1), int(scan0), int(n_scans), _p(out))
    return np.stack([x, y, z], axis=1), int(out[0]), float(out[1])
