"""Pins of the oracle's Metropolis-Hastings potential-energy initialisation
(Sec. 4: sequential random displacements of at most dx in random directions,
accepted if the crystal's potential energy falls or with probability
exp(-dE / k_B T)).

Each pin ties it to something other than itself:
  * energy bookkeeping: the accepted energy changes add up to the change of
    the rotating-frame potential energy computed independently by
    orc_energy_rot (itself pinned in test_oracle_push.py), with the wall on and
    an arbitrary wall phase -- a dropped, mis-signed or self-including term in
    dE breaks it;
  * T -> 0: only downhill moves survive, so the potential energy never rises
    from one scan to the next;
  * one ion, no Coulomb partner, axially symmetric trap: the chain samples the
    Boltzmann distribution of a 3D harmonic well, <z^2> = k_B T / (m w_z^2)
    and <x^2 + y^2> = 2 k_B T / k_r with k_r = q B w_r - m w_r^2 - m w_z^2 / 2
    (equipartition, separately per direction);
  * dx = 0: every move is accepted and nothing moves.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

KB = 1.380649e-23


@pytest.fixture(scope="module")
def small_crystal():
    cr = W.crystal_sphere_1k(seed=11)
    return cr["pos"][:60].copy(), cr["q"][:60].copy(), cr["trap"]


def pot(pos, q, trap, t):
    e = oracle.energy_rot(pos, np.zeros_like(pos), q, trap, t)
    return e[1] + e[2]


def test_accepted_changes_add_up_to_the_energy_change(small_crystal):
    pos, q, trap = small_crystal
    trap = dict(trap, delta=0.02)
    t = 3.7e-7
    cs = (math.cos(trap["omega_r"] * t), math.sin(trap["omega_r"] * t))
    p2, acc, de = oracle.mh_scans(pos, q, trap, 10e-3, 1e-6, 5, 0, 4, cs)
    assert 0 < acc < 4 * len(q)
    assert not np.array_equal(p2, pos)
    dE = pot(p2, q, trap, t) - pot(pos, q, trap, t)
    assert abs(de - dE) <= 1e-9 * abs(dE) + 1e-30, (de, dE)


def test_zero_temperature_only_descends(small_crystal):
    pos, q, trap = small_crystal
    e_prev = pot(pos, q, trap, 0.0)
    p = pos
    total = 0
    for sc in range(4):
        p, acc, de = oracle.mh_scans(p, q, trap, 1e-30, 1e-6, 9, sc, 1, (1.0, 0.0))
        e = pot(p, q, trap, 0.0)
        assert de <= 0.0 and e <= e_prev + 1e-12 * abs(e_prev)
        e_prev = e
        total += acc
    assert total > 0


def test_single_ion_equipartition():
    tr = W.trap(aspect=0.3)  # oblate: the radial and axial springs differ
    tr = dict(tr, delta=0.0)
    m, q, B = tr["mass"], tr["charge"], tr["B"]
    wz, wr = tr["omega_z"], tr["omega_r"]
    kr = q * B * wr - m * wr * wr - 0.5 * m * wz * wz
    assert kr > 0 and abs(kr / (m * wz * wz) - 1.0) > 0.5
    T = 10e-3
    sz2 = KB * T / (m * wz * wz)
    sr2 = 2.0 * KB * T / kr
    dx = 3.0 * math.sqrt(min(sz2, 0.5 * sr2))
    pos = np.zeros((1, 3))
    qq = np.array([q])
    p = pos
    z2, r2 = [], []
    p, _, _ = oracle.mh_scans(p, qq, tr, T, dx, 21, 0, 2000, (1.0, 0.0))   # burn-in
    for k in range(40):
        # 500 scans at a time, sampling the end of each block of 25
        for j in range(20):
            p, _, _ = oracle.mh_scans(p, qq, tr, T, dx, 21, 2000 + 1000 * k + 25 * j, 25, (1.0, 0.0))
            z2.append(p[0, 2] ** 2)
            r2.append(p[0, 0] ** 2 + p[0, 1] ** 2)
    mz, mr = np.mean(z2) / sz2, np.mean(r2) / sr2
    assert abs(mz - 1.0) < 0.1 and abs(mr - 1.0) < 0.1, (mz, mr)


def test_zero_step_accepts_and_keeps(small_crystal):
    pos, q, trap = small_crystal
    p2, acc, de = oracle.mh_scans(pos, q, trap, 10e-3, 0.0, 3, 0, 2, (1.0, 0.0))
    assert acc == 2 * len(q) and de == 0.0
    assert np.array_equal(p2, pos)


def test_counter_stream_is_deterministic(small_crystal):
    pos, q, trap = small_crystal
    a = oracle.mh_scans(pos, q, trap, 10e-3, 1e-6, 5, 10, 2, (1.0, 0.0))
    b = oracle.mh_scans(pos, q, trap, 10e-3, 1e-6, 5, 10, 2, (1.0, 0.0))
    c = oracle.mh_scans(pos, q, trap, 10e-3, 1e-6, 5, 11, 2, (1.0, 0.0))
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    assert not np.array_equal(a[0], c[0])
