"""Pins of the oracle's Coulomb sums and octree keys against closed forms.

Closed forms used: the two-ion field, the field on a charge of a regular
polygon of equal charges, the field on a vertex of a cube of equal charges,
Newton's third law, E = -grad(phi) (finite differences of the oracle's own
potential, a second output computed by a different expression), the interior
field of a uniform spheroid (Sec. 4 shape law) and hand-worked Morton keys.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

KE = 1.0 / (4.0 * math.pi * W.EPS0)
Q = W.E_CHARGE


def test_two_ions():
    r = 7.3e-6
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    E, phi = oracle.coulomb_direct(pos, [Q, 2 * Q])
    assert E[0, 0] == pytest.approx(-KE * 2 * Q / r**2, rel=1e-15)
    assert E[1, 0] == pytest.approx(KE * Q / r**2, rel=1e-15)
    assert np.all(E[:, 1:] == 0.0)
    assert phi[0] == pytest.approx(KE * 2 * Q / r, rel=1e-15)
    assert phi[1] == pytest.approx(KE * Q / r, rel=1e-15)


@pytest.mark.parametrize("n", [3, 7, 12])
def test_regular_polygon(n):
    R = 20e-6
    th = 2 * math.pi * np.arange(n) / n
    pos = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(n)], 1)
    E, phi = oracle.coulomb_direct(pos, np.full(n, Q))
    s = sum(1.0 / math.sin(math.pi * k / n) for k in range(1, n))
    e_rad = KE * Q / (4 * R * R) * s
    radial = np.stack([np.cos(th), np.sin(th), np.zeros(n)], 1)
    assert np.allclose(E, e_rad * radial, rtol=0, atol=1e-13 * e_rad)
    assert np.allclose(phi, KE * Q / (2 * R) * s, rtol=1e-14)


def test_cube_vertices():
    a = 3e-6
    pos = np.array([[sx, sy, sz] for sx in (-a, a) for sy in (-a, a) for sz in (-a, a)])
    E, _ = oracle.coulomb_direct(pos, np.full(8, Q))
    mag = KE * Q / a**2 * (0.25 + 0.25 / math.sqrt(2) + 1 / (12 * math.sqrt(3)))
    assert np.allclose(E, mag * np.sign(pos), rtol=1e-14, atol=0)


def test_newton_third_law_and_permutation():
    rng = np.random.default_rng(4)
    pos = rng.normal(size=(200, 3)) * 30e-6
    q = rng.choice([Q, 2 * Q, 3 * Q], size=200)
    E, phi = oracle.coulomb_direct(pos, q)
    F = q[:, None] * E
    assert np.abs(F.sum(0)).max() < 1e-13 * np.abs(F).sum()
    perm = rng.permutation(200)
    E2, phi2 = oracle.coulomb_direct(pos[perm], q[perm])
    assert np.allclose(E2, E[perm], rtol=1e-13, atol=1e-13 * np.abs(E).max())
    assert np.allclose(phi2, phi[perm], rtol=1e-13)


def test_field_is_minus_gradient_of_potential():
    rng = np.random.default_rng(5)
    n = 30
    pos = rng.normal(size=(n, 3)) * 10e-6
    q = np.full(n, Q)
    E, _ = oracle.coulomb_direct(pos, q)
    h = 1e-11
    for i in (0, 7, 29):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            _, php = oracle.coulomb_direct(pp, q)
            _, phm = oracle.coulomb_direct(pm, q)
            g = (php[i] - phm[i]) / (2 * h)
            assert -g == pytest.approx(E[i, a], rel=2e-6, abs=1e-6 * np.abs(E[i]).max())


@pytest.mark.slow
def test_uniform_spheroid_interior_field_matches_depolarization_factors():
    # Uniform spheroid of density n0 and aspect 0.3: interior field
    # (q n0 / eps0)(N_x x, N_y y, N_z z) with N_x = N_y = (1 - N_z)/2.
    aspect = 0.3
    n = 12000
    tr = W.trap(aspect=aspect, delta=0.0)
    n0 = W.rigid_rotor_density(tr["omega_r"])
    a_r = (3 * n / (4 * math.pi * n0 * aspect)) ** (1 / 3)
    pos = W.spheroid(n, a_r, aspect * a_r, seed=6)
    E, _ = oracle.coulomb_direct(pos, np.full(n, Q))
    nz = W.axial_depolarization(aspect)
    nx = (1 - nz) / 2
    rho = np.sqrt((pos[:, 0] / a_r) ** 2 + (pos[:, 1] / a_r) ** 2 + (pos[:, 2] / (aspect * a_r)) ** 2)
    inner = rho < 0.7
    pref = Q * n0 / W.EPS0
    for a, nfac in ((0, nx), (1, nx), (2, nz)):
        slope = np.sum(E[inner, a] * pos[inner, a]) / np.sum(pos[inner, a] ** 2)
        assert slope == pytest.approx(pref * nfac, rel=0.03), (a, slope / (pref * nfac))
    # the spheroid at the beta of its aspect is in rigid-rotor balance:
    # q E_coulomb balances the effective confinement m w_z^2 (beta r, z)
    assert pref * nz * Q == pytest.approx(W.MASS * W.OMEGA_Z**2, rel=1e-12)
    assert pref * nx * Q == pytest.approx(W.MASS * W.OMEGA_Z**2 * tr["beta"], rel=1e-12)


def test_depolarization_limits():
    assert W.axial_depolarization(1.0) == pytest.approx(1 / 3)
    assert W.axial_depolarization(0.999999) == pytest.approx(1 / 3, rel=1e-5)
    assert W.axial_depolarization(1.000001) == pytest.approx(1 / 3, rel=1e-5)
    assert W.axial_depolarization(1e-4) == pytest.approx(1.0, rel=1e-3)
    assert W.beta_for_aspect(1.0) == pytest.approx(1.0)


def test_root_cube_and_hand_worked_keys():
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.1, 0.6, 0.9], [0.99, 0.01, 0.5]])
    lo, side = oracle.root_cube(pos)
    assert np.array_equal(lo, [0.0, 0.0, 0.0]) and side == 1.0
    k1, _, _ = oracle.leaf_keys(pos, 1)
    # depth 1: (ix,iy,iz) = (0,0,0), (1,1,1) clamped, (0,1,1), (1,0,1)
    assert list(k1) == [0, 7, 3, 5]
    k2, _, _ = oracle.leaf_keys(pos, 2)
    # depth 2, ion 2: (0,2,3) -> b0 (0,0,1) = 1, b1 (0,1,1) = 24;  ion 3: (3,0,2)
    assert list(k2) == [0, 63, 25, (1 << 2) | (1 << 5) | (1 << 3)]
    # parent key is the child key shifted by 3
    rng = np.random.default_rng(7)
    p = rng.normal(size=(500, 3))
    k5, _, _ = oracle.leaf_keys(p, 5)
    k4, _, _ = oracle.leaf_keys(p, 4)
    assert np.array_equal(k5 >> 3, k4)


def test_root_cube_is_smallest_centred_cube():
    rng = np.random.default_rng(8)
    p = rng.normal(size=(300, 3)) * [1.0, 3.0, 0.5] + [5.0, -2.0, 1.0]
    lo, side = oracle.root_cube(p)
    assert side == (p.max(0) - p.min(0)).max()
    assert np.allclose(lo + side / 2, (p.max(0) + p.min(0)) / 2, rtol=0, atol=1e-15 * 10)
    # degenerate: a single ion gives a unit cube around it
    lo1, s1 = oracle.root_cube(np.array([[2.0, 3.0, 4.0]]))
    assert s1 == 1.0 and np.array_equal(lo1, [1.5, 2.5, 3.5])


def test_near_field_membership():
    # depth <= 1: every pair of leaves is adjacent -> near field = direct sum
    rng = np.random.default_rng(9)
    pos = rng.random((60, 3))
    q = np.full(60, Q)
    Ed, pd = oracle.coulomb_direct(pos, q)
    for d in (0, 1):
        En, pn = oracle.coulomb_near(pos, q, d)
        assert np.array_equal(En, Ed) and np.array_equal(pn, pd)
    # root cube [0.1, 1]^3, depth 2 (cells of 0.225): ions 0 and 1 share leaf
    # (0,0,0), ion 2 is in (3,0,0), ion 3 in (3,3,3) -> only ions 0 and 1 interact
    pos = np.array([[0.1, 0.1, 0.1], [0.3, 0.1, 0.1], [0.9, 0.1, 0.1], [1.0, 1.0, 1.0]])
    q = np.full(4, Q)
    En, pn = oracle.coulomb_near(pos, q, 2)
    assert pn[0] == pytest.approx(KE * Q / 0.2, rel=1e-15)
    assert pn[1] == pytest.approx(KE * Q / 0.2, rel=1e-15)
    assert pn[2] == 0.0 and En[2, 0] == 0.0


def test_sampled_targets_reproduce_the_full_sum():
    # The sampled-target sum is the same definition restricted to chosen
    # targets: at every sampled ion it equals the all-pairs sum exactly
    # (same pair expression, same ascending source order), and it sees the
    # ion's own charge nowhere.
    rng = np.random.default_rng(17)
    n = 300
    pos = rng.normal(size=(n, 3)) * 1e-5
    q = W.E_CHARGE * (1.0 + rng.random(n))
    E, phi = oracle.coulomb_direct(pos, q)
    idx = np.array([0, 7, 299, 150, 7])
    Es, ps = oracle.coulomb_targets(pos, q, idx)
    assert np.array_equal(Es, E[idx]) and np.array_equal(ps, phi[idx])
    # removing the target ion's charge changes nothing at that target
    q2 = q.copy()
    q2[150] = 0.0
    Es2, ps2 = oracle.coulomb_targets(pos, q2, np.array([150]))
    assert np.array_equal(Es2[0], E[150]) and ps2[0] == phi[150]
