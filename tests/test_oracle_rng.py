"""Pins of the oracle's random numbers, exponential and photon-kick sampling.

Each check compares against something other than the oracle itself: cuRAND's
host-side Philox4x32-10 generator (a library implementation of the same
published generator), numpy's exp, scipy's Poisson quantile function, and the
closed-form moments of Poisson counts and isotropic unit vectors.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

CURAND = "/usr/local/cuda/lib64/libcurand.so"


def _curand_blocks(seed, n_blocks):
    try:
        lib = ctypes.CDLL(CURAND if os.path.exists(CURAND) else "libcurand.so")
    except OSError:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    buf = np.zeros(4 * n_blocks, np.uint32)
    assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p),
                              ctypes.c_size_t(buf.size)) == 0
    lib.curandDestroyGenerator(gen)
    return buf.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEFCAFEBABE, 2**63 + 12345])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host Philox4x32-10 emits block b from counter (0, 0, b, 0) with
    # key (seed lo, seed hi).  Agreement over many blocks and keys pins the
    # round function, the multipliers and the key schedule.
    blocks = _curand_blocks(seed, 512)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in list(range(0, 512, 7)) + [511]:
        assert oracle.philox4x32_10([0, 0, b, 0], key) == [int(v) for v in blocks[b]]


def test_u01_is_exact_53_bit_grid():
    assert oracle.u01(0, 0) == 0.0
    assert oracle.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0**-53
    assert oracle.u01(1 << 31, 0) == 0.5
    assert oracle.u01(0, 1 << 6) == 2.0**-53


def test_exp_against_numpy_within_two_ulp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-700, 700, 4000), rng.uniform(-1, 1, 4000),
                         rng.uniform(-1e-6, 1e-6, 500), np.array([0.0, 1.0, -1.0, 0.5, -0.5])])
    worst = 0.0
    for x in xs:
        ref = math.exp(x)
        got = oracle.exp(x)
        worst = max(worst, abs(got - ref) / math.ulp(ref))
    assert worst <= 2.0, worst
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-800.0) == 0.0
    assert oracle.exp(800.0) == math.inf
    # subnormal range stays within a relative 1e-12 of libm
    for x in (-710.0, -720.0, -740.0):
        assert abs(oracle.exp(x) - math.exp(x)) <= 1e-12 * math.exp(x) + 5e-324


def test_poisson_inversion_matches_scipy_quantile():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(1)
    for lam in (1e-3, 3e-2, 1.0, 4.0, 15.0):
        us = rng.random(3000)
        for u in us:
            k = oracle.poisson(lam, u)
            # smallest k with CDF(k) > u; skip u within 1e-12 of a step
            cdf_k = stats.poisson.cdf(k, lam)
            cdf_km1 = stats.poisson.cdf(k - 1, lam) if k > 0 else 0.0
            if min(abs(cdf_k - u), abs(cdf_km1 - u)) < 1e-12:
                continue
            assert cdf_km1 <= u < cdf_k, (lam, u, k)


def _rate_closed_form_beam(S0):
    return {"s0": S0, "detuning": -0.5 * W.GAMMA0, "k": (0.0, 0.0, W.K_313), "uniform": True}


def test_scattering_rate_closed_forms():
    g0 = W.GAMMA0
    # uniform axial beam, Delta = -gamma0/2, v = 0: gamma = gamma0 S / (2 + 2S)
    for S in (5e-3, 0.5, 2.0):
        b = _rate_closed_form_beam(S)
        got = oracle.scatter_rate(b, g0, 0.0, 0.0, (0.0, 0.0, 0.0))
        assert got == pytest.approx(g0 * S / (2 + 2 * S), rel=1e-14)
    # on Doppler resonance Delta = k.v: gamma = gamma0 S / (1 + 2S)
    b = _rate_closed_form_beam(0.3)
    vz = -0.5 * W.GAMMA0 / W.K_313
    got = oracle.scatter_rate(b, g0, 0.0, 0.0, (0.0, 0.0, vz))
    assert got == pytest.approx(g0 * 0.3 / 1.6, rel=1e-12)
    # far off resonance the rate falls as the Lorentzian tail
    got = oracle.scatter_rate(b, g0, 0.0, 0.0, (0.0, 0.0, 1e4))
    det = -0.5 * g0 - W.K_313 * 1e4
    assert got == pytest.approx(0.3 * g0 * (g0 / 2) ** 2 / ((g0 / 2) ** 2 * 1.6 + det * det), rel=1e-12)


def test_planar_profile_is_gaussian_in_y_and_z():
    b = W.planar_beam(s0=0.5)
    d, wy, wz = b["offset_d"], b["waist_y"], b["waist_z"]
    assert oracle.saturation(b, d, 0.0) == pytest.approx(0.5, rel=1e-15)
    assert oracle.saturation(b, d + wy, 0.0) == pytest.approx(0.5 / math.e, rel=1e-14)
    assert oracle.saturation(b, d - 2 * wy, 0.0) == pytest.approx(0.5 * math.exp(-4), rel=1e-14)
    assert oracle.saturation(b, d, wz) == pytest.approx(0.5 / math.e, rel=1e-14)


def _big_beam(S, det, k):
    return {"s0": S, "detuning": det, "k": k, "uniform": True}


def test_photon_counts_are_poisson_with_the_rate():
    # one uniform beam, v = 0, rate from the closed form; lambda = rate * dt ~ 0.7
    n = 40000
    beam = _big_beam(1.0, -0.5 * W.GAMMA0, (0.0, 0.0, W.K_313))
    rate = W.GAMMA0 * 1.0 / 4.0
    dt = 0.7 / rate
    pos = np.zeros((n, 3))
    vel = np.zeros((n, 3))
    counts, dv = oracle.laser_kick(pos, vel, [beam], W.GAMMA0, W.MASS, 99, 5, dt)
    lam = rate * dt
    c = counts[:, 0].astype(float)
    assert abs(c.mean() - lam) < 5 * math.sqrt(lam / n)
    # variance of a Poisson count equals its mean (5 sigma on the variance estimator)
    assert abs(c.var() - lam) < 5 * math.sqrt((lam + 2 * lam * lam) / n)
    # P(0) = exp(-lambda)
    p0 = (c == 0).mean()
    assert abs(p0 - math.exp(-lam)) < 5 * math.sqrt(p0 * (1 - p0) / n)


def test_recoil_is_absorption_plus_isotropic_emission():
    n = 60000
    k = W.K_313
    beam = _big_beam(1.0, -0.5 * W.GAMMA0, (k, 0.0, 0.0))
    rate = W.GAMMA0 / 4.0
    dt = 1.0 / rate
    counts, dv = oracle.laser_kick(np.zeros((n, 3)), np.zeros((n, 3)), [beam], W.GAMMA0, W.MASS,
                                   7, 11, dt)
    rk = 1.054571817e-34 / W.MASS
    one = counts[:, 0] == 1
    # single-photon ions: dv = hbar k/m x_hat + hbar |k|/m q_hat, |q_hat| = 1
    qhat = (dv[one] - np.array([rk * k, 0, 0])) / (rk * k)
    assert np.allclose(np.linalg.norm(qhat, axis=1), 1.0, atol=1e-12)
    m = len(qhat)
    assert np.all(np.abs(qhat.mean(0)) < 5 * math.sqrt(1 / 3 / m))
    second = qhat.T @ qhat / m
    assert np.allclose(second, np.eye(3) / 3, atol=5 * math.sqrt(2 / 15 / m) + 5e-3)
    # mean momentum per absorbed photon is hbar k (emission averages out)
    total = counts[:, 0].sum()
    mean_dv = dv.sum(0) / total
    sig = rk * k * math.sqrt(1 / 3 / total)
    assert abs(mean_dv[0] - rk * k) < 5 * sig
    assert abs(mean_dv[1]) < 5 * sig and abs(mean_dv[2]) < 5 * sig
    # ions without photons get no kick
    assert np.all(dv[counts[:, 0] == 0] == 0.0)


def test_kicks_depend_only_on_seed_step_ion_beam():
    beams = W.cooling_beams(planar_s0=0.5)
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(300, 3)) * 5e-6
    vel = rng.normal(size=(300, 3)) * 3.0
    a = oracle.laser_kick(pos, vel, beams, W.GAMMA0, W.MASS, 123, 77, 1e-6)
    b = oracle.laser_kick(pos, vel, beams, W.GAMMA0, W.MASS, 123, 77, 1e-6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # a subset of ions (same indices) sees the same draws
    c = oracle.laser_kick(pos[:100], vel[:100], beams, W.GAMMA0, W.MASS, 123, 77, 1e-6)
    assert np.array_equal(a[0][:100], c[0]) and np.array_equal(a[1][:100], c[1])
    d = oracle.laser_kick(pos, vel, beams, W.GAMMA0, W.MASS, 123, 78, 1e-6)
    assert not np.array_equal(a[0], d[0])


def test_paper_parameters_in_presets():
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))
    assert W.GAMMA0 == pytest.approx(2 * math.pi * gold["gamma0_over_2pi_hz"]["value"], rel=1e-15)
    ax = W.axial_beams()
    assert ax[0]["s0"] == gold["axial_saturation"]["value"]
    assert ax[0]["detuning"] == pytest.approx(gold["axial_detuning_over_gamma0"]["value"] * W.GAMMA0)
    pb = W.paper_beams()[2]
    assert pb["s0"] == gold["planar_saturation_paper"]["value"]
    assert pb["offset_d"] == gold["planar_offset_d_m"]["value"]
    assert pb["waist_y"] == gold["planar_waist_y_m"]["value"]
    assert pb["detuning"] == pytest.approx(2 * math.pi * gold["planar_detuning_over_2pi_hz"]["value"])
