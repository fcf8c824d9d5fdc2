"""GPU parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances (relative RMS over ions, Err = sqrt(sum |a-b|^2 / sum |b|^2)):
  * FP64 direct sum vs oracle direct sum: 1e-13 (rounding order only);
  * near field (adjacent-leaf pair sum) FP64: 1e-12; FP32: 3e-6 (FP32
    pair arithmetic in leaf-relative coordinates, ~2^-23 per pair);
  * FMM vs the direct sum: the truncation error of order p, decreasing
    geometrically, with the p = 10 bound measured on the same inputs;
  * integer and index results (octree keys, permutation, photon counts) and
    the FP64 push of a lone ion: bit-exact.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2405_13973_gb300 as pt
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def dev_pos(pos):
    return torch.tensor(np.ascontiguousarray(pos.T), dtype=torch.float64, device=DEV)


def dev_vec(v):
    return torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def sphere4k():
    w = W.sphere_sweep(4000, seed=21)
    Eo, phio = oracle.coulomb_direct(w["pos"], w["q"])
    return w["pos"], w["q"], Eo, phio


def test_direct_matches_oracle(sphere4k):
    pos, q, Eo, phio = sphere4k
    E, phi = pt.direct(dev_pos(pos), dev_vec(q))
    torch.cuda.synchronize()
    assert rel(E.cpu().numpy().T, Eo) < 1e-13
    assert rel(phi.cpu().numpy(), phio) < 1e-13


@pytest.mark.parametrize("n,depth", [(1, 0), (2, 1), (37, 2), (3000, 4), (5000, 5)])
def test_tree_keys_and_permutation_bit_exact(n, depth):
    rng = np.random.default_rng(n)
    pos = rng.normal(size=(n, 3)) * [30e-6, 20e-6, 10e-6]
    q = np.full(n, W.E_CHARGE)
    plan = pt.Plan(n, p=4, depth=depth, precision="fp64")
    plan.forces(dev_pos(pos), dev_vec(q))
    root, perm, keys = plan.tree_info(n)
    ko, lo, side = oracle.leaf_keys(pos, depth)
    assert root[:3] == list(lo) and root[3] == side
    assert np.array_equal(keys.cpu().numpy().astype(np.uint32).astype(np.uint64), ko)
    assert np.array_equal(perm.cpu().numpy(), np.argsort(ko, kind="stable"))
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("depth", [2, 3, 4])
def test_near_field_matches_oracle(sphere4k, precision, tol, depth):
    pos, q, _, _ = sphere4k
    plan = pt.Plan(len(q), p=6, depth=depth, precision=precision)
    plan.set_phases(pt.PT_PHASE_NEAR)
    E, phi = plan.forces(dev_pos(pos), dev_vec(q))
    En, pn = oracle.coulomb_near(pos, q, depth)
    assert rel(E.cpu().numpy().T, En) < tol
    assert rel(phi.cpu().numpy(), pn) < tol
    plan.close()


def test_fmm_fp64_converges_geometrically_in_p(sphere4k):
    pos, q, Eo, phio = sphere4k
    errs = []
    for p in (4, 6, 8, 10, 12):
        plan = pt.Plan(len(q), p=p, depth=3, precision="fp64")
        E, phi = plan.forces(dev_pos(pos), dev_vec(q))
        errs.append((rel(E.cpu().numpy().T, Eo), rel(phi.cpu().numpy(), phio)))
        plan.close()
    eF = [e[0] for e in errs]
    assert all(b < a * 0.6 for a, b in zip(eF, eF[1:])), errs
    # p = 10 at depth 3 on this sphere: truncation error of the one-cell-gap
    # FMM (measured ~2.6e-6 for the force, ~4e-8 for the potential)
    assert eF[3] < 5e-6, errs
    assert errs[3][1] < 1e-7, errs


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_fmm_auto_depth_error(sphere4k, precision):
    pos, q, Eo, phio = sphere4k
    plan = pt.Plan(len(q), p=10, leaf_max=32, depth=-1, precision=precision)
    E, phi = plan.forces(dev_pos(pos), dev_vec(q))
    d = plan.last_depth
    ko, _, _ = oracle.leaf_keys(pos, d)
    assert len(q) / len(np.unique(ko)) <= 32
    if d > 0:
        kp, _, _ = oracle.leaf_keys(pos, d - 1)
        assert len(q) / len(np.unique(kp)) > 32
    eF = rel(E.cpu().numpy().T, Eo)
    assert eF < {"fp64": 1e-5, "fp32": 2e-5, "tf32x3": 2e-5, "bf16x3": 2e-5}[precision], (d, eF)
    plan.close()


@pytest.mark.parametrize("tc", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("depth", [2, 3, 4])
def test_tensor_core_m2l_matches_cuda_core_m2l(sphere4k, depth, tc):
    # Far field (P2M, M2M, M2L, L2L, L2P) with M2M/M2L/L2L on the tensor cores
    # vs the same stages in FP32 on the CUDA cores: they differ only by the
    # split-product rounding (about 2^-21 per 3xTF32 product, 2^-24 per
    # BF16x3 product, the same as an FP32 multiply) and the FP32 sums.
    pos, q, Eo, _ = sphere4k
    out = {}
    for prec in ("fp32", tc):
        plan = pt.Plan(len(q), p=10, depth=depth, precision=prec)
        plan.set_phases(pt.PT_PHASE_FAR)
        E, _ = plan.forces(dev_pos(pos), dev_vec(q))
        out[prec] = E.cpu().numpy().T
        plan.close()
    assert rel(out[tc], out["fp32"]) < {"tf32x3": 1e-5, "bf16x3": 5e-6}[tc]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp32", "fp64"])
@pytest.mark.parametrize("depth", [2, 3, 4, 5])
def test_pair_schedule_equals_tile_schedule(sphere4k, depth, prec):
    # The two M2L schedules compute the same translations and differ only in
    # the order of the sums (tensor cores: FP32 in tensor memory over runs of
    # offsets vs one partial per pair, summed in offset order; CUDA cores:
    # per-target loops over the offsets vs the same per-pair partials): the
    # far fields agree to the arithmetic's rounding, and the pair schedule is
    # deterministic (bitwise equal on a second evaluation).
    # The rotation schedule (CUDA cores) factors every translation as rotate,
    # translate along z, rotate back: equal to the dense operator up to
    # rounding.
    pos, q, Eo, _ = sphere4k
    out = {}
    scheds = ("tiles", "pairs") if prec in ("tf32x3", "bf16x3") else ("tiles", "pairs", "rotation")
    for sched in scheds:
        plan = pt.Plan(len(q), p=10, depth=depth, precision=prec)
        plan.set_m2l_schedule(sched)
        assert plan.m2l_schedule == sched
        plan.set_phases(pt.PT_PHASE_FAR)
        E, _ = plan.forces(dev_pos(pos), dev_vec(q))
        out[sched] = E.cpu().numpy().T
        if sched != "tiles":
            E2, _ = plan.forces(dev_pos(pos), dev_vec(q))
            assert np.array_equal(E2.cpu().numpy().T, out[sched])
        plan.close()
    for sched in scheds[1:]:
        assert rel(out[sched], out["tiles"]) < (1e-12 if prec == "fp64" else 2e-6), sched


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-7), ("fp32", 1e-6)])
def test_rotation_m2l_at_p16_against_the_oracle(sphere4k, precision, tol):
    # Order 16 (beyond the tensor-core paths): the rotation-based M2L, and
    # the dense per-pair M2L beside it, against the oracle's direct sum; the
    # two factorisations of the same operator agree to rounding.
    pos, q, Eo, _ = sphere4k
    out = {}
    for sched in ("rotation", "pairs"):
        plan = pt.Plan(len(q), p=16, depth=3, precision=precision)
        plan.set_m2l_schedule(sched)
        E, _ = plan.forces(dev_pos(pos), dev_vec(q))
        out[sched] = E.cpu().numpy().T
        plan.close()
    assert rel(out["rotation"], Eo) < tol
    assert rel(out["rotation"], out["pairs"]) < (1e-13 if precision == "fp64" else 1e-6)


def test_fp64_error_keeps_falling_through_order_16_on_a_planar_crystal():
    # In a planar crystal the ions sit where the sectoral harmonics Y_n^n are
    # largest, so the last column of an order-16 expansion (m = 16, degree 16
    # only) carries a large share of its degree-16 terms: were it dropped
    # anywhere on the path, the error would stall between p = 15 and 16.
    n = 4000
    pos = W.spheroid(n, 100e-6, 0.1e-6, seed=31)
    q = W.charges(n)
    Eo, _ = oracle.coulomb_direct(pos, q, want_phi=False)
    errs = []
    for p in (14, 15, 16):
        plan = pt.Plan(n, p=p, depth=3, precision="fp64")
        E, _ = plan.forces(dev_pos(pos), dev_vec(q), want_phi=False)
        errs.append(rel(E.cpu().numpy().T, Eo))
        plan.close()
    assert errs[1] < 0.9 * errs[0] and errs[2] < 0.9 * errs[1], errs


def test_rotation_schedule_is_refused_on_the_tensor_cores():
    plan = pt.Plan(100, p=8, precision="bf16x3")
    with pytest.raises(pt.PenningError) as ei:
        plan.set_m2l_schedule("rotation")
    assert ei.value.status == pt.PT_ERR_UNSUPPORTED
    plan.close()


def test_field_of_one_and_two_ions():
    for precision in ("fp64", "fp32", "tf32x3", "bf16x3"):
        plan = pt.Plan(2, p=6, precision=precision)
        E, phi = plan.forces(dev_pos(np.array([[1e-5, -2e-5, 3e-5]])), dev_vec([W.E_CHARGE]))
        assert torch.all(E == 0) and torch.all(phi == 0)
        r = 7e-6
        pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        E, phi = plan.forces(dev_pos(pos), dev_vec([W.E_CHARGE, W.E_CHARGE]))
        ke = 1 / (4 * math.pi * W.EPS0)
        want = ke * W.E_CHARGE / r**2
        e = E.cpu().numpy()
        tol = 1e-14 if precision == "fp64" else 1e-6
        assert abs(e[0, 1] - want) < tol * want and abs(e[0, 0] + want) < tol * want
        plan.close()


def _laser(seed=9, s0=0.5):
    beams = W.cooling_beams(planar_s0=s0)
    return beams, pt.make_laser(beams, seed=seed, gamma0=W.GAMMA0)


def test_laser_kicks_bit_exact():
    n = 20000
    rng = np.random.default_rng(5)
    pos = np.stack([rng.normal(size=n) * 20e-6, 5e-6 + rng.normal(size=n) * 3e-6,
                    rng.normal(size=n) * 20e-6], 1)
    vel = rng.normal(size=(n, 3)) * 20.0
    beams = W.cooling_beams(planar_s0=2.0)
    laser = pt.make_laser(beams, seed=0xABCDEF1234, gamma0=W.GAMMA0)
    dt = 2e-7  # large rates: many multi-photon steps
    counts, dv = pt.laser_kicks(laser, W.MASS, dev_pos(pos), dev_pos(vel), 123456789, dt)
    co, dvo = oracle.laser_kick(pos, vel, beams, W.GAMMA0, W.MASS, 0xABCDEF1234, 123456789, dt)
    c = counts.cpu().numpy()
    assert c.sum() > n  # the test exercises multi-photon kicks
    assert np.array_equal(c, co)
    assert np.array_equal(dv.cpu().numpy().T, dvo)


@pytest.mark.parametrize("laser_on", [False, True])
def test_lone_ion_trajectory_bit_exact(laser_on):
    tr = W.trap(beta=0.6, delta=0.02)
    pos = np.array([[12e-6, 4e-6, -3e-6]])
    vel = W.rotating_maxwellian(pos, tr["omega_r"], 10e-3, seed=2)
    beams, laser = _laser(seed=17, s0=5.0)
    plan = pt.Plan(1, p=4, precision="fp64")
    st = pt.State.from_numpy(pos, vel, [W.E_CHARGE], device=DEV, t=1.5e-6, step=40)
    plan.step(st, tr, laser if laser_on else None, 1e-9, 700)
    po, vo = oracle.step(pos, vel, [W.E_CHARGE], tr, 1e-9, 700, t0=1.5e-6, step0=40,
                         beams=beams if laser_on else (), gamma0=W.GAMMA0, seed=17,
                         laser_on=laser_on)
    assert np.array_equal(st.pos().cpu().numpy(), po)
    assert np.array_equal(st.vel().cpu().numpy(), vo)
    assert st.step == 740 and st.t == 1.5e-6 + 700 * 1e-9
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_one_step_is_the_drift_plus_the_fmm_field_kick(precision):
    # After one step the GPU and oracle states differ only through the field:
    # v_gpu - v_oracle = R(w_c dt/2) (q/m) dt (E_fmm(x_mid) - E_direct(x_mid)),
    # with E_fmm the plan's own field at the midpoint (Eq. time_ev2).
    cr = W.crystal_sphere_1k(seed=4)
    n = 600
    pos, vel, q, tr = cr["pos"][:n], cr["vel"][:n], cr["q"][:n], cr["trap"]
    dt = 1e-9
    plan = pt.Plan(n, p=12, depth=2, precision=precision)
    st = pt.State.from_numpy(pos, vel, q, device=DEV)
    plan.step(st, tr, None, dt, 1)
    po, vo = oracle.step(pos, vel, q, tr, dt, 1)
    wc = W.omega_c()
    xm, _ = oracle.u0(pos, vel, 0.5 * dt, wc)
    Ef, _ = plan.forces(dev_pos(xm), dev_vec(q))
    Ed, _ = oracle.coulomb_direct(xm, q)
    dE = Ef.cpu().numpy().T - Ed
    kick = (q / tr["mass"])[:, None] * dE * dt
    c, s_ = math.cos(wc * 0.5 * dt), math.sin(wc * 0.5 * dt)
    want = np.stack([kick[:, 0] * c + kick[:, 1] * s_, -kick[:, 0] * s_ + kick[:, 1] * c,
                     kick[:, 2]], 1)
    got = st.vel().cpu().numpy() - vo
    assert np.abs(got - want).max() < 1e-6 * np.abs(want).max() + 1e-12, (
        np.abs(got - want).max(), np.abs(want).max())
    gotx = st.pos().cpu().numpy() - po
    assert np.abs(gotx).max() < 0.5 * dt * 1.01 * np.abs(want).max() + 1e-18
    plan.close()


@pytest.mark.slow
def test_rotating_frame_energy_over_a_thousand_steps():
    # Cooling off, a start without close pairs (jittered lattice at the
    # rigid-rotor density): the GPU conserves the rotating-frame energy as the
    # oracle does (bounded splitting oscillation, no secular drift), and the
    # energies of the two trajectories agree (Eq. rms_en, GPU vs oracle).
    cr = W.crystal_lattice_1k()
    pos, vel, q, tr = cr["pos"], cr["vel"], cr["q"], cr["trap"]
    plan = pt.Plan(1000, p=12, precision="fp64")
    st = pt.State.from_numpy(pos, vel, q, device=DEV)
    e0 = oracle.energy_rot(pos, vel, q, tr, 0.0)[3]
    p, v = pos, vel
    drifts, errs = [], []
    for k in range(5):
        plan.step(st, tr, None, 1e-9, 200)
        p, v = oracle.step(p, v, q, tr, 1e-9, 200, t0=k * 200e-9, step0=k * 200)
        eg = pt.energy(st, tr)[3]
        eo = oracle.energy_rot(p, v, q, tr, (k + 1) * 200e-9)[3]
        drifts.append(abs(eg - e0) / abs(e0))
        errs.append(abs(eg - eo) / abs(eo))
    assert max(drifts) < 3e-7, drifts
    assert max(errs) < 1e-8, errs
    plan.close()


def test_energy_matches_oracle():
    cr = W.crystal_sphere_1k(seed=6)
    st = pt.State.from_numpy(cr["pos"], cr["vel"], cr["q"], device=DEV, t=3.3e-7)
    e = pt.energy(st, cr["trap"])
    eo = oracle.energy_rot(cr["pos"], cr["vel"], cr["q"], cr["trap"], 3.3e-7)
    for a, b in zip(e, eo):
        assert a == pytest.approx(b, rel=1e-12, abs=1e-12 * abs(eo[3]))
    plan = pt.Plan(1000, p=10, precision="fp64")
    ef = pt.energy(st, cr["trap"], plan)
    assert ef[2] == pytest.approx(eo[2], rel=1e-7)
    plan.close()


def test_nonfinite_position_is_reported():
    pos = np.random.default_rng(1).normal(size=(50, 3)) * 1e-5
    pos[7, 1] = np.nan
    plan = pt.Plan(50, p=4, precision="fp64")
    with pytest.raises(pt.PenningError) as ei:
        plan.forces(dev_pos(pos), dev_vec(np.full(50, W.E_CHARGE)))
        torch.cuda.synchronize()
    assert ei.value.status == pt.PT_ERR_NONFINITE
    # the plan stays usable
    pos[7, 1] = 0.0
    E, _ = plan.forces(dev_pos(pos), dev_vec(np.full(50, W.E_CHARGE)))
    assert torch.isfinite(E).all()
    plan.close()
