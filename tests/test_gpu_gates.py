"""The accuracy gates of the hot path, through the C ABI, against the FP64
oracle (or the FP64 GPU direct sum, itself pinned to the oracle's to 1e-13 by
test_gpu_core.test_direct_matches_oracle).

  * Force: relative RMS error Err_F = sqrt(sum |F - F_ref|^2 / sum |F_ref|^2)
    (the vector analogue of the paper's potential error, Eq. rms_pot) at most
    1e-6 for the benchmark crystal (10,000 ions, aspect-0.3 spheroid) at the
    operating order p = 12, for the mixed BF16x3 path and the FP64 path, and
    for the 1e5-ion sweep sphere.  p = 10 does not reach 1e-6 on these
    crystals with the one-cell-gap interaction list (its FP64 truncation
    error alone is about 3e-6), so p = 12 is the operating point.
  * Energy: Error_en(t) = |E_r^gpu(t) - E_r^oracle(t)| / |E_r^oracle(t)|
    (Eq. rms_en, the rotating-frame energy of the two trajectories from the
    same start) at most 1e-8 over 1e4 steps with cooling off, from a start
    without close pairs (a jittered lattice at the rigid-rotor density),
    for the FP64 and the BF16x3 paths.
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
def spheroid10k():
    cr = W.crystal_spheroid_10k()
    Eo, _ = oracle.coulomb_direct(cr["pos"], cr["q"], want_phi=False)
    return cr["pos"], cr["q"], Eo


@pytest.mark.parametrize("precision,schedule", [("bf16x3", "pairs"), ("bf16x3", "tiles"),
                                                 ("fp64", "rotation"), ("fp64", "pairs")])
def test_benchmark_crystal_force_error_at_most_1e6(spheroid10k, precision, schedule):
    pos, q, Eo = spheroid10k
    plan = pt.Plan(len(q), p=12, leaf_max=32, depth=-1, precision=precision)
    plan.set_m2l_schedule(schedule)
    E, _ = plan.forces(dev_pos(pos), dev_vec(q), want_phi=False)
    err = rel(E.cpu().numpy().T, Eo)
    plan.close()
    assert err <= 1e-6, err


@pytest.mark.parametrize("precision", ["bf16x3", "fp64"])
def test_sweep_sphere_1e5_force_error_at_most_1e6(precision):
    w = W.sphere_sweep(100000)
    pd, qd = dev_pos(w["pos"]), dev_vec(w["q"])
    Ed, _ = pt.direct(pd, qd, want_phi=False)
    plan = pt.Plan(len(w["q"]), p=12, leaf_max=32, depth=-1, precision=precision)
    E, _ = plan.forces(pd, qd, want_phi=False)
    err = rel(E.cpu().numpy(), Ed.cpu().numpy())
    plan.close()
    assert err <= 1e-6, err


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_two_ions_in_one_leaf(precision):
    # two ions share the only leaf: the field is the FP32 (or FP64) pair sum
    # in leaf-relative fixed-point coordinates, exact separations rounded
    # once, so the closed form k_e q / r^2 holds to a few FP32 roundings
    plan = pt.Plan(2, p=6, precision=precision)
    r = 7e-6
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    E, _ = plan.forces(dev_pos(pos), dev_vec([W.E_CHARGE, W.E_CHARGE]))
    want = W.E_CHARGE / (4 * math.pi * W.EPS0) / r**2
    e = E.cpu().numpy()
    tol = 1e-14 if precision == "fp64" else 1e-6
    assert abs(e[0, 1] - want) <= tol * want and abs(e[0, 0] + want) <= tol * want
    assert e[1, 0] == e[2, 0] == e[1, 1] == e[2, 1] == 0.0
    plan.close()


@pytest.fixture(scope="module")
def lattice_trajectory():
    """Oracle trajectory of the 1,000-ion lattice start, energies every 1,000
    steps up to 1e4 (cooling off, dt = 1 ns)."""
    cr = W.crystal_lattice_1k()
    pos, vel, q, tr = cr["pos"], cr["vel"], cr["q"], cr["trap"]
    p, v = pos, vel
    energies = []
    for k in range(10):
        p, v = oracle.step(p, v, q, tr, 1e-9, 1000, t0=k * 1000e-9, step0=k * 1000)
        energies.append(oracle.energy_rot(p, v, q, tr, (k + 1) * 1000e-9)[3])
    return cr, energies


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_energy_error_over_1e4_steps(lattice_trajectory, precision):
    cr, eo = lattice_trajectory
    pos, vel, q, tr = cr["pos"], cr["vel"], cr["q"], cr["trap"]
    plan = pt.Plan(len(q), p=12, leaf_max=32, depth=-1, precision=precision)
    st = pt.State.from_numpy(pos, vel, q, device=DEV)
    errs = []
    for k in range(10):
        plan.step(st, tr, None, 1e-9, 1000)
        eg = pt.energy(st, tr)[3]
        errs.append(abs(eg - eo[k]) / abs(eo[k]))
    plan.close()
    assert st.step == 10000
    assert max(errs) <= 1e-8, errs
