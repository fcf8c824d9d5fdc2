"""GPU Metropolis-Hastings potential-energy initialisation (Sec. 4) against the
oracle's sequential scans, through the C ABI.

The proposals (Philox stream, Marsaglia direction, distance) and the external
energy are the same IEEE sequences on both sides; the Coulomb change is a
parallel FP64 sum on the GPU and a sequential one in the oracle, so the two
dE differ in the last bits only and every accept decision agrees unless a
uniform falls within ~1e-16 of its threshold.  So positions and accept counts
are compared exactly, and the sums of accepted energy changes to 1e-9.  Both
kernels are covered: the 8-CTA cluster (up to 4096 ions) and one block.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2405_13973_gb300 as pt
import workloads as W

pytestmark = pytest.mark.gpu


def crystal(n):
    cr = W.crystal_sphere_1k(seed=11)
    if n <= 1000:
        return cr["pos"][:n].copy(), cr["q"][:n].copy(), dict(cr["trap"], delta=0.02)
    w = W.sphere_sweep(n, seed=4)
    return w["pos"], w["q"], dict(cr["trap"], delta=0.02)


@pytest.mark.parametrize("n,scans", [(300, 3), (1500, 2), (5000, 1)])  # cluster path up to 4096
def test_mh_scans_match_the_oracle(n, scans):
    pos, q, trap = crystal(n)
    t = 3.7e-7
    cs = (math.cos(trap["omega_r"] * t), math.sin(trap["omega_r"] * t))
    po, acc_o, de_o = oracle.mh_scans(pos, q, trap, 10e-3, 1e-6, 17, 5, scans, cs)
    st = pt.State.from_numpy(pos, np.zeros_like(pos), q, t=t)
    acc, de = pt.mh_scans(st, trap, 10e-3, 1e-6, 17, 5, scans)
    assert 0 < acc_o < n * scans
    assert acc == acc_o
    assert np.array_equal(st.pos().cpu().numpy(), po)
    assert abs(de - de_o) <= 1e-9 * abs(de_o)


def test_mh_resumes_by_scan_index():
    pos, q, trap = crystal(200)
    a = pt.State.from_numpy(pos, np.zeros_like(pos), q)
    b = pt.State.from_numpy(pos, np.zeros_like(pos), q)
    n1, _ = pt.mh_scans(a, trap, 10e-3, 1e-6, 3, 0, 3)
    m1, _ = pt.mh_scans(b, trap, 10e-3, 1e-6, 3, 0, 2)
    m2, _ = pt.mh_scans(b, trap, 10e-3, 1e-6, 3, 2, 1)
    assert n1 == m1 + m2
    assert torch.equal(a.pos(), b.pos())


def test_mh_rejects_bad_arguments():
    pos, q, trap = crystal(10)
    st = pt.State.from_numpy(pos, np.zeros_like(pos), q)
    with pytest.raises(pt.PenningError):
        pt.mh_scans(st, trap, 0.0, 1e-6, 1, 0, 1)
    with pytest.raises(pt.PenningError):
        pt.mh_scans(st, trap, 10e-3, -1e-6, 1, 0, 1)
