"""GPU force evaluation at the sweep sizes (N = 1e5 and 1e6 ions uniform in a
sphere at 2e14 m^-3 plus 1% jitter), through the C ABI.

References: at N = 1e5 the FP64 direct sum on the GPU (itself checked against
the oracle's direct sum at N = 4000 in test_gpu_core); at N = 1e6 the
oracle's direct sum at 512 sampled ions (the full O(N^2) sum is out of reach
on the host).

Tolerances, relative RMS force error (Err = sqrt(sum|E - E_ref|^2 /
sum|E_ref|^2), the force analogue of Eq. rms_pot):
  * FP64 FMM, automatic depth (5 at 1e5): about twice the truncation error of
    order p (measured 7.6e-4, 7.9e-6, 3.5e-7 at p = 4, 8, 12), falling by more
    than an order of magnitude per four orders;
  * FP32 CUDA cores and BF16x3 tensor cores at p = 12: the 1e-6 force-error
    target (measured 4.6e-7 and 5.6e-7 at 1e5, BF16x3 6.9e-7 at 1e6 on the
    sampled ions).
"""
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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def sphere100k():
    w = W.sphere_sweep(100000, seed=3)
    pos, q = w["pos"], w["q"]
    pd, qd = dev(pos.T), dev(q)
    Ed, _ = pt.direct(pd, qd, want_phi=False)
    return pd, qd, Ed.cpu().numpy().T


def fmm_field(pd, qd, n, p, precision):
    plan = pt.Plan(n, p=p, leaf_max=32, depth=-1, precision=precision)
    E, _ = plan.forces(pd, qd, want_phi=False)
    depth = plan.last_depth
    plan.close()
    return E.cpu().numpy().T, depth


def test_fp64_fmm_error_falls_with_order_at_1e5(sphere100k):
    pd, qd, Ed = sphere100k
    errs = {}
    for p in (4, 8, 12):
        E, depth = fmm_field(pd, qd, 100000, p, "fp64")
        errs[p] = rel(E, Ed)
    assert depth == 5
    assert errs[4] < 1.5e-3 and errs[8] < 1.6e-5 and errs[12] < 7e-7, errs
    assert errs[8] < errs[4] / 10 and errs[12] < errs[8] / 10, errs


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-6), ("bf16x3", 1e-6)])
def test_mixed_precision_at_1e5(sphere100k, precision, tol):
    pd, qd, Ed = sphere100k
    E, _ = fmm_field(pd, qd, 100000, 12, precision)
    assert rel(E, Ed) < tol


def test_bf16x3_at_1e6_on_sampled_ions():
    n = 1000000
    w = W.sphere_sweep(n, seed=3)
    pos, q = w["pos"], w["q"]
    idx = np.random.default_rng(0).choice(n, 512, replace=False)
    Eo, _ = oracle.coulomb_targets(pos, q, idx, want_phi=False)
    E, depth = fmm_field(dev(pos.T), dev(q), n, 12, "bf16x3")
    assert depth == 6
    assert np.all(np.isfinite(E))
    assert rel(E[idx], Eo) < 1e-6
