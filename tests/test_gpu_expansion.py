"""Ancestor expansions of the tensor-core paths computed two ways (Sec. 2.3.1):
the passes (P2M at the leaves, M2M shifts up, M2L, L2L shifts down, L2P at the
leaves) and directly (P2M of every ion about each of its ancestor cells, M2L,
L2P of every ancestor's own M2L sum at the ion).  M2M and L2L shift truncated
expansions exactly, so both give the same far field up to rounding.

Tolerances (relative RMS over ions): both routes round like FP32 (the split
tensor-core products of the shifts are FP32-grade for BF16x3, about 2^-21 for
3xTF32; the direct route evaluates the harmonics in FP32 at the ancestor's
scale), the same bounds as the tensor-core vs CUDA-core comparison.
"""
import numpy as np
import pytest
import torch

import paper_2405_13973_gb300 as pt
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = {"tf32x3": 1e-5, "bf16x3": 5e-6}


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.fixture(scope="module")
def sphere4k():
    w = W.sphere_sweep(4000, seed=21)
    pos = torch.tensor(np.ascontiguousarray(w["pos"].T), dtype=torch.float64, device=DEV)
    q = torch.tensor(w["q"], dtype=torch.float64, device=DEV)
    return pos, q


def far_field(pos, q, depth, precision, mode=None, p=10):
    plan = pt.Plan(q.numel(), p=p, depth=depth, precision=precision)
    plan.set_phases(pt.PT_PHASE_FAR)
    if mode is not None:
        plan.set_expansion(mode)
    E, phi = plan.forces(pos, q)
    out = (E.cpu().numpy().T, phi.cpu().numpy())
    plan.close()
    return out


@pytest.mark.parametrize("tc", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("depth", [2, 3, 4, 5])
def test_direct_ancestor_expansions_equal_the_passes(sphere4k, depth, tc):
    pos, q = sphere4k
    Et, pt_ = far_field(pos, q, depth, tc, pt.EXPAND_TREE)
    Ed, pd = far_field(pos, q, depth, tc, pt.EXPAND_DIRECT)
    Ef, pf = far_field(pos, q, depth, "fp32")
    assert np.all(np.isfinite(Ed))
    assert rel(Ed, Et) < TOL[tc], (rel(Ed, Et), rel(pd, pt_))
    assert rel(pd, pt_) < TOL[tc]
    # and both against the FP32 CUDA-core passes
    assert rel(Ed, Ef) < TOL[tc] and rel(Et, Ef) < TOL[tc], (rel(Ed, Ef), rel(Et, Ef))


def test_tree_is_the_default(sphere4k):
    pos, q = sphere4k
    Ea, _ = far_field(pos, q, 4, "bf16x3")
    Em, _ = far_field(pos, q, 4, "bf16x3", pt.EXPAND_TREE)
    assert np.array_equal(Ea, Em)


def test_bad_expansion_mode_is_rejected():
    plan = pt.Plan(100, p=4, depth=2, precision="bf16x3")
    with pytest.raises(pt.PenningError):
        plan.set_expansion(7)
    plan.close()
