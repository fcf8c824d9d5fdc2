"""Work accounting of the octree (Sec. 2.3): the interaction counts that
fmm_plan_stats reports, and the tensor-core M2L work list that
fmm_plan_tc_stats reports, against counts built here from the oracle's leaf
keys (plain numpy over the cells of each level).

Definitions counted:
  * M2L pairs: (target cell, source cell) at levels >= 2 where the source is
    a child of a neighbour of the target's parent, not a neighbour of the
    target, and holds ions (Sec. 2.3, the interaction list);
  * P2P pairs: ordered ion pairs i != j in the same or adjacent leaves;
  * shifts: one per cell at levels >= 3 (its M2M into the parent and its L2L
    from the parent);
  * tensor-core tiles: per level, cells in (child octant, parent Morton code)
    order, cut into 128-row tiles, per octant on levels holding at least 512
    cells and across octants below; a tile's products are the offsets with at
    least one admitted target row whose source cell holds ions;
  * pair-packed products: per offset, its pairs over every level, cut into
    runs of 128; with mirroring (the BF16x3 default), per pair of offsets
    {o, -o}, their pairs together.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2405_13973_gb300 as pt
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
ROWS = 128
MIXED_BELOW = 512


def decode(codes, l):
    """Cell coordinates of level-l Morton codes (bit 3i + a -> bit i of axis a)."""
    c = np.zeros((len(codes), 3), np.int64)
    for i in range(l):
        for a in range(3):
            c[:, a] |= ((codes >> np.uint64(3 * i + a)) & np.uint64(1)).astype(np.int64) << i
    return c


def expected_counts(pos, D):
    keys, _, _ = oracle.leaf_keys(pos, D)
    out = {"cells": 0, "m2l_pairs": 0, "shifts": 0, "tiles": 0, "products": 0, "rows": 0}
    offs = [(ox, oy, oz) for ox in range(-3, 4) for oy in range(-3, 4) for oz in range(-3, 4)
            if max(abs(ox), abs(oy), abs(oz)) > 1]
    per_offset = np.zeros(len(offs), np.int64)
    for l in range(2, D + 1):
        codes = np.unique(keys >> np.uint64(3 * (D - l)))
        oct_ = (codes & np.uint64(7)).astype(np.int64)
        order = np.lexsort((codes >> np.uint64(3), oct_))
        codes, oct_ = codes[order], oct_[order]
        xyz = decode(codes, l)
        lim = 1 << l
        occ = np.zeros((lim + 6,) * 3, bool)
        occ[xyz[:, 0] + 3, xyz[:, 1] + 3, xyz[:, 2] + 3] = True
        b = xyz & 1
        valid = np.zeros((len(codes), len(offs)), bool)
        for k, o in enumerate(offs):
            o = np.array(o)
            adm = np.all((o >= b - 3) & (o <= b + 2), axis=1)
            s = xyz - o + 3
            valid[:, k] = adm & occ[s[:, 0], s[:, 1], s[:, 2]]
        per_offset += valid.sum(0)
        out["cells"] += len(codes)
        out["m2l_pairs"] += int(valid.sum())
        out["shifts"] += len(codes) if l >= 3 else 0
        groups = ([np.arange(len(codes))] if len(codes) < MIXED_BELOW
                  else [np.where(oct_ == o)[0] for o in range(8)])
        for g in groups:
            for t0 in range(0, len(g), ROWS):
                rows = g[t0:t0 + ROWS]
                out["tiles"] += 1
                out["rows"] += len(rows)
                out["products"] += int(valid[rows].any(axis=0).sum())
    leaf = decode(np.unique(keys), D)
    cnt = {tuple(c): 0 for c in leaf}
    for c in decode(keys, D):
        cnt[tuple(c)] += 1
    p2p = 0
    for c, m in cnt.items():
        nb = sum(cnt.get((c[0] + dx, c[1] + dy, c[2] + dz), 0)
                 for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1))
        p2p += m * nb - m
    out["p2p_pairs"] = p2p
    out["leaves"] = len(cnt)
    out["pair_offsets"] = int((per_offset > 0).sum())
    out["pair_products"] = int(((per_offset + ROWS - 1) // ROWS).sum())
    # offsets o and -o as one (T_{-o} = (-1)^(j+l) T_o): each unordered pair once
    index = {o: k for k, o in enumerate(offs)}
    merged = np.array([per_offset[k] + per_offset[index[(-o[0], -o[1], -o[2])]]
                       for k, o in enumerate(offs) if o < (0, 0, 0)])
    assert len(merged) == len(offs) // 2
    out["pair_offsets_mirrored"] = int((merged > 0).sum())
    out["pair_products_mirrored"] = int(((merged + ROWS - 1) // ROWS).sum())
    return out


@pytest.mark.parametrize("crystal,D", [("spheroid10k", 4), ("sphere3k", 3), ("sphere3k", 5)])
def test_interaction_and_work_list_counts(crystal, D):
    if crystal == "spheroid10k":
        pos = W.crystal_spheroid_10k()["pos"]
    else:
        pos = W.sphere_sweep(3000, seed=5)["pos"]
    n = len(pos)
    q = np.full(n, W.E_CHARGE)
    plan = pt.Plan(n, p=12, depth=D, precision="bf16x3")
    plan.set_m2l_schedule("tiles")
    pd = torch.tensor(np.ascontiguousarray(pos.T), dtype=torch.float64, device=DEV)
    plan.forces(pd, torch.tensor(q, dtype=torch.float64, device=DEV), want_phi=False)
    st, tc = plan.stats(), plan.tc_stats()
    plan.set_m2l_schedule("pairs")
    qd = torch.tensor(q, dtype=torch.float64, device=DEV)
    e_mirrored = plan.forces(pd, qd, want_phi=False)[0].cpu().numpy()
    tm = plan.tc_stats()
    plan.set_m2l_mirror(False)
    e_plain = plan.forces(pd, qd, want_phi=False)[0].cpu().numpy()
    tp = plan.tc_stats()
    plan.close()
    ex = expected_counts(pos, D)
    # pair-packed work list: offsets with pairs, 128-row runs per offset, every pair once
    assert tp == {"tiles": ex["pair_offsets"], "products": ex["pair_products"],
                  "items": ex["pair_products"], "rows": ex["m2l_pairs"]}
    # mirrored: the runs of each offset pair {o, -o}, every pair once
    assert tm == {"tiles": ex["pair_offsets_mirrored"], "products": ex["pair_products_mirrored"],
                  "items": ex["pair_products_mirrored"], "rows": ex["m2l_pairs"]}
    # both negations of a mirrored pair are exact, so the field is that of the
    # plain work list (the same products, up to the sign of each term)
    assert np.all(np.isfinite(e_mirrored))
    diff = np.sqrt(((e_mirrored - e_plain) ** 2).sum() / (e_plain ** 2).sum())
    assert diff <= 1e-7, diff
    assert (st["n"], st["depth"], st["leaves"], st["cells"]) == (n, D, ex["leaves"], ex["cells"])
    assert st["m2l_pairs"] == ex["m2l_pairs"]
    assert st["p2p_pairs"] == ex["p2p_pairs"]
    assert st["l2l_shifts"] == st["m2m_shifts"] == ex["shifts"]
    assert (tc["tiles"], tc["products"], tc["rows"]) == (ex["tiles"], ex["products"], ex["rows"])
    # every tile with a product yields at least one work item, each item at least one product
    assert ex["tiles"] <= tc["items"] <= tc["products"]
    # each pair lies in one row of one product
    assert tc["products"] * ROWS >= st["m2l_pairs"]


def test_cuda_core_path_has_no_work_list():
    pos = W.sphere_sweep(3000, seed=5)["pos"]
    q = np.full(len(pos), W.E_CHARGE)
    plan = pt.Plan(len(pos), p=6, depth=3, precision="fp32")
    pd = torch.tensor(np.ascontiguousarray(pos.T), dtype=torch.float64, device=DEV)
    plan.forces(pd, torch.tensor(q, dtype=torch.float64, device=DEV), want_phi=False)
    assert plan.tc_stats() == {"tiles": 0, "products": 0, "items": 0, "rows": 0}
    plan.close()
