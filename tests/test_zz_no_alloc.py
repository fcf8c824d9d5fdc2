"""pt_energy_noalloc: the rotating-frame energy for callers that cannot
allocate device memory (real-time loops that cannot take cudaMalloc's device
synchronisation mid-run, programs whose device memory is all reserved by
their own allocator).  Its scratch is a fixed array inside the library, so
it must give the same energies as pt_energy with the direct sum, call after
call, and refuse states larger than that array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes run alone.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2405_13973_gb300 as pt
import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, st, trap):
    out = (ctypes.c_double * 4)()
    c = st._c()
    status = lib.pt_energy_noalloc(ctypes.byref(c), ctypes.byref(trap), out,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return status, list(out)


def test_noalloc_energy_matches_pt_energy_twice_in_a_row():
    lib = pt.load()
    for seed, n in ((6, 1000), (7, 3001)):
        cr = W.crystal_sphere_1k(seed=seed) if n == 1000 else None
        if cr is None:
            rng = np.random.default_rng(seed)
            pos = rng.normal(size=(n, 3)) * 40e-6
            tr_d = W.trap(beta=0.8)
            vel = W.rotating_maxwellian(pos, tr_d["omega_r"], 10e-3, seed)
            cr = {"pos": pos, "vel": vel, "q": W.charges(n), "trap": tr_d}
        st = pt.State.from_numpy(cr["pos"], cr["vel"], cr["q"], t=2.5e-7)
        trap = pt.make_trap(cr["trap"])
        ref = pt.energy(st, trap)                     # allocating path, direct sum
        for _ in range(2):                            # two calls in a row
            status, got = _noalloc(lib, st, trap)
            assert status == pt.PT_OK, pt.status_str(status)
            for a, b in zip(got, ref):
                assert a == pytest.approx(b, rel=1e-12, abs=1e-12 * abs(ref[3]))


def test_noalloc_rejects_states_beyond_its_scratch():
    lib = pt.load()
    n = 65537
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = pt.State(z, z, z, z, z, z, z + W.E_CHARGE)
    status, _ = _noalloc(lib, st, pt.make_trap(W.trap()))
    assert status == pt.PT_ERR_ARG
