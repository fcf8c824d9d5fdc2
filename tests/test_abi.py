"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/penning.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2405_13973_gb300 as pt
from paper_2405_13973_gb300 import _build


def test_header_declares_the_boundary_calls():
    names = pt.exported_functions()
    for must in ("fmm_plan_create", "fmm_plan_destroy", "fmm_forces", "pt_step", "pt_energy",
                 "pt_status_str", "fmm_direct", "pt_laser_kicks", "fmm_tree_info"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [f for f in pt.exported_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_library_is_sm_103a_code():
    # the build passes exactly one -gencode for sm_103a
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_without_gpu():
    lib = pt.load()
    assert pt.status_str(0) == "ok"
    assert "argument" in pt.status_str(pt.PT_ERR_ARG)
    assert "non-finite" in pt.status_str(pt.PT_ERR_NONFINITE)


def test_struct_layouts_match_the_header():
    # pt_beam: 8 doubles + 2 int32; pt_laser: 2 int32, u64, double, 8 beams
    assert ctypes.sizeof(pt.pt_beam) == 72
    assert ctypes.sizeof(pt.pt_laser) == 24 + 8 * 72
    assert ctypes.sizeof(pt.pt_trap) == 48
    assert ctypes.sizeof(pt.pt_state) == 24 + 7 * 8


def test_argument_errors_are_reported_not_raised():
    lib = pt.load()
    h = ctypes.c_void_p()
    # invalid order / size are rejected before any CUDA call
    assert lib.fmm_plan_create(0, 8, 32, -1, 0, ctypes.byref(h)) == pt.PT_ERR_ARG
    assert lib.fmm_plan_create(100, 1, 32, -1, 0, ctypes.byref(h)) == pt.PT_ERR_ARG
    assert lib.fmm_plan_create(100, 17, 32, -1, 0, ctypes.byref(h)) == pt.PT_ERR_ARG
    assert lib.fmm_plan_create(100, 8, 32, 9, 0, ctypes.byref(h)) == pt.PT_ERR_ARG
    assert lib.fmm_plan_create(100, 8, 32, -1, 7, ctypes.byref(h)) == pt.PT_ERR_ARG
    assert lib.fmm_forces(None, 10, None, None, None, None, None) == pt.PT_ERR_ARG
    assert lib.pt_step(None, None, None, None, 1e-9, 1, None) == pt.PT_ERR_ARG
