"""Python binding of libpenning: the FMM Coulomb field of a Penning-trap ion
crystal fused with the cyclotronic push, for GB300 (sm_103a).

Argument marshalling only: every step of the computation runs in the CUDA
library behind the C ABI of ``include/penning.h``; PyTorch supplies device
memory and the current stream.  There is no CPU fallback: importing works
without a GPU (the library is only loaded), but every call that computes
needs CUDA and the compiled ``libpenning.so``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpenning.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "penning.h")

PT_OK, PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CUDA = 0, -1, -2, -3
PT_ERR_NONFINITE, PT_ERR_ESCAPED, PT_ERR_TIMEOUT, PT_ERR_COINCIDENT, PT_ERR_UNSUPPORTED = (
    -4, -5, -6, -7, -8)
PT_FP64, PT_MIXED_TF32X3, PT_MIXED_BF16X3, PT_FP32 = 0, 1, 2, 3
PT_PHASE_NEAR, PT_PHASE_FAR, PT_PHASE_ALL = 1, 2, 3
EXPAND_TREE, EXPAND_DIRECT = 0, 1
M2L_TILES, M2L_PAIRS, M2L_ROTATION = 0, 1, 2
PT_MAX_BEAMS = 8
PRECISIONS = {"fp64": PT_FP64, "tf32x3": PT_MIXED_TF32X3, "bf16x3": PT_MIXED_BF16X3,
              "fp32": PT_FP32}


class PenningError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


class pt_trap(ctypes.Structure):
    _fields_ = [("B", ctypes.c_double), ("omega_z", ctypes.c_double),
                ("omega_r", ctypes.c_double), ("delta", ctypes.c_double),
                ("mass", ctypes.c_double), ("charge", ctypes.c_double)]


class pt_beam(ctypes.Structure):
    _fields_ = [("s0", ctypes.c_double), ("detuning", ctypes.c_double),
                ("kx", ctypes.c_double), ("ky", ctypes.c_double), ("kz", ctypes.c_double),
                ("waist_y", ctypes.c_double), ("waist_z", ctypes.c_double),
                ("offset_d", ctypes.c_double), ("uniform", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class pt_laser(ctypes.Structure):
    _fields_ = [("n_beams", ctypes.c_int32), ("enabled", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("gamma0", ctypes.c_double),
                ("beam", pt_beam * PT_MAX_BEAMS)]


class pt_state(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("t", ctypes.c_double), ("step", ctypes.c_int64)] + [
        (k, ctypes.c_void_p) for k in ("x", "y", "z", "vx", "vy", "vz", "q")]


_lib = None
_lock = threading.Lock()
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def exported_functions() -> list[str]:
    """Names of the functions declared in include/penning.h."""
    import re
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def load(build_if_missing: bool = True):
    """Load libpenning.so (compiling it first if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import _build
            try:
                _build.build()
            except RuntimeError:
                if not os.path.exists(LIB_PATH):
                    raise
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpenning.so is not built ({LIB_PATH}); run "
                              "python -c 'import __graft_entry__ as g; g.build()'")
        L = ctypes.CDLL(LIB_PATH)
        L.pt_status_str.argtypes = [ctypes.c_int]
        L.pt_status_str.restype = ctypes.c_char_p
        L.fmm_plan_create.argtypes = [_I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(_VP)]
        L.fmm_plan_destroy.argtypes = [_VP]
        L.fmm_plan_set_phases.argtypes = [_VP, ctypes.c_int]
        L.fmm_plan_last_depth.argtypes = [_VP]
        L.fmm_forces.argtypes = [_VP, _I64, _VP, _VP, _VP, _VP, _VP]
        L.fmm_direct.argtypes = [_I64, _VP, _VP, _VP, _VP, _VP]
        L.pt_step.argtypes = [_VP, ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap),
                              ctypes.POINTER(pt_laser), _D, _I64, _VP]
        L.pt_laser_kicks.argtypes = [ctypes.POINTER(pt_laser), _D, _I64, _VP, _VP, _VP, _VP, _VP,
                                     _VP, _I64, _D, _VP, _VP, _VP]
        L.pt_energy.argtypes = [_VP, ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap),
                                ctypes.POINTER(_D), _VP]
        L.fmm_tree_info.argtypes = [_VP, ctypes.POINTER(_D), _VP, _VP, _VP]
        L.pt_step_async.argtypes = L.pt_step.argtypes
        L.pt_sync.argtypes = [_VP, _VP]
        L.fmm_plan_profile.argtypes = [_VP, ctypes.c_int]
        L.fmm_plan_phase_times.argtypes = [_VP, ctypes.POINTER(_D)]
        L.fmm_plan_kernel_times.argtypes = [_VP, ctypes.POINTER(_D)]
        L.fmm_plan_stats.argtypes = [_VP, ctypes.POINTER(_I64), _VP]
        L.fmm_plan_tc_stats.argtypes = [_VP, ctypes.POINTER(_I64), _VP]
        L.fmm_plan_set_expansion.argtypes = [_VP, ctypes.c_int]
        L.fmm_plan_set_m2l_schedule.argtypes = [_VP, ctypes.c_int]
        L.fmm_plan_m2l_schedule.argtypes = [_VP]
        L.fmm_plan_set_m2l_ctas.argtypes = [_VP, ctypes.c_int]
        L.fmm_plan_set_m2l_mirror.argtypes = [_VP, ctypes.c_int]
        L.pt_energy_noalloc.argtypes = [ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap),
                                        ctypes.POINTER(_D), _VP]
        L.fmm_plan_footprint.argtypes = [_I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(_I64), ctypes.POINTER(_I64)]
        L.pt_set_damping.argtypes = [_VP, _D]
        L.pt_temperatures.argtypes = [ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap),
                                      ctypes.POINTER(_D), _VP]
        L.pt_position_moments.argtypes = [ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap),
                                          _VP, _VP]
        L.pt_rms_displacement.argtypes = [_I64, _VP, _I64, _VP, _VP]
        L.pt_potential_temperature.argtypes = [_VP, ctypes.POINTER(pt_state),
                                               ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap),
                                               ctypes.POINTER(_D), _VP]
        L.pt_mh_scans.argtypes = [ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap), _D, _D,
                                  ctypes.c_uint64, _I64, _I64, ctypes.POINTER(_I64),
                                  ctypes.POINTER(_D), _VP]
        L.pt_ensemble_create.argtypes = [ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]
        L.pt_ensemble_step.argtypes = [_VP, ctypes.POINTER(pt_state), ctypes.POINTER(pt_trap),
                                       ctypes.POINTER(pt_laser), ctypes.POINTER(_D), _I64, _VP]
        L.pt_ensemble_sync.argtypes = [_VP, _VP]
        L.pt_ensemble_set_joined_m2l.argtypes = [_VP, ctypes.c_int]
        L.pt_ensemble_joined_m2l.argtypes = [_VP, ctypes.POINTER(ctypes.c_int)]
        L.pt_ensemble_destroy.argtypes = [_VP]
        _lib = L
        return L


def status_str(status: int) -> str:
    return load(build_if_missing=False).pt_status_str(int(status)).decode()


def _check(status: int, what: str):
    if status != PT_OK:
        raise PenningError(status, what)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev_f64(t, shape=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return t


def make_trap(tr) -> pt_trap:
    return pt_trap(tr["B"], tr["omega_z"], tr["omega_r"], tr["delta"], tr["mass"], tr["charge"])


def make_laser(beams, seed=0, gamma0=None, enabled=True) -> pt_laser:
    if len(beams) > PT_MAX_BEAMS:
        raise ValueError("too many beams")
    L = pt_laser()
    L.n_beams = len(beams)
    L.enabled = 1 if (enabled and len(beams)) else 0
    L.seed = int(seed) & (2**64 - 1)
    L.gamma0 = float(gamma0 if gamma0 is not None else 2 * 3.141592653589793 * 18e6)
    for i, b in enumerate(beams):
        L.beam[i] = pt_beam(b["s0"], b["detuning"], b["k"][0], b["k"][1], b["k"][2],
                            b.get("waist_y", 1.0), b.get("waist_z", 1.0), b.get("offset_d", 0.0),
                            1 if b.get("uniform", False) else 0, 0)
    return L


@dataclass
class State:
    """Ion state on the device (each tensor (n,) float64 CUDA) plus t and step."""
    x: torch.Tensor
    y: torch.Tensor
    z: torch.Tensor
    vx: torch.Tensor
    vy: torch.Tensor
    vz: torch.Tensor
    q: torch.Tensor
    t: float = 0.0
    step: int = 0

    @classmethod
    def from_numpy(cls, pos, vel, q, device="cuda", t=0.0, step=0):
        def col(a, i):
            return torch.tensor(a[:, i], dtype=torch.float64, device=device).contiguous()
        return cls(col(pos, 0), col(pos, 1), col(pos, 2), col(vel, 0), col(vel, 1), col(vel, 2),
                   torch.tensor(q, dtype=torch.float64, device=device).contiguous(), t, step)

    @property
    def n(self) -> int:
        return self.x.numel()

    def pos(self):
        return torch.stack([self.x, self.y, self.z], 1)

    def vel(self):
        return torch.stack([self.vx, self.vy, self.vz], 1)

    def _c(self) -> pt_state:
        for t in (self.x, self.y, self.z, self.vx, self.vy, self.vz, self.q):
            _dev_f64(t, (self.n,))
        return pt_state(self.n, float(self.t), int(self.step), *[
            t.data_ptr() for t in (self.x, self.y, self.z, self.vx, self.vy, self.vz, self.q)])


class Plan:
    """An FMM plan: octree, expansion and operator workspace on the device."""

    def __init__(self, n_max: int, p: int = 10, leaf_max: int = 32, depth: int = -1,
                 precision="fp64"):
        L = load()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        _check(L.fmm_plan_create(int(n_max), int(p), int(leaf_max), int(depth), prec,
                                 ctypes.byref(h)), "fmm_plan_create")
        self._h = h
        self.n_max, self.p, self.precision = int(n_max), int(p), prec

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load(False).fmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_phases(self, phases: int):
        _check(load(False).fmm_plan_set_phases(self._h, int(phases)), "fmm_plan_set_phases")

    def set_expansion(self, mode: int):
        """EXPAND_TREE (default: P2M at the leaves and their parents, the
        M2M / L2L passes above) or EXPAND_DIRECT (every ion expanded about,
        and evaluated in, each ancestor cell) for the tensor-core
        precisions."""
        _check(load(False).fmm_plan_set_expansion(self._h, int(mode)), "fmm_plan_set_expansion")

    def set_m2l_schedule(self, schedule):
        """M2L_TILES, M2L_PAIRS or M2L_ROTATION ("tiles" / "pairs" /
        "rotation") (fmm_plan_set_m2l_schedule)."""
        if isinstance(schedule, str):
            schedule = {"tiles": M2L_TILES, "pairs": M2L_PAIRS, "rotation": M2L_ROTATION}[schedule]
        _check(load(False).fmm_plan_set_m2l_schedule(self._h, int(schedule)),
               "fmm_plan_set_m2l_schedule")

    def set_m2l_ctas(self, ctas: int):
        """At most `ctas` CTAs for the persistent tensor-core M2L kernel (0:
        one per SM)."""
        _check(load(False).fmm_plan_set_m2l_ctas(self._h, int(ctas)), "fmm_plan_set_m2l_ctas")

    def set_m2l_mirror(self, on: bool):
        """Pairs of offsets o and -o in the same BF16x3 products, with the
        operator of o (default on; fmm_plan_set_m2l_mirror)."""
        _check(load(False).fmm_plan_set_m2l_mirror(self._h, 1 if on else 0),
               "fmm_plan_set_m2l_mirror")

    @property
    def m2l_schedule(self) -> str:
        return {M2L_TILES: "tiles", M2L_PAIRS: "pairs",
                M2L_ROTATION: "rotation"}[int(load(False).fmm_plan_m2l_schedule(self._h))]

    @property
    def last_depth(self) -> int:
        return int(load(False).fmm_plan_last_depth(self._h))

    def forces(self, pos, q, E=None, phi=None, want_phi=True, stream=None):
        """Coulomb field (3, n) V/m and potential (n,) V of every ion; pos (3, n) m."""
        n = q.numel()
        _dev_f64(pos, (3, n))
        _dev_f64(q, (n,))
        if E is None:
            E = torch.empty((3, n), dtype=torch.float64, device=pos.device)
        if want_phi and phi is None:
            phi = torch.empty(n, dtype=torch.float64, device=pos.device)
        _check(load(False).fmm_forces(self._h, n, _ptr(pos), _ptr(q), _ptr(E),
                                      _ptr(phi) if want_phi else None, _stream(stream)),
               "fmm_forces")
        return E, phi

    def step(self, state: State, trap, laser: pt_laser | None, dt: float, n_steps: int,
             stream=None):
        """Advance state by n_steps cyclotronic steps (in place; t and step advanced)."""
        st = state._c()
        tr = trap if isinstance(trap, pt_trap) else make_trap(trap)
        _check(load(False).pt_step(self._h, ctypes.byref(st), ctypes.byref(tr),
                                   ctypes.byref(laser) if laser is not None else None,
                                   float(dt), int(n_steps), _stream(stream)), "pt_step")
        state.t, state.step = st.t, st.step
        return state

    def step_async(self, state: State, trap, laser: pt_laser | None, dt: float, n_steps: int,
                   stream=None):
        """Enqueue n_steps steps without synchronising (fixed or previously chosen depth)."""
        st = state._c()
        tr = trap if isinstance(trap, pt_trap) else make_trap(trap)
        _check(load(False).pt_step_async(self._h, ctypes.byref(st), ctypes.byref(tr),
                                         ctypes.byref(laser) if laser is not None else None,
                                         float(dt), int(n_steps), _stream(stream)),
               "pt_step_async")
        state.t, state.step = st.t, st.step
        return state

    def sync(self, stream=None):
        _check(load(False).pt_sync(self._h, _stream(stream)), "pt_sync")

    def set_damping(self, gamma: float):
        """Artificial damping rate (1/s) of the rotating-frame velocity; 0 = off."""
        _check(load(False).pt_set_damping(self._h, float(gamma)), "pt_set_damping")

    def profile(self, enable: bool = True):
        _check(load(False).fmm_plan_profile(self._h, 1 if enable else 0), "fmm_plan_profile")

    PHASES = ("drift_bbox", "tree", "upward", "m2l", "near_far", "kick_drift")

    def phase_times(self) -> dict:
        out = (ctypes.c_double * 6)()
        _check(load(False).fmm_plan_phase_times(self._h, out), "fmm_plan_phase_times")
        return dict(zip(self.PHASES, list(out)))

    def kernel_times(self) -> dict:
        """Device ms of the M2L kernel and the P2P kernel alone in the last
        profiled step or force evaluation."""
        out = (ctypes.c_double * 2)()
        _check(load(False).fmm_plan_kernel_times(self._h, out), "fmm_plan_kernel_times")
        return {"m2l_kernel": out[0], "p2p_kernel": out[1]}

    def stats(self, stream=None) -> dict:
        out = (ctypes.c_int64 * 8)()
        _check(load(False).fmm_plan_stats(self._h, out, _stream(stream)), "fmm_plan_stats")
        keys = ("n", "depth", "leaves", "cells", "m2l_pairs", "p2p_pairs", "l2l_shifts",
                "m2m_shifts")
        return dict(zip(keys, [int(v) for v in out]))

    def tc_stats(self, stream=None) -> dict:
        """Tensor-core M2L work list of the last evaluation (zeros off the
        tensor-core path): tiles, tile-offset products, work items, rows."""
        out = (ctypes.c_int64 * 4)()
        _check(load(False).fmm_plan_tc_stats(self._h, out, _stream(stream)), "fmm_plan_tc_stats")
        return dict(zip(("tiles", "products", "items", "rows"), [int(v) for v in out]))

    def tree_info(self, n: int, device="cuda", stream=None):
        root = (ctypes.c_double * 4)()
        perm = torch.empty(n, dtype=torch.int32, device=device)
        keys = torch.empty(n, dtype=torch.int32, device=device)
        _check(load(False).fmm_tree_info(self._h, root, _ptr(perm), _ptr(keys), _stream(stream)),
               "fmm_tree_info")
        return list(root), perm, keys.view(torch.int32)


def direct(pos, q, want_phi=True, stream=None):
    """FP64 O(N^2) Coulomb field (3, n) and potential on the GPU."""
    n = q.numel()
    _dev_f64(pos, (3, n))
    _dev_f64(q, (n,))
    E = torch.empty((3, n), dtype=torch.float64, device=pos.device)
    phi = torch.empty(n, dtype=torch.float64, device=pos.device) if want_phi else None
    _check(load().fmm_direct(n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi), _stream(stream)),
           "fmm_direct")
    return E, phi


def laser_kicks(laser: pt_laser, mass: float, pos, vel, step: int, dt: float, stream=None):
    """Photon counts (n, n_beams) int32 and recoil dv (3, n) for a midpoint state."""
    n = pos.shape[1]
    _dev_f64(pos, (3, n))
    _dev_f64(vel, (3, n))
    counts = torch.zeros((n, max(laser.n_beams, 1)), dtype=torch.int32, device=pos.device)
    dv = torch.empty((3, n), dtype=torch.float64, device=pos.device)
    p = [_ptr(pos[i]) for i in range(3)] + [_ptr(vel[i]) for i in range(3)]
    _check(load().pt_laser_kicks(ctypes.byref(laser), float(mass), n, *p, int(step), float(dt),
                                 _ptr(counts), _ptr(dv), _stream(stream)), "pt_laser_kicks")
    return counts[:, :laser.n_beams], dv


def energy(state: State, trap, plan: Plan | None = None, stream=None):
    """Rotating-frame energy parts [kinetic, external, Coulomb, total] (J)."""
    st = state._c()
    tr = trap if isinstance(trap, pt_trap) else make_trap(trap)
    out = (ctypes.c_double * 4)()
    _check(load().pt_energy(plan._h if plan is not None else None, ctypes.byref(st),
                            ctypes.byref(tr), out, _stream(stream)), "pt_energy")
    return list(out)


def temperatures(state: State, trap, stream=None):
    """(T_par, T_perp) in K of the motion relative to the rigid rotation."""
    st = state._c()
    tr = trap if isinstance(trap, pt_trap) else make_trap(trap)
    out = (ctypes.c_double * 2)()
    _check(load().pt_temperatures(ctypes.byref(st), ctypes.byref(tr), out, _stream(stream)),
           "pt_temperatures")
    return out[0], out[1]


def mh_scans(state: State, trap, temperature: float, dx: float, seed: int, scan0: int,
             n_scans: int, stream=None):
    """Metropolis-Hastings potential-energy scans on the state's positions (in
    place); returns (accepted moves, sum of the accepted energy changes in J)."""
    st = state._c()
    tr = trap if isinstance(trap, pt_trap) else make_trap(trap)
    acc = _I64(0)
    de = _D(0.0)
    _check(load().pt_mh_scans(ctypes.byref(st), ctypes.byref(tr), float(temperature), float(dx),
                              int(seed) & (2**64 - 1), int(scan0), int(n_scans),
                              ctypes.byref(acc), ctypes.byref(de), _stream(stream)),
           "pt_mh_scans")
    return int(acc.value), float(de.value)


def position_moments(state: State, trap, acc, stream=None):
    """acc (4, n) float64 CUDA += rotating-frame (x_r, y_r, z, |x_r|^2) at state.t."""
    st = state._c()
    tr = trap if isinstance(trap, pt_trap) else make_trap(trap)
    _dev_f64(acc, (4, state.n))
    _check(load().pt_position_moments(ctypes.byref(st), ctypes.byref(tr), _ptr(acc),
                                      _stream(stream)), "pt_position_moments")
    return acc


def rms_displacement(acc, samples: int, out=None, stream=None):
    """Delta r_rms (n,) of every ion (Eq. rms_disp) from K = samples
    accumulations of position_moments (pt_rms_displacement)."""
    _dev_f64(acc)
    n = acc.shape[1]
    _dev_f64(acc, (4, n))
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=acc.device)
    _check(load().pt_rms_displacement(n, _ptr(acc), int(samples), _ptr(out), _stream(stream)),
           "pt_rms_displacement")
    return out


def potential_temperature(state: State, trap, reference: State, plan: Plan | None = None,
                          stream=None):
    """T_PE in K (Eq. temp_pe) of state against the reference configuration
    (pt_potential_temperature)."""
    st, ref = state._c(), reference._c()
    tr = trap if isinstance(trap, pt_trap) else make_trap(trap)
    out = _D(0.0)
    _check(load().pt_potential_temperature(plan._h if plan is not None else None,
                                           ctypes.byref(st), ctypes.byref(ref),
                                           ctypes.byref(tr), ctypes.byref(out), _stream(stream)),
           "pt_potential_temperature")
    return float(out.value)


def plan_footprint(n_max: int, p: int, leaf_max: int = 32, depth: int = -1,
                   precision="fp64") -> tuple[int, int]:
    """(plan workspace bytes, shared operator bytes) that Plan(...) would take."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().fmm_plan_footprint(int(n_max), int(p), int(leaf_max), int(depth), prec,
                                     ctypes.byref(a), ctypes.byref(b)), "fmm_plan_footprint")
    return a.value, b.value


class Ensemble:
    """Independent crystals advanced together: every step of all members is
    one launch of one CUDA graph (members as parallel branches; the BF16x3
    pair-packed members' M2L as one joined launch).  The plans stay the
    caller's; a member's result equals its plan stepped alone."""

    def __init__(self, plans, share_sms: bool = False, joined_m2l: bool = True):
        """share_sms: each member's persistent M2L kernel takes one CTA per
        256 ions (at least 2) instead of one per SM, so that the members' M2L
        kernels run side by side (results do not depend on it).  Measured on
        256 crystals of 100-20,000 ions: slower with the pair-packed schedule
        (41.9 against 27.1 ms a step), about even with the tile schedule, so
        off by default."""
        self.plans = list(plans)
        if share_sms:
            for pl in self.plans:
                pl.set_m2l_ctas(max(2, min(1024, (pl.n_max + 255) // 256)))
        arr = (_VP * len(self.plans))(*[pl._h.value for pl in self.plans])
        h = ctypes.c_void_p()
        _check(load(False).pt_ensemble_create(len(self.plans), arr, ctypes.byref(h)),
               "pt_ensemble_create")
        self._h = h
        if not joined_m2l:
            self.set_joined_m2l(False)

    def set_joined_m2l(self, on: bool):
        """One M2L launch for all BF16x3 pair-packed members (default) or one
        per member; takes effect at the next step."""
        _check(load(False).pt_ensemble_set_joined_m2l(self._h, 1 if on else 0),
               "pt_ensemble_set_joined_m2l")

    def joined_m2l(self) -> int:
        """Members covered by the joined M2L launch of the current graph."""
        k = ctypes.c_int()
        _check(load(False).pt_ensemble_joined_m2l(self._h, ctypes.byref(k)), "pt_ensemble_joined_m2l")
        return k.value

    def step(self, states, traps, lasers, dts, n_steps: int, stream=None):
        """Enqueue n_steps steps of every member (asynchronous; see sync)."""
        m = len(self.plans)
        if not (len(states) == len(traps) == len(dts) == m) or (lasers is not None and len(lasers) != m):
            raise ValueError("one state, trap, dt (and laser) per member")
        st = (pt_state * m)(*[s._c() for s in states])
        tr = (pt_trap * m)(*[t if isinstance(t, pt_trap) else make_trap(t) for t in traps])
        lz = (pt_laser * m)(*lasers) if lasers is not None else None
        dt = (ctypes.c_double * m)(*[float(d) for d in dts])
        _check(load(False).pt_ensemble_step(self._h, st, tr, lz, dt, int(n_steps),
                                            _stream(stream)), "pt_ensemble_step")
        for s, c in zip(states, st):
            s.t, s.step = c.t, c.step
        return states

    def sync(self, stream=None):
        _check(load(False).pt_ensemble_sync(self._h, _stream(stream)), "pt_ensemble_sync")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load(False).pt_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
