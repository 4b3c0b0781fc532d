"""Thin ctypes binding of libsph.so (include/sph.h). Argument marshalling only:
every step of the computation runs in the library's CUDA kernels. Functions
keep the C names; arrays may be numpy arrays (host) or torch tensors (host or
CUDA), converted to float64 / int32 contiguous buffers as the ABI requires.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

SPH_OK = 0
SPH_E_INVALID = -1
SPH_E_CUDA = -2
SPH_E_OOM = -3
SPH_E_DOMAIN = -4
SPH_E_UNSTABLE = -5
SPH_E_CAPACITY = -6
SPH_E_TIMEOUT = -7
SPH_E_BOUNDS = -8
SPH_FLAG_GRAPH = 1
SPH_FLAG_KEEP_ACC = 2
SPH_FLAG_FROZEN_GEOMETRY = 4
SPH_FLAG_DEBUG_BOUNDS = 8
SPH_FLAG_PERSISTENT = 16
SPH_FLAG_HALF_PAIR = 32
SPH_DEBUG_NEIGHBOUR = 1
SPH_DEBUG_WALL_OFFSET = 2

ERROR_NAMES = {0: "SPH_OK", -1: "SPH_E_INVALID", -2: "SPH_E_CUDA", -3: "SPH_E_OOM",
               -4: "SPH_E_DOMAIN", -5: "SPH_E_UNSTABLE", -6: "SPH_E_CAPACITY", -7: "SPH_E_TIMEOUT",
               -8: "SPH_E_BOUNDS"}

# every function declared in include/sph.h
EXPORTS = [
    "sph_params_check", "sph_create", "sph_destroy", "sph_last_error", "sph_get_info",
    "sph_build_cells", "sph_advection_step", "sph_acoustic_substep", "sph_step",
    "sph_diagnostics", "sph_get_state", "sph_set_state", "sph_get_acceleration",
    "sph_get_permutation", "sph_get_neighbours", "sph_pair_count", "sph_kernel_launches",
    "sph_set_kernel_timing", "sph_kernel_times", "sph_diagnostics_noalloc",
    "sph_get_launch_config", "sph_set_launch_config", "sph_autotune", "sph_gather_ceiling", "sph_set_gravity",
    "sph_learned_weight_count", "sph_learned_create", "sph_learned_destroy",
    "sph_learned_last_error", "sph_learned_set_weights", "sph_learned_get_weights",
    "sph_learned_set_fused", "sph_learned_predict", "sph_learned_train_step", "sph_learned_step",
    "sph_species_create", "sph_species_destroy", "sph_species_last_error", "sph_species_set",
    "sph_species_get", "sph_diffusion_step", "sph_species_set_gate", "sph_species_get_gate",
    "sph_reaction_step", "sph_species_set_scale", "sph_species_set_correction", "sph_species_set_tensors", "sph_clear_error", "sph_debug_write",
    "sph_gradient_diagnostics", "sph_solid_create", "sph_solid_destroy", "sph_solid_last_error", "sph_solid_size",
    "sph_solid_get_state",
]


class SphParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("free_surface", ctypes.c_int32),
        ("h", ctypes.c_double), ("dp", ctypes.c_double),
        ("rho0", ctypes.c_double), ("c0", ctypes.c_double),
        ("cfl_ad", ctypes.c_double), ("cfl_ac", ctypes.c_double),
        ("u_ref", ctypes.c_double), ("nu", ctypes.c_double),
        ("gravity", ctypes.c_double * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("periodic", ctypes.c_int32 * 3), ("capacity", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("p_transport", ctypes.c_double), ("max_substeps", ctypes.c_int32),
    ]


class SphDiag(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("kinetic", ctypes.c_double), ("potential", ctypes.c_double),
        ("internal", ctypes.c_double), ("energy", ctypes.c_double),
        ("max_rho_dev", ctypes.c_double), ("mean_rho_dev", ctypes.c_double),
        ("front_x", ctypes.c_double), ("t", ctypes.c_double), ("dt_ad", ctypes.c_double),
        ("n_fluid", ctypes.c_int64), ("advection_steps", ctypes.c_int64),
        ("substeps", ctypes.c_int64),
    ]

    def as_dict(self):
        return {"mass": self.mass, "momentum": np.array(self.momentum[:]), "kinetic": self.kinetic,
                "potential": self.potential, "internal": self.internal, "energy": self.energy,
                "max_rho_dev": self.max_rho_dev, "mean_rho_dev": self.mean_rho_dev,
                "front_x": self.front_x, "t": self.t, "dt_ad": self.dt_ad,
                "n_fluid": self.n_fluid, "advection_steps": self.advection_steps,
                "substeps": self.substeps}


class SphInfo(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("n_instances", ctypes.c_int32), ("capacity", ctypes.c_int32),
        ("bits", ctypes.c_int32), ("n_fluid", ctypes.c_int64), ("n_wall", ctypes.c_int64),
        ("n_cells", ctypes.c_int64), ("cell", ctypes.c_double), ("dq", ctypes.c_double),
        ("sigma0", ctypes.c_double), ("R2", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
    ]


_lib = None


SPH_REACTION_FN, SPH_REACTION_AP = 1, 2


class SphReaction(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32)] + [(f, ctypes.c_double) for f in
                                               ("a", "b", "k", "eps0", "mu1", "mu2", "beta", "gamma", "sigma")]


SPH_SOLID_LINEAR, SPH_SOLID_NEO_HOOKEAN = 1, 2


class SphSolidParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("rho0", ctypes.c_double), ("youngs", ctypes.c_double),
                ("poisson", ctypes.c_double), ("h", ctypes.c_double), ("single_step", ctypes.c_int32)]


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def load():
    """Load libsph.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsph.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sph_params_check": (i32, [ctypes.POINTER(SphParams)]),
        "sph_create": (i32, [ctypes.POINTER(SphParams), i32, P, P, i64, P, P, P, P, i64, P, P, P, P,
                             ctypes.POINTER(P)]),
        "sph_destroy": (None, [P]),
        "sph_last_error": (ctypes.c_char_p, [P]),
        "sph_get_info": (i32, [P, ctypes.POINTER(SphInfo)]),
        "sph_build_cells": (i32, [P, P]),
        "sph_set_gravity": (i32, [P, i32, P, P]),
        "sph_advection_step": (i32, [P, ctypes.POINTER(dbl), P]),
        "sph_acoustic_substep": (i32, [P, ctypes.POINTER(i32), ctypes.POINTER(dbl), P]),
        "sph_step": (i32, [P, i32, P]),
        "sph_diagnostics": (i32, [P, ctypes.POINTER(SphDiag), P]),
        "sph_get_state": (i32, [P, P, P, P, P, P]),
        "sph_set_state": (i32, [P, P, P, P, P, dbl, P]),
        "sph_get_acceleration": (i32, [P, P, P]),
        "sph_get_permutation": (i32, [P, P, P]),
        "sph_get_neighbours": (i32, [P, P, P, P, P, i32, P]),
        "sph_pair_count": (i32, [P, ctypes.POINTER(i64), ctypes.POINTER(i64), P]),
        "sph_kernel_launches": (i32, [P, ctypes.POINTER(i64)]),
        "sph_set_kernel_timing": (i32, [P, i32]),
        "sph_kernel_times": (i32, [P, ctypes.POINTER(dbl), ctypes.POINTER(i64)]),
        "sph_diagnostics_noalloc": (i32, [ctypes.POINTER(SphParams), i64, P, P, P, P,
                                          ctypes.POINTER(SphDiag), P]),
        "sph_get_launch_config": (i32, [P, ctypes.POINTER(i32)]),
        "sph_set_launch_config": (i32, [P, ctypes.POINTER(i32)]),
        "sph_autotune": (i32, [P, ctypes.POINTER(i32), ctypes.POINTER(dbl), P]),
        "sph_gather_ceiling": (i32, [P, i32, ctypes.POINTER(dbl), P]),
        "sph_learned_weight_count": (i32, [ctypes.POINTER(i64)]),
        "sph_learned_create": (i32, [i32, P, ctypes.POINTER(P)]),
        "sph_learned_destroy": (None, [P]),
        "sph_learned_last_error": (ctypes.c_char_p, [P]),
        "sph_learned_set_weights": (i32, [P, P]),
        "sph_learned_get_weights": (i32, [P, P]),
        "sph_learned_set_fused": (i32, [P, i32]),
        "sph_learned_predict": (i32, [P, P, P, P]),
        "sph_learned_train_step": (i32, [P, P, P, dbl, ctypes.POINTER(dbl), P, P]),
        "sph_learned_step": (i32, [P, P, dbl, dbl, ctypes.POINTER(i32), P]),
        "sph_species_create": (i32, [P, P, ctypes.POINTER(P)]),
        "sph_species_destroy": (None, [P]),
        "sph_species_last_error": (ctypes.c_char_p, [P]),
        "sph_species_set": (i32, [P, P, P, P]),
        "sph_species_get": (i32, [P, P, P, P]),
        "sph_diffusion_step": (i32, [P, P, dbl, i32, P]),
        "sph_species_set_gate": (i32, [P, P, P, P]),
        "sph_species_get_gate": (i32, [P, P, P, P]),
        "sph_reaction_step": (i32, [P, P, ctypes.POINTER(SphReaction), dbl, i32, P]),
        "sph_species_set_scale": (i32, [P, P, P, P]),
        "sph_species_set_correction": (i32, [P, P, i32]),
        "sph_species_set_tensors": (i32, [P, P, P, P]),
        "sph_clear_error": (i32, [P, P]),
        "sph_debug_write": (i32, [P, i32, i64, i32, i64, P]),
        "sph_gradient_diagnostics": (i32, [P, P, P, P, P, P]),
        "sph_solid_create": (i32, [P, ctypes.POINTER(SphSolidParams), i64, P, P, P, P, ctypes.POINTER(P)]),
        "sph_solid_destroy": (None, [P]),
        "sph_solid_last_error": (ctypes.c_char_p, [P]),
        "sph_solid_size": (i64, [P]),
        "sph_solid_get_state": (i32, [P, P, P, P, P, P, ctypes.POINTER(i64), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ------------------------------------------------------------------------------ helpers
def _ptr(a):
    """Raw address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()            # torch tensor (host or device)


def _f64(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    import torch
    return a.to(torch.float64).contiguous()


def _count(a):
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _sized(a, count, what):
    """The C side reads exactly `count` values of a caller array (it cannot check): reject
    any other size, and a CUDA tensor on another device, before the call."""
    if a is None:
        return a
    if _count(a) != count:
        raise SphError(SPH_E_INVALID, f"{what}: {count} values expected, {_count(a)} given")
    if not isinstance(a, np.ndarray) and a.is_cuda:
        import torch
        if a.device.index != torch.cuda.current_device():
            raise SphError(SPH_E_INVALID, f"{what}: the tensor is not on the current device")
    return a


def _out(a, count, what):
    """A caller's output array: `count` float64 values, contiguous (the C side writes them)."""
    ok = (a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]) if isinstance(a, np.ndarray) else \
        (str(a.dtype) == "torch.float64" and a.is_contiguous())
    if not ok:
        raise SphError(SPH_E_INVALID, f"{what}: a contiguous float64 array is expected")
    return _sized(a, count, what)


def _handle_shape(h, n=None, dim=None, what="array"):
    """(fluid particles, dim) of handle h; given n or dim must match them."""
    info = sph_get_info(h)
    nh, dh = int(info.n_fluid), int(info.dim)
    if (n is not None and int(n) != nh) or (dim is not None and int(dim) != dh):
        raise SphError(SPH_E_INVALID, f"{what}: the handle holds {nh} fluid particles in {dh}D, "
                                      f"not {n} in {dim}D")
    return nh, dh


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream       # torch.cuda.Stream


def params_from(problem, flags=0, capacity=0, max_substeps=0) -> SphParams:
    """Build the C parameter struct from any object carrying the problem's attributes."""
    p = SphParams()
    p.dim = int(problem.dim)
    p.free_surface = int(problem.free_surface)
    p.h, p.dp = float(problem.h), float(problem.dp)
    p.rho0, p.c0 = float(problem.rho0), float(problem.c0)
    p.cfl_ad, p.cfl_ac = float(problem.cfl_ad), float(problem.cfl_ac)
    p.u_ref, p.nu = float(problem.u_ref), float(problem.nu)
    for a in range(3):
        p.gravity[a] = float(problem.gravity[a])
        p.lo[a] = float(problem.lo[a])
        p.hi[a] = float(problem.hi[a])
        p.periodic[a] = int(problem.periodic[a])
    p.capacity = int(capacity)
    p.p_transport = float(getattr(problem, "p_transport", 0.0))
    p.flags = int(flags)
    p.max_substeps = int(max_substeps)
    return p


def check(lib, h, code):
    if code != SPH_OK:
        msg = lib.sph_last_error(h).decode() if h else ""
        raise SphError(code, msg)


# ------------------------------------------------------------------------------ C names
def sph_params_check(params: SphParams) -> int:
    return load().sph_params_check(ctypes.byref(params))


def sph_create(params, pos, vel, rho, mass, wall_pos, wall_normal, wall_vol,
               fluid_offsets=None, wall_offsets=None, stream=None):
    """params: one SphParams or a list (one per tank). Returns the opaque handle."""
    lib = load()
    plist = params if isinstance(params, (list, tuple)) else [params]
    arr = (SphParams * len(plist))(*plist)
    pos, vel, rho, mass = _f64(pos), _f64(vel), _f64(rho), _f64(mass)
    wall_pos, wall_normal, wall_vol = _f64(wall_pos), _f64(wall_normal), _f64(wall_vol)
    dim = int(plist[0].dim)
    n_, nw_ = _count(rho), _count(wall_vol)
    for a, c, w in ((pos, n_ * dim, "pos"), (vel, n_ * dim, "vel"), (mass, n_, "mass"),
                    (wall_pos, nw_ * dim, "wall_pos"), (wall_normal, nw_ * dim, "wall_normal")):
        _sized(a, c, "sph_create: " + w)
    fo = None if fluid_offsets is None else np.ascontiguousarray(fluid_offsets, dtype=np.int64)
    wo = None if wall_offsets is None else np.ascontiguousarray(wall_offsets, dtype=np.int64)
    n = int(rho.shape[0])
    nw = int(wall_vol.shape[0])
    h = ctypes.c_void_p()
    code = lib.sph_create(arr, len(plist), _ptr(fo), _ptr(wo), n, _ptr(pos), _ptr(vel), _ptr(rho),
                          _ptr(mass), nw, _ptr(wall_pos), _ptr(wall_normal), _ptr(wall_vol),
                          _stream(stream), ctypes.byref(h))
    if code != SPH_OK:
        msg = lib.sph_last_error(h).decode() if h.value else ""
        if h.value:
            lib.sph_destroy(h)
        raise SphError(code, msg)
    return h


def sph_destroy(h):
    load().sph_destroy(h)


def sph_get_info(h) -> SphInfo:
    lib = load()
    info = SphInfo()
    check(lib, h, lib.sph_get_info(h, ctypes.byref(info)))
    return info


def sph_clear_error(h, stream=None):
    lib = load()
    check(lib, h, lib.sph_clear_error(h, _stream(stream)))


def sph_debug_write(h, what, index, slot, value, stream=None):
    """Overwrite one table entry (test aid; needs a SPH_FLAG_DEBUG_BOUNDS handle)."""
    lib = load()
    check(lib, h, lib.sph_debug_write(h, int(what), int(index), int(slot), int(value), _stream(stream)))


def sph_build_cells(h, stream=None):
    lib = load()
    check(lib, h, lib.sph_build_cells(h, _stream(stream)))


def sph_advection_step(h, stream=None, want_dt=True):
    lib = load()
    dt = ctypes.c_double(0.0)
    check(lib, h, lib.sph_advection_step(h, ctypes.byref(dt) if want_dt else None, _stream(stream)))
    return dt.value


def sph_acoustic_substep(h, stream=None, sync=True):
    lib = load()
    done = ctypes.c_int32(0)
    dt = ctypes.c_double(0.0)
    if sync:
        check(lib, h, lib.sph_acoustic_substep(h, ctypes.byref(done), ctypes.byref(dt), _stream(stream)))
        return bool(done.value), dt.value
    check(lib, h, lib.sph_acoustic_substep(h, None, None, _stream(stream)))
    return None, None


def sph_step(h, n_advection_steps=1, stream=None):
    lib = load()
    check(lib, h, lib.sph_step(h, int(n_advection_steps), _stream(stream)))


def sph_diagnostics(h, n_instances=1, stream=None):
    lib = load()
    out = (SphDiag * n_instances)()
    check(lib, h, lib.sph_diagnostics(h, out, _stream(stream)))
    return [d.as_dict() for d in out]


def sph_get_state(h, n, dim, stream=None, out=None):
    """Returns (pos, vel, rho, drho_dt) float64 numpy arrays in id order (or fills `out`)."""
    lib = load()
    n, dim = _handle_shape(h, n, dim, "sph_get_state")
    if out is None:
        out = (np.empty((n, dim)), np.empty((n, dim)), np.empty(n), np.empty(n))
    for a, c, w in zip(out, (n * dim, n * dim, n, n), ("pos", "vel", "rho", "drho_dt")):
        _out(a, c, "sph_get_state: " + w)
    check(lib, h, lib.sph_get_state(h, *[_ptr(a) for a in out], _stream(stream)))
    return out


def sph_set_state(h, pos, vel, rho, drho_dt=None, t=-1.0, stream=None):
    lib = load()
    pos, vel, rho, drho_dt = _f64(pos), _f64(vel), _f64(rho), _f64(drho_dt)
    n, dim = _handle_shape(h)
    for a, c, w in ((pos, n * dim, "pos"), (vel, n * dim, "vel"), (rho, n, "rho"), (drho_dt, n, "drho_dt")):
        _sized(a, c, "sph_set_state: " + w)
    check(lib, h, lib.sph_set_state(h, _ptr(pos), _ptr(vel), _ptr(rho), _ptr(drho_dt), float(t),
                                    _stream(stream)))


def sph_gradient_diagnostics(h, n, dim, stream=None):
    """Strong- and weak-form gradients of rho and p per fluid particle (caller order):
    dict of four (n, dim) float64 arrays."""
    lib = load()
    n, dim = _handle_shape(h, n, dim, "sph_gradient_diagnostics")
    out = {k: np.empty((n, dim)) for k in ("rho_strong", "rho_weak", "p_strong", "p_weak")}
    check(lib, h, lib.sph_gradient_diagnostics(h, _ptr(out["rho_strong"]), _ptr(out["rho_weak"]),
                                               _ptr(out["p_strong"]), _ptr(out["p_weak"]), _stream(stream)))
    return out


def sph_get_acceleration(h, n, dim, stream=None):
    lib = load()
    n, dim = _handle_shape(h, n, dim, "sph_get_acceleration")
    acc = np.empty((n, dim))
    check(lib, h, lib.sph_get_acceleration(h, _ptr(acc), _stream(stream)))
    return acc


def sph_get_permutation(h, n, stream=None):
    lib = load()
    n, _ = _handle_shape(h, n, None, "sph_get_permutation")
    ids = np.empty(n, dtype=np.int32)
    check(lib, h, lib.sph_get_permutation(h, _ptr(ids), _stream(stream)))
    return ids


def sph_get_neighbours(h, n, stride, stream=None):
    """Returns (fluid_count, wall_count, fluid_ids[n, stride], wall_ids[n, stride])."""
    lib = load()
    n, _ = _handle_shape(h, n, None, "sph_get_neighbours")
    fc = np.empty(n, dtype=np.int32)
    wc = np.empty(n, dtype=np.int32)
    fi = np.empty((n, stride), dtype=np.int32)
    wi = np.empty((n, stride), dtype=np.int32)
    check(lib, h, lib.sph_get_neighbours(h, _ptr(fc), _ptr(wc), _ptr(fi), _ptr(wi), int(stride),
                                         _stream(stream)))
    return fc, wc, fi, wi


def sph_pair_count(h, stream=None):
    lib = load()
    f = ctypes.c_int64(0)
    w = ctypes.c_int64(0)
    check(lib, h, lib.sph_pair_count(h, ctypes.byref(f), ctypes.byref(w), _stream(stream)))
    return int(f.value), int(w.value)


def sph_kernel_launches(h) -> int:
    lib = load()
    v = ctypes.c_int64(0)
    check(lib, h, lib.sph_kernel_launches(h, ctypes.byref(v)))
    return int(v.value)


def sph_set_kernel_timing(h, enable=True):
    lib = load()
    check(lib, h, lib.sph_set_kernel_timing(h, 1 if enable else 0))


def sph_kernel_times(h):
    lib = load()
    ms = (ctypes.c_double * 2)()
    cnt = (ctypes.c_int64 * 2)()
    check(lib, h, lib.sph_kernel_times(h, ms, cnt))
    return list(ms), list(cnt)


def sph_get_launch_config(h):
    lib = load()
    cfg = (ctypes.c_int32 * 4)()
    check(lib, h, lib.sph_get_launch_config(h, cfg))
    return list(cfg)


def sph_set_launch_config(h, cfg):
    lib = load()
    arr = (ctypes.c_int32 * 4)(*[int(c) for c in cfg])
    check(lib, h, lib.sph_set_launch_config(h, arr))


def sph_autotune(h, stream=None):
    """Tune the relaxation kernels' launch variants during one advection step; returns
    (cfg, times in ms: [kernel][variant], variants 0-8 = 3 tpp_index + block_index, 9 = the
    row-task form, -1 where it does not apply)."""
    lib = load()
    cfg = (ctypes.c_int32 * 4)()
    ms = (ctypes.c_double * 20)()
    check(lib, h, lib.sph_autotune(h, cfg, ms, _stream(stream)))
    return list(cfg), np.array(ms[:]).reshape(2, 10)


def sph_set_gravity(h, g, instance=-1, stream=None):
    """Replace the gravity of one tank (every tank when instance < 0), e.g. g - a_tank(t)."""
    lib = load()
    gv = np.zeros(3, dtype=np.float64)
    gv[:len(g)] = np.asarray(g, dtype=np.float64)
    check(lib, h, lib.sph_set_gravity(h, int(instance), _ptr(gv), _stream(stream)))


def sph_gather_ceiling(h, reps=10, stream=None) -> float:
    """Mean ms of the gather-only walk of the current neighbour table."""
    lib = load()
    ms = ctypes.c_double(0)
    check(lib, h, lib.sph_gather_ceiling(h, int(reps), ctypes.byref(ms), _stream(stream)))
    return float(ms.value)


def sph_diagnostics_noalloc(params: SphParams, pos, vel, rho, mass, stream=None):
    """FP64 diagnostics of caller-owned DEVICE arrays (torch CUDA float64 tensors, caller
    order) without any device allocation by the library. Returns a dict like
    sph_diagnostics."""
    lib = load()
    import torch
    dim = int(params.dim)
    arrays = {"pos": pos, "vel": vel, "rho": rho, "mass": mass}
    for name, a in arrays.items():
        # the library cannot see array sizes: a short or mistyped array would be read past
        # its end on the device, so the binding checks what the C call takes on trust
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64
                and a.is_contiguous()):
            raise SphError(SPH_E_INVALID, f"sph_diagnostics_noalloc: {name} must be a contiguous "
                                          "float64 CUDA tensor")
        if a.device.index != torch.cuda.current_device():
            raise SphError(SPH_E_INVALID, f"sph_diagnostics_noalloc: {name} is not on the current device")
    n = int(rho.numel())
    if rho.dim() != 1 or mass.dim() != 1 or mass.numel() != n:
        raise SphError(SPH_E_INVALID, "sph_diagnostics_noalloc: rho and mass must have shape [n]")
    if pos.numel() != n * dim or vel.numel() != n * dim:
        raise SphError(SPH_E_INVALID, "sph_diagnostics_noalloc: pos and vel must hold n * dim values")
    out = SphDiag()
    code = lib.sph_diagnostics_noalloc(ctypes.byref(params), n, _ptr(pos), _ptr(vel), _ptr(rho),
                                       _ptr(mass), ctypes.byref(out), _stream(stream))
    if code != SPH_OK:
        raise SphError(code, lib.sph_last_error(None).decode())
    return out.as_dict()


# ------------------------------------------------------------------------------ learned
def _lcheck(lib, net, code):
    if code != SPH_OK:
        msg = lib.sph_learned_last_error(net).decode() if net else ""
        raise SphError(code, msg)


def sph_learned_weight_count() -> int:
    lib = load()
    v = ctypes.c_int64(0)
    check(lib, None, lib.sph_learned_weight_count(ctypes.byref(v)))
    return int(v.value)


def sph_learned_create(dim, weights=None):
    lib = load()
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    _sized(w, sph_learned_weight_count(), "sph_learned_create: weights")
    net = ctypes.c_void_p()
    code = lib.sph_learned_create(int(dim), _ptr(w), ctypes.byref(net))
    if code != SPH_OK:
        msg = lib.sph_learned_last_error(net).decode() if net.value else ""
        if net.value:
            lib.sph_learned_destroy(net)
        raise SphError(code, msg)
    return net


def sph_learned_destroy(net):
    load().sph_learned_destroy(net)


def sph_learned_set_weights(net, weights):
    lib = load()
    w = _sized(np.ascontiguousarray(weights, dtype=np.float32), sph_learned_weight_count(),
               "sph_learned_set_weights")
    _lcheck(lib, net, lib.sph_learned_set_weights(net, _ptr(w)))


def sph_learned_get_weights(net):
    lib = load()
    w = np.empty(sph_learned_weight_count(), dtype=np.float32)
    _lcheck(lib, net, lib.sph_learned_get_weights(net, _ptr(w)))
    return w


def sph_learned_set_fused(net, enabled):
    lib = load()
    _lcheck(lib, net, lib.sph_learned_set_fused(net, int(enabled)))


def sph_learned_predict(h, net, n, dim, stream=None):
    lib = load()
    n, dim = _handle_shape(h, n, dim, "sph_learned_predict")
    y = np.empty((n, dim + 1))
    _lcheck(lib, net, lib.sph_learned_predict(h, net, _ptr(y), _stream(stream)))
    return y


def sph_learned_train_step(h, net, target, lr, want_grad=False, stream=None):
    """Returns (loss, gradient or None)."""
    lib = load()
    n, dim = _handle_shape(h)
    t = _sized(_f64(target), n * (dim + 1), "sph_learned_train_step: target")
    loss = ctypes.c_double(0.0)
    g = np.empty(sph_learned_weight_count(), dtype=np.float32) if want_grad else None
    _lcheck(lib, net, lib.sph_learned_train_step(h, net, _ptr(t), float(lr), ctypes.byref(loss), _ptr(g),
                                                 _stream(stream)))
    return loss.value, g


def sph_learned_step(h, net, max_mean_rho_dev=0.01, max_energy_drift=0.005, stream=None):
    lib = load()
    used = ctypes.c_int32(0)
    code = lib.sph_learned_step(h, net, float(max_mean_rho_dev), float(max_energy_drift),
                                ctypes.byref(used), _stream(stream))
    if code != SPH_OK:
        msg = lib.sph_learned_last_error(net).decode() or lib.sph_last_error(h).decode()
        raise SphError(code, msg)
    return bool(used.value)


# ------------------------------------------------------------------------------ convenience
# ------------------------------------------------------------------------ species diffusion
def _scheck(lib, sp, code):
    if code != SPH_OK:
        raise SphError(code, lib.sph_species_last_error(sp).decode() if sp else "")


def sph_species_create(h, D, dim):
    """Species object on handle h with diffusion tensor D (dim x dim, SPD)."""
    lib = load()
    Dm = np.ascontiguousarray(np.asarray(D, dtype=np.float64)[:dim, :dim])
    sp = ctypes.c_void_p()
    code = lib.sph_species_create(h, _ptr(Dm), ctypes.byref(sp))
    if code != SPH_OK:
        msg = lib.sph_species_last_error(sp).decode() if sp.value else ""
        if sp.value:
            lib.sph_species_destroy(sp)
        raise SphError(code, msg)
    return sp


def sph_species_destroy(sp):
    load().sph_species_destroy(sp)


def sph_species_set(h, sp, C, stream=None):
    lib = load()
    C = _sized(_f64(C), _handle_shape(h)[0], "sph_species_set")
    _scheck(lib, sp, lib.sph_species_set(h, sp, _ptr(C), _stream(stream)))


def sph_species_get(h, sp, n, stream=None, out=None):
    lib = load()
    n, _ = _handle_shape(h, n, None, "sph_species_get")
    C = np.empty(n, dtype=np.float64) if out is None else _out(out, n, "sph_species_get")
    _scheck(lib, sp, lib.sph_species_get(h, sp, _ptr(C), _stream(stream)))
    return C


def sph_species_set_gate(h, sp, w, stream=None):
    lib = load()
    w = _sized(_f64(w), _handle_shape(h)[0], "sph_species_set_gate")
    _scheck(lib, sp, lib.sph_species_set_gate(h, sp, _ptr(w), _stream(stream)))


def sph_species_get_gate(h, sp, n, stream=None, out=None):
    lib = load()
    n, _ = _handle_shape(h, n, None, "sph_species_get_gate")
    w = np.empty(n, dtype=np.float64) if out is None else _out(out, n, "sph_species_get_gate")
    _scheck(lib, sp, lib.sph_species_get_gate(h, sp, _ptr(w), _stream(stream)))
    return w


def sph_species_set_scale(h, sp, s, stream=None):
    """Per-particle diffusivity factors (caller row order, positive)."""
    lib = load()
    s = _sized(_f64(s), _handle_shape(h)[0], "sph_species_set_scale")
    _scheck(lib, sp, lib.sph_species_set_scale(h, sp, _ptr(s), _stream(stream)))


def sph_species_set_tensors(h, sp, Dp, stream=None):
    """Per-particle diffusion tensors (n, dim, dim) in caller row order, or None to return to
    the species' own tensor."""
    lib = load()
    if Dp is None:
        _scheck(lib, sp, lib.sph_species_set_tensors(h, sp, None, _stream(stream)))
        return
    n, dim = _handle_shape(h)
    Dp = _sized(_f64(Dp), n * dim * dim, "sph_species_set_tensors")
    _scheck(lib, sp, lib.sph_species_set_tensors(h, sp, _ptr(Dp), _stream(stream)))


def sph_species_set_correction(h, sp, on=True):
    """The kernel-corrected diffusion form (Eq. grad-laplace-renormalize) on or off."""
    lib = load()
    _scheck(lib, sp, lib.sph_species_set_correction(h, sp, 1 if on else 0))


def reaction_from(model, **params) -> SphReaction:
    """SphReaction for model SPH_REACTION_FN or SPH_REACTION_AP; other fields default to 0."""
    r = SphReaction()
    r.model = int(model)
    for k, v in params.items():
        setattr(r, k, float(v))
    return r


def sph_reaction_step(h, sp, reaction, dt, n_steps=1, stream=None):
    lib = load()
    _scheck(lib, sp, lib.sph_reaction_step(h, sp, ctypes.byref(reaction), float(dt), int(n_steps),
                                           _stream(stream)))


def sph_diffusion_step(h, sp, dt, n_steps=1, stream=None):
    lib = load()
    _scheck(lib, sp, lib.sph_diffusion_step(h, sp, float(dt), int(n_steps), _stream(stream)))


class Simulation:
    """One handle over one or more tanks built from workload objects (marshalling only)."""

    def __init__(self, problems, flags=0, capacity=0, stream=None, max_substeps=0):
        probs = problems if isinstance(problems, (list, tuple)) else [problems]
        self.problems = probs
        self.dim = int(probs[0].dim)
        self.stream = stream
        params = [params_from(p, flags=flags, capacity=capacity, max_substeps=max_substeps) for p in probs]
        pos = np.concatenate([np.asarray(p.pos, dtype=np.float64).reshape(-1, self.dim) for p in probs])
        vel = np.concatenate([np.asarray(p.vel, dtype=np.float64).reshape(-1, self.dim) for p in probs])
        rho = np.concatenate([np.asarray(p.rho, dtype=np.float64) for p in probs])
        mass = np.concatenate([np.asarray(p.mass, dtype=np.float64) for p in probs])
        wpos = np.concatenate([np.asarray(p.wall_pos, dtype=np.float64).reshape(-1, self.dim) for p in probs])
        wnrm = np.concatenate([np.asarray(p.wall_normal, dtype=np.float64).reshape(-1, self.dim) for p in probs])
        wvol = np.concatenate([np.asarray(p.wall_vol, dtype=np.float64) for p in probs])
        fo = np.cumsum([0] + [len(p.rho) for p in probs])
        wo = np.cumsum([0] + [len(p.wall_vol) for p in probs])
        self.n = int(rho.shape[0])
        self.n_wall = int(wvol.shape[0])
        self.n_instances = len(probs)
        self.fluid_offsets = fo
        self.handle = sph_create(params, pos, vel, rho, mass, wpos, wnrm, wvol,
                                 fo if len(probs) > 1 else None, wo if len(probs) > 1 else None,
                                 stream=stream)

    def close(self):
        if self.handle is not None:
            sph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return sph_get_info(self.handle)

    def build_cells(self):
        sph_build_cells(self.handle, self.stream)

    def advection_step(self):
        return sph_advection_step(self.handle, self.stream)

    def acoustic_substep(self):
        return sph_acoustic_substep(self.handle, self.stream)

    def step(self, n=1):
        sph_step(self.handle, n, self.stream)

    def diagnostics(self):
        d = sph_diagnostics(self.handle, self.n_instances, self.stream)
        return d if self.n_instances > 1 else d[0]

    def state(self):
        return sph_get_state(self.handle, self.n, self.dim, self.stream)

    def set_state(self, pos, vel, rho, drho_dt=None, t=-1.0):
        sph_set_state(self.handle, pos, vel, rho, drho_dt, t, self.stream)

    def acceleration(self):
        return sph_get_acceleration(self.handle, self.n, self.dim, self.stream)

    def permutation(self):
        return sph_get_permutation(self.handle, self.n, self.stream)

    def neighbours(self):
        cap = self.info().capacity
        return sph_get_neighbours(self.handle, self.n, cap, self.stream)

    def kernel_launches(self):
        return sph_kernel_launches(self.handle)

    def pair_count(self):
        return sph_pair_count(self.handle, self.stream)


# ------------------------------------------------------------------------ fluid-structure
def sph_solid_create(h, model, rho0, youngs, poisson, h_s, pos, vol, normal, fixed=None, single_step=False):
    """Attach an elastic solid to handle h; returns the opaque solid."""
    lib = load()
    p = SphSolidParams(int(model), float(rho0), float(youngs), float(poisson), float(h_s), 1 if single_step else 0)
    pos, vol, normal = _f64(pos), _f64(vol), _f64(normal)
    fx = None if fixed is None else np.ascontiguousarray(np.asarray(fixed).astype(np.int32))
    n = int(vol.shape[0])
    dim = sph_get_info(h).dim
    for a, c, w in ((pos, n * dim, "pos"), (normal, n * dim, "normal"), (fx, n, "fixed")):
        _sized(a, c, "sph_solid_create: " + w)
    s = ctypes.c_void_p()
    code = lib.sph_solid_create(h, ctypes.byref(p), n, _ptr(pos), _ptr(vol), _ptr(normal), _ptr(fx), ctypes.byref(s))
    if code != SPH_OK:
        msg = lib.sph_solid_last_error(s).decode() if s.value else ""
        if s.value:
            lib.sph_solid_destroy(s)
        raise SphError(code, msg)
    return s


def sph_solid_destroy(s):
    load().sph_solid_destroy(s)


def sph_solid_size(s) -> int:
    return int(load().sph_solid_size(s))


def sph_solid_get_state(h, s, n=None, dim=None, stream=None):
    """Returns dict(pos, vel, force (n, dim), F (n, dim, dim), solid_steps). n and dim are the
    solid's own (its particle count and the handle's dimension); given ones must match."""
    lib = load()
    n_s, dim_h = sph_solid_size(s), sph_get_info(h).dim
    if (n is not None and n != n_s) or (dim is not None and dim != dim_h):
        raise ValueError(f"the solid has {n_s} particles in {dim_h}D, not {n} in {dim}D")
    n, dim = n_s, dim_h
    out = {"pos": np.empty((n, dim)), "vel": np.empty((n, dim)), "force": np.empty((n, dim)),
           "F": np.empty((n, dim, dim))}
    steps = ctypes.c_int64(0)
    code = lib.sph_solid_get_state(h, s, _ptr(out["pos"]), _ptr(out["vel"]), _ptr(out["force"]), _ptr(out["F"]),
                                   ctypes.byref(steps), _stream(stream))
    if code != SPH_OK:
        raise SphError(code, lib.sph_solid_last_error(s).decode())
    out["solid_steps"] = int(steps.value)
    return out


def solid_from(sim, problem, single_step=False):
    """Attach the solid a workload describes (solid_* attributes) to a Simulation."""
    return sph_solid_create(sim.handle, problem.solid_model, problem.solid_rho0, problem.solid_youngs,
                            problem.solid_poisson, problem.solid_h, problem.solid_pos, problem.solid_vol,
                            problem.solid_normal, problem.solid_fixed, single_step)
