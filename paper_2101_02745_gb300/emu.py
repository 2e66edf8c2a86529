"""ctypes binding of the C ABI in include/emu.h (argument marshalling only).

Every function here forwards to the ``emu_*`` function of the same name in
libemu_gb300.so; all arithmetic runs in the CUDA kernels.  If the library is
missing, loading fails with an error: there is no CPU path.

``Box`` is a convenience holder that allocates the caller-owned device arrays
the ABI expects as torch tensors and passes their raw pointers.
"""
from __future__ import annotations

import ctypes
from pathlib import Path
from typing import Optional

import numpy as np

from . import build as _build

EMU_OK = 0
EMU_EINVAL = -1
EMU_ECUDA = -2
EMU_ENUMERIC = -3
EMU_ETIMEOUT = -4
EMU_ELATTICE = -5
N_DIAG = 63
AUTOTUNE_CANDIDATES = 17   # EMU_AUTOTUNE_CANDIDATES


class EmuError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"emu error {code}: {message}")
        self.code = code


class emu_config(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int32),
        ("ndir", ctypes.c_int32),
        ("Lz", ctypes.c_double),
        ("area", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("c_light", ctypes.c_double),
        ("cfl_adv", ctypes.c_double),
        ("cfl_flavor", ctypes.c_double),
        ("shape_order", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class emu_oscillation(ctypes.Structure):
    _fields_ = [("mass_eV", ctypes.c_double * 3)] + [(k, ctypes.c_double) for k in
                ("theta12", "theta13", "theta23", "delta_cp", "energy_erg", "n_e", "hbar", "erg_per_eV")]


class emu3_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("ndir", ctypes.c_int32),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("kappa", ctypes.c_double), ("c_light", ctypes.c_double), ("cfl_adv", ctypes.c_double),
                ("cfl_flavor", ctypes.c_double), ("shape_order", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class emu_particles(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("z", "ox", "oy", "oz", "N", "Nbar", "rho", "rhobar", "acc", "stage")] + [("P", ctypes.c_int64)]


_lib = None


def lib_path() -> Path:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libemu_gb300.so and declare the ABI.  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build.stale():
        _build.build()
    if not path.exists():
        raise RuntimeError(f"CUDA library {path} is not built; run paper_2101_02745_gb300.build.build()")
    L = ctypes.CDLL(str(path))
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    cfgp = ctypes.POINTER(emu_config)
    sig = {
        "emu_workspace_bytes": (i64, [cfgp]),
        "emu_create": (i32, [cfgp, ctypes.POINTER(vp)]),
        "emu_bind": (i32, [vp, ctypes.POINTER(emu_particles), vp, i64, vp]),
        "emu_init_particles": (i32, [vp, vp, vp, vp, vp, vp, dbl, ctypes.c_uint64]),
        "emu_set_particles": (i32, [vp] + [vp] * 8 + [i32]),
        "emu_get_particles": (i32, [vp] + [vp] * 8 + [i32]),
        "emu_deposit": (i32, [vp, i32, dbl, vp, i32]),
        "emu_interpolate_H": (i32, [vp, dbl, vp, i32]),
        "emu_rk_stage": (i32, [vp, i32, dbl]),
        "emu_step": (i32, [vp, i64, dbl]),
        "emu_moments": (i32, [vp, vp, i32]),
        "emu_diagnostics": (i32, [vp, vp, i32]),
        "emu_timestep": (i32, [vp, ctypes.POINTER(dbl)]),
        "emu_sync": (i32, [vp]),
        "emu_kernel_launches": (i64, [vp]),
        "emu_profile": (i32, [vp, i32]),
        "emu_kernel_times": (i32, [vp, vp, vp]),
        "emu_deposit_static": (i32, [cfgp] + [vp] * 8 + [dbl, vp, vp]),
        "emu_batch_particles": (i64, [cfgp, ctypes.c_int32]),
        "emu_batch_cells": (i64, [cfgp, ctypes.c_int32]),
        "emu_batch_workspace_bytes": (i64, [cfgp, ctypes.c_int32]),
        "emu_batch_create": (i32, [cfgp, ctypes.c_int32, ctypes.POINTER(vp)]),
        "emu_batch_init_particles": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "emu_batch_timestep": (i32, [vp, vp]),
        "emu_batch_set_dt": (i32, [vp, vp]),
        "emu_batch_step": (i32, [vp, i64]),
        "emu_batch_diagnostics": (i32, [vp, vp, i32]),
        "emu_autotune": (i32, [vp, i32, vp, vp]),
        "emu_set_grid": (i32, [vp, ctypes.c_int32]),
        "emu_set_rk_form": (i32, [vp, ctypes.c_int32]),
        "emu_set_deposit_form": (i32, [vp, ctypes.c_int32]),
        "emu_set_step_form": (i32, [vp, ctypes.c_int32]),
        "emu_set_barrier_timeout": (i32, [vp, i64]),
        "emu_set_layout": (i32, [vp, ctypes.c_int32]),
        "emu_get_layout": (i32, [vp, ctypes.POINTER(ctypes.c_int32)]),
        "emu_set_oscillation": (i32, [vp, ctypes.c_int32, ctypes.POINTER(emu_oscillation)]),
        "emu_adjoint_workspace_bytes": (i64, [cfgp]),
        "emu_batch_adjoint_workspace_bytes": (i64, [cfgp, ctypes.c_int32]),
        "emu_adjoint_seed": (i32, [vp, vp, vp, vp, vp]),
        "emu_adjoint_step": (i32, [vp, dbl, vp, vp, vp, vp, i64]),
        "emu_batch_adjoint_record_bytes": (i64, [cfgp, ctypes.c_int32]),
        "emu_adjoint_record_step": (i32, [vp, dbl, vp, i64]),
        "emu_adjoint_step_recorded": (i32, [vp, dbl, vp, vp, vp, vp, vp, i64]),
        "emu_weight_gradient": (i32, [vp, vp, vp, vp, i32]),
        "emu3_workspace_bytes": (i64, [ctypes.POINTER(emu3_config)]),
        "emu3_create": (i32, [ctypes.POINTER(emu3_config), ctypes.POINTER(vp)]),
        "emu3_bind": (i32, [vp, ctypes.POINTER(emu_particles), vp, vp, vp, i64, vp]),
        "emu3_init_particles": (i32, [vp, vp, vp, vp, vp, vp, dbl, ctypes.c_uint64]),
        "emu3_get_positions": (i32, [vp, vp, vp, i32]),
        "emu3_set_positions": (i32, [vp, vp, vp, i32]),
        "emu_last_error": (ctypes.c_char_p, [vp]),
        "emu_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(box, rc: int):
    if rc != EMU_OK:
        msg = load().emu_last_error(box)
        raise EmuError(rc, msg.decode() if msg else "")


def _host_ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def make_config(nz, ndir, Lz, kappa, c_light, cfl_adv=0.4, cfl_flavor=0.4, area=1.0, shape_order=2) -> emu_config:
    return emu_config(int(nz), int(ndir), float(Lz), float(area), float(kappa), float(c_light), float(cfl_adv),
                      float(cfl_flavor), int(shape_order), 0)


# ----------------------------------------------------------- thin wrappers

def emu_workspace_bytes(cfg: emu_config) -> int:
    n = load().emu_workspace_bytes(ctypes.byref(cfg))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu_create(cfg: emu_config):
    box = ctypes.c_void_p()
    rc = load().emu_create(ctypes.byref(cfg), ctypes.byref(box))
    _check(None, rc)
    return box


def emu_bind(box, parts: emu_particles, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    _check(box, load().emu_bind(box, ctypes.byref(parts), workspace_ptr, workspace_bytes, stream_ptr))


def emu_init_particles(box, n_nu, n_nubar, f_nu, f_nubar, dirs, alpha: float, seed: int):
    arrs = [np.ascontiguousarray(a, np.float64) for a in (n_nu, n_nubar, f_nu, f_nubar)]
    d = None if dirs is None else np.ascontiguousarray(dirs, np.float64)
    _check(box, load().emu_init_particles(box, *map(_host_ptr, arrs), _host_ptr(d), float(alpha), int(seed)))


def emu_set_particles(box, z, ox, oy, oz, N, Nbar, rho, rhobar, on_host: int):
    _check(box, load().emu_set_particles(box, z, ox, oy, oz, N, Nbar, rho, rhobar, int(on_host)))


def emu_get_particles(box, z, ox, oy, oz, N, Nbar, rho, rhobar, on_host: int):
    _check(box, load().emu_get_particles(box, z, ox, oy, oz, N, Nbar, rho, rhobar, int(on_host)))


def emu_deposit(box, src: int, pos_dt: float, A_out, on_host: int):
    _check(box, load().emu_deposit(box, int(src), float(pos_dt), A_out, int(on_host)))


def emu_interpolate_H(box, pos_dt: float, H_out, on_host: int):
    _check(box, load().emu_interpolate_H(box, float(pos_dt), H_out, int(on_host)))


def emu_rk_stage(box, s: int, dt: float):
    _check(box, load().emu_rk_stage(box, int(s), float(dt)))


def emu_step(box, nsteps: int, dt: float):
    _check(box, load().emu_step(box, int(nsteps), float(dt)))


def emu_moments(box, out, on_host: int):
    _check(box, load().emu_moments(box, out, int(on_host)))


def emu_diagnostics(box, out, on_host: int):
    _check(box, load().emu_diagnostics(box, out, int(on_host)))


def emu_timestep(box) -> float:
    dt = ctypes.c_double()
    _check(box, load().emu_timestep(box, ctypes.byref(dt)))
    return dt.value


def emu_sync(box):
    _check(box, load().emu_sync(box))


def emu_kernel_launches(box) -> int:
    return int(load().emu_kernel_launches(box))


KERNEL_CLASSES = ("shifts", "deposit", "rk_stage", "combine", "other", "step", "rk_deposit")


def emu_profile(box, enable: bool):
    _check(box, load().emu_profile(box, int(bool(enable))))


def emu_kernel_times(box):
    """{class: (total_ms, launches)} recorded since profiling was enabled."""
    ms = np.zeros(len(KERNEL_CLASSES))
    cnt = np.zeros(len(KERNEL_CLASSES), np.int64)
    _check(box, load().emu_kernel_times(box, _host_ptr(ms), cnt.ctypes.data_as(ctypes.c_void_p)))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}


def emu_deposit_static(cfg: emu_config, z, ox, oy, oz, N, Nbar, rho, rhobar, pos_dt: float, A_out, stream_ptr):
    """Deposit into A_out ([36][nz], device) using the library's static scratch
    instead of a caller workspace, for callers that cannot allocate device
    memory.  Synchronises the stream.  Calls that overlap on the GPU race."""
    rc = load().emu_deposit_static(ctypes.byref(cfg), z, ox, oy, oz, N, Nbar, rho, rhobar, float(pos_dt),
                                   A_out, stream_ptr)
    _check(None, rc)


def _cfg_array(cfgs):
    arr = (emu_config * len(cfgs))(*cfgs)
    return arr, ctypes.cast(arr, ctypes.POINTER(emu_config))


def emu_batch_particles(cfgs) -> int:
    arr, ptr = _cfg_array(cfgs)
    n = load().emu_batch_particles(ptr, len(cfgs))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu_batch_cells(cfgs) -> int:
    arr, ptr = _cfg_array(cfgs)
    n = load().emu_batch_cells(ptr, len(cfgs))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu_batch_workspace_bytes(cfgs) -> int:
    arr, ptr = _cfg_array(cfgs)
    n = load().emu_batch_workspace_bytes(ptr, len(cfgs))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu_batch_create(cfgs):
    arr, ptr = _cfg_array(cfgs)
    box = ctypes.c_void_p()
    _check(None, load().emu_batch_create(ptr, len(cfgs), ctypes.byref(box)))
    return box


def emu_batch_init_particles(box, n_nu, n_nubar, f_nu, f_nubar, dirs, alpha, seed):
    arrs = [np.ascontiguousarray(a, np.float64) for a in (n_nu, n_nubar, f_nu, f_nubar, alpha)]
    sd = np.ascontiguousarray(seed, np.uint64)
    d = None if dirs is None else np.ascontiguousarray(dirs, np.float64)
    _check(box, load().emu_batch_init_particles(box, *map(_host_ptr, arrs[:4]), _host_ptr(d), _host_ptr(arrs[4]),
                                                sd.ctypes.data_as(ctypes.c_void_p)))


def emu_batch_timestep(box, nbox: int) -> np.ndarray:
    out = np.zeros(nbox)
    _check(box, load().emu_batch_timestep(box, _host_ptr(out)))
    return out


def emu_batch_set_dt(box, dt):
    dt = np.ascontiguousarray(dt, np.float64)
    _check(box, load().emu_batch_set_dt(box, _host_ptr(dt)))


def emu_batch_step(box, nsteps: int):
    _check(box, load().emu_batch_step(box, int(nsteps)))


def emu_batch_diagnostics(box, out, on_host: int):
    _check(box, load().emu_batch_diagnostics(box, out, int(on_host)))


def emu_autotune(box, trial_steps: int):
    """(choice index, per-step ms of the candidates; see AUTOTUNE_GRID_FORMS)."""
    choice = ctypes.c_int32()
    ms = np.zeros(AUTOTUNE_CANDIDATES)
    _check(box, load().emu_autotune(box, int(trial_steps), ctypes.byref(choice), _host_ptr(ms)))
    return int(choice.value), ms


def emu_set_grid(box, blocks: int):
    _check(box, load().emu_set_grid(box, int(blocks)))


def emu_set_rk_form(box, form: int):
    _check(box, load().emu_set_rk_form(box, int(form)))


def emu_set_step_form(box, form: int):
    _check(box, load().emu_set_step_form(box, int(form)))


def emu_set_deposit_form(box, form: int):
    _check(box, load().emu_set_deposit_form(box, int(form)))


def emu_set_barrier_timeout(box, ns: int):
    _check(box, load().emu_set_barrier_timeout(box, int(ns)))


def emu_set_layout(box, layout: int):
    """0: particles on their lattice sites, 1: anywhere, -1: checked when particles are installed."""
    _check(box, load().emu_set_layout(box, int(layout)))


def emu_get_layout(box) -> int:
    """1 if the box steps with the path for particles anywhere, else 0."""
    g = ctypes.c_int32()
    _check(box, load().emu_get_layout(box, ctypes.byref(g)))
    return int(g.value)


# (step form, grid blocks, RK form, deposit form) of each autotuner candidate, as emu.h lists them
AUTOTUNE_GRID_FORMS = tuple((0, g, f, 0) for g in (304, 152, 608) for f in (0, 1)) + \
    tuple((1, g, f, 0) for g in (304, 152) for f in (0, 1)) + tuple((2, g, -1, 0) for g in (304, 152, 608)) + \
    tuple((0, 304, c % 2, 1 if c < 15 else 2) for c in range(13, 17))


def apply_choice(box, choice: int):
    """Set a box to autotuner candidate `choice` (e.g. the choice made on a twin box)."""
    form, grid, rk, dep = AUTOTUNE_GRID_FORMS[choice]
    emu_set_grid(box, grid)
    emu_set_rk_form(box, rk)
    emu_set_step_form(box, form)
    emu_set_deposit_form(box, dep)


def make_oscillation(d: dict) -> emu_oscillation:
    o = emu_oscillation()
    for i, m in enumerate(d["mass_eV"]):
        o.mass_eV[i] = float(m)
    for k in ("theta12", "theta13", "theta23", "delta_cp", "energy_erg", "n_e", "hbar", "erg_per_eV"):
        setattr(o, k, float(d[k]))
    return o


def emu_set_oscillation(box, box_index: int, osc):
    """osc: emu_oscillation, dict of its fields, or None (remove the terms)."""
    if isinstance(osc, dict):
        osc = make_oscillation(osc)
    ptr = ctypes.byref(osc) if osc is not None else None
    _check(box, load().emu_set_oscillation(box, int(box_index), ptr))


def emu_adjoint_workspace_bytes(cfg: emu_config) -> int:
    n = load().emu_adjoint_workspace_bytes(ctypes.byref(cfg))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu_batch_adjoint_workspace_bytes(cfgs) -> int:
    arr, ptr = _cfg_array(cfgs)
    n = load().emu_batch_adjoint_workspace_bytes(ptr, len(cfgs))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu_adjoint_seed(box, dmom, lam, gN, gNbar):
    _check(box, load().emu_adjoint_seed(box, dmom, lam, gN, gNbar))


def emu_adjoint_step(box, dt: float, lam, gN, gNbar, adj_ws, adj_ws_bytes: int):
    _check(box, load().emu_adjoint_step(box, float(dt), lam, gN, gNbar, adj_ws, int(adj_ws_bytes)))


def emu_batch_adjoint_record_bytes(cfgs) -> int:
    arr, ptr = _cfg_array(cfgs)
    n = load().emu_batch_adjoint_record_bytes(ptr, len(cfgs))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu_adjoint_record_step(box, dt: float, rec, rec_bytes: int):
    _check(box, load().emu_adjoint_record_step(box, float(dt), rec, int(rec_bytes)))


def emu_adjoint_step_recorded(box, dt: float, rec, lam, gN, gNbar, adj_ws, adj_ws_bytes: int):
    _check(box, load().emu_adjoint_step_recorded(box, float(dt), rec, lam, gN, gNbar, adj_ws, int(adj_ws_bytes)))


def emu_weight_gradient(box, gN, gNbar, out, on_host: int):
    _check(box, load().emu_weight_gradient(box, gN, gNbar, out, on_host))


def emu_last_error(box) -> str:
    m = load().emu_last_error(box)
    return m.decode() if m else ""


def emu_destroy(box):
    load().emu_destroy(box)


# ------------------------------------------------------------ convenience

def _no_dirs(M):
    raise ValueError("explicit directions for some boxes of a batch need explicit directions for all")

def _ordered(fn):
    """Box methods run the library on the box's stream: order that stream after
    the caller's current stream (tensors torch just filled) and the current
    stream after it (results, and memory torch may reuse).  No-op when the
    box uses the current stream."""
    import functools

    @functools.wraps(fn)
    def wrapper(self, *args, **kwargs):
        cur = self.torch.cuda.current_stream(self.device)
        same = cur == self.stream
        if not same:
            self.stream.wait_stream(cur)
        out = fn(self, *args, **kwargs)
        if not same:
            cur.wait_stream(self.stream)
        return out
    return wrapper


class Box:
    """One box with its caller-owned device memory held as torch tensors."""

    FIELDS = ("z", "ox", "oy", "oz", "N", "Nbar")

    def __init__(self, nz, ndir, Lz, kappa, c_light, cfl_adv=0.4, cfl_flavor=0.4, area=1.0,
                 device="cuda", stream=None, cfgs=None, shape_order=2):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        if cfgs is None:
            self.cfgs = [make_config(nz, ndir, Lz, kappa, c_light, cfl_adv, cfl_flavor, area, shape_order)]
        else:
            self.cfgs = list(cfgs)
        self.cfg = self.cfgs[0]
        self.nbox = len(self.cfgs)
        self.nz = emu_batch_cells(self.cfgs)
        self.P = emu_batch_particles(self.cfgs)
        self.ndir = self.cfg.ndir if self.nbox == 1 else None
        f64 = dict(dtype=torch.float64, device=self.device)
        self.t = {k: torch.zeros(self.P, **f64) for k in self.FIELDS}
        self.t["rho"] = torch.zeros(9, self.P, **f64)
        self.t["rhobar"] = torch.zeros(9, self.P, **f64)
        self.t["acc"] = torch.zeros(18, self.P, **f64)
        self.t["stage"] = torch.zeros(18, self.P, **f64)
        self.ws_bytes = emu_batch_workspace_bytes(self.cfgs)
        self._ws_raw = torch.zeros(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws_raw.data_ptr()
        self.ws_ptr = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.parts = emu_particles(*[self.t[k].data_ptr() for k in
                                     ("z", "ox", "oy", "oz", "N", "Nbar", "rho", "rhobar", "acc", "stage")],
                                   self.P)
        self.box = emu_batch_create(self.cfgs)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))   # the zero fills above
        emu_bind(self.box, self.parts, self.ws_ptr, self.ws_bytes, self.stream.cuda_stream)

    @classmethod
    def from_workloads(cls, wls, device="cuda", init=True, stream=None):
        """A batch of the given workloads (one box each), initialised together."""
        cfgs = [make_config(w.nz, w.ndir, w.Lz, w.kappa, w.c_light, w.cfl_adv, w.cfl_flavor, w.area, w.shape_order)
                for w in wls]
        b = cls(0, 0, 0, 0, 0, device=device, cfgs=cfgs, stream=stream)
        if init:
            dirs = None
            if any(w.dirs is not None for w in wls):
                dirs = np.concatenate([np.asarray(w.dirs if w.dirs is not None else _no_dirs(w.ndir)).reshape(-1)
                                       for w in wls])
            emu_batch_init_particles(b.box, np.concatenate([w.n_nu for w in wls]),
                                     np.concatenate([w.n_nubar for w in wls]),
                                     np.concatenate([np.asarray(w.f_nu).reshape(-1) for w in wls]),
                                     np.concatenate([np.asarray(w.f_nubar).reshape(-1) for w in wls]), dirs,
                                     np.array([w.alpha for w in wls]), np.array([w.seed for w in wls], np.uint64))
        return b

    @classmethod
    def from_workload(cls, wl, device="cuda", init=True, stream=None):
        b = cls(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area, device=device,
                shape_order=wl.shape_order, stream=stream)
        if init:
            b.init(wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.dirs, wl.alpha, wl.seed)
        return b

    def __del__(self):
        try:
            if getattr(self, "box", None) is not None:
                emu_destroy(self.box)
                self.box = None
        except Exception:
            pass

    # -- ABI calls
    @_ordered
    def init(self, n_nu, n_nubar, f_nu, f_nubar, dirs=None, alpha=1e-6, seed=0):
        nz = self.nz
        emu_init_particles(self.box, np.broadcast_to(np.asarray(n_nu, float), (nz,)),
                           np.broadcast_to(np.asarray(n_nubar, float), (nz,)),
                           np.broadcast_to(np.asarray(f_nu, float), (nz, 3)),
                           np.broadcast_to(np.asarray(f_nubar, float), (nz, 3)), dirs, alpha, seed)

    @_ordered
    def deposit(self, src=0, pos_dt=0.0):
        out = self.torch.empty(36, self.nz, dtype=self.torch.float64, device=self.device)
        emu_deposit(self.box, src, pos_dt, out.data_ptr(), 0)
        return out

    @_ordered
    def interpolate_H(self, pos_dt=0.0):
        out = self.torch.empty(9, self.P, dtype=self.torch.float64, device=self.device)
        emu_interpolate_H(self.box, pos_dt, out.data_ptr(), 0)
        return out

    @_ordered
    def rk_stage(self, s, dt):
        emu_rk_stage(self.box, s, dt)

    @_ordered
    def step(self, nsteps, dt=0.0):
        emu_step(self.box, nsteps, dt)

    @_ordered
    def moments(self):
        out = self.torch.empty(72, self.nz, dtype=self.torch.float64, device=self.device)
        emu_moments(self.box, out.data_ptr(), 0)
        return out

    @_ordered
    def diagnostics(self) -> np.ndarray:
        out = np.zeros(N_DIAG)
        emu_diagnostics(self.box, _host_ptr(out), 1)
        return out

    @_ordered
    def timestep(self) -> float:
        return emu_timestep(self.box)

    def sync(self):
        emu_sync(self.box)

    # -- batch calls
    @_ordered
    def batch_timestep(self) -> np.ndarray:
        return emu_batch_timestep(self.box, self.nbox)

    @_ordered
    def batch_set_dt(self, dt):
        emu_batch_set_dt(self.box, dt)

    @_ordered
    def batch_step(self, nsteps):
        emu_batch_step(self.box, nsteps)

    @_ordered
    def batch_diagnostics(self) -> np.ndarray:
        out = np.zeros((self.nbox, N_DIAG))
        emu_batch_diagnostics(self.box, _host_ptr(out), 1)
        return out

    @_ordered
    def autotune(self, trial_steps=2):
        return emu_autotune(self.box, trial_steps)

    def set_grid(self, blocks: int):
        emu_set_grid(self.box, blocks)

    def set_rk_form(self, form: int):
        """1: RK stage with 32 cells per warp, 0: halo-lane form, -1: by units per warp."""
        emu_set_rk_form(self.box, form)

    def set_step_form(self, form: int):
        """0: one launch per phase, 1: one cooperative launch per step, 2: RK
        stages that deposit the next stage (shape orders 0-2)."""
        emu_set_step_form(self.box, form)

    def set_deposit_form(self, form: int):
        """0: per-warp partial sums and their combination, 1, 2: thread-block
        clusters of 8, 16 blocks that write the potential (step form 0 and the
        stage calls)."""
        emu_set_deposit_form(self.box, form)

    def set_barrier_timeout(self, ns: int):
        emu_set_barrier_timeout(self.box, ns)

    @_ordered
    def set_layout(self, layout: int):
        emu_set_layout(self.box, layout)

    def general(self) -> bool:
        return bool(emu_get_layout(self.box))

    def apply_choice(self, choice: int):
        apply_choice(self.box, choice)

    @_ordered
    def set_oscillation(self, osc, box=-1):
        emu_set_oscillation(self.box, box, osc)

    def launches(self) -> int:
        return emu_kernel_launches(self.box)

    # -- adjoint (single box; device tensors)
    def _f64(self, *shape):
        return self.torch.zeros(*shape, dtype=self.torch.float64, device=self.device)

    @_ordered
    def save_state(self, out=None):
        """Positions and density matrices (the evolving state) copied into a
        (19, P) device tensor: row 0 z, rows 1-9 rho, rows 10-18 rhobar."""
        if out is None:
            out = self.torch.empty(19, self.P, dtype=self.torch.float64, device=self.device)
        emu_get_particles(self.box, out[0].data_ptr(), None, None, None, None, None, out[1].data_ptr(),
                          out[10].data_ptr(), 0)
        return out

    @_ordered
    def load_state(self, st):
        emu_set_particles(self.box, st[0].data_ptr(), None, None, None, None, None, st[1].data_ptr(),
                          st[10].data_ptr(), 0)

    @_ordered
    def adjoint_seed(self, dmom, lam, gN, gNbar):
        """lam (18, P) = dL/d(rho, rhobar) from dmom = dL/d(moments) (72, nz);
        adds the direct terms to gN, gNbar (P,)."""
        dmom = dmom.to(dtype=self.torch.float64, device=self.device).contiguous()
        emu_adjoint_seed(self.box, dmom.data_ptr(), lam.data_ptr(), gN.data_ptr(), gNbar.data_ptr())

    def _adjoint_ws(self):
        if getattr(self, "_adj_ws", None) is None:
            n = emu_batch_adjoint_workspace_bytes(self.cfgs)
            self._adj_raw = self.torch.empty(n + 256, dtype=self.torch.uint8, device=self.device)
            self._adj_ws = ((self._adj_raw.data_ptr() + 255) & ~255, n)
        return self._adj_ws

    @_ordered
    def adjoint_step(self, dt, lam, gN, gNbar):
        """One adjoint RK4 step from the step's start state (held by the box);
        dt = 0: every box's own step size (batches)."""
        ptr, n = self._adjoint_ws()
        emu_adjoint_step(self.box, dt, lam.data_ptr(), gN.data_ptr(), gNbar.data_ptr(), ptr, n)

    def record_stride(self) -> int:
        """Bytes of one step's adjoint record, rounded up to 256."""
        return (emu_batch_adjoint_record_bytes(self.cfgs) + 255) & ~255

    def record_buffer(self, nsteps: int):
        """(raw tensor, base pointer, slot stride): device memory for the records
        of nsteps steps in 256-byte aligned slots.  The box keeps the largest
        one asked for and hands it out again (the library replays one graph per
        slot, keyed on its address)."""
        stride = self.record_stride()
        c = getattr(self, "_rec", None)
        if c is None or c[3] < nsteps:
            self._rec = None
            raw = self.torch.empty(nsteps * stride + 256, dtype=self.torch.uint8, device=self.device)
            c = self._rec = (raw, (raw.data_ptr() + 255) & ~255, stride, nsteps)
        return c[:3]

    def adjoint_buffers(self):
        """(lam (18, P), gN (P,), gNbar (P,)) device buffers kept by the box
        (the adjoint steps' graphs are keyed on them); gN and gNbar are zeroed."""
        c = getattr(self, "_adj_bufs", None)
        if c is None:
            c = self._adj_bufs = (self._f64(18, self.P), self._f64(self.P), self._f64(self.P))
        else:
            c[1].zero_()
            c[2].zero_()
        return c

    @_ordered
    def adjoint_record_step(self, dt, buf, slot: int):
        """One forward step (the state advances) that writes its adjoint record
        into slot `slot` of a record_buffer."""
        raw, base, stride = buf
        emu_adjoint_record_step(self.box, dt, base + slot * stride, stride)

    @_ordered
    def adjoint_step_recorded(self, dt, buf, slot: int, lam, gN, gNbar):
        """adjoint_step from the record in slot `slot` (no recomputed stages);
        the box holds that step's start state."""
        raw, base, stride = buf
        ptr, n = self._adjoint_ws()
        emu_adjoint_step_recorded(self.box, dt, base + slot * stride, lam.data_ptr(), gN.data_ptr(),
                                  gNbar.data_ptr(), ptr, n)

    @_ordered
    def weight_gradient(self, gN, gNbar):
        """(8, nz): dL/dn_nu, dL/dn_nubar, dL/df_nu (x, y, z), dL/df_nubar (x, y, z) per cell."""
        out = self._f64(8, self.nz)
        emu_weight_gradient(self.box, gN.data_ptr(), gNbar.data_ptr(), out.data_ptr(), 0)
        return out

    @_ordered
    def get_host(self) -> dict:
        """All particle fields copied to host numpy arrays (rho, rhobar as (9, P))."""
        h = {k: np.zeros(self.P) for k in self.FIELDS}
        h["rho"] = np.zeros((9, self.P))
        h["rhobar"] = np.zeros((9, self.P))
        emu_get_particles(self.box, *[_host_ptr(h[k]) for k in self.FIELDS + ("rho", "rhobar")], 1)
        return h

    @_ordered
    def set_host(self, **fields):
        args = []
        for k in self.FIELDS + ("rho", "rhobar"):
            a = fields.get(k)
            if a is not None:
                a = np.ascontiguousarray(a, np.float64)
                fields[k] = a
            args.append(_host_ptr(a))
        emu_set_particles(self.box, *args, 1)


class PingPongFeed:
    """Per-step particle state from host memory for two boxes of one
    configuration that take turns, through the host-buffer path of the C ABI
    (emu_set_particles with host pointers).  While one box steps, the next
    step's state (z, rho, rhobar) is copied from the host into the other box's
    particle arrays on that box's own stream, so the copy overlaps the step.
    The boxes need distinct streams; the host arrays should be pinned (page-
    locked) for the copy to run asynchronously.

    `prime()` installs the first step's state in box 0; `step(enqueue)` calls
    enqueue(box) on the box that holds this step's state (the caller enqueues
    that box's work, asynchronously), then installs the next step's state in
    the other box and returns the box that was stepped.  The install returns
    once the copy is done (on_host = 1), or with asynchronous=True once it is
    enqueued (on_host = 2): then the host arrays must stay unchanged until the
    boxes' streams have passed the copies, and the boxes should have a fixed
    particle layout (emu_set_layout 0 or 1), since choosing one synchronises."""

    KEYS = ("z", "rho", "rhobar")

    def __init__(self, boxes, host: dict, asynchronous: bool = False):
        if len(boxes) != 2 or boxes[0].P != boxes[1].P:
            raise ValueError("two boxes of the same configuration")
        if boxes[0].stream == boxes[1].stream:
            raise ValueError("the two boxes need distinct streams")
        self.boxes = list(boxes)
        self.host = {k: host[k] for k in self.KEYS}
        self.on_host = 2 if asynchronous else 1
        self.turn = 0

    @staticmethod
    def _ptr(a):
        return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)

    @property
    def h2d_bytes(self) -> int:
        return sum(int(v.numel() * v.element_size()) if hasattr(v, "numel") else int(v.nbytes)
                   for v in self.host.values())

    def install(self, k: int):
        h = self.host
        emu_set_particles(self.boxes[k].box, self._ptr(h["z"]), None, None, None, None, None, self._ptr(h["rho"]),
                          self._ptr(h["rhobar"]), self.on_host)

    def prime(self):
        self.install(0)

    def step(self, enqueue) -> "Box":
        k = self.turn % 2
        b = self.boxes[k]
        enqueue(b)
        self.install(1 - k)
        self.turn += 1
        return b


# ------------------------------------------------------------------ 3D boxes

def make_config3(nx, ny, nz, ndir, Lx, Ly, Lz, kappa, c_light, cfl_adv=0.4, cfl_flavor=0.4,
                 shape_order=2) -> emu3_config:
    return emu3_config(int(nx), int(ny), int(nz), int(ndir), float(Lx), float(Ly), float(Lz), float(kappa),
                       float(c_light), float(cfl_adv), float(cfl_flavor), int(shape_order), 0)


def emu3_workspace_bytes(cfg: emu3_config) -> int:
    n = load().emu3_workspace_bytes(ctypes.byref(cfg))
    if n < 0:
        raise EmuError(int(n), "invalid configuration")
    return int(n)


def emu3_create(cfg: emu3_config):
    box = ctypes.c_void_p()
    _check(None, load().emu3_create(ctypes.byref(cfg), ctypes.byref(box)))
    return box


def emu3_bind(box, parts: emu_particles, x_ptr: int, y_ptr: int, workspace_ptr: int, workspace_bytes: int,
              stream_ptr: int):
    _check(box, load().emu3_bind(box, ctypes.byref(parts), x_ptr, y_ptr, workspace_ptr, workspace_bytes,
                                 stream_ptr))


def emu3_init_particles(box, n_nu, n_nubar, f_nu, f_nubar, dirs, alpha: float, seed: int):
    arrs = [np.ascontiguousarray(a, np.float64) for a in (n_nu, n_nubar, f_nu, f_nubar)]
    d = None if dirs is None else np.ascontiguousarray(dirs, np.float64)
    _check(box, load().emu3_init_particles(box, *map(_host_ptr, arrs), _host_ptr(d), float(alpha), int(seed)))


def emu3_get_positions(box, x, y, on_host: int):
    _check(box, load().emu3_get_positions(box, x, y, int(on_host)))


def emu3_set_positions(box, x, y, on_host: int):
    _check(box, load().emu3_set_positions(box, x, y, int(on_host)))


class Box3D(Box):
    """One 3D box (emu3_create) with its caller-owned device memory as torch
    tensors; the Box methods that the C ABI supports for 3D boxes apply."""

    FIELDS = ("z", "ox", "oy", "oz", "N", "Nbar")

    def __init__(self, nx, ny, nz, ndir, Lx, Ly, Lz, kappa, c_light, cfl_adv=0.4, cfl_flavor=0.4,
                 device="cuda", stream=None, shape_order=2):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.cfg3 = make_config3(nx, ny, nz, ndir, Lx, Ly, Lz, kappa, c_light, cfl_adv, cfl_flavor, shape_order)
        self.cfgs = []
        self.nbox = 1
        self.C = nx * ny * nz
        self.nz = self.C            # cells: the moments are [72][C]
        self.ndir = ndir
        self.P = self.C * ndir
        f64 = dict(dtype=torch.float64, device=self.device)
        self.t = {k: torch.zeros(self.P, **f64) for k in self.FIELDS + ("x", "y")}
        self.t["rho"] = torch.zeros(9, self.P, **f64)
        self.t["rhobar"] = torch.zeros(9, self.P, **f64)
        self.t["acc"] = torch.zeros(18, self.P, **f64)
        self.t["stage"] = torch.zeros(18, self.P, **f64)
        self.ws_bytes = emu3_workspace_bytes(self.cfg3)
        self._ws_raw = torch.zeros(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self._ws_raw.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.parts = emu_particles(*[self.t[k].data_ptr() for k in
                                     ("z", "ox", "oy", "oz", "N", "Nbar", "rho", "rhobar", "acc", "stage")],
                                   self.P)
        self.box = emu3_create(self.cfg3)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        emu3_bind(self.box, self.parts, self.t["x"].data_ptr(), self.t["y"].data_ptr(), self.ws_ptr, self.ws_bytes,
                  self.stream.cuda_stream)

    @classmethod
    def from_workload(cls, wl, device="cuda", init=True, stream=None):
        b = cls(wl.nx, wl.ny, wl.nz, wl.ndir, wl.Lx, wl.Ly, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor,
                device=device, stream=stream, shape_order=wl.shape_order)
        if init:
            b.init(wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.dirs, wl.alpha, wl.seed)
        return b

    @_ordered
    def init(self, n_nu, n_nubar, f_nu, f_nubar, dirs=None, alpha=1e-6, seed=0):
        C = self.C
        emu3_init_particles(self.box, np.broadcast_to(np.asarray(n_nu, float), (C,)),
                            np.broadcast_to(np.asarray(n_nubar, float), (C,)),
                            np.broadcast_to(np.asarray(f_nu, float), (C, 3)),
                            np.broadcast_to(np.asarray(f_nubar, float), (C, 3)), dirs, alpha, seed)

    @_ordered
    def get_host(self) -> dict:
        h = Box.get_host.__wrapped__(self)
        x, y = np.zeros(self.P), np.zeros(self.P)
        emu3_get_positions(self.box, _host_ptr(x), _host_ptr(y), 1)
        h["x"], h["y"] = x, y
        return h
