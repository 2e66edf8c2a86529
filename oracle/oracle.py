"""ctypes binding of the plain C FP64 oracle (emu_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package entry point's
smoke check and the benchmark's CPU-baseline leg may import this module.  The
product library never loads it, and it never loads the product library.

The oracle keeps particles as an array of structs with full complex 3x3
matrices (numpy structured dtype ``PARTICLE``) and the grid as one struct per
cell (``CELL``).  Every function below forwards to the C routine of the same
name without touching the arithmetic; see emu_oracle.c for the paper
passages each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "emu_oracle.c"
_SRCS = (_SRC, _HERE / "emu_oracle3d.c")
_HDR = _HERE / "emu_oracle.h"
_LIB = _HERE / "liboracle.so"

PARTICLE = np.dtype(
    [
        ("z", "f8"),
        ("omega", "f8", (3,)),
        ("N", "f8"),
        ("Nbar", "f8"),
        ("rho", "c16", (3, 3)),
        ("rhobar", "c16", (3, 3)),
    ],
    align=True,
)
CELL = np.dtype(
    [
        ("n", "c16", (3, 3)),
        ("nbar", "c16", (3, 3)),
        ("f", "c16", (3, 3, 3)),
        ("fbar", "c16", (3, 3, 3)),
    ],
    align=True,
)


class OrConfig(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int32),
        ("ndir", ctypes.c_int32),
        ("Lz", ctypes.c_double),
        ("area", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("c_light", ctypes.c_double),
        ("cfl_adv", ctypes.c_double),
        ("cfl_flavor", ctypes.c_double),
        ("osc_on", ctypes.c_int32),
        ("shape_order", ctypes.c_int32),
        ("mass_eV", ctypes.c_double * 3),
        ("theta12", ctypes.c_double),
        ("theta13", ctypes.c_double),
        ("theta23", ctypes.c_double),
        ("delta_cp", ctypes.c_double),
        ("energy_erg", ctypes.c_double),
        ("n_e", ctypes.c_double),
        ("hbar", ctypes.c_double),
        ("erg_per_eV", ctypes.c_double),
    ]


def build(force: bool = False) -> Path:
    """Compile emu_oracle.c and emu_oracle3d.c with gcc (-O2, no fast-math) into liboracle.so."""
    newest = max(f.stat().st_mtime for f in _SRCS + (_HDR,))
    if force or not _LIB.exists() or _LIB.stat().st_mtime < newest:
        tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
             "-o", str(tmp), *map(str, _SRCS), "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        vp, i64, dbl, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        cfgp = ctypes.POINTER(OrConfig)
        L.or_splitmix64.argtypes = [u64, u64]; L.or_splitmix64.restype = u64
        L.or_uniform.argtypes = [u64, i64, ctypes.c_int]; L.or_uniform.restype = dbl
        L.or_fibonacci_direction.argtypes = [ctypes.c_int, ctypes.c_int, vp]; L.or_fibonacci_direction.restype = None
        L.or_wrap.argtypes = [cfgp, dbl]; L.or_wrap.restype = dbl
        L.or_shape.argtypes = [cfgp, dbl, vp, vp]; L.or_shape.restype = ctypes.c_int
        L.or_bspline.argtypes = [ctypes.c_int, dbl]; L.or_bspline.restype = dbl
        L.or_init.argtypes = [cfgp, vp, vp, vp, vp, vp, dbl, u64, vp]; L.or_init.restype = ctypes.c_int
        L.or_deposit.argtypes = [cfgp, vp, i64, vp]; L.or_deposit.restype = None
        L.or_hamiltonian.argtypes = [cfgp, vp, vp, vp]; L.or_hamiltonian.restype = None
        L.or_hamiltonian_bar.argtypes = [vp, vp]; L.or_hamiltonian_bar.restype = None
        L.or_commutator_rhs.argtypes = [vp, vp, vp]; L.or_commutator_rhs.restype = None
        L.or_rhs.argtypes = [cfgp, vp, i64, vp, vp, vp]; L.or_rhs.restype = None
        L.or_rk4_step.argtypes = [cfgp, vp, i64, dbl]; L.or_rk4_step.restype = ctypes.c_int
        L.or_run.argtypes = [cfgp, vp, i64, dbl, i64]; L.or_run.restype = ctypes.c_int
        L.or_timestep.argtypes = [cfgp, vp]; L.or_timestep.restype = dbl
        L.or_eln_matrix.argtypes = [vp, i64, vp]; L.or_eln_matrix.restype = None
        L.or_mixing_matrix.argtypes = [cfgp, vp]; L.or_mixing_matrix.restype = None
        L.or_vacuum_matter.argtypes = [cfgp, vp, vp]; L.or_vacuum_matter.restype = None
        L.or_domain_averages.argtypes = [cfgp, vp, vp, vp]; L.or_domain_averages.restype = None
        cfg3p = ctypes.POINTER(OrConfig3)
        L.or3_shape.argtypes = [cfg3p, vp, vp, vp]; L.or3_shape.restype = ctypes.c_int
        L.or3_cell_volume.argtypes = [cfg3p]; L.or3_cell_volume.restype = dbl
        L.or3_init.argtypes = [cfg3p, vp, vp, vp, vp, vp, dbl, u64, vp]; L.or3_init.restype = ctypes.c_int
        L.or3_deposit.argtypes = [cfg3p, vp, i64, vp]; L.or3_deposit.restype = None
        L.or3_hamiltonian.argtypes = [cfg3p, vp, vp, vp]; L.or3_hamiltonian.restype = None
        L.or3_rhs.argtypes = [cfg3p, vp, i64, vp, vp, vp]; L.or3_rhs.restype = None
        L.or3_rk4_step.argtypes = [cfg3p, vp, i64, dbl]; L.or3_rk4_step.restype = ctypes.c_int
        L.or3_run.argtypes = [cfg3p, vp, i64, dbl, i64]; L.or3_run.restype = ctypes.c_int
        L.or3_timestep.argtypes = [cfg3p, vp]; L.or3_timestep.restype = dbl
        for name in ("or_sizeof_particle", "or_sizeof_cell", "or_sizeof_config", "or3_sizeof_particle",
                     "or3_sizeof_config"):
            getattr(L, name).restype = ctypes.c_int32
        assert L.or_sizeof_particle() == PARTICLE.itemsize, "particle struct mismatch"
        assert L.or_sizeof_cell() == CELL.itemsize, "cell struct mismatch"
        assert L.or_sizeof_config() == ctypes.sizeof(OrConfig), "config struct mismatch"
        assert L.or3_sizeof_particle() == PARTICLE3.itemsize, "3D particle struct mismatch"
        assert L.or3_sizeof_config() == ctypes.sizeof(OrConfig3), "3D config struct mismatch"
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def config(nz, ndir, Lz, kappa, c_light, cfl_adv=0.4, cfl_flavor=0.4, area=1.0, osc=None,
           shape_order=2) -> OrConfig:
    """osc: None, or a dict with mass_eV (3), theta12, theta13, theta23, delta_cp [rad],
    energy_erg, n_e [cm^-3], hbar [erg s], erg_per_eV (vacuum and matter terms of Eq. 2).
    shape_order: degree 0..3 of the B-spline particle shape (Sec. 2.2.1)."""
    if shape_order not in (0, 1, 2, 3):
        raise ValueError("shape_order must be 0, 1, 2 or 3")
    c = OrConfig(int(nz), int(ndir), float(Lz), float(area), float(kappa), float(c_light),
                 float(cfl_adv), float(cfl_flavor))
    c.shape_order = int(shape_order)
    if osc is not None:
        c.osc_on = 1
        for i, m in enumerate(osc["mass_eV"]):
            c.mass_eV[i] = float(m)
        for k in ("theta12", "theta13", "theta23", "delta_cp", "energy_erg", "n_e", "hbar", "erg_per_eV"):
            setattr(c, k, float(osc[k]))
    return c


def mixing_matrix(cfg: OrConfig) -> np.ndarray:
    U = np.zeros((3, 3), complex)
    lib().or_mixing_matrix(ctypes.byref(cfg), _ptr(U))
    return U


def vacuum_matter(cfg: OrConfig):
    """(H_vacuum, H_matter) / hbar [1/s] of Eq. 2."""
    a = np.zeros((3, 3), complex)
    b = np.zeros((3, 3), complex)
    lib().or_vacuum_matter(ctypes.byref(cfg), _ptr(a), _ptr(b))
    return a, b


def splitmix64(seed: int, n: int) -> int:
    return int(lib().or_splitmix64(seed, n))


def uniform(seed: int, p: int, k: int) -> float:
    return float(lib().or_uniform(seed, p, k))


def fibonacci_direction(d: int, M: int) -> np.ndarray:
    out = np.zeros(3)
    lib().or_fibonacci_direction(d, M, _ptr(out))
    return out


def wrap(cfg: OrConfig, z: float) -> float:
    """z mapped into [0, Lz) (periodic domain)."""
    return float(lib().or_wrap(ctypes.byref(cfg), float(z)))


def shape(cfg: OrConfig, z: float):
    """(cells, weights) of a particle at z: shape_order + 1 of each."""
    cells = np.zeros(4, np.int32)
    w = np.zeros(4)
    n = lib().or_shape(ctypes.byref(cfg), float(z), _ptr(cells), _ptr(w))
    return cells[:n], w[:n]


def bspline(n: int, x: float) -> float:
    return float(lib().or_bspline(int(n), float(x)))


def init(cfg: OrConfig, n_nu, n_nubar, f_nu, f_nubar, alpha=1e-6, seed=0, dirs=None):
    """Particles of Eq. 8/9 (one per direction per cell), numbered p = d*nz + j0."""
    nz, M = cfg.nz, cfg.ndir
    n_nu = np.ascontiguousarray(np.broadcast_to(np.asarray(n_nu, float), (nz,)))
    n_nubar = np.ascontiguousarray(np.broadcast_to(np.asarray(n_nubar, float), (nz,)))
    f_nu = np.ascontiguousarray(np.broadcast_to(np.asarray(f_nu, float), (nz, 3)))
    f_nubar = np.ascontiguousarray(np.broadcast_to(np.asarray(f_nubar, float), (nz, 3)))
    parts = np.zeros(nz * M, PARTICLE)
    dptr = None
    if dirs is not None:
        dirs = np.ascontiguousarray(np.asarray(dirs, float).reshape(M, 3))
        dptr = _ptr(dirs)
    rc = lib().or_init(ctypes.byref(cfg), dptr, _ptr(n_nu), _ptr(n_nubar), _ptr(f_nu),
                       _ptr(f_nubar), float(alpha), int(seed), _ptr(parts))
    if rc != 0:
        raise ValueError("negative particle weight: a flux factor exceeds 1/3")
    return parts


def deposit(cfg: OrConfig, parts: np.ndarray) -> np.ndarray:
    grid = np.zeros(cfg.nz, CELL)
    lib().or_deposit(ctypes.byref(cfg), _ptr(parts), len(parts), _ptr(grid))
    return grid


def hamiltonian(cfg: OrConfig, grid: np.ndarray, parts: np.ndarray) -> np.ndarray:
    """H/hbar [1/s] at every particle (Eq. 6 then Eq. 2), shape (P, 3, 3)."""
    H = np.zeros((len(parts), 3, 3), complex)
    L = lib()
    for p in range(len(parts)):
        L.or_hamiltonian(ctypes.byref(cfg), _ptr(grid), _ptr(parts[p:p + 1]), _ptr(H[p]))
    return H


def hamiltonian_bar(H: np.ndarray) -> np.ndarray:
    H = np.ascontiguousarray(H, complex)
    out = np.zeros_like(H)
    L = lib()
    for p in range(H.shape[0]):
        L.or_hamiltonian_bar(_ptr(H[p]), _ptr(out[p]))
    return out


def commutator_rhs(H: np.ndarray, rho: np.ndarray) -> np.ndarray:
    H = np.ascontiguousarray(H, complex); rho = np.ascontiguousarray(rho, complex)
    out = np.zeros((3, 3), complex)
    lib().or_commutator_rhs(_ptr(H), _ptr(rho), _ptr(out))
    return out


def rhs(cfg: OrConfig, parts: np.ndarray):
    P = len(parts)
    grid = np.zeros(cfg.nz, CELL)
    dr = np.zeros((P, 3, 3), complex)
    db = np.zeros((P, 3, 3), complex)
    lib().or_rhs(ctypes.byref(cfg), _ptr(parts), P, _ptr(grid), _ptr(dr), _ptr(db))
    return dr, db, grid


def rk4_step(cfg: OrConfig, parts: np.ndarray, dt: float) -> None:
    if lib().or_rk4_step(ctypes.byref(cfg), _ptr(parts), len(parts), float(dt)) != 0:
        raise MemoryError("oracle scratch allocation failed")


def run(cfg: OrConfig, parts: np.ndarray, dt: float, nsteps: int) -> None:
    if lib().or_run(ctypes.byref(cfg), _ptr(parts), len(parts), float(dt), int(nsteps)) != 0:
        raise MemoryError("oracle scratch allocation failed")


def timestep(cfg: OrConfig, grid: np.ndarray) -> float:
    return float(lib().or_timestep(ctypes.byref(cfg), _ptr(grid)))


def eln_matrix(parts: np.ndarray) -> np.ndarray:
    E = np.zeros((3, 3), complex)
    lib().or_eln_matrix(_ptr(parts), len(parts), _ptr(E))
    return E


def domain_averages(cfg: OrConfig, grid: np.ndarray):
    """(abs_avgs[4,3,3] = <|n|>, <|nbar|>, <|f_x|>, <|fbar_x|>;  avg[2,3,3] = <n>, <nbar>)."""
    a = np.zeros((4, 3, 3))
    m = np.zeros((2, 3, 3), complex)
    lib().or_domain_averages(ctypes.byref(cfg), _ptr(grid), _ptr(a), _ptr(m))
    return a, m


# ------------------------------------------------------------------ 3D grid

PARTICLE3 = np.dtype(
    [
        ("x", "f8", (3,)),
        ("omega", "f8", (3,)),
        ("N", "f8"),
        ("Nbar", "f8"),
        ("rho", "c16", (3, 3)),
        ("rhobar", "c16", (3, 3)),
    ],
    align=True,
)


class OrConfig3(ctypes.Structure):
    _fields_ = [("c", OrConfig), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("Lx", ctypes.c_double),
                ("Ly", ctypes.c_double)]


def config3(nx, ny, nz, ndir, Lx, Ly, Lz, kappa, c_light, cfl_adv=0.4, cfl_flavor=0.4, osc=None,
            shape_order=2) -> OrConfig3:
    """3D periodic box of nx x ny x nz cells (see emu_oracle3d.c)."""
    c = OrConfig3()
    c.c = config(nz, ndir, Lz, kappa, c_light, cfl_adv, cfl_flavor, Lx * Ly, osc, shape_order)
    c.nx, c.ny, c.Lx, c.Ly = int(nx), int(ny), float(Lx), float(Ly)
    return c


def ncells3(cfg: OrConfig3) -> int:
    return cfg.nx * cfg.ny * cfg.c.nz


def cell_volume3(cfg: OrConfig3) -> float:
    return float(lib().or3_cell_volume(ctypes.byref(cfg)))


def shape3(cfg: OrConfig3, x):
    """(cell indices, weights) of the tensor-product shape of a particle at x (3,)."""
    x = np.ascontiguousarray(x, float)
    cells = np.zeros(64, np.int32)
    w = np.zeros(64)
    n = lib().or3_shape(ctypes.byref(cfg), _ptr(x), _ptr(cells), _ptr(w))
    return cells[:n], w[:n]


def init3(cfg: OrConfig3, n_nu, n_nubar, f_nu, f_nubar, alpha=1e-6, seed=0, dirs=None):
    """Particles of Eq. 8/9 on the 3D lattice, numbered p = d * ncells + c0."""
    C, M = ncells3(cfg), cfg.c.ndir
    n_nu = np.ascontiguousarray(np.broadcast_to(np.asarray(n_nu, float), (C,)))
    n_nubar = np.ascontiguousarray(np.broadcast_to(np.asarray(n_nubar, float), (C,)))
    f_nu = np.ascontiguousarray(np.broadcast_to(np.asarray(f_nu, float), (C, 3)))
    f_nubar = np.ascontiguousarray(np.broadcast_to(np.asarray(f_nubar, float), (C, 3)))
    parts = np.zeros(C * M, PARTICLE3)
    dptr = None
    if dirs is not None:
        dirs = np.ascontiguousarray(np.asarray(dirs, float).reshape(M, 3))
        dptr = _ptr(dirs)
    rc = lib().or3_init(ctypes.byref(cfg), dptr, _ptr(n_nu), _ptr(n_nubar), _ptr(f_nu), _ptr(f_nubar),
                        float(alpha), int(seed), _ptr(parts))
    if rc != 0:
        raise ValueError("negative particle weight: a flux factor exceeds 1/3")
    return parts


def deposit3(cfg: OrConfig3, parts: np.ndarray) -> np.ndarray:
    grid = np.zeros(ncells3(cfg), CELL)
    lib().or3_deposit(ctypes.byref(cfg), _ptr(parts), len(parts), _ptr(grid))
    return grid


def hamiltonian3(cfg: OrConfig3, grid: np.ndarray, parts: np.ndarray) -> np.ndarray:
    H = np.zeros((len(parts), 3, 3), complex)
    L = lib()
    for p in range(len(parts)):
        L.or3_hamiltonian(ctypes.byref(cfg), _ptr(grid), _ptr(parts[p:p + 1]), _ptr(H[p]))
    return H


def rhs3(cfg: OrConfig3, parts: np.ndarray):
    P = len(parts)
    grid = np.zeros(ncells3(cfg), CELL)
    dr = np.zeros((P, 3, 3), complex)
    db = np.zeros((P, 3, 3), complex)
    lib().or3_rhs(ctypes.byref(cfg), _ptr(parts), P, _ptr(grid), _ptr(dr), _ptr(db))
    return dr, db, grid


def rk4_step3(cfg: OrConfig3, parts: np.ndarray, dt: float) -> None:
    if lib().or3_rk4_step(ctypes.byref(cfg), _ptr(parts), len(parts), float(dt)) != 0:
        raise MemoryError("oracle scratch allocation failed")


def run3(cfg: OrConfig3, parts: np.ndarray, dt: float, nsteps: int) -> None:
    if lib().or3_run(ctypes.byref(cfg), _ptr(parts), len(parts), float(dt), int(nsteps)) != 0:
        raise MemoryError("oracle scratch allocation failed")


def timestep3(cfg: OrConfig3, grid: np.ndarray) -> float:
    return float(lib().or3_timestep(ctypes.byref(cfg), _ptr(grid)))
