"""Seeded synthetic inputs for the particle step (no method arithmetic here).

This module only fixes physical constants and draws the per-cell input
densities and fluxes of the workloads; both the CUDA library (through its
binding) and the CPU oracle (in the tests and the CPU baseline) take these
arrays as inputs.  Particle weights (Eq. 8), directions and the random
perturbations of the initial flavour state (Eq. 9) are computed by each side
on its own.

The paper releases no input data: these synthetic workloads stand in for its
runs (Sec. 3.1, App. B), with the grid sizes, direction counts, densities and
flux factors its text gives.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# CODATA 2018 / PDG values.  kappa = sqrt(2) G_F / hbar with G_F in erg cm^3
# (Eq. 2 carries sqrt(2) G_F (hbar c)^3 with G_F/(hbar c)^3 in GeV^-2).
GF_GEV2 = 1.1663787e-5          # G_F / (hbar c)^3  [GeV^-2]
HBARC_GEV_CM = 197.3269804e-3 * 1e-13  # hbar c [GeV cm]
ERG_PER_GEV = 1.602176634e-3
HBAR_ERG_S = 1.054571817e-27
C_LIGHT = 2.99792458e10         # [cm/s]
KAPPA = math.sqrt(2.0) * GF_GEV2 * HBARC_GEV_CM ** 3 * ERG_PER_GEV / HBAR_ERG_S  # [cm^3/s]
ERG_PER_EV = 1.602176634e-12
ATOMIC_MASS_G = 1.66053906660e-24   # atomic mass unit [g]


@dataclass
class Workload:
    """One 1D periodic box: grid, directions and per-cell species inputs."""
    name: str
    nz: int
    ndir: int
    Lz: float                      # [cm]
    n_nu: np.ndarray               # (nz,)   nu_e number density [cm^-3]
    n_nubar: np.ndarray            # (nz,)   nubar_e number density [cm^-3]
    f_nu: np.ndarray               # (nz, 3) nu_e number flux [cm^-3]
    f_nubar: np.ndarray            # (nz, 3) nubar_e number flux [cm^-3]
    dirs: Optional[np.ndarray] = None   # (ndir, 3) or None = Fibonacci sphere
    alpha: float = 1e-6            # perturbation strength of Eq. 9
    seed: int = 0                  # seed of the Eq. 9 perturbations
    steps: int = 100
    cfl_adv: float = 0.4
    cfl_flavor: float = 0.4
    area: float = 1.0              # transverse cell area [cm^2]
    kappa: float = KAPPA
    c_light: float = C_LIGHT
    shape_order: int = 2           # degree of the B-spline particle shape (Sec. 2.2.1)
    meta: dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return self.nz * self.ndir

    @property
    def dz(self) -> float:
        return self.Lz / self.nz


def _uniform_species(nz, n, nbar, fvec, fbarvec):
    return (np.full(nz, float(n)), np.full(nz, float(nbar)),
            np.tile(np.asarray(fvec, float), (nz, 1)), np.tile(np.asarray(fbarvec, float), (nz, 1)))


def tiny_fiducial(seed: int = 0) -> Workload:
    """32 cells over 4 fastest-growing wavelengths (Lz = 13.42 cm), 16 Fibonacci
    directions, n_nue = 4.9e32, n_nuebar = 6.1e32 cm^-3, isotropic nu_e and
    nubar_e flux factor 1/3 along -z, 100 steps at C = C_F = 0.4."""
    nz, n, nb = 32, 4.9e32, 6.1e32
    sp = _uniform_species(nz, n, nb, (0, 0, 0), (0, 0, -nb / 3.0))
    return Workload("tiny_fiducial_32x16", nz, 16, 13.42, *sp, seed=seed, steps=100)


def paper_1d(asymmetric: bool = False, seed: int = 0) -> Workload:
    """The paper's 1D run shape (Sec. 3.1): 64 cm, 1024 cells, 378 directions
    per cell (387,072 particles), species of tiny_fiducial; optionally the
    nubar flux tilted to normalize(0.1, 0, -1) with flux factor 1/3."""
    nz, n, nb = 1024, 4.9e32, 6.1e32
    if asymmetric:
        u = np.array([0.1, 0.0, -1.0]); u /= np.linalg.norm(u)
        fb = nb / 3.0 * u
    else:
        fb = np.array([0.0, 0.0, -nb / 3.0])
    sp = _uniform_species(nz, n, nb, (0, 0, 0), fb)
    name = "paper_1d_1024x378" + ("_asym" if asymmetric else "")
    return Workload(name, nz, 378, 64.0, *sp, seed=seed, steps=20000)


def throughput_1d(nz: int = 16384, ndir: int = 1000, seed: int = 0) -> Workload:
    """Throughput-scale 1D box: dz = 1/16 cm, per-cell n ~ U[1e32, 1e33] and
    flux factor ~ U[0, 0.3] for each species, flux along +z or -z (random sign),
    all drawn from numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.uniform(1e32, 1e33, nz)
    nb = rng.uniform(1e32, 1e33, nz)
    ff = rng.uniform(0.0, 0.3, nz)
    ffb = rng.uniform(0.0, 0.3, nz)
    sg = rng.choice([-1.0, 1.0], nz)
    sgb = rng.choice([-1.0, 1.0], nz)
    f = np.zeros((nz, 3)); f[:, 2] = sg * ff * n
    fb = np.zeros((nz, 3)); fb[:, 2] = sgb * ffb * nb
    return Workload(f"throughput_1d_{nz}x{ndir}", nz, ndir, nz / 16.0, n, nb, f, fb, seed=seed, steps=200)


def random_box(nz: int, ndir: int, seed: int = 0, Lz: Optional[float] = None) -> Workload:
    """Small randomised box for parity tests: per-cell densities in [1e32, 1e33],
    flux factors in [0, 1/3) with random 3D directions (so the x and y flux
    terms are exercised)."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    n = rng.uniform(1e32, 1e33, nz)
    nb = rng.uniform(1e32, 1e33, nz)

    def flux(dens):
        v = rng.normal(size=(nz, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * (rng.uniform(0.0, 0.33, nz) * dens)[:, None]

    f, fb = flux(n), flux(nb)
    return Workload(f"random_{nz}x{ndir}_s{seed}", nz, ndir, Lz if Lz else nz / 16.0, n, nb, f, fb,
                    seed=seed, steps=10)


def adjoint_box(alpha: float = 1e-20, seed: int = 0, nz: int = 256, ndir: int = 96, steps: int = 400) -> Workload:
    """Box for gradients of the growth phase: tiny_fiducial's species and cell
    size (dz = 13.42/32 cm) over nz cells (nz/8 fastest-growing wavelengths),
    ndir Fibonacci directions, `steps` steps; alpha small enough that the
    instability is still in its linear phase at the last step."""
    n, nb = 4.9e32, 6.1e32
    sp = _uniform_species(nz, n, nb, (0, 0, 0), (0, 0, -nb / 3.0))
    return Workload(f"adjoint_{nz}x{ndir}", nz, ndir, 13.42 / 32 * nz, *sp, alpha=alpha, seed=seed, steps=steps,
                    meta={"checkpoint_every": 20})


def two_beam(nz: int = 64, n: float = 4.89e32) -> Workload:
    """Inhomogeneous two-beam test (App. A.4): a 1 cm box, one nu_e beam along
    +z and one nubar_e beam along -z of equal density n.  With two directions
    +-z, flux factors of +-1/3 put all neutrinos in the +z particle and all
    antineutrinos in the -z particle (Eq. 8)."""
    sp = _uniform_species(nz, n, n, (0, 0, n / 3.0), (0, 0, -n / 3.0))
    dirs = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    return Workload(f"two_beam_{nz}", nz, 2, 1.0, *sp, dirs=dirs, steps=200)


def sweep(nbox: int = 256, seed: int = 0, nz_range=(64, 1024), ndir_range=(48, 378)) -> list:
    """Parameter sweep of independent boxes (the density, flux-magnitude and
    flux-direction sweeps of Sec. 4): per box, from numpy PCG64(seed),
    nz ~ U{nz_range}, ndir ~ U{ndir_range}, n, nbar ~ U[1e32, 1e33] cm^-3,
    flux factors |f|/n, |fbar|/nbar ~ U[0, 1/3], nu flux along +z and nubar flux
    at an angle ~ U[0, pi] from it; dz = 1/16 cm; Eq. 9 seed = box index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(nbox):
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        M = int(rng.integers(ndir_range[0], ndir_range[1] + 1))
        n, nb = rng.uniform(1e32, 1e33, 2)
        ff, ffb = rng.uniform(0.0, 1.0 / 3.0, 2)
        ang = rng.uniform(0.0, np.pi)
        fv = np.array([0.0, 0.0, ff * n])
        fbv = ffb * nb * np.array([np.sin(ang), 0.0, np.cos(ang)])
        sp = _uniform_species(nz, n, nb, fv, fbv)
        out.append(Workload(f"sweep{b}_{nz}x{M}", nz, M, nz / 16.0, *sp, seed=b, steps=2000,
                            meta={"flux_angle": ang, "ff": ff, "ffb": ffb}))
    return out


def head(wl: Workload, nz: int) -> Workload:
    """The first nz cells of a workload (same per-cell inputs, cell size and
    directions): a bounded sample of it."""
    nz = min(nz, wl.nz)
    return Workload(f"{wl.name}[:{nz}]", nz, wl.ndir, wl.dz * nz, wl.n_nu[:nz].copy(), wl.n_nubar[:nz].copy(),
                    wl.f_nu[:nz].copy(), wl.f_nubar[:nz].copy(), dirs=wl.dirs, alpha=wl.alpha, seed=wl.seed,
                    steps=wl.steps, cfl_adv=wl.cfl_adv, cfl_flavor=wl.cfl_flavor, area=wl.area, kappa=wl.kappa,
                    c_light=wl.c_light, shape_order=wl.shape_order)


def oscillation(mass_eV=(0.0, 0.0, 0.0), theta12=0.0, theta13=0.0, theta23=0.0, delta_cp=0.0,
                energy_MeV=50.0, rho_g_cm3=0.0, Ye=0.5) -> dict:
    """Vacuum and matter parameters of Eq. 2: masses m_i c^2 [eV], mixing angles
    and phase [rad], neutrino energy, matter density and electron fraction
    (net electron density n_e = rho Ye / m_u)."""
    return {"mass_eV": tuple(float(m) for m in mass_eV), "theta12": float(theta12), "theta13": float(theta13),
            "theta23": float(theta23), "delta_cp": float(delta_cp), "energy_erg": energy_MeV * 1e6 * ERG_PER_EV,
            "n_e": rho_g_cm3 * Ye / ATOMIC_MASS_G, "hbar": HBAR_ERG_S, "erg_per_eV": ERG_PER_EV}


def msw_test() -> tuple:
    """App. A.1: one 1 cm zone, matter of 1.35e9 g/cm^3 with Ye = 1, m1 = 8.6e-3 eV,
    m2 = 0, theta12 = 33.82 deg, E = 0.138 eV; two particles, one neutrino and one
    antineutrino each (negligible self-interaction)."""
    osc = oscillation(mass_eV=(8.6e-3, 0.0, 0.0), theta12=math.radians(33.82), energy_MeV=0.138e-6,
                      rho_g_cm3=1.35e9, Ye=1.0)
    dirs = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    # one physical (anti)neutrino per particle: n = N * M / dV = 2 cm^-3, isotropic
    sp = _uniform_species(1, 2.0, 2.0, (0, 0, 0), (0, 0, 0))
    return Workload("msw_1zone", 1, 2, 1.0, *sp, dirs=dirs, alpha=0.0, steps=0, meta={"osc": osc}), osc


def bipolar() -> tuple:
    """App. A.2: one zone, one particle along +z and one along -z, each carrying
    nu_e and nubar_e of equal density n = nbar with sqrt(2) G_F n / hbar = 10 x
    the vacuum frequency |dm^2| c^4 / (2 E hbar) (m1 = 8.6e-3 eV, m2 = 0,
    theta12 = 0.01 rad, E = 50 MeV, no matter)."""
    osc = oscillation(mass_eV=(8.6e-3, 0.0, 0.0), theta12=0.01, energy_MeV=50.0)
    dm2 = (osc["mass_eV"][0] * ERG_PER_EV) ** 2
    w_vac = dm2 / (2.0 * osc["energy_erg"]) / HBAR_ERG_S
    n = 10.0 * w_vac / KAPPA
    dirs = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    sp = _uniform_species(1, n, n, (0, 0, 0), (0, 0, 0))
    return (Workload("bipolar_1zone", 1, 2, 1.0, *sp, dirs=dirs, alpha=0.0, steps=0,
                     meta={"omega": w_vac, "mu": KAPPA * n}), osc)


def homogeneous_two_beam() -> tuple:
    """App. A.3: one zone, a nu_e beam along +z and a nubar_e beam along -z of
    equal density n = |dm^2| c^4 / (4 sqrt(2) G_F E) with m1 = 8.6e-3 eV, m2 = 0,
    theta12 = 1e-6 deg, E = 50 MeV, no matter."""
    osc = oscillation(mass_eV=(8.6e-3, 0.0, 0.0), theta12=math.radians(1e-6), energy_MeV=50.0)
    dm2 = (osc["mass_eV"][0] * ERG_PER_EV) ** 2
    w_vac = dm2 / (2.0 * osc["energy_erg"]) / HBAR_ERG_S
    n = w_vac / (2.0 * KAPPA)
    dirs = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    sp = _uniform_species(1, n, n, (0, 0, n / 3.0), (0, 0, -n / 3.0))
    return Workload("two_beam_homogeneous", 1, 2, 1.0, *sp, dirs=dirs, alpha=0.0, steps=0,
                    meta={"osc": osc, "growth": w_vac}), osc


def with_shape(wl: Workload, order: int) -> Workload:
    """The same workload with particles of shape order `order` (0..3)."""
    import dataclasses
    return dataclasses.replace(wl, name=f"{wl.name}_o{order}", shape_order=int(order))


def by_name(name: str) -> Workload:
    table = {
        "tiny_fiducial": tiny_fiducial,
        "paper_1d": paper_1d,
        "paper_1d_asym": lambda: paper_1d(True),
        "throughput_1d": throughput_1d,
    }
    return table[name]()


@dataclass
class Workload3:
    """One 3D periodic box: nx x ny x nz cells, directions and per-cell
    species inputs in cell-index order c = (jx * ny + jy) * nz + jz."""
    name: str
    nx: int
    ny: int
    nz: int
    ndir: int
    Lx: float
    Ly: float
    Lz: float
    n_nu: np.ndarray               # (C,)
    n_nubar: np.ndarray            # (C,)
    f_nu: np.ndarray               # (C, 3)
    f_nubar: np.ndarray            # (C, 3)
    dirs: Optional[np.ndarray] = None
    alpha: float = 1e-6
    seed: int = 0
    steps: int = 10
    cfl_adv: float = 0.4
    cfl_flavor: float = 0.4
    kappa: float = KAPPA
    c_light: float = C_LIGHT
    shape_order: int = 2
    meta: dict = field(default_factory=dict)

    @property
    def C(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def P(self) -> int:
        return self.C * self.ndir


def random_box3(nx: int, ny: int, nz: int, ndir: int, seed: int = 0, h: float = 1.0 / 16.0,
                shape_order: int = 2) -> Workload3:
    """Randomised 3D box: cells of edge h (the paper's converged 1D resolution
    by default), per-cell densities in [1e32, 1e33] and flux factors in
    [0, 1/3) with random 3D directions, numpy PCG64(2000 + seed)."""
    rng = np.random.Generator(np.random.PCG64(2000 + seed))
    C = nx * ny * nz
    n = rng.uniform(1e32, 1e33, C)
    nb = rng.uniform(1e32, 1e33, C)

    def flux(dens):
        v = rng.normal(size=(C, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * (rng.uniform(0.0, 0.33, C) * dens)[:, None]

    f, fb = flux(n), flux(nb)
    return Workload3(f"random3_{nx}x{ny}x{nz}x{ndir}_s{seed}", nx, ny, nz, ndir, nx * h, ny * h, nz * h, n, nb, f, fb,
                     seed=seed, shape_order=shape_order)


def fiducial_3d(nx: int = 32, ny: int = 32, nz: int = 32, ndir: int = 16) -> Workload3:
    """3D box of tiny_fiducial's species (n = 4.9e32, nbar = 6.1e32 cm^-3,
    nubar flux -nbar/3 along z, the ELN crossing of Sec. 3.2) with its cell
    edge (13.42/32 cm) on every axis."""
    C = nx * ny * nz
    n, nb = 4.9e32, 6.1e32
    sp = (np.full(C, n), np.full(C, nb), np.zeros((C, 3)), np.tile([0.0, 0.0, -nb / 3.0], (C, 1)))
    h = 13.42 / 32
    return Workload3(f"fiducial3d_{nx}x{ny}x{nz}x{ndir}", nx, ny, nz, ndir, nx * h, ny * h, nz * h, *sp, steps=50)
