"""Two-flavour limit of the oracle against a separately written 2x2 integration.

With rho_etau = rho_mutau = rho_tautau = 0 (and the same for rhobar) the tau
row and column of every density matrix stay zero under Eq. 4 with the
self-interaction Hamiltonian of Eq. 2 (H's e-tau and mu-tau entries are
deposits of zero entries), so the e-mu block evolves as a two-flavour system.
This file integrates that system on its own, written from Eq. 4-6 and
Sec. 2.3 with 2x2 complex matrices (numpy, vectorised over particles: the
quadratic B-spline weights of Sec. 2.2.1, the deposit of Eq. 5 with
B = N rho - Nbar rhobar^*, H = kappa sum_j w (A0_j - Omega . A_j), Hbar = -H^*,
K = -i[H, rho], the classic RK4 tableau, positions advanced with the stages),
and checks the oracle's e-mu block against it.  A mistake shared by every
flavour pair of the oracle's 3x3 code (a sign of the commutator's diagonal
terms, a transposed product, a missing conjugate) fails here; the relabelling
test of the pins cannot see it."""
import numpy as np

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W


def _quadratic_weights(z, dz, nz):
    """Cells and weights of the quadratic B-spline centred on z (three cells)."""
    xi = z / dz - 0.5
    j = np.floor(xi + 0.5)
    d = xi - j
    w = np.stack([0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2], axis=1)
    cells = np.stack([j - 1, j, j + 1], axis=1).astype(np.int64) % nz
    return cells, w


class TwoFlavourPIC:
    """1D periodic two-flavour particle step with 2x2 complex matrices."""

    def __init__(self, nz, Lz, kappa, c_light, area, omega, N, Nbar):
        self.nz, self.Lz, self.kappa, self.c = nz, Lz, kappa, c_light
        self.dz = Lz / nz
        self.dV = self.dz * area
        self.omega, self.N, self.Nbar = omega, N, Nbar

    def derivatives(self, z, rho, rhobar):
        cells, w = _quadratic_weights(z, self.dz, self.nz)
        B = self.N[:, None, None] * rho - self.Nbar[:, None, None] * np.conj(rhobar)   # (P, 2, 2)
        A0 = np.zeros((self.nz, 2, 2), complex)
        A = np.zeros((self.nz, 3, 2, 2), complex)
        for k in range(3):
            np.add.at(A0, cells[:, k], w[:, k, None, None] * B)
            np.add.at(A, cells[:, k], w[:, k, None, None, None] * self.omega[:, :, None, None] * B[:, None])
        A0 *= self.kappa / self.dV
        A *= self.kappa / self.dV
        H = np.zeros_like(rho)
        for k in range(3):
            H += w[:, k, None, None] * (A0[cells[:, k]] - np.einsum("pi,pirs->prs", self.omega, A[cells[:, k]]))
        Hbar = -np.conj(H)
        K = -1j * (H @ rho - rho @ H)
        Kbar = -1j * (Hbar @ rhobar - rhobar @ Hbar)
        return K, Kbar

    def step(self, z, rho, rhobar, dt):
        vz = self.c * self.omega[:, 2]
        k1, l1 = self.derivatives(z, rho, rhobar)
        k2, l2 = self.derivatives(z + 0.5 * dt * vz, rho + 0.5 * dt * k1, rhobar + 0.5 * dt * l1)
        k3, l3 = self.derivatives(z + 0.5 * dt * vz, rho + 0.5 * dt * k2, rhobar + 0.5 * dt * l2)
        k4, l4 = self.derivatives(z + dt * vz, rho + dt * k3, rhobar + dt * l3)
        rho = rho + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        rhobar = rhobar + dt / 6.0 * (l1 + 2.0 * l2 + 2.0 * l3 + l4)
        z = z + dt * vz
        z = z - self.Lz * np.floor(z / self.Lz)
        return z, rho, rhobar


def _two_flavour_start(wl, alpha):
    cfg = O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, alpha, wl.seed, wl.dirs)
    for key in ("rho", "rhobar"):
        r = parts[key]
        r[:, 0, 2] = r[:, 2, 0] = r[:, 1, 2] = r[:, 2, 1] = r[:, 2, 2] = 0.0
        r[:, 0, 0] = 1.0 - r[:, 1, 1].real          # unit trace, eps_mu = |rho_emu|^2 as in Eq. 9
    return cfg, parts


def _check(wl, alpha, steps):
    cfg, parts = _two_flavour_start(wl, alpha)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    two = TwoFlavourPIC(wl.nz, wl.Lz, wl.kappa, wl.c_light, wl.area, parts["omega"].copy(), parts["N"].copy(),
                        parts["Nbar"].copy())
    z, rho, rhobar = parts["z"].copy(), parts["rho"][:, :2, :2].copy(), parts["rhobar"][:, :2, :2].copy()
    emu0 = np.abs(rho[:, 0, 1]).max()
    for n in range(steps):
        O.run(cfg, parts, dt, 1)
        z, rho, rhobar = two.step(z, rho, rhobar, dt)
        for key, mine in (("rho", rho), ("rhobar", rhobar)):
            r = parts[key]
            assert np.all(r[:, 2, :] == 0) and np.all(r[:, :, 2] == 0), (n, key)   # tau stays exactly empty
            block = r[:, :2, :2]
            scale = np.sqrt((np.abs(block) ** 2).sum(axis=(1, 2))).max()
            assert np.abs(block - mine).max() <= 1e-13 * scale, (n, key, np.abs(block - mine).max() / scale)
            off = np.abs(block[:, 0, 1]).max()
            assert np.abs(block[:, 0, 1] - mine[:, 0, 1]).max() <= 1e-9 * off, (n, key)
        assert np.abs(parts["z"] - z).max() <= 1e-13 * wl.Lz
    return emu0, np.abs(rho[:, 0, 1]).max()


def test_two_flavour_block_matches_2x2_integration_fiducial():
    """The 32 x 16 fiducial box (ELN crossing, Sec. 3.2), 100 steps in the
    linear phase (alpha = 1e-10): the unstable e-mu block grows ~1e4-fold."""
    emu0, emu1 = _check(W.tiny_fiducial(), 1e-10, 100)
    assert emu1 > 1e3 * emu0          # the instability is exercised, not a static state


def test_two_flavour_block_matches_2x2_integration_random_3d_fluxes():
    """A box with per-cell densities and 3D flux directions (every component of
    Omega . A enters), 60 steps from alpha = 1e-6."""
    _check(W.random_box(24, 10, seed=8), 1e-6, 60)
