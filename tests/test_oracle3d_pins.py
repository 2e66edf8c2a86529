"""Pins of the 3D oracle (emu_oracle3d.c) against things other than itself.

- The 1D oracle: with nx = ny = 1 the 3D box is the 1D box along z; with the
  problem turned so that the old z axis runs along x (or y) and nx = 32
  (or ny = 32) it is the same physical system, so it must give the 1D run's
  states up to rounding.  Together these pin the handling of every axis.
- Brute force: one particle in a box with three different cell counts and
  edges, next to a corner (periodic wrap on every axis), against the
  quadratic B-spline weights written out here.
- Exact properties: deposit and interpolation are adjoint (the same weights);
  a constant field interpolates to itself; a state without spatial structure
  stays homogeneous; the trace of rho and the domain lepton matrix
  sum_p (N rho - Nbar rhobar^*) are conserved (Sec. 3.3, Eq. 18).
- Linear stability: the fastest box mode along x grows at the rate of the
  discrete dispersion solve (Sec. 3.2), as in 1D.
"""
import numpy as np
import pytest

from oracle import dispersion as D
from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import family_err, pack


def _qweights(x, h):
    """Cells (unwrapped) and weights of the quadratic B-spline at x on an axis of cell width h."""
    xi = x / h - 0.5
    j = np.floor(xi + 0.5)
    d = xi - j
    return [int(j) - 1, int(j), int(j) + 1], [0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2]


def _rand_herm(rng):
    a = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    h = a @ a.conj().T
    return h / np.trace(h).real


def _turn(v, axis):
    """Components of v (..., 3) with the old z axis turned onto `axis` (0 = x,
    1 = y), by a cyclic permutation (a rotation)."""
    v = np.asarray(v, float)
    return v[..., [2, 0, 1]] if axis == 0 else v[..., [1, 2, 0]]


def _fibonacci(M):
    return np.array([O.fibonacci_direction(d, M) for d in range(M)])


def _one_d(wl, steps):
    cfg = O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    O.run(cfg, parts, dt, steps)
    return parts, dt


def test_reduces_to_1d_along_z():
    wl = W.random_box(29, 7, seed=4)
    ref, dt1 = _one_d(wl, 12)
    cfg = O.config3(1, 1, wl.nz, wl.ndir, 1.0, wl.area, wl.Lz, wl.kappa, wl.c_light)
    parts = O.init3(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    dt = O.timestep3(cfg, O.deposit3(cfg, parts))
    assert abs(dt - dt1) <= 1e-15 * dt1
    O.run3(cfg, parts, dt1, 12)
    for key in ("rho", "rhobar"):
        assert family_err(pack(parts[key]), pack(ref[key])) < 1e-13, key
    assert np.abs(parts["x"][:, 2] - ref["z"]).max() <= 1e-13 * wl.Lz
    assert np.all(parts["N"] == ref["N"]) and np.all(parts["Nbar"] == ref["Nbar"])


@pytest.mark.parametrize("axis", [0, 1])
def test_turned_box_along_x_or_y_equals_1d(axis):
    wl = W.random_box(24, 9, seed=5)
    ref, dt = _one_d(wl, 15)
    # the two one-cell axes span the 1D box's cross-section (area), so that
    # the cells have the 1D cell's volume
    L = [0.8, wl.area / 0.8, 0.8]
    L[(axis + 1) % 3] = wl.area / 0.8
    L[(axis + 2) % 3] = 0.8
    n = [1, 1, 1]
    n[axis], L[axis] = wl.nz, wl.Lz
    dirs = _turn(wl.dirs if wl.dirs is not None else _fibonacci(wl.ndir), axis)
    cfg = O.config3(n[0], n[1], n[2], wl.ndir, L[0], L[1], L[2], wl.kappa, wl.c_light)
    assert abs(O.cell_volume3(cfg) / (wl.Lz / wl.nz * wl.area) - 1) < 1e-15
    parts = O.init3(cfg, wl.n_nu, wl.n_nubar, _turn(wl.f_nu, axis), _turn(wl.f_nubar, axis), wl.alpha, wl.seed,
                    dirs)
    assert np.abs(parts["N"] - ref["N"]).max() <= 1e-14 * np.abs(ref["N"]).max()
    O.run3(cfg, parts, dt, 15)
    for key in ("rho", "rhobar"):
        assert family_err(pack(parts[key]), pack(ref[key])) < 1e-12, key
    assert np.abs(parts["x"][:, axis] - ref["z"]).max() <= 1e-12 * wl.Lz


def test_single_particle_deposit_brute_force_3d():
    rng = np.random.default_rng(11)
    nx, ny, nz = 5, 4, 7
    Lx, Ly, Lz = 2.5, 1.0, 4.9
    cfg = O.config3(nx, ny, nz, 1, Lx, Ly, Lz, W.KAPPA, W.C_LIGHT)
    parts = np.zeros(1, O.PARTICLE3)
    pos = np.array([0.07, 0.98, 4.85])          # next to a corner: wraps on every axis
    parts["x"] = pos
    om = rng.normal(size=3)
    parts["omega"] = om / np.linalg.norm(om)
    parts["N"], parts["Nbar"] = 2.0e30, 1.5e30
    parts["rho"] = _rand_herm(rng)
    parts["rhobar"] = _rand_herm(rng)
    grid = O.deposit3(cfg, parts)
    dV = (Lx / nx) * (Ly / ny) * (Lz / nz)
    expect = np.zeros(nx * ny * nz)
    for ci, wi in zip(*_qweights(pos[0], Lx / nx)):
        for cj, wj in zip(*_qweights(pos[1], Ly / ny)):
            for ck, wk in zip(*_qweights(pos[2], Lz / nz)):
                expect[((ci % nx) * ny + cj % ny) * nz + ck % nz] += wi * wj * wk
    assert np.count_nonzero(expect) == 27
    q = parts[0]
    # the oracle evaluates the B-spline from its truncated-power form, whose
    # small weights (a particle near a face) carry cancellation: compare at
    # 1e-14 of the largest contribution; untouched cells must be exactly 0
    an = 1e-14 * q["N"] * np.abs(q["rho"]).max() / dV
    ab = 1e-14 * q["Nbar"] * np.abs(q["rhobar"]).max() / dV
    for c in range(nx * ny * nz):
        if expect[c] == 0.0:
            assert not np.any(grid["n"][c]) and not np.any(grid["f"][c]) and not np.any(grid["nbar"][c])
            continue
        assert np.allclose(grid["n"][c], q["N"] * expect[c] * q["rho"] / dV, rtol=1e-14, atol=an)
        assert np.allclose(grid["nbar"][c], q["Nbar"] * expect[c] * q["rhobar"] / dV, rtol=1e-14, atol=ab)
        for i in range(3):
            assert np.allclose(grid["f"][c, i], q["N"] * expect[c] * q["rho"] * q["omega"][i] / dV, rtol=1e-14,
                               atol=an)


def test_deposit_interpolation_adjoint_and_constants_3d():
    rng = np.random.default_rng(12)
    nx, ny, nz, P = 4, 6, 5, 60
    L = np.array([1.2, 2.4, 3.5])
    cfg = O.config3(nx, ny, nz, 1, *L, W.KAPPA, W.C_LIGHT)
    parts = np.zeros(P, O.PARTICLE3)
    parts["x"] = rng.uniform(0, 1, size=(P, 3)) * L
    om = rng.normal(size=(P, 3))
    parts["omega"] = om / np.linalg.norm(om, axis=1, keepdims=True)
    parts["N"] = rng.uniform(1, 2, size=P) * 1e30
    parts["rho"] = np.array([_rand_herm(rng) for _ in range(P)])
    grid = O.deposit3(cfg, parts)
    C = nx * ny * nz
    G = np.zeros(C, O.CELL)
    G["n"] = rng.normal(size=(C, 3, 3)) + 1j * rng.normal(size=(C, 3, 3))
    H = O.hamiltonian3(cfg, G, parts) / W.KAPPA      # = interpolation of G["n"] (Eq. 6)
    dV = O.cell_volume3(cfg)
    lhs = np.sum(grid["n"] * G["n"])
    rhs = np.sum(parts["N"][:, None, None] * parts["rho"] * H) / dV
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    K = np.zeros(C, O.CELL)
    M0 = _rand_herm(rng) * 3.0
    K["n"] = M0
    assert np.allclose(O.hamiltonian3(cfg, K, parts) / W.KAPPA, M0[None], rtol=1e-14, atol=1e-15)


def _small_3d(seed=0, n=(4, 3, 5), M=6, alpha=1e-6, L=(1.6, 1.2, 2.0)):
    rng = np.random.default_rng(seed)
    C = n[0] * n[1] * n[2]
    cfg = O.config3(*n, M, *L, W.KAPPA, W.C_LIGHT)
    nn = rng.uniform(1e32, 1e33, C)
    nb = rng.uniform(1e32, 1e33, C)
    fu = rng.normal(size=(C, 3))
    fb = rng.normal(size=(C, 3))
    fu *= (rng.uniform(0, 0.3, C) * nn / np.linalg.norm(fu, axis=1))[:, None]
    fb *= (rng.uniform(0, 0.3, C) * nb / np.linalg.norm(fb, axis=1))[:, None]
    parts = O.init3(cfg, nn, nb, fu, fb, alpha, seed)
    return cfg, parts


def test_trace_and_lepton_matrix_conserved_3d():
    cfg, parts = _small_3d(seed=3, alpha=1e-2)
    E0 = np.sum(parts["N"][:, None, None] * parts["rho"] - parts["Nbar"][:, None, None] * parts["rhobar"].conj(),
                axis=0)
    dt = O.timestep3(cfg, O.deposit3(cfg, parts))
    O.run3(cfg, parts, dt, 25)
    E1 = np.sum(parts["N"][:, None, None] * parts["rho"] - parts["Nbar"][:, None, None] * parts["rhobar"].conj(),
                axis=0)
    scale = np.abs(parts["N"]).sum() + np.abs(parts["Nbar"]).sum()
    assert np.abs(E1 - E0).max() <= 1e-12 * scale
    for key in ("rho", "rhobar"):
        tr = np.trace(parts[key], axis1=1, axis2=2)
        assert np.abs(tr - 1.0).max() <= 1e-12
    # the state did change (off-diagonals grew or rotated)
    assert np.abs(E1[0, 1]) > 0


def test_homogeneous_state_stays_homogeneous_3d():
    n = (3, 4, 5)
    C = n[0] * n[1] * n[2]
    M = 8
    cfg = O.config3(*n, M, 1.5, 2.0, 2.5, W.KAPPA, W.C_LIGHT)
    parts = O.init3(cfg, 4.9e32, 6.1e32, [0.05e32, 0.0, 0.1e32], [0.0, -0.3e32, -2.0e32], 1e-4, 2)
    for key in ("rho", "rhobar"):
        r = parts[key].reshape(M, C, 3, 3)
        r[:] = r[:, :1]
    O.run3(cfg, parts, O.timestep3(cfg, O.deposit3(cfg, parts)), 30)
    g = O.deposit3(cfg, parts)
    for key in ("n", "nbar"):
        v = g[key]
        assert np.abs(v - v.mean(axis=0, keepdims=True)).max() <= 1e-10 * np.abs(v).max()
    assert np.abs(g["n"][:, 0, 1]).max() > 0


def test_growth_along_x_matches_discrete_dispersion():
    """The fiducial species turned onto x in a 32 x 1 x 1 box: the fastest box
    mode along x grows at the discrete dispersion solve's rate (same 16
    directions, box wavenumbers, quadratic shape transfer averaged over the
    particles' offsets) within 2%, as the 1D box does along z."""
    wl = W.tiny_fiducial()
    dirs1 = _fibonacci(wl.ndir)
    cfg = O.config3(wl.nz, 1, 1, wl.ndir, wl.Lz, 1.0, 1.0, wl.kappa, wl.c_light)
    parts = O.init3(cfg, wl.n_nu, wl.n_nubar, _turn(wl.f_nu, 0), _turn(wl.f_nubar, 0), wl.alpha, wl.seed,
                    _turn(dirs1, 0))
    g = (wl.n_nu[0] + 3 * dirs1 @ wl.f_nu[0]) / wl.ndir
    gb = (wl.n_nubar[0] + 3 * dirs1 @ wl.f_nubar[0]) / wl.ndir
    rates = {}
    for m in range(1, wl.nz // 2):
        k = 2 * np.pi * m / wl.Lz
        rates[m] = D.discrete_growth(k, dirs1, g, gb, W.KAPPA, W.C_LIGHT,
                                     S=D.shape_transfer(k, wl.Lz / wl.nz, 2, spread=True))
    mbest = max(rates, key=rates.get)
    dt = O.timestep3(cfg, O.deposit3(cfg, parts))
    amp = []
    for _ in range(81):
        gr = O.deposit3(cfg, parts)
        amp.append(abs(np.fft.fft(gr["n"][:, 0, 1])[mbest]))
        O.rk4_step3(cfg, parts, dt)
    ts = np.arange(81) * dt
    slope = np.polyfit(ts[30:], np.log(amp)[30:], 1)[0]
    assert abs(slope / rates[mbest] - 1) < 0.02, (mbest, slope, rates[mbest])
