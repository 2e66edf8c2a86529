"""Particles anywhere: positions jittered off the lattice and a direction of
their own per particle (no rings), through the C ABI, against the oracle,
which takes any positions and directions (Eq. 5, 6 per particle).

The box notices on its own (emu_set_particles checks the lattice contract)
and switches to the sorted path: per stage a stable radix sort by cell and a
deposit by one warp per cell in that order.  Tolerances as on the lattice:
one deposit, moments, interpolation 1e-12; every one of the first steps
1e-10; runs bitwise reproducible."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import density_scales, family_err, moment_families, oracle_moments, oracle_potential, pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_02745_gb300 import build
    build.build()
    return torch


def _cfg(wl):
    return O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area,
                    shape_order=wl.shape_order)


def _scatter(wl, seed, jitter=0.45, own_dirs=True):
    """Oracle particles of wl with every position moved by U(-jitter, jitter)
    cells and (own_dirs) every direction replaced by a random unit vector,
    and the same arrays for the GPU machine (inputs of both sides)."""
    cfg = _cfg(wl)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    rng = np.random.default_rng(seed)
    z = parts["z"] + rng.uniform(-jitter, jitter, len(parts)) * wl.dz
    z = z - wl.Lz * np.floor(z / wl.Lz)
    parts["z"] = np.where(z >= wl.Lz, z - wl.Lz, z)
    if own_dirs:
        om = rng.normal(size=(len(parts), 3))
        parts["omega"] = om / np.linalg.norm(om, axis=1, keepdims=True)
    return cfg, parts


def _box(wl, parts):
    from paper_2101_02745_gb300.emu import Box
    box = Box.from_workload(wl)
    assert not box.general()
    box.set_host(z=parts["z"].copy(), ox=parts["omega"][:, 0].copy(), oy=parts["omega"][:, 1].copy(),
                 oz=parts["omega"][:, 2].copy())
    return box


def _moment_errs(box, grid):
    got = box.moments().cpu().numpy()
    ref = oracle_moments(grid)
    sn, snb, _ = density_scales(grid)
    return [family_err(g, r, s) for g, r, s in zip(moment_families(got), moment_families(ref), [sn] * 4 + [snb] * 4)]


CASES = [(67, 9, 2), (31, 4, 0), (31, 4, 1), (40, 6, 3), (2, 30, 2), (1, 20, 2), (5000, 7, 2)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_deposit_moments_interpolation_anywhere(torch, case):
    nz, M, order = case
    wl = W.with_shape(W.random_box(nz, M, seed=nz + M), order)
    cfg, parts = _scatter(wl, seed=1)
    box = _box(wl, parts)
    # one cell: every ring is one particle, so any positions and directions
    # keep the lattice contract; take the sorted path on purpose there
    assert box.general() == (nz > 1)
    if nz == 1:
        box.set_layout(1)
        assert box.general()
    grid = O.deposit(cfg, parts)
    A = box.deposit(0, 0.0).cpu().numpy()
    Aref = oracle_potential(grid, wl.kappa)
    s = wl.kappa * density_scales(grid)[2]
    assert max(family_err(A[9 * f:9 * (f + 1)], Aref[9 * f:9 * (f + 1)], s) for f in range(4)) < 1e-12
    assert max(_moment_errs(box, grid)) < 1e-12
    H = box.interpolate_H(0.0).cpu().numpy()
    assert family_err(H, pack(O.hamiltonian(cfg, grid, parts)), s) < 1e-12
    box.sync()


@pytest.mark.parametrize("case", [(67, 9, 2), (31, 4, 0), (40, 6, 3), (2, 30, 2)], ids=lambda c: "x".join(map(str, c)))
def test_steps_anywhere_match_oracle(torch, case):
    nz, M, order = case
    wl = W.with_shape(W.random_box(nz, M, seed=3 * nz + M), order)
    cfg, parts = _scatter(wl, seed=2)
    box = _box(wl, parts)
    dt = O.timestep(cfg, O.deposit(cfg, parts)) * (0.917 if order == 0 else 1.0)
    assert abs(box.timestep() - dt / (0.917 if order == 0 else 1.0)) <= 1e-13 * dt
    for n in range(50 if nz < 1000 else 10):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
        h = box.get_host()
        errs = [family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"]))]
        assert max(errs) < 1e-10, (n, errs)
        assert np.abs(h["z"] - parts["z"]).max() <= 1e-13 * wl.Lz
    assert max(_moment_errs(box, O.deposit(cfg, parts))) < 1e-10
    box.sync()


def test_anywhere_bitwise_reproducible_and_invariants(torch):
    wl = W.random_box(301, 12, seed=4)
    wl.alpha = 1e-3
    out = []
    for _ in range(2):
        cfg, parts = _scatter(wl, seed=3)
        box = _box(wl, parts)
        d0 = box.diagnostics()
        box.step(40)
        d1 = box.diagnostics()
        scale = np.abs(d0[36:45]).max() + np.abs(d0[45:54]).max()
        assert np.abs(d1[54:63] - d0[54:63]).max() < 1e-12 * scale      # Eq. 18
        out.append(box.get_host())
        box.sync()
    for k in ("rho", "rhobar", "z"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_lattice_particles_on_either_path_agree(torch):
    """Particles on the lattice run the same steps on the sorted path (forced
    with emu_set_layout) as on the lattice path, to rounding."""
    from paper_2101_02745_gb300.emu import Box
    wl = W.random_box(67, 37, seed=5)
    a, b = Box.from_workload(wl), Box.from_workload(wl)
    b.set_layout(1)
    assert b.general() and not a.general()
    dt = a.timestep()
    assert abs(b.timestep() - dt) <= 1e-13 * dt
    a.step(20, dt)
    b.step(20, dt)
    ha, hb = a.get_host(), b.get_host()
    assert family_err(hb["rho"], ha["rho"]) < 1e-12
    assert family_err(hb["rhobar"], ha["rhobar"]) < 1e-12
    assert np.array_equal(ha["z"], hb["z"])
    b.set_layout(-1)                  # checked again: on the lattice
    assert not b.general()
    a.sync()
    b.sync()


def test_batch_with_scattered_box(torch):
    """A batch whose middle box has scattered particles: the batch takes the
    sorted path and every box still matches its own oracle run."""
    from paper_2101_02745_gb300.emu import Box
    wls = [W.random_box(40, 5, seed=11), W.random_box(23, 8, seed=12), W.random_box(57, 3, seed=13)]
    box = Box.from_workloads(wls)
    refs = []
    z = []
    om = []
    for i, w in enumerate(wls):
        cfg, parts = _scatter(w, seed=20 + i) if i == 1 else (_cfg(w), O.init(_cfg(w), w.n_nu, w.n_nubar, w.f_nu,
                                                                                w.f_nubar, w.alpha, w.seed))
        refs.append((cfg, parts))
        z.append(parts["z"])
        om.append(parts["omega"])
    z, om = np.concatenate(z), np.concatenate(om)
    box.set_host(z=z, ox=om[:, 0].copy(), oy=om[:, 1].copy(), oz=om[:, 2].copy())
    assert box.general()
    dts = box.batch_timestep()
    box.batch_step(15)
    h = box.get_host()
    off = 0
    for (cfg, parts), dt, w in zip(refs, dts, wls):
        O.run(cfg, parts, dt, 15)
        assert family_err(h["rho"][:, off:off + w.P], pack(parts["rho"])) < 1e-10
        assert family_err(h["rhobar"][:, off:off + w.P], pack(parts["rhobar"])) < 1e-10
        off += w.P
    box.sync()


def test_anywhere_refuses_lattice_only_calls(torch):
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(31, 4, seed=6)
    cfg, parts = _scatter(wl, seed=4)
    box = _box(wl, parts)
    lam = box._f64(18, box.P)
    gN, gNb = box._f64(box.P), box._f64(box.P)
    dmom = box._f64(72, box.nz)
    with pytest.raises(E.EmuError) as ei:
        E.emu_adjoint_seed(box.box, dmom.data_ptr(), lam.data_ptr(), gN.data_ptr(), gNb.data_ptr())
    assert ei.value.code == E.EMU_EINVAL and "lattice" in str(ei.value)
    with pytest.raises(E.EmuError):
        box.set_step_form(1)
    with pytest.raises(E.EmuError):
        box.set_layout(2)
    box.set_layout(0)                 # the lattice path on scattered particles: reported
    with pytest.raises(E.EmuError) as ei:
        box.step(1, 1e-13)
        box.sync()
    assert ei.value.code == E.EMU_ELATTICE


def test_anywhere_paper_shape_full_size(torch):
    """The benchmark's scattered workload at full size: the paper's 1024 x 378
    run shape (387,072 particles), every position moved by U(-0.45, 0.45)
    cells and every direction replaced (the same draws as the benchmark):
    deposit, moments and H at 1e-12, then each of 10 steps at 1e-10 against
    the oracle."""
    wl = W.paper_1d()
    cfg, parts = _scatter(wl, seed=0)
    box = _box(wl, parts)
    assert box.general()
    grid = O.deposit(cfg, parts)
    A = box.deposit(0, 0.0).cpu().numpy()
    Aref = oracle_potential(grid, wl.kappa)
    s = wl.kappa * density_scales(grid)[2]
    assert max(family_err(A[9 * f:9 * (f + 1)], Aref[9 * f:9 * (f + 1)], s) for f in range(4)) < 1e-12
    assert max(_moment_errs(box, grid)) < 1e-12
    H = box.interpolate_H(0.0).cpu().numpy()
    assert family_err(H, pack(O.hamiltonian(cfg, grid, parts)), s) < 1e-12
    dt = O.timestep(cfg, grid)
    assert abs(box.timestep() - dt) <= 1e-13 * dt
    for n in range(10):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
        h = box.get_host()
        errs = [family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"]))]
        assert max(errs) < 1e-10, (n, errs)
        assert np.abs(h["z"] - parts["z"]).max() <= 1e-13 * wl.Lz
    box.sync()
