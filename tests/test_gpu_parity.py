"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Both sides start from their own initialisation of the same seeded inputs and
run their own arithmetic; nothing computed on the GPU feeds the oracle.
Tolerances (readings of "1e-10 relative on every grid moment and particle
matrix": per element the requirement is ill-posed where a value is 0, such as
rho_mutau at the start, so it is read per family of matrices):
  - per family the error is max_item ||gpu - ref||_F over a scale: for rho and
    rhobar the max_item ||ref||_F; for the grid families n, f_i (nbar, fbar_i)
    the max over cells of ||n||_F (||nbar||_F); for A and H, which contain the
    cancelling difference n - nbar^*, kappa max_j (||n_j||_F + ||nbar_j||_F):
    a sum's rounding error scales with its summands, not with its result;
  - deposit, moments, interpolation of one state: 1e-12;
  - every step of the first 50 steps: 1e-10;
  - init: weights and directions to a few ulp, random draws bitwise.
"""
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


def _oracle_init(wl):
    return O.init(_cfg(wl), wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)


def _box(wl):
    from paper_2101_02745_gb300.emu import Box
    return Box.from_workload(wl)


def _state_errs(h, parts):
    return (family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"])))


def _moment_errs(box, cfg, parts):
    got = box.moments().cpu().numpy()
    grid = O.deposit(cfg, parts)
    ref = oracle_moments(grid)
    sn, snb, _ = density_scales(grid)
    scales = [sn] * 4 + [snb] * 4
    return [family_err(g, r, s) for g, r, s in zip(moment_families(got), moment_families(ref), scales)]


def _potential_err(A, grid, kappa):
    Aref = oracle_potential(grid, kappa)
    s = kappa * density_scales(grid)[2]
    return max(family_err(A[9 * f:9 * (f + 1)], Aref[9 * f:9 * (f + 1)], s) for f in range(4))


SMALL = [W.tiny_fiducial(), W.random_box(67, 37, seed=1), W.random_box(31, 9, seed=2), W.two_beam(nz=40)]


@pytest.mark.parametrize("wl", SMALL, ids=lambda w: w.name)
def test_init_parity(torch, wl):
    box = _box(wl)
    h = box.get_host()
    parts = _oracle_init(wl)
    assert np.array_equal(h["z"], parts["z"])
    for i, k in enumerate(("ox", "oy", "oz")):
        assert np.abs(h[k] - parts["omega"][:, i]).max() <= 4e-16
    for k in ("N", "Nbar"):
        ref = parts[k]
        assert np.all(np.abs(h[k] - ref) <= 4e-16 * np.abs(ref).max())
    if wl.dirs is not None:
        assert np.array_equal(h["N"], parts["N"]) and np.array_equal(h["Nbar"], parts["Nbar"])
    assert np.array_equal(h["rho"], pack(parts["rho"]))
    assert np.array_equal(h["rhobar"], pack(parts["rhobar"]))


@pytest.mark.parametrize("wl", SMALL, ids=lambda w: w.name)
def test_deposit_moments_interpolation_parity(torch, wl):
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    grid = O.deposit(cfg, parts)
    A = box.deposit(0, 0.0).cpu().numpy()
    assert _potential_err(A, grid, wl.kappa) < 1e-12
    assert max(_moment_errs(box, cfg, parts)) < 1e-12
    H = box.interpolate_H(0.0).cpu().numpy()
    Href = pack(O.hamiltonian(cfg, grid, parts))
    assert family_err(H, Href, wl.kappa * density_scales(grid)[2]) < 1e-12
    box.sync()


def test_timestep_parity(torch):
    wl = W.random_box(67, 37, seed=3)
    box = _box(wl)
    cfg = _cfg(wl)
    dt_ref = O.timestep(cfg, O.deposit(cfg, _oracle_init(wl)))
    assert abs(box.timestep() - dt_ref) <= 1e-13 * dt_ref


@pytest.mark.parametrize("wl", [W.tiny_fiducial(), W.random_box(67, 37, seed=1)], ids=lambda w: w.name)
def test_first_50_steps_parity(torch, wl):
    """Every one of the first 50 RK4 steps: rho, rhobar and all grid moments
    within 1e-10 of the oracle (family-wise relative)."""
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    worst = 0.0
    for n in range(50):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
        h = box.get_host()
        errs = list(_state_errs(h, parts)) + _moment_errs(box, cfg, parts)
        worst = max(worst, max(errs))
        assert max(errs) < 1e-10, (n, errs)
        assert np.abs(h["z"] - parts["z"]).max() <= 1e-13 * wl.Lz
    box.sync()
    print(f"{wl.name}: worst family error over 50 steps {worst:.2e}")


@pytest.mark.parametrize("nz,ndir", [(1, 3), (2, 5), (3, 1), (29, 17), (30, 8), (31, 9), (61, 40), (90, 2)])
def test_edge_and_ragged_sizes(torch, nz, ndir):
    wl = W.random_box(nz, ndir, seed=nz + ndir)
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    for _ in range(5):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
    h = box.get_host()
    assert max(_state_errs(h, parts)) < 1e-10
    assert max(_moment_errs(box, cfg, parts)) < 1e-10
    box.sync()


def test_stage_api_equals_step_and_is_deterministic(torch):
    wl = W.random_box(61, 23, seed=4)
    a, b, c = _box(wl), _box(wl), _box(wl)
    dt = a.timestep()
    for _ in range(7):
        a.step(1, dt)
        b.step(1, dt)
        for s in (1, 2, 3, 4):
            c.rk_stage(s, dt)
    ha, hb, hc = a.get_host(), b.get_host(), c.get_host()
    for k in ha:
        assert np.array_equal(ha[k], hb[k]), k       # run-to-run bitwise reproducible
        assert np.array_equal(ha[k], hc[k]), k       # stage calls == step
    assert np.array_equal(a.moments().cpu().numpy(), b.moments().cpu().numpy())


def test_timed_launch_path_equals_graph_replay(torch):
    """The benchmark times steps with per-kernel CUDA events, which launches the
    step kernels one by one (programmatic dependent launch, events between
    kernels) instead of replaying the captured graph: both give bitwise the
    same states, on the default grid and on the 32-cell RK form."""
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(200, 40, seed=12)
    for form in (-1, 1):
        a, b = _box(wl), _box(wl)
        for x in (a, b):
            x.set_rk_form(form)
        dt = a.timestep()
        E.emu_profile(b.box, True)
        a.step(6, dt)
        b.step(6, dt)
        times = E.emu_kernel_times(b.box)
        E.emu_profile(b.box, False)
        assert times["rk_stage"][1] == 24 and times["deposit"][1] == 24
        ha, hb = a.get_host(), b.get_host()
        for k in ha:
            assert np.array_equal(ha[k], hb[k]), (form, k)


def test_invariants_on_gpu(torch):
    wl = W.tiny_fiducial()
    box = _box(wl)
    d0 = box.diagnostics()
    E0 = d0[54:63]
    scale = np.abs(d0[36:45]).max() + np.abs(d0[45:54]).max()
    box.step(100)
    d1 = box.diagnostics()
    assert np.abs(d1[54:63] - E0).max() < 1e-12 * scale
    h = box.get_host()
    for k in ("rho", "rhobar"):
        assert np.abs(h[k][0] + h[k][1] + h[k][2] - 1.0).max() < 1e-12
    # the instability grew: <|n_emu|> (Eq. 10, row-major entry (0, 1))
    assert d1[1] > 1e3 * d0[1]
    box.sync()


@pytest.mark.parametrize("dep_form", [0, 1])
def test_unperturbed_state_stays_exactly_diagonal(torch, dep_form):
    """Degenerate case: no perturbation (alpha = 0).  Every rho starts as
    diag(1, 0, 0) exactly (Eq. 9 with eps_x = 0), every deposit of the
    off-diagonal components is a sum of exact zeros, so H stays diagonal,
    commutes with rho (Eq. 4) and nothing evolves: after 20 steps every
    density matrix is bitwise its initial value, while the positions move."""
    wl = W.random_box(67, 21, seed=11)
    wl.alpha = 0.0
    box = _box(wl)
    box.set_deposit_form(dep_form)
    h0 = box.get_host()
    assert np.all(h0["rho"][0] == 1.0) and not h0["rho"][1:].any() and not h0["rhobar"][1:].any()
    box.step(20, box.timestep())
    h = box.get_host()
    box.sync()
    for k in ("rho", "rhobar"):
        assert np.array_equal(h[k], h0[k]), k
    assert not np.array_equal(h["z"], h0["z"])


@pytest.mark.parametrize("order", [2, 0, 1, 3])
def test_diagnostics_match_oracle(torch, order):
    """The one-pass deposit of n, f_x, nbar, fbar_x behind the diagnostics, at
    every shape order (steps at 0.917 x Eq. 7: no order-0 stage position on a face)."""
    wl = W.with_shape(W.random_box(67, 37, seed=5), order)
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    dt = 0.917 * O.timestep(cfg, O.deposit(cfg, parts))
    box.step(10, dt)
    O.run(cfg, parts, dt, 10)
    d = box.diagnostics()
    g = O.deposit(cfg, parts)
    a, m = O.domain_averages(cfg, g)
    for blk in range(4):
        assert np.allclose(d[9 * blk:9 * (blk + 1)].reshape(3, 3), a[blk], rtol=1e-10, atol=1e-10 * a[blk].max())
    assert family_err(d[36:45, None], pack(m[0])[:, None]) < 1e-10
    assert family_err(d[45:54, None], pack(m[1])[:, None]) < 1e-10
    eln = pack(np.mean(g["n"] - np.conj(g["nbar"]), axis=0))
    assert family_err(d[54:63, None], eln[:, None]) < 1e-10


def test_lattice_violation_is_reported(torch):
    """With the lattice layout fixed (emu_set_layout 0), a particle off its
    site is reported; with the default (checked when particles are installed)
    the box takes the path for particles anywhere instead."""
    from paper_2101_02745_gb300.emu import EmuError, EMU_ELATTICE
    wl = W.random_box(31, 4, seed=6)
    box = _box(wl)
    box.set_layout(0)
    h = box.get_host()
    z = h["z"].copy()
    z[40] += 0.7 * wl.dz      # out of the cell its ring position assigns
    box.set_host(z=z)
    assert not box.general()
    box.step(1, 1e-13)
    with pytest.raises(EmuError) as ei:
        box.sync()
    assert ei.value.code == EMU_ELATTICE
    box.sync()  # the error word was cleared
    auto = _box(wl)
    auto.set_host(z=z)
    assert auto.general()
    auto.step(1, 1e-13)
    auto.sync()


def test_lattice_with_per_direction_offsets_and_ties(torch):
    """Each ring shifted by its own offset in [-1/2, 1/2) cells, several exactly
    at the cell boundary (a tie of the shape function), then stepped: same as
    the oracle, which places each particle by floor()."""
    wl = W.random_box(37, 11, seed=9)
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    u = np.linspace(-0.5, 0.45, wl.ndir)
    u[[0, 3, 7]] = -0.5
    z = parts["z"].reshape(wl.ndir, wl.nz) + u[:, None] * wl.dz
    z = np.where(z < 0, z + wl.Lz, z).reshape(-1)
    parts["z"] = z
    box.set_host(z=z)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    for _ in range(8):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
    h = box.get_host()
    assert max(_state_errs(h, parts)) < 1e-10
    assert max(_moment_errs(box, cfg, parts)) < 1e-10
    box.sync()


def test_nonfinite_state_is_reported(torch):
    from paper_2101_02745_gb300.emu import EmuError, EMU_ENUMERIC
    wl = W.random_box(31, 4, seed=7)
    box = _box(wl)
    h = box.get_host()
    r = h["rho"].copy()
    r[3, 17] = np.nan
    box.set_host(rho=r)
    box.step(1, 1e-13)
    with pytest.raises(EmuError) as ei:
        box.sync()
    assert ei.value.code == EMU_ENUMERIC


def test_bad_calls_are_rejected(torch):
    from paper_2101_02745_gb300.emu import EmuError, EMU_EINVAL
    box = _box(W.random_box(31, 4, seed=8))
    with pytest.raises(EmuError) as ei:
        box.rk_stage(2, 1e-13)
    assert ei.value.code == EMU_EINVAL
    box.rk_stage(1, 1e-13)
    with pytest.raises(EmuError):
        box.rk_stage(2, 2e-13)
    with pytest.raises(EmuError):
        box.step(1, 1e-13)          # a step is in progress
    for s in (2, 3, 4):
        box.rk_stage(s, 1e-13)
    wl = W.tiny_fiducial()
    with pytest.raises(EmuError):
        box2 = _box(wl)
        box2.init(wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar * 1.5)   # flux factor > 1/3
    box.sync()


# ------------------------------------------------------------ full sizes ---

def test_paper_1d_full_size_50_steps(torch):
    """The paper's 1D run shape (1024 cells x 378 directions, the tilted nubar
    flux): init and deposit, then every one of the first 50 RK4 steps against
    the oracle on all 387,072 particles, in the launch configuration the
    benchmark picks for this shape (autotuned): rho, rhobar and every grid
    moment within 1e-10 (family-wise relative), positions within 1e-13 Lz."""
    wl = W.paper_1d(asymmetric=True)
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    h = box.get_host()
    assert np.array_equal(h["rho"], pack(parts["rho"]))
    grid = O.deposit(cfg, parts)
    A = box.deposit(0, 0.0).cpu().numpy()
    assert _potential_err(A, grid, wl.kappa) < 1e-12
    dt = O.timestep(cfg, grid)
    box.timestep()
    box.autotune(trial_steps=1)
    worst = 0.0
    for n in range(50):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
        h = box.get_host()
        errs = list(_state_errs(h, parts)) + _moment_errs(box, cfg, parts)
        worst = max(worst, max(errs))
        assert max(errs) < 1e-10, (n, errs)
        assert np.abs(h["z"] - parts["z"]).max() <= 1e-13 * wl.Lz
    box.sync()
    print(f"{wl.name}: worst family error over 50 steps {worst:.2e}")


def test_throughput_full_size_sampled(torch):
    """The throughput workload at full size (16384 cells x 1000 directions,
    16.4M particles), in the launch configuration the benchmark times: the
    full deposit against the oracle, then each of the four RK stages on 2000
    sampled particles against the oracle.  Every stage's expected values come
    from the oracle alone: its right-hand side (deposit of the whole stage
    state, per-particle H and commutators) at the stage states of the classic
    tableau built from its own derivatives.  Then two full steps checked
    through the exact invariants."""
    wl = W.throughput_1d()
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    grid = O.deposit(cfg, parts)
    A = box.deposit(0, 0.0).cpu().numpy()
    assert _potential_err(A, grid, wl.kappa) < 1e-12
    dt = O.timestep(cfg, grid)
    del grid
    assert abs(box.timestep() - dt) <= 1e-13 * dt
    box.autotune(trial_steps=1)   # the benchmark's launch configuration (dry steps: state untouched)
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(wl.P, 2000, replace=False))
    cstage = (0.0, 0.5, 0.5, 1.0)
    bweight = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)
    y0r, y0b = parts["rho"][sample].copy(), parts["rhobar"][sample].copy()
    acc_r, acc_b = y0r.copy(), y0b.copy()
    ystage = parts.copy()
    step_z = parts["z"] + dt * wl.c_light * parts["omega"][:, 2]
    for s in range(1, 5):
        dr, db, _ = O.rhs(cfg, ystage)          # k_s at the stage state (the oracle's deposit and commutators)
        box.rk_stage(s, dt)
        acc_r = acc_r + bweight[s - 1] * dt * dr[sample]
        acc_b = acc_b + bweight[s - 1] * dt * db[sample]
        if s < 4:
            c = cstage[s]
            ystage["rho"] = parts["rho"] + c * dt * dr
            ystage["rhobar"] = parts["rhobar"] + c * dt * db
            zs = parts["z"] + c * dt * wl.c_light * parts["omega"][:, 2]
            zs = zs - wl.Lz * np.floor(zs / wl.Lz)
            ystage["z"] = np.where(zs >= wl.Lz, zs - wl.Lz, zs)
            stage = box.t["stage"][:, sample].cpu().numpy()
            accv = box.t["acc"][:, sample].cpu().numpy()
            assert family_err(stage[:9], pack(ystage["rho"][sample])) < 1e-13, s
            assert family_err(stage[9:], pack(ystage["rhobar"][sample])) < 1e-13, s
            assert family_err(accv[:9], pack(acc_r)) < 1e-13, s
            assert family_err(accv[9:], pack(acc_b)) < 1e-13, s
        del dr, db
    got_r = box.t["rho"][:, sample].cpu().numpy()
    got_b = box.t["rhobar"][:, sample].cpu().numpy()
    got_z = box.t["z"][sample].cpu().numpy()
    assert family_err(got_r, pack(acc_r)) < 1e-13
    assert family_err(got_b, pack(acc_b)) < 1e-13
    zn = step_z[sample] - wl.Lz * np.floor(step_z[sample] / wl.Lz)
    assert np.abs(got_z - zn).max() <= 1e-13 * wl.Lz
    del parts, ystage
    d0 = box.diagnostics()
    box.step(2, dt)
    d1 = box.diagnostics()
    scale = np.abs(d0[36:45]).max() + np.abs(d0[45:54]).max()
    assert np.abs(d1[54:63] - d0[54:63]).max() < 1e-12 * scale
    h = box.get_host()
    for k in ("rho", "rhobar"):
        assert np.abs(h[k][0] + h[k][1] + h[k][2] - 1.0).max() < 1e-12
    box.sync()


def test_post_saturation_abundances(torch):
    """Through saturation and kinematic decoherence: the flavour abundances
    a = <n_ee>/<Tr n> and abar = <nbar_ee>/<Tr nbar>, averaged over cells and over
    every step with t >= 3 ns (App. B, Eq. B1), agree with the oracle within 2e-2
    relative.  The trajectories are chaotic after saturation (Sec. 3.3), so only
    these statistics are compared.  Reduced box (the paper-shaped run is too long
    for the oracle): 128 cells x 48 directions over 32 cm, species of the tiny
    fiducial box, 1800 steps (6 ns)."""
    n, nb, nz, M = 4.9e32, 6.1e32, 128, 48
    wl = W.Workload("saturation_128x48", nz, M, 32.0, np.full(nz, n), np.full(nz, nb), np.zeros((nz, 3)),
                    np.tile([0.0, 0.0, -nb / 3.0], (nz, 1)), seed=0)
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    steps = 1800
    ga, gab, oa, oab = [], [], [], []
    for s in range(steps):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
        if (s + 1) * dt >= 3e-9:
            d = box.diagnostics()
            ga.append(d[36] / (d[36] + d[37] + d[38]))
            gab.append(d[45] / (d[45] + d[46] + d[47]))
            g = O.deposit(cfg, parts)
            m = g["n"].real.mean(axis=0)
            mb = g["nbar"].real.mean(axis=0)
            oa.append(m[0, 0] / np.trace(m))
            oab.append(mb[0, 0] / np.trace(mb))
    box.sync()
    a, ab, ra, rab = np.mean(ga), np.mean(gab), np.mean(oa), np.mean(oab)
    print(f"post-saturation <N_ee>/Tr: gpu {a:.4f} oracle {ra:.4f}; nubar gpu {ab:.4f} oracle {rab:.4f}")
    assert abs(a - ra) <= 2e-2 * ra
    assert abs(ab - rab) <= 2e-2 * rab
    assert a < 0.9 and ab < 0.9                  # flavour transformation happened
    # Eq. 18 on both sides: the same number of neutrinos and antineutrinos changed flavour
    assert abs(n * (1 - a) - nb * (1 - ab)) <= 1e-3 * n
