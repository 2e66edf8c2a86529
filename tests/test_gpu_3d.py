"""The particle step on a 3D periodic grid through the C ABI (emu3_create and the
shared calls), against the 3D oracle (emu_oracle3d.c).

Both sides start from their own initialisation of the same seeded inputs.
Tolerances as in 1D: one deposit, moments or interpolation 1e-12 (family-wise,
against the density scale of the summands); every one of the first steps
1e-10; initial positions and random draws bitwise, weights and directions to
a few ulp.  Boxes cover ragged z tiles, one-cell and two-cell axes (the
stencil wraps onto the same cells), every shape order, and the vacuum and
matter terms."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import density_scales, family_err, moment_families, oracle_moments, oracle_potential, pack

pytestmark = pytest.mark.gpu

OSC = W.oscillation(mass_eV=(0.01, 0.02, 0.05), theta12=0.59, theta13=0.15, theta23=0.84, delta_cp=1.0,
                    energy_MeV=5e-5, rho_g_cm3=1e8, Ye=0.4)


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_02745_gb300 import build
    build.build()
    return torch


def _cfg(wl, osc=None):
    return O.config3(wl.nx, wl.ny, wl.nz, wl.ndir, wl.Lx, wl.Ly, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv,
                     wl.cfl_flavor, osc=osc, shape_order=wl.shape_order)


def _oracle(wl, osc=None):
    cfg = _cfg(wl, osc)
    return cfg, O.init3(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)


def _box(wl, osc=None):
    from paper_2101_02745_gb300.emu import Box3D
    box = Box3D.from_workload(wl)
    if osc is not None:
        box.set_oscillation(osc)
    return box


def _potential_err(A, grid, kappa):
    Aref = oracle_potential(grid, kappa)
    s = kappa * density_scales(grid)[2]
    return max(family_err(A[9 * f:9 * (f + 1)], Aref[9 * f:9 * (f + 1)], s) for f in range(4))


def _moment_errs(box, grid):
    got = box.moments().cpu().numpy()
    ref = oracle_moments(grid)
    sn, snb, _ = density_scales(grid)
    scales = [sn] * 4 + [snb] * 4
    return [family_err(g, r, s) for g, r, s in zip(moment_families(got), moment_families(ref), scales)]


# (nx, ny, nz, ndir, order): ragged z tiles (33, 31), a one-cell axis (the
# stencil's three cells are the same cell), two-cell axes, tiny z rows
BOXES = [(4, 3, 33, 5, 2), (1, 1, 29, 7, 2), (5, 1, 7, 6, 2), (2, 2, 31, 4, 2), (3, 4, 5, 6, 0), (3, 4, 5, 6, 1),
         (4, 3, 9, 5, 3), (6, 5, 2, 4, 2)]


def _wl(case, seed=0):
    nx, ny, nz, M, order = case
    return W.random_box3(nx, ny, nz, M, seed=seed + nx + 7 * ny + 31 * nz, shape_order=order)


@pytest.mark.parametrize("case", BOXES, ids=lambda c: "x".join(map(str, c)))
def test_init_parity_3d(torch, case):
    wl = _wl(case)
    box = _box(wl)
    h = box.get_host()
    box.sync()
    _, parts = _oracle(wl)
    for i, k in enumerate(("x", "y", "z")):
        assert np.array_equal(h[k], parts["x"][:, i]), k
    for i, k in enumerate(("ox", "oy", "oz")):
        assert np.abs(h[k] - parts["omega"][:, i]).max() <= 4e-16
    for k in ("N", "Nbar"):
        assert np.all(np.abs(h[k] - parts[k]) <= 4e-16 * np.abs(parts[k]).max())
    assert np.array_equal(h["rho"], pack(parts["rho"]))
    assert np.array_equal(h["rhobar"], pack(parts["rhobar"]))


@pytest.mark.parametrize("case", BOXES, ids=lambda c: "x".join(map(str, c)))
def test_deposit_moments_interpolation_parity_3d(torch, case):
    wl = _wl(case, seed=1)
    box = _box(wl)
    cfg, parts = _oracle(wl)
    grid = O.deposit3(cfg, parts)
    A = box.deposit(0, 0.0).cpu().numpy()
    assert _potential_err(A, grid, wl.kappa) < 1e-12
    assert max(_moment_errs(box, grid)) < 1e-12
    H = box.interpolate_H(0.0).cpu().numpy()
    Href = pack(O.hamiltonian3(cfg, grid, parts))
    assert family_err(H, Href, wl.kappa * density_scales(grid)[2]) < 1e-12
    box.sync()


def test_timestep_parity_3d(torch):
    wl = _wl((4, 3, 33, 5, 2), seed=3)
    box = _box(wl)
    cfg, parts = _oracle(wl)
    dt_ref = O.timestep3(cfg, O.deposit3(cfg, parts))
    assert abs(box.timestep() - dt_ref) <= 1e-13 * dt_ref
    box.sync()


@pytest.mark.parametrize("case", [(4, 3, 33, 5, 2), (3, 4, 5, 6, 0), (3, 4, 5, 6, 1), (4, 3, 9, 5, 3),
                                  (1, 1, 29, 7, 2)], ids=lambda c: "x".join(map(str, c)))
def test_steps_parity_3d(torch, case):
    """Every one of the first 20 steps (order 0: 0.917 x Eq. 7, so no stage
    position sits exactly on a cell face, where that shape is discontinuous)."""
    wl = _wl(case, seed=2)
    box = _box(wl)
    cfg, parts = _oracle(wl)
    dt = O.timestep3(cfg, O.deposit3(cfg, parts)) * (0.917 if wl.shape_order == 0 else 1.0)
    for n in range(20):
        box.step(1, dt)
        O.rk4_step3(cfg, parts, dt)
        h = box.get_host()
        errs = [family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"]))]
        errs += _moment_errs(box, O.deposit3(cfg, parts))
        assert max(errs) < 1e-10, (n, errs)
        for i, k in enumerate(("x", "y", "z")):
            L = (wl.Lx, wl.Ly, wl.Lz)[i]
            assert np.abs(h[k] - parts["x"][:, i]).max() <= 1e-13 * L, (n, k)
    box.sync()


def test_stage_calls_equal_step_3d(torch):
    wl = _wl((4, 3, 33, 5, 2), seed=4)
    a, b = _box(wl), _box(wl)
    dt = a.timestep()
    b.timestep()
    a.step(2, dt)
    for _ in range(2):
        for s in (1, 2, 3, 4):
            b.rk_stage(s, dt)
    ha, hb = a.get_host(), b.get_host()
    for k in ("rho", "rhobar", "x", "y", "z"):
        assert np.array_equal(ha[k], hb[k]), k
    a.sync()
    b.sync()


def test_vacuum_and_matter_3d(torch):
    wl = _wl((4, 3, 13, 5, 2), seed=5)
    box = _box(wl, OSC)
    cfg, parts = _oracle(wl, OSC)
    dt = O.timestep3(cfg, O.deposit3(cfg, parts))
    assert abs(box.timestep() - dt) <= 1e-13 * dt
    for n in range(12):
        box.step(1, dt)
        O.rk4_step3(cfg, parts, dt)
    h = box.get_host()
    assert family_err(h["rho"], pack(parts["rho"])) < 1e-10
    assert family_err(h["rhobar"], pack(parts["rhobar"])) < 1e-10
    box.sync()


def test_invariants_and_determinism_3d(torch):
    """A 12 x 10 x 40 box of 8 directions (38,400 particles), 30 steps: the
    trace of every rho and the domain lepton matrix (Eq. 18) conserved to
    rounding; two runs bitwise equal."""
    wl = W.random_box3(12, 10, 40, 8, seed=9)
    wl.alpha = 1e-3
    runs = []
    for _ in range(2):
        box = _box(wl)
        d0 = box.diagnostics()
        box.step(30)
        d1 = box.diagnostics()
        scale = np.abs(d0[36:45]).max() + np.abs(d0[45:54]).max()
        assert np.abs(d1[54:63] - d0[54:63]).max() < 1e-12 * scale
        h = box.get_host()
        for k in ("rho", "rhobar"):
            assert np.abs(h[k][0] + h[k][1] + h[k][2] - 1.0).max() < 1e-12
        runs.append(h)
        box.sync()
    for k in ("rho", "rhobar", "x", "y", "z"):
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_lattice_violation_and_unsupported_calls_3d(torch):
    from paper_2101_02745_gb300 import emu as E
    wl = _wl((3, 4, 5, 6, 2), seed=6)
    box = _box(wl)
    h = box.get_host()
    x = h["x"].copy()
    x[7] += 0.7 * wl.Lx / wl.nx          # off its lattice site on the x axis
    E.emu3_set_positions(box.box, x.ctypes.data, None, 1)
    with pytest.raises(E.EmuError) as ei:
        box.step(1, 1e-13)
        box.sync()
    assert ei.value.code == E.EMU_ELATTICE
    lam = box._f64(18, box.P)
    gN, gNb = box._f64(box.P), box._f64(box.P)
    with pytest.raises(E.EmuError) as ei:
        E.emu_adjoint_step(box.box, 1e-13, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), 0, 0)
    assert ei.value.code == E.EMU_EINVAL and "3D" in str(ei.value)
    with pytest.raises(E.EmuError):
        box.set_step_form(1)
    with pytest.raises(E.EmuError):
        E.emu3_create(E.make_config3(0, 1, 1, 1, 1.0, 1.0, 1.0, wl.kappa, wl.c_light))


def test_box3d_full_size_sampled(torch):
    """The 3D benchmark box at full size (64^3 cells x 16 directions, 4.19M
    particles) in the launch configuration the benchmark times: the full
    deposit against the oracle, then each of the four RK stages on 2000
    sampled particles against the oracle's right-hand side (its deposit of the
    whole stage state, per-particle H and commutators) at the stage states of
    the classic tableau built from its own derivatives; then two full steps
    checked through the exact invariants."""
    wl = W.random_box3(64, 64, 64, 16, seed=0)
    box = _box(wl)
    cfg, parts = _oracle(wl)
    grid = O.deposit3(cfg, parts)
    A = box.deposit(0, 0.0).cpu().numpy()
    assert _potential_err(A, grid, wl.kappa) < 1e-12
    dt = O.timestep3(cfg, grid)
    del grid, A
    assert abs(box.timestep() - dt) <= 1e-13 * dt
    box.autotune(trial_steps=1)   # dry steps: the state is untouched
    P = len(parts)
    sample = np.sort(np.random.default_rng(1).choice(P, 2000, replace=False))
    cstage = (0.0, 0.5, 0.5, 1.0)
    bweight = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)
    L = np.array([wl.Lx, wl.Ly, wl.Lz])
    acc_r, acc_b = parts["rho"][sample].copy(), parts["rhobar"][sample].copy()
    ystage = parts.copy()
    for s in range(1, 5):
        dr, db, _ = O.rhs3(cfg, ystage)
        box.rk_stage(s, dt)
        acc_r = acc_r + bweight[s - 1] * dt * dr[sample]
        acc_b = acc_b + bweight[s - 1] * dt * db[sample]
        if s < 4:
            c = cstage[s]
            ystage["rho"] = parts["rho"] + c * dt * dr
            ystage["rhobar"] = parts["rhobar"] + c * dt * db
            xs = parts["x"] + c * dt * wl.c_light * parts["omega"]
            xs = xs - L * np.floor(xs / L)
            ystage["x"] = np.where(xs >= L, xs - L, xs)
            stage = box.t["stage"][:, sample].cpu().numpy()
            accv = box.t["acc"][:, sample].cpu().numpy()
            assert family_err(stage[:9], pack(ystage["rho"][sample])) < 1e-13, s
            assert family_err(stage[9:], pack(ystage["rhobar"][sample])) < 1e-13, s
            assert family_err(accv[:9], pack(acc_r)) < 1e-13, s
            assert family_err(accv[9:], pack(acc_b)) < 1e-13, s
        del dr, db
    h = box.get_host()
    assert family_err(h["rho"][:, sample], pack(acc_r)) < 1e-13
    assert family_err(h["rhobar"][:, sample], pack(acc_b)) < 1e-13
    xn = parts["x"][sample] + dt * wl.c_light * parts["omega"][sample]
    xn = xn - L * np.floor(xn / L)
    for i, k in enumerate(("x", "y", "z")):
        assert np.abs(h[k][sample] - xn[:, i]).max() <= 1e-13 * L[i], k
    del parts, ystage, h
    d0 = box.diagnostics()
    box.step(2, dt)
    d1 = box.diagnostics()
    scale = np.abs(d0[36:45]).max() + np.abs(d0[45:54]).max()
    assert np.abs(d1[54:63] - d0[54:63]).max() < 1e-12 * scale
    h = box.get_host()
    for k in ("rho", "rhobar"):
        assert np.abs(h[k][0] + h[k][1] + h[k][2] - 1.0).max() < 1e-12
    box.sync()
