"""Step form 2: every RK stage also deposits (Eq. 5) the state it has just
computed at the next stage's positions (stage 4: the next step's first), so a
step is four (combination, RK stage) launch pairs; the first step of a call
deposits its state first.  The warps sum their deposits per 32-cell tile over
a frame of 36 cells, k_frame_sum adds the warps' frames of each tile, and the
next RK stage adds the frame entries that cover each cell.

The summation order differs from the separate deposit's, so the form matches
the other forms to rounding (not bitwise), and the oracle at the usual
tolerances (every step 1e-10); for a fixed grid it is bitwise reproducible.
Boxes cover ragged last tiles of 1 to 31 cells (so that a tile two tiles away
reaches a cell across the periodic end), rings of one and two cells, shape
orders 0-2 and the vacuum and matter terms.  Step sizes with dt c >= 1.9 dz
run form 0 instead (bitwise form 0's results); the cubic shape is refused."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import density_scales, family_err, moment_families, oracle_moments, pack

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
    return O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area, osc=osc,
                    shape_order=wl.shape_order)


def _box(wl, step_form, blocks=304, osc=None):
    from paper_2101_02745_gb300.emu import Box
    box = Box.from_workload(wl)
    if osc is not None:
        box.set_oscillation(osc)
    box.set_grid(blocks)
    box.set_step_form(step_form)
    return box


def _dt_scale(order):
    # order 0: 0.917 x Eq. 7, so that no stage position sits on a cell face,
    # where that shape is discontinuous
    return 0.917 if order == 0 else 1.0


# (cells, directions, order): ragged last tiles of 3, 4, 1 and 1 cells (65:
# three tiles; 97: four, so a cell of tile 2 receives from tile 0 across the
# periodic end), rings of 1, 2 and 5 cells, full tiles
CASES = [(32, 16, 2), (67, 37, 2), (100, 9, 2), (65, 5, 2), (97, 3, 2), (31, 4, 0), (31, 4, 1), (2, 30, 2),
         (1, 20, 2), (5, 7, 1), (256, 24, 2)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_rk_deposit_matches_oracle(torch, case):
    """One call of 30 steps (the deposits carried from stage to stage and
    from step to step inside the call), then single-step calls: every state
    against the oracle's at 1e-10, positions at 1e-13 Lz."""
    nz, M, order = case
    wl = W.with_shape(W.random_box(nz, M, seed=7 * nz + M), order)
    cfg = _cfg(wl)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    box = _box(wl, 2)
    dt = O.timestep(cfg, O.deposit(cfg, parts)) * _dt_scale(order)
    box.step(30, dt)
    O.run(cfg, parts, dt, 30)
    for n in range(6):
        h = box.get_host()
        errs = [family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"]))]
        assert max(errs) < 1e-10, (n, errs)
        dz = np.abs(h["z"] - parts["z"])
        assert np.minimum(dz, wl.Lz - dz).max() <= 1e-13 * wl.Lz   # (periodic: 0 and Lz are one point)
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
    got = box.moments().cpu().numpy()
    grid = O.deposit(cfg, parts)
    ref = oracle_moments(grid)
    sn, snb, _ = density_scales(grid)
    assert max(family_err(g, r, s) for g, r, s in zip(moment_families(got), moment_families(ref),
                                                       [sn] * 4 + [snb] * 4)) < 1e-10
    box.sync()


@pytest.mark.parametrize("order", [0, 1, 2])
def test_rk_deposit_agrees_with_separate_launches(torch, order):
    """A batch of uneven boxes, 20 steps in one call: form 2 against form 0
    (other deposit summation order) to 1e-13; two runs of form 2 bitwise."""
    from paper_2101_02745_gb300.emu import Box
    wls = [W.with_shape(W.random_box(nz, M, seed=nz + M), order) for nz, M in ((40, 5), (23, 8), (129, 3), (3, 11))]
    runs = {}
    for form, rep in ((0, 0), (2, 0), (2, 1)):
        box = Box.from_workloads(wls)
        box.set_grid(152)
        box.set_step_form(form)
        dts = box.batch_timestep()
        box.batch_set_dt([d * _dt_scale(order) for d in dts])
        box.batch_step(20)
        runs[(form, rep)] = box.get_host()
        box.sync()
    for k in ("rho", "rhobar"):
        assert family_err(runs[(2, 0)][k], runs[(0, 0)][k]) < 1e-13, k
        assert np.array_equal(runs[(2, 0)][k], runs[(2, 1)][k]), k
    assert np.array_equal(runs[(2, 0)]["z"], runs[(0, 0)]["z"])


def test_rk_deposit_with_vacuum_and_matter(torch):
    wl = W.random_box(67, 30, seed=5)
    cfg = _cfg(wl, OSC)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    box = _box(wl, 2, osc=OSC)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    assert abs(box.timestep() - dt) <= 1e-13 * dt
    box.step(12, dt)
    O.run(cfg, parts, dt, 12)
    h = box.get_host()
    assert family_err(h["rho"], pack(parts["rho"])) < 1e-10
    assert family_err(h["rhobar"], pack(parts["rhobar"])) < 1e-10
    box.sync()


@pytest.mark.parametrize("blocks", [152, 304, 608])
def test_rk_deposit_grids(torch, blocks):
    """Every grid of the autotuner: the paper's direction count on a short
    box, 10 steps, against form 0 to 1e-13."""
    wl = W.random_box(96, 378, seed=3)
    a, b = _box(wl, 0, blocks), _box(wl, 2, blocks)
    dt = a.timestep()
    a.step(10, dt)
    b.step(10, dt)
    ha, hb = a.get_host(), b.get_host()
    for k in ("rho", "rhobar"):
        assert family_err(hb[k], ha[k]) < 1e-13, k
    assert np.array_equal(ha["z"], hb["z"])
    a.sync()
    b.sync()


def test_rk_deposit_large_step_runs_form_0(torch):
    """dt c >= 1.9 dz: a ring could move two cells between stages, so the
    steps run form 0, bitwise its results."""
    wl = W.random_box(40, 6, seed=9)
    a, b = _box(wl, 0), _box(wl, 2)
    dt = 2.0 * wl.dz / wl.c_light
    a.step(3, dt)
    b.step(3, dt)
    ha, hb = a.get_host(), b.get_host()
    for k in ("rho", "rhobar", "z"):
        assert np.array_equal(ha[k], hb[k]), k
    # and back below the limit: form 2 again (agrees to rounding)
    dt2 = 0.5 * wl.dz / wl.c_light
    a.step(3, dt2)
    b.step(3, dt2)
    ha, hb = a.get_host(), b.get_host()
    for k in ("rho", "rhobar"):
        assert family_err(hb[k], ha[k]) < 1e-13, k
    a.sync()
    b.sync()


def test_rk_deposit_kernel_classes(torch):
    """Per-kernel timing: a call of n steps launches 4 n RK-deposit kernels,
    4 n combinations, n shift tables and one first deposit."""
    from paper_2101_02745_gb300 import emu as E
    box = _box(W.random_box(64, 12, seed=2), 2)
    dt = box.timestep()
    E.emu_profile(box.box, True)
    box.step(3, dt)
    t = E.emu_kernel_times(box.box)
    E.emu_profile(box.box, False)
    box.sync()
    assert t["rk_deposit"][1] == 12 and t["combine"][1] == 12 and t["shifts"][1] == 3 and t["deposit"][1] == 1
    assert t["rk_stage"][1] == 0


def test_rk_deposit_refusals_and_autotune(torch):
    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300.emu import Box
    cubic = Box.from_workload(W.with_shape(W.random_box(40, 6, seed=1), 3))
    with pytest.raises(E.EmuError) as ei:
        cubic.set_step_form(2)
    assert ei.value.code == E.EMU_EINVAL
    choice, ms = cubic.autotune()
    assert list(ms[10:13]) == [-1.0, -1.0, -1.0] and not 10 <= choice < 13
    cubic.sync()
    box = Box.from_workload(W.random_box(256, 96, seed=4))
    choice, ms = box.autotune()
    assert len(ms) == E.AUTOTUNE_CANDIDATES == 17
    assert all(m > 0 for m in ms[10:])
    assert ms[choice] == min(m for m in ms if m > 0)
    box.step(5)
    box.sync()
