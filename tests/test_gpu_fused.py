"""The fused step: all phases of an RK4 step (lattice shifts, and per stage the
deposit of Eq. 5, its combination, and the RK stage with Eq. 6, Eq. 2 and
Eq. 4) in one persistent cooperative launch with grid barriers between them.

It must give bitwise the results of the separate launches with the same grid
(same arithmetic, same summation order), match the oracle, and report a grid
barrier that gives up (a host-chosen wait limit of 0) as EMU_ETIMEOUT, after
which the box steps normally again."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import family_err, pack

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


def _box(wl, blocks, rk_form, step_form, osc=None):
    from paper_2101_02745_gb300.emu import Box
    box = Box.from_workload(wl)
    if osc is not None:
        box.set_oscillation(osc)
    box.set_grid(blocks)
    box.set_rk_form(rk_form)
    box.set_step_form(step_form)
    return box


def _steps(wl, blocks, rk_form, step_form, steps, osc=None, dt_scale=1.0):
    box = _box(wl, blocks, rk_form, step_form, osc)
    dt = dt_scale * box.timestep()
    box.step(steps, dt)
    h = box.get_host()
    box.sync()
    return h, box


# (cells, directions): ragged tiles, fewer units than warps (one unit per
# busy warp), rings shorter than the stencil, long rings of few directions
CASES = [(67, 30), (31, 4), (2, 40), (256, 96), (1000, 3)]


@pytest.mark.parametrize("order", [0, 1, 2, 3])
@pytest.mark.parametrize("nz,M", CASES)
def test_fused_equals_separate_launches(torch, order, nz, M):
    wl = W.with_shape(W.random_box(nz, M, seed=nz + M), order)
    for blocks in (304, 152):
        for rk_form in (0, 1):
            ref, _ = _steps(wl, blocks, rk_form, 0, 4, dt_scale=0.917)
            got, box = _steps(wl, blocks, rk_form, 1, 4, dt_scale=0.917)
            for k in ("rho", "rhobar", "z"):
                assert np.array_equal(got[k], ref[k]), (blocks, rk_form, k)


@pytest.mark.parametrize("order", [2, 3])
def test_fused_with_vacuum_and_matter_equals_separate(torch, order):
    wl = W.with_shape(W.random_box(67, 30, seed=5), order)
    for rk_form in (0, 1):
        ref, _ = _steps(wl, 304, rk_form, 0, 6, osc=OSC)
        got, _ = _steps(wl, 304, rk_form, 1, 6, osc=OSC)
        for k in ("rho", "rhobar", "z"):
            assert np.array_equal(got[k], ref[k]), (rk_form, k)


def test_fused_matches_oracle_50_steps(torch):
    """The 32 x 16 fiducial box, every one of the first 50 steps at 1e-10."""
    wl = W.tiny_fiducial()
    box = _box(wl, 304, -1, 1)
    cfg = O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    for _ in range(50):
        box.step(1, dt)
        O.run(cfg, parts, dt, 1)
        h = box.get_host()
        assert family_err(h["rho"], pack(parts["rho"])) < 1e-10
        assert family_err(h["rhobar"], pack(parts["rhobar"])) < 1e-10
        assert np.abs(h["z"] - parts["z"]).max() < 1e-13 * wl.Lz
    box.sync()


def test_fused_batch_equals_separate(torch):
    from paper_2101_02745_gb300.emu import Box
    wls = W.sweep(7, seed=4, nz_range=(20, 97), ndir_range=(3, 41))
    out = []
    for form in (0, 1):
        box = Box.from_workloads(wls)
        box.set_step_form(form)
        box.batch_timestep()
        box.batch_step(5)
        out.append(box.get_host())
        box.sync()
    for k in ("rho", "rhobar", "z"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_fused_one_launch_per_step_and_graph_equals_eager(torch):
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(96, 24, seed=9)
    a = _box(wl, 304, -1, 1)
    b = _box(wl, 304, -1, 1)
    dt = a.timestep()
    b.timestep()
    n0 = a.launches()
    a.step(6, dt)                      # graph replay
    assert a.launches() - n0 == 6
    E.emu_profile(b.box, True)         # direct launches
    b.step(6, dt)
    t = E.emu_kernel_times(b.box)
    E.emu_profile(b.box, False)
    assert t["step"][1] == 6 and t["rk_stage"][1] == 0 and t["deposit"][1] == 0
    ha, hb = a.get_host(), b.get_host()
    for k in ("rho", "rhobar", "z"):
        assert np.array_equal(ha[k], hb[k]), k
    a.sync()
    b.sync()


def test_barrier_timeout_reports_and_recovers(torch):
    """A wait limit of 0 makes every barrier wait give up at once: the launch
    stops, the next synchronising call returns EMU_ETIMEOUT, no kernel is left
    waiting, and the box then steps exactly as the separate launches do."""
    from paper_2101_02745_gb300.emu import EMU_ETIMEOUT, EmuError
    wl = W.random_box(67, 30, seed=2)
    box = _box(wl, 304, -1, 1)
    dt = box.timestep()
    box.set_barrier_timeout(0)
    box.step(1, dt)
    with pytest.raises(EmuError) as ei:
        box.sync()
    assert ei.value.code == EMU_ETIMEOUT
    box.step(1, dt)                    # the limit is still 0: the next step gives up the same way
    with pytest.raises(EmuError) as ei:
        box.sync()
    assert ei.value.code == EMU_ETIMEOUT
    box.set_barrier_timeout(10 ** 9)
    box.init(wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.dirs, wl.alpha, wl.seed)
    box.step(3, dt)
    got = box.get_host()
    box.sync()
    ref, _ = _steps(wl, 304, -1, 0, 3)
    for k in ("rho", "rhobar", "z"):
        assert np.array_equal(got[k], ref[k]), k


def test_step_form_validation(torch):
    from paper_2101_02745_gb300.emu import EmuError
    box = _box(W.random_box(40, 8, seed=1), 304, -1, 0)
    for bad in (-1, 3):
        with pytest.raises(EmuError):
            box.set_step_form(bad)
    with pytest.raises(EmuError):
        box.set_barrier_timeout(-1)
    box.set_grid(608)                  # two waves of blocks: cannot all be resident
    with pytest.raises(EmuError):
        box.set_step_form(1)
    box.set_grid(304)
    box.set_step_form(1)
    box.set_grid(608)                  # a grid too large for the fused form drops it
    box.step(1, box.timestep())
    box.sync()


def test_fused_equals_separate_on_the_paper_shape(torch):
    """The paper's 1024 x 378 run shape (387,072 particles), 3 steps: the fused
    step with the 32-cell and the halo-lane RK stage equals the separate
    launches of the same grid bitwise."""
    wl = W.paper_1d()
    for rk_form in (1, 0):
        ref, _ = _steps(wl, 304, rk_form, 0, 3)
        got, _ = _steps(wl, 304, rk_form, 1, 3)
        for k in ("rho", "rhobar", "z"):
            assert np.array_equal(got[k], ref[k]), (rk_form, k)
