"""The RK stage with 32 cells per warp (every shape order; the cubic shape
reaches two cells past a tile's ends).  It runs when every
warp of the grid walks at least 8 units; a one-block grid (8 warps) makes small
boxes take it.  Parity with the oracle for every order with and without the
vacuum and matter terms, ragged and tiny boxes, batches; agreement with the
halo-lane form of the stage."""
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


def _units32(nz, M):
    return (nz + 31) // 32 * M


def _run(wl, osc, steps, blocks):
    from paper_2101_02745_gb300.emu import Box
    box = Box.from_workload(wl)
    if osc is not None:
        box.set_oscillation(osc)
    box.set_grid(blocks)
    cfg = O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area, osc=osc,
                   shape_order=wl.shape_order)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    # 0.917 x Eq. 7: at Eq. 7's advective limit some directions move particles exactly
    # onto cell faces at stage positions, where the order-0 shape is discontinuous
    dt = 0.917 * O.timestep(cfg, O.deposit(cfg, parts))
    box.step(steps, dt)
    O.run(cfg, parts, dt, steps)
    return box, box.get_host(), parts


# (cells, directions): partial tiles (33 and 65: a last tile of one cell, shorter
# than the cubic stencil's reach), fewer cells than a tile, fewer cells than the
# stencil (1, 2), one cell, one full tile per ring (32), long rings of few
# directions (1000 x 2: warp ranges that start and end inside rings); at least
# 64 units
CASES = [(67, 30), (33, 40), (96, 30), (1, 70), (2, 70), (5, 70), (31, 64), (65, 32), (32, 64), (1000, 2)]


@pytest.mark.parametrize("order", [0, 1, 2, 3])
@pytest.mark.parametrize("nz,M", CASES)
def test_rk32_parity(torch, order, nz, M):
    assert _units32(nz, M) >= 64
    wl = W.with_shape(W.random_box(nz, M, seed=nz + M + order), order)
    box, h, parts = _run(wl, None, 12, 1)
    assert family_err(h["rho"], pack(parts["rho"])) < 1e-10
    assert family_err(h["rhobar"], pack(parts["rhobar"])) < 1e-10
    assert np.abs(h["z"] - parts["z"]).max() <= 1e-13 * wl.Lz
    box.sync()


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_rk32_with_vacuum_and_matter(torch, order):
    wl = W.with_shape(W.random_box(67, 30, seed=5), order)
    box, h, parts = _run(wl, OSC, 12, 1)
    assert family_err(h["rho"], pack(parts["rho"])) < 1e-10
    assert family_err(h["rhobar"], pack(parts["rhobar"])) < 1e-10
    box.sync()


@pytest.mark.parametrize("order", [2, 3])
def test_rk32_agrees_with_halo_form(torch, order):
    """The 32-cell form (one block: 90 units over 8 warps) and the halo-lane
    form (two blocks: fewer than 8 units per warp) of the same steps agree to
    rounding (their deposits sum the same terms in different warp orders)."""
    from paper_2101_02745_gb300.emu import Box
    wl = W.with_shape(W.random_box(67, 30, seed=9), order)
    a = Box.from_workload(wl)
    a.set_grid(1)
    b = Box.from_workload(wl)
    b.set_grid(2)
    dt = a.timestep()
    a.step(6, dt)
    b.step(6, dt)
    ha, hb = a.get_host(), b.get_host()
    assert family_err(ha["rho"], hb["rho"]) < 1e-13
    assert family_err(ha["rhobar"], hb["rhobar"]) < 1e-13
    assert np.array_equal(ha["z"], hb["z"])
    a.sync()
    b.sync()


def test_rk32_batch(torch):
    from paper_2101_02745_gb300.emu import Box
    wls = W.sweep(3, seed=31, nz_range=(20, 90), ndir_range=(20, 40))
    box = Box.from_workloads(wls)
    box.set_grid(1)
    dts = box.batch_timestep()
    box.batch_step(8)
    h = box.get_host()
    off = 0
    for w, dt in zip(wls, dts):
        cfg = O.config(w.nz, w.ndir, w.Lz, w.kappa, w.c_light, w.cfl_adv, w.cfl_flavor, w.area)
        parts = O.init(cfg, w.n_nu, w.n_nubar, w.f_nu, w.f_nubar, w.alpha, w.seed)
        O.run(cfg, parts, dt, 8)
        sl = slice(off, off + w.P)
        assert family_err(h["rho"][:, sl], pack(parts["rho"])) < 1e-10
        assert family_err(h["rhobar"][:, sl], pack(parts["rhobar"])) < 1e-10
        off += w.P
    box.sync()


def test_set_grid_validation(torch):
    from paper_2101_02745_gb300.emu import Box, EmuError
    box = Box.from_workload(W.random_box(20, 4, seed=1))
    for bad in (0, -1, 609):
        with pytest.raises(EmuError):
            box.set_grid(bad)
    box.set_grid(608)
    box.sync()


@pytest.mark.parametrize("order", [2, 3])
def test_rk32_with_few_units_per_warp(torch, order):
    """The 32-cell form forced on the default grid, where warps walk one unit or
    none (every tile end computed directly): parity with the oracle and bitwise
    the halo-lane form's results."""
    from paper_2101_02745_gb300.emu import Box
    wl = W.with_shape(W.random_box(67, 30, seed=13), order)
    out = []
    for form in (1, 0):
        box = Box.from_workload(wl)
        box.set_rk_form(form)
        dt = 0.917 * box.timestep()
        box.step(10, dt)
        out.append(box.get_host())
        box.sync()
    for k in ("rho", "rhobar", "z"):
        assert np.array_equal(out[0][k], out[1][k]), k
    cfg = O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area,
                   shape_order=order)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    O.run(cfg, parts, dt, 10)
    assert family_err(out[0]["rho"], pack(parts["rho"])) < 1e-10
    assert family_err(out[0]["rhobar"], pack(parts["rhobar"])) < 1e-10


def test_set_rk_form_validation(torch):
    from paper_2101_02745_gb300.emu import Box, EmuError
    box = Box.from_workload(W.random_box(20, 4, seed=1))
    for bad in (-2, 2):
        with pytest.raises(EmuError):
            box.set_rk_form(bad)
    box.set_rk_form(-1)
    box.sync()


def test_every_launch_configuration_agrees(torch):
    """The six configurations the autotuner chooses from (three grids, two RK
    stage forms): the two forms of one grid give bitwise the same steps; the
    grids differ only in the deposit's summation order (1e-13)."""
    from paper_2101_02745_gb300.emu import Box
    wl = W.random_box(200, 24, seed=21)
    out = {}
    for blocks in (304, 152, 608):
        for form in (0, 1):
            box = Box.from_workload(wl)
            box.set_grid(blocks)
            box.set_rk_form(form)
            dt = box.timestep()
            box.step(5, dt)
            out[blocks, form] = box.get_host()
            box.sync()
    ref = out[304, 0]
    for (blocks, form), h in out.items():
        other = out[blocks, 1 - form]
        for k in ("rho", "rhobar", "z"):
            assert np.array_equal(h[k], other[k]), (blocks, k)
        assert family_err(h["rho"], ref["rho"]) < 1e-13
        assert family_err(h["rhobar"], ref["rhobar"]) < 1e-13
