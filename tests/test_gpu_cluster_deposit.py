"""Deposit forms 1 and 2: the step's deposit (Eq. 5) by thread-block clusters
of 8 or 16 blocks.  Each cluster takes one tile at a time; its warps split the
tile's rings, their sums are added in warp order through shared memory and in
block-rank order through distributed shared memory, and the potential is
written in the same launch (no second, combining launch).

The summation order differs from the per-warp deposit's, so the forms match
form 0 to rounding (not bitwise) and the oracle at the usual tolerances
(every step 1e-10); the order depends only on the box and the cluster size,
so runs are bitwise reproducible.  Boxes cover ragged last tiles, rings
shorter than the stencil, fewer rings than a cluster has warps, every shape
order, the vacuum and matter terms and a batch of uneven boxes."""
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


def _box(wl, dep_form, osc=None):
    from paper_2101_02745_gb300.emu import Box
    box = Box.from_workload(wl)
    if osc is not None:
        box.set_oscillation(osc)
    box.set_deposit_form(dep_form)
    return box


def _dt_scale(order):
    # order 0: 0.917 x Eq. 7, so that no stage position sits on a cell face,
    # where that shape is discontinuous
    return 0.917 if order == 0 else 1.0


# (cells, directions, order): ragged last tiles, fewer rings than the 64 or
# 128 warps of a cluster (3, 9), rings of 1 and 2 cells, every shape order
CASES = [(67, 37, 2), (31, 9, 2), (1000, 3, 2), (2, 40, 2), (1, 20, 2), (31, 4, 0), (40, 6, 1), (45, 7, 3),
         (256, 96, 2)]


@pytest.mark.parametrize("dep_form", [1, 2])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_cluster_deposit_matches_oracle(torch, case, dep_form):
    """20 steps, every state against the oracle's at 1e-10 (positions 1e-13
    Lz), then the moments."""
    nz, M, order = case
    wl = W.with_shape(W.random_box(nz, M, seed=5 * nz + M), order)
    cfg = _cfg(wl)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    box = _box(wl, dep_form)
    dt = O.timestep(cfg, O.deposit(cfg, parts)) * _dt_scale(order)
    for n in range(20):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
        h = box.get_host()
        errs = [family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"]))]
        assert max(errs) < 1e-10, (n, errs)
        dz = np.abs(h["z"] - parts["z"])
        assert np.minimum(dz, wl.Lz - dz).max() <= 1e-13 * wl.Lz   # (periodic: 0 and Lz are one point)
    got = box.moments().cpu().numpy()
    grid = O.deposit(cfg, parts)
    ref = oracle_moments(grid)
    sn, snb, _ = density_scales(grid)
    assert max(family_err(g, r, s) for g, r, s in zip(moment_families(got), moment_families(ref),
                                                       [sn] * 4 + [snb] * 4)) < 1e-10
    box.sync()


def test_cluster_deposit_with_vacuum_and_matter(torch):
    wl = W.random_box(67, 30, seed=5)
    cfg = _cfg(wl, OSC)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    box = _box(wl, 1, osc=OSC)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    box.step(12, dt)
    O.run(cfg, parts, dt, 12)
    h = box.get_host()
    assert family_err(h["rho"], pack(parts["rho"])) < 1e-10
    assert family_err(h["rhobar"], pack(parts["rhobar"])) < 1e-10
    box.sync()


def test_cluster_deposit_paper_shape_agrees_and_is_reproducible(torch):
    """The paper's 1024 x 378 run shape, 10 steps: each cluster size twice
    (bitwise equal), against the per-warp deposit to 1e-13; positions equal."""
    wl = W.paper_1d()
    runs = {}
    for form, rep in ((0, 0), (1, 0), (1, 1), (2, 0), (2, 1)):
        box = _box(wl, form)
        box.set_rk_form(1)
        box.step(10, box.timestep())
        runs[(form, rep)] = box.get_host()
        box.sync()
    for form in (1, 2):
        for k in ("rho", "rhobar"):
            assert np.array_equal(runs[(form, 0)][k], runs[(form, 1)][k]), (form, k)
            assert family_err(runs[(form, 0)][k], runs[(0, 0)][k]) < 1e-13, (form, k)
        assert np.array_equal(runs[(form, 0)]["z"], runs[(0, 0)]["z"])


def test_cluster_deposit_batch(torch):
    """A batch of uneven boxes (clusters walk all boxes' tiles): every box
    against its own oracle run at 1e-10 after 10 steps."""
    from paper_2101_02745_gb300.emu import Box
    wls = [W.random_box(nz, M, seed=nz + M) for nz, M in ((40, 5), (23, 80), (129, 3), (3, 11), (64, 48))]
    box = Box.from_workloads(wls)
    box.set_deposit_form(1)
    dts = box.batch_timestep()
    box.batch_step(10)
    h = box.get_host()
    box.sync()
    p0 = 0
    for wl, dt in zip(wls, dts):
        cfg = _cfg(wl)
        parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
        assert abs(O.timestep(cfg, O.deposit(cfg, parts)) - dt) <= 1e-13 * dt
        O.run(cfg, parts, dt, 10)
        P = wl.P
        assert family_err(h["rho"][:, p0:p0 + P], pack(parts["rho"])) < 1e-10, wl.name
        assert family_err(h["rhobar"][:, p0:p0 + P], pack(parts["rhobar"])) < 1e-10, wl.name
        p0 += P


def test_cluster_deposit_stage_calls_and_launches(torch):
    """Stage calls equal the step bitwise; per step one shift table, 4
    deposits, 4 RK stages and no combination."""
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(96, 24, seed=9)
    a, b = _box(wl, 1), _box(wl, 1)
    dt = a.timestep()
    b.timestep()
    E.emu_profile(a.box, True)
    a.step(3, dt)
    t = E.emu_kernel_times(a.box)
    E.emu_profile(a.box, False)
    assert t["deposit"][1] == 12 and t["rk_stage"][1] == 12 and t["combine"][1] == 0 and t["shifts"][1] == 3
    for _ in range(3):
        for s in (1, 2, 3, 4):
            b.rk_stage(s, dt)
    ha, hb = a.get_host(), b.get_host()
    for k in ("rho", "rhobar", "z"):
        assert np.array_equal(ha[k], hb[k]), k
    a.sync()
    b.sync()


def test_cluster_deposit_refusals_and_autotune(torch):
    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300.emu import Box, Box3D
    box = Box.from_workload(W.random_box(256, 96, seed=4))
    for bad in (-1, 3):
        with pytest.raises(E.EmuError) as ei:
            box.set_deposit_form(bad)
        assert ei.value.code == E.EMU_EINVAL
    box.rk_stage(1, 1e-13)
    with pytest.raises(E.EmuError):
        box.set_deposit_form(1)        # a step is in progress
    for s in (2, 3, 4):
        box.rk_stage(s, 1e-13)
    choice, ms = box.autotune()
    assert len(ms) == E.AUTOTUNE_CANDIDATES == 17
    assert all(m > 0 for m in ms[13:])
    assert ms[choice] == min(m for m in ms if m > 0)
    box.step(2)
    box.sync()
    b3 = Box3D.from_workload(W.random_box3(4, 3, 33, 5, seed=1))
    with pytest.raises(E.EmuError) as ei:
        b3.set_deposit_form(1)
    assert ei.value.code == E.EMU_EINVAL
    choice, ms = b3.autotune()
    assert list(ms[13:]) == [-1.0] * 4 and choice < 13
    b3.sync()
