"""Vacuum and matter terms of Eq. 2 on the GPU path: parity with the oracle
for a three-flavour box with every mixing parameter non-zero, and the
paper's closed-form tests (App. A.1 MSW, App. A.3 homogeneous two-beam)
run through the C ABI."""
import json
from pathlib import Path

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import family_err, pack

pytestmark = pytest.mark.gpu
GOLD = json.loads((Path(__file__).parent / "golden" / "paper_numbers.json").read_text())


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_02745_gb300 import build
    build.build()
    return torch


# vacuum term comparable to the self-interaction (low energy), all angles and the phase on, matter on
OSC3 = W.oscillation(mass_eV=(0.01, 0.02, 0.05), theta12=0.59, theta13=0.15, theta23=0.84, delta_cp=1.0,
                     energy_MeV=5e-5, rho_g_cm3=1e8, Ye=0.4)


def _cfg(wl, osc):
    return O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area, osc=osc)


def test_three_flavour_oscillation_parity(torch):
    from paper_2101_02745_gb300.emu import Box
    wl = W.random_box(43, 11, seed=31)
    box = Box.from_workload(wl)
    box.set_oscillation(OSC3)
    cfg = _cfg(wl, OSC3)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    assert abs(box.timestep() - dt) <= 1e-13 * dt
    Hv, Hm = O.vacuum_matter(cfg)
    assert 0.05 < np.abs(Hv).max() / (W.KAPPA * wl.n_nu.max()) < 1.0   # the vacuum term matters here
    for n in range(20):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
    h = box.get_host()
    assert family_err(h["rho"], pack(parts["rho"])) < 1e-10
    assert family_err(h["rhobar"], pack(parts["rhobar"])) < 1e-10
    # removing the terms restores the plain path
    box.set_oscillation(None)
    box.step(1, dt)
    O.rk4_step(O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light), parts, dt)
    assert family_err(box.get_host()["rho"], pack(parts["rho"])) < 1e-10
    box.sync()


def test_msw_on_gpu(torch):
    from paper_2101_02745_gb300.emu import Box
    g = GOLD["msw_max_error"]
    wl, osc = W.msw_test()
    box = Box.from_workload(wl)
    box.set_oscillation(osc)
    D = -(osc["mass_eV"][0] * W.ERG_PER_EV) ** 2 / (2 * osc["energy_erg"]) / W.HBAR_ERG_S
    V = W.KAPPA * osc["n_e"]
    th = osc["theta12"]

    def pee(t, v):
        w = np.sqrt((v - D * np.cos(2 * th)) ** 2 + (D * np.sin(2 * th)) ** 2)
        return 1 - (D * np.sin(2 * th) / w) ** 2 * np.sin(w * t / 2) ** 2

    dt, t, err = g["dt_s"], 0.0, 0.0
    while t * W.C_LIGHT < g["ct_cm"]:
        box.step(1, dt)
        t += dt
        h = box.get_host()
        err = max(err, np.abs(h["rho"][0] - pee(t, V)).max(), np.abs(h["rhobar"][0] - pee(t, -V)).max())
    assert err <= g["max_abs_error"], err
    box.sync()


def test_bipolar_on_gpu(torch):
    """App. A.2 through the ABI: the bipolar run agrees with the oracle to 1e-10
    through the first full conversion and its return (2.6 ms, 13000 steps)."""
    from paper_2101_02745_gb300.emu import Box
    wl, osc = W.bipolar()
    box = Box.from_workload(wl)
    box.set_oscillation(osc)
    cfg = _cfg(wl, osc)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, 0.0, 0, wl.dirs)
    dt, chunk, worst, lowest = 2e-7, 500, 0.0, 1.0
    for _ in range(26):
        box.step(chunk, dt)
        O.run(cfg, parts, dt, chunk)
        h = box.get_host()
        worst = max(worst, family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"])))
        lowest = min(lowest, h["rho"][0].min())
    assert worst < 1e-10, worst
    assert lowest < 0.2                     # the pendulum swung through (full conversion near 1.21 ms)
    box.sync()


def test_homogeneous_two_beam_on_gpu(torch):
    from paper_2101_02745_gb300.emu import Box
    g = GOLD["two_beam_homogeneous_growth"]
    wl, osc = W.homogeneous_two_beam()
    box = Box.from_workload(wl)
    box.set_oscillation(osc)
    dt, t, ts, amp = 2e-6, 0.0, [], []
    while t < g["fit_window_s"][1] + dt / 2:
        box.step(1, dt)
        t += dt
        if t >= g["fit_window_s"][0] - dt:
            h = box.get_host()
            ts.append(t)
            amp.append(np.hypot(h["rho"][3, 0], h["rho"][4, 0]))
    ts, amp = np.array(ts), np.array(amp)
    sel = (ts >= g["fit_window_s"][0]) & (ts <= g["fit_window_s"][1])
    slope = np.polyfit(ts[sel], np.log(amp[sel]), 1)[0]
    assert abs(slope / wl.meta["growth"] - 1) <= g["relative_error_reported"], slope
    box.sync()


def test_batch_with_and_without_potentials(torch):
    from paper_2101_02745_gb300.emu import Box
    wls = W.sweep(4, seed=13, nz_range=(20, 70), ndir_range=(4, 19))
    box = Box.from_workloads(wls)
    box.set_oscillation(OSC3, box=1)
    box.set_oscillation(OSC3, box=3)
    dts = box.batch_timestep()
    box.batch_step(8)
    h = box.get_host()
    off = 0
    for b, (w, dt) in enumerate(zip(wls, dts)):
        cfg = _cfg(w, OSC3 if b in (1, 3) else None)
        parts = O.init(cfg, w.n_nu, w.n_nubar, w.f_nu, w.f_nubar, w.alpha, w.seed)
        dref = O.timestep(cfg, O.deposit(cfg, parts))
        assert abs(dt - dref) <= 1e-13 * dref
        O.run(cfg, parts, dt, 8)
        assert family_err(h["rho"][:, off:off + w.P], pack(parts["rho"])) < 1e-10
        assert family_err(h["rhobar"][:, off:off + w.P], pack(parts["rhobar"])) < 1e-10
        off += w.P
    box.sync()
