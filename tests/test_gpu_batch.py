"""Batched independent boxes (the parameter-sweep pattern of Sec. 4): one set of
launches per step covers every box, replayed from a CUDA graph.

Every box of a batch must evolve as the oracle evolves it alone, and as the
single-box path evolves it; graph replay must equal direct launches bitwise;
the autotuner must leave the particle state untouched."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import pack, family_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_02745_gb300 import build
    build.build()
    return torch


def _small_sweep(nbox=9, seed=3):
    return W.sweep(nbox, seed=seed, nz_range=(20, 97), ndir_range=(3, 41))


def _cfg(wl):
    return O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area)


def _split(h, wls):
    """Per-box views of a batch's host state."""
    out, off = [], 0
    for w in wls:
        out.append({k: (v[..., off:off + w.P]) for k, v in h.items()})
        off += w.P
    return out


def test_batch_boxes_match_oracle(torch):
    from paper_2101_02745_gb300.emu import Box
    wls = _small_sweep()
    box = Box.from_workloads(wls)
    dts = box.batch_timestep()
    ref = []
    for w, dt in zip(wls, dts):
        cfg = _cfg(w)
        parts = O.init(cfg, w.n_nu, w.n_nubar, w.f_nu, w.f_nubar, w.alpha, w.seed)
        dref = O.timestep(cfg, O.deposit(cfg, parts))
        assert abs(dt - dref) <= 1e-13 * dref
        ref.append((cfg, parts))
    steps = 12
    box.batch_step(steps)
    for cfg, parts in ref:
        O.run(cfg, parts, O.timestep(cfg, O.deposit(cfg, parts)), steps)
    h = box.get_host()
    for (cfg, parts), hb in zip(ref, _split(h, wls)):
        assert family_err(hb["rho"], pack(parts["rho"])) < 1e-10
        assert family_err(hb["rhobar"], pack(parts["rhobar"])) < 1e-10
        assert np.abs(hb["z"] - parts["z"]).max() <= 1e-13 * cfg.Lz
    d = box.batch_diagnostics()
    for b, (cfg, parts) in enumerate(ref):
        a, m = O.domain_averages(cfg, O.deposit(cfg, parts))
        assert np.allclose(d[b, :9].reshape(3, 3), a[0], rtol=1e-9, atol=1e-9 * a[0].max())
    box.sync()


def test_batch_equals_single_boxes_and_graph_equals_eager(torch):
    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300.emu import Box
    wls = _small_sweep(nbox=6, seed=5)
    g = Box.from_workloads(wls)       # graph replay
    e = Box.from_workloads(wls)       # direct launches (timing on forces them)
    dts = g.batch_timestep()
    e.batch_set_dt(dts)
    E.emu_profile(e.box, True)
    g.batch_step(7)
    e.batch_step(7)
    E.emu_kernel_times(e.box)
    hg, he = g.get_host(), e.get_host()
    for k in hg:
        assert np.array_equal(hg[k], he[k]), k
    singles = []
    for w, dt in zip(wls, dts):
        s = Box.from_workload(w)
        s.step(7, dt)
        singles.append(s.get_host())
    for hb, hs in zip(_split(hg, wls), singles):
        assert family_err(hb["rho"], hs["rho"]) < 1e-12
        assert family_err(hb["rhobar"], hs["rhobar"]) < 1e-12
        assert np.abs(hb["z"] - hs["z"]).max() == 0.0
    g.sync()


def test_autotune_leaves_state_and_keeps_parity(torch):
    from paper_2101_02745_gb300.emu import Box
    wls = _small_sweep(nbox=5, seed=7)
    box = Box.from_workloads(wls)
    h0 = box.get_host()
    choice, ms = box.autotune(trial_steps=2)
    assert 0 <= choice < len(ms) and ms[choice] > 0 and np.all((ms > 0) | (ms == -1.0))
    h1 = box.get_host()
    for k in h0:
        assert np.array_equal(h0[k], h1[k]), k
    box.batch_step(5)
    h = box.get_host()
    for w, hb in zip(wls, _split(h, wls)):
        cfg = _cfg(w)
        parts = O.init(cfg, w.n_nu, w.n_nubar, w.f_nu, w.f_nubar, w.alpha, w.seed)
        O.run(cfg, parts, O.timestep(cfg, O.deposit(cfg, parts)), 5)
        assert family_err(hb["rho"], pack(parts["rho"])) < 1e-10
    box.sync()


def test_batch_invariants_each_box(torch):
    from paper_2101_02745_gb300.emu import Box
    wls = _small_sweep(nbox=8, seed=11)
    box = Box.from_workloads(wls)
    d0 = box.batch_diagnostics()
    box.batch_step(40)
    d1 = box.batch_diagnostics()
    for b in range(len(wls)):
        scale = np.abs(d0[b, 36:45]).max() + np.abs(d0[b, 45:54]).max()
        assert np.abs(d1[b, 54:63] - d0[b, 54:63]).max() < 1e-12 * scale
    box.sync()


def test_full_sweep_sampled_boxes(torch):
    """The benchmark's sweep at full size (256 boxes, 31.7M particles) in its
    launch configuration (autotuned grid, graph replay): two steps of the whole
    batch, then the smallest, the largest and two other boxes against the
    oracle run of each box alone."""
    from paper_2101_02745_gb300.emu import Box
    wls = W.sweep(256, seed=0)
    box = Box.from_workloads(wls)
    dts = box.batch_timestep()
    box.autotune(trial_steps=1)
    box.batch_step(2)
    sizes = [w.P for w in wls]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 200})
    offs = np.concatenate([[0], np.cumsum(sizes)])
    P = offs[-1]
    for b in picks:
        w = wls[b]
        cfg = _cfg(w)
        parts = O.init(cfg, w.n_nu, w.n_nubar, w.f_nu, w.f_nubar, w.alpha, w.seed)
        assert abs(dts[b] / O.timestep(cfg, O.deposit(cfg, parts)) - 1) < 1e-14
        O.run(cfg, parts, dts[b], 2)
        # this box's slice of the batch state (device to host, this box only)
        sl = slice(int(offs[b]), int(offs[b + 1]))
        rho = box.t["rho"][:, sl].cpu().numpy()
        rhob = box.t["rhobar"][:, sl].cpu().numpy()
        z = box.t["z"][sl].cpu().numpy()
        assert family_err(rho, pack(parts["rho"])) < 1e-10, w.name
        assert family_err(rhob, pack(parts["rhobar"])) < 1e-10, w.name
        assert np.abs(z - parts["z"]).max() <= 1e-13 * w.Lz
    assert P == box.P
    box.sync()
