"""Boxes bound to a caller's own CUDA stream (graphs captured and replayed on
that stream) give bitwise the results of boxes on the default stream: single
boxes, batches and the adjoint."""
import numpy as np
import pytest

from paper_2101_02745_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_02745_gb300 import build
    build.build()
    return torch


def _on_stream(wl, stream):
    from paper_2101_02745_gb300.emu import Box
    b = Box(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area, stream=stream,
            shape_order=wl.shape_order)
    b.init(wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.dirs, wl.alpha, wl.seed)
    return b


def test_single_box_on_user_stream(torch):
    from paper_2101_02745_gb300.emu import Box
    wl = W.random_box(53, 9, seed=11)
    ref = Box.from_workload(wl)
    dt = ref.timestep()
    ref.step(6, dt)
    box = _on_stream(wl, torch.cuda.Stream())
    assert box.timestep() == dt
    box.step(2, dt)
    box.step(4, dt)            # graph replays on the user stream
    hr, hb = ref.get_host(), box.get_host()
    for k in hr:
        assert np.array_equal(hr[k], hb[k]), k
    assert torch.equal(box.moments(), ref.moments())
    assert np.array_equal(box.diagnostics(), ref.diagnostics())
    box.sync()


def test_batch_on_user_stream(torch):
    from paper_2101_02745_gb300.emu import Box, make_config
    wls = W.sweep(3, seed=21, nz_range=(20, 70), ndir_range=(4, 12))
    ref = Box.from_workloads(wls)
    dts = ref.batch_timestep()
    ref.batch_step(5)
    cfgs = [make_config(w.nz, w.ndir, w.Lz, w.kappa, w.c_light, w.cfl_adv, w.cfl_flavor, w.area) for w in wls]
    box = Box(0, 0, 0, 0, 0, cfgs=cfgs, stream=torch.cuda.Stream())
    from paper_2101_02745_gb300 import emu as E
    E.emu_batch_init_particles(box.box, np.concatenate([w.n_nu for w in wls]),
                               np.concatenate([w.n_nubar for w in wls]),
                               np.concatenate([w.f_nu.reshape(-1) for w in wls]),
                               np.concatenate([w.f_nubar.reshape(-1) for w in wls]), None,
                               np.array([w.alpha for w in wls]), np.array([w.seed for w in wls], np.uint64))
    assert np.array_equal(box.batch_timestep(), dts)
    box.batch_step(5)
    hr, hb = ref.get_host(), box.get_host()
    for k in hr:
        assert np.array_equal(hr[k], hb[k]), k
    box.sync()


def test_adjoint_on_user_stream(torch):
    from paper_2101_02745_gb300.adjoint import Evolve, Simulation, objectives
    from paper_2101_02745_gb300.emu import Box
    wl = W.adjoint_box(nz=32, ndir=16, steps=12)
    grads = []
    for stream in (None, torch.cuda.Stream()):
        box = Box(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, stream=stream)
        sim = Simulation(box, 12, 3.4e-12, every=5, alpha=wl.alpha, seed=wl.seed)
        leaves = [torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True)
                  for a in (wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar)]
        objectives(Evolve.apply(*leaves, sim))[1].backward()
        grads.append([l.grad.cpu().numpy() for l in leaves])
    for a, b in zip(*grads):
        assert np.array_equal(a, b)
