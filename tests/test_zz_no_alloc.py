"""The allocation-free deposit (emu_deposit_static) against the regular one.

Callers that cannot allocate device memory but may still enqueue stream work
(allocator-free sections of other libraries, code running while a memory
pool is resized) use emu_deposit_static, which keeps its scratch
in a static device array of the library.  This file is collected last so that
a stop at the first failure has already run every other test; it must pass
both alone in a fresh process and after the rest of the suite."""
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


def _scale(A):
    # the potential's natural scale: kappa times the densities it is summed from
    return np.abs(A).max()


def test_static_deposit_matches_workspace_deposit_twice(torch):
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(67, 37, seed=21)
    box = E.Box.from_workload(wl)
    dt = box.timestep()
    t = box.t
    ptrs = [t[k].data_ptr() for k in ("z", "ox", "oy", "oz", "N", "Nbar", "rho", "rhobar")]
    stream = box.stream.cuda_stream
    for pos_dt in (0.0, 0.5 * dt):
        ref = box.deposit(0, pos_dt).cpu().numpy()
        out = torch.full((36, wl.nz), np.nan, dtype=torch.float64, device=box.device)
        E.emu_deposit_static(box.cfg, *ptrs, pos_dt, out.data_ptr(), stream)
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * _scale(ref)
    box.sync()


def test_static_deposit_at_chunked_size_and_rejects_oversize(torch):
    from paper_2101_02745_gb300 import emu as E
    wl = W.paper_1d()          # 35 cell tiles x 18 direction chunks: uses the partial sums
    box = E.Box.from_workload(wl)
    t = box.t
    ptrs = [t[k].data_ptr() for k in ("z", "ox", "oy", "oz", "N", "Nbar", "rho", "rhobar")]
    ref = box.deposit(0, 0.0).cpu().numpy()
    out = torch.zeros((36, wl.nz), dtype=torch.float64, device=box.device)
    for _ in range(2):
        out.zero_()
        E.emu_deposit_static(box.cfg, *ptrs, 0.0, out.data_ptr(), box.stream.cuda_stream)
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * _scale(ref)
    big = E.make_config(1, 600000, 1.0, wl.kappa, wl.c_light)
    with pytest.raises(E.EmuError) as ei:
        E.emu_deposit_static(big, *ptrs, 0.0, out.data_ptr(), box.stream.cuda_stream)
    assert ei.value.code == E.EMU_EINVAL and "static array" in str(ei.value)
    box.sync()


def test_static_deposit_refuses_a_capturing_stream(torch):
    """Every call copies its error word to the host and synchronises, which a
    stream capture cannot hold: on a capturing stream the call returns
    EMU_EINVAL before any device work, and the capture stays valid."""
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(31, 5, seed=2)
    box = E.Box.from_workload(wl)
    t = box.t
    ptrs = [t[k].data_ptr() for k in ("z", "ox", "oy", "oz", "N", "Nbar", "rho", "rhobar")]
    out = torch.zeros((36, wl.nz), dtype=torch.float64, device=box.device)
    box.sync()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        graph.capture_begin()
        try:
            with pytest.raises(E.EmuError) as ei:
                E.emu_deposit_static(box.cfg, *ptrs, 0.0, out.data_ptr(), side.cuda_stream)
            out.add_(1.0)      # the capture still records work
        finally:
            graph.capture_end()
    assert ei.value.code == E.EMU_EINVAL and "captured" in str(ei.value)
    graph.replay()
    torch.cuda.synchronize()
    assert float(out.min()) == 1.0
    E.emu_deposit_static(box.cfg, *ptrs, 0.0, out.data_ptr(), box.stream.cuda_stream)
    assert np.abs(out.cpu().numpy() - box.deposit(0, 0.0).cpu().numpy()).max() <= 1e-12 * _scale(out.cpu().numpy())
    box.sync()
