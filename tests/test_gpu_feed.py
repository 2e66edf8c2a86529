"""PingPongFeed: per-step particle state from pinned host memory through the
host-buffer path of the C ABI (emu_set_particles, on_host = 1, or 2 for the
asynchronous copy), two boxes taking turns: every step equals a plain upload
and step, bitwise."""
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


@pytest.mark.parametrize("asynchronous", [False, True])
def test_ping_pong_feed_steps_match(torch, asynchronous):
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(61, 9, seed=5)
    a = E.Box.from_workload(wl, stream=torch.cuda.Stream())
    b = E.Box.from_workload(wl, stream=torch.cuda.Stream())
    dt = a.timestep()
    a.step(2, dt)
    host = a.get_host()
    pin = {k: torch.from_numpy(host[k].copy()).pin_memory() for k in ("z", "rho", "rhobar")}
    ref = E.Box.from_workload(wl)
    ref.set_host(z=host["z"], rho=host["rho"], rhobar=host["rhobar"])
    ref.step(1, dt)
    want, want_h = ref.diagnostics(), ref.get_host()
    if asynchronous:   # the uploads keep the lattice: no check (and no synchronisation) per upload
        a.set_layout(0)
        b.set_layout(0)
    feed = E.PingPongFeed([a, b], pin, asynchronous=asynchronous)
    assert feed.h2d_bytes == 19 * 8 * a.P
    feed.prime()
    seen = []
    for _ in range(4):
        d = np.zeros(E.N_DIAG)
        box = feed.step(lambda bx: E.emu_step(bx.box, 1, dt))
        E.emu_diagnostics(box.box, d.ctypes.data, 1)
        assert np.array_equal(d, want)
        h = box.get_host()
        for k in ("rho", "rhobar", "z"):
            assert np.array_equal(h[k], want_h[k]), k
        seen.append(box)
    assert seen[0] is seen[2] and seen[1] is seen[3] and seen[0] is not seen[1]
    a.sync()
    b.sync()


def test_ping_pong_feed_needs_two_streams(torch):
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(20, 3, seed=1)
    a, b = E.Box.from_workload(wl), E.Box.from_workload(wl)
    with pytest.raises(ValueError):
        E.PingPongFeed([a, b], {k: np.zeros(1) for k in ("z", "rho", "rhobar")})


def test_set_particles_rejects_unknown_copy_mode(torch):
    from paper_2101_02745_gb300 import emu as E
    box = E.Box.from_workload(W.random_box(20, 3, seed=2))
    z = np.zeros(box.P)
    with pytest.raises(E.EmuError) as ei:
        E.emu_set_particles(box.box, z.ctypes.data, None, None, None, None, None, None, None, 3)
    assert ei.value.code == E.EMU_EINVAL
    box.sync()
