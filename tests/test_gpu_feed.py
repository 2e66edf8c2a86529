"""HostFeed (double-buffered host-to-device state feed) through the C ABI:
the state it installs equals the host arrays, and steps fed this way equal
steps after a plain host upload, bitwise."""
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


def test_feed_installs_host_state_and_steps_match(torch):
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(61, 9, seed=4)
    box = E.Box.from_workload(wl)
    dt = box.timestep()
    box.step(3, dt)
    host = box.get_host()
    pin = {k: torch.from_numpy(host[k].copy()).pin_memory() for k in ("z", "rho", "rhobar")}
    # reference: plain upload then two steps, diagnostics after each
    ref = E.Box.from_workload(wl)
    diags_ref = []
    for _ in range(2):
        ref.set_host(z=host["z"], rho=host["rho"], rhobar=host["rhobar"])
        ref.step(1, dt)
        diags_ref.append(ref.diagnostics())
    feed = E.HostFeed(box, pin)
    assert feed.h2d_bytes == 19 * 8 * box.P
    feed.prefetch()
    diags = []
    for _ in range(2):
        feed.load()
        got = box.get_host()
        for k in ("z", "rho", "rhobar"):
            assert np.array_equal(got[k], host[k])
        feed.prefetch()
        box.step(1, dt)
        diags.append(box.diagnostics())
    for a, b in zip(diags, diags_ref):
        assert np.array_equal(a, b)
    box.sync()


def test_ping_pong_feed_steps_match(torch):
    """Two boxes taking turns, each step's state copied from the host straight
    into the idle box: every step equals a plain upload and step, bitwise."""
    from paper_2101_02745_gb300 import emu as E
    wl = W.random_box(61, 9, seed=5)
    a, b = E.Box.from_workload(wl), E.Box.from_workload(wl)
    dt = a.timestep()
    a.step(2, dt)
    host = a.get_host()
    pin = {k: torch.from_numpy(host[k].copy()).pin_memory() for k in ("z", "rho", "rhobar")}
    ref = E.Box.from_workload(wl)
    ref.set_host(z=host["z"], rho=host["rho"], rhobar=host["rhobar"])
    ref.step(1, dt)
    want, want_h = ref.diagnostics(), ref.get_host()
    feed = E.PingPongFeed([a, b], pin)
    assert feed.h2d_bytes == 19 * 8 * a.P
    feed.prefetch(0)
    seen = []
    for _ in range(4):
        box = feed.next_box()
        E.emu_step(box.box, 1, dt)
        d = np.zeros(E.N_DIAG)
        E.emu_diagnostics(box.box, d.ctypes.data, 1)
        assert np.array_equal(d, want)
        h = box.get_host()
        for k in ("rho", "rhobar", "z"):
            assert np.array_equal(h[k], want_h[k]), k
        seen.append(box)
    assert seen[0] is seen[2] and seen[1] is seen[3] and seen[0] is not seen[1]
    a.sync()
    b.sync()
