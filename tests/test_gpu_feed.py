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
