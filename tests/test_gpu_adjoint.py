"""Parity of the hand-written adjoint (emu_adjoint_seed / emu_adjoint_step /
emu_weight_gradient behind paper_2101_02745_gb300.adjoint.Evolve) against
central finite differences of the GPU forward path and the oracle's
reference gradient (oracle/gradient.py).

Objectives: final <n_ee> and log <|n_emu|> (Eq. 10); parameters: the species
inputs of Eq. 8; the time step is held fixed.  Bar: 1e-5 relative (row norm)."""
import json
import time
from pathlib import Path

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gradient as og  # noqa: E402
from paper_2101_02745_gb300 import workloads as W  # noqa: E402
from paper_2101_02745_gb300.adjoint import Evolve, Simulation, objectives  # noqa: E402
from paper_2101_02745_gb300.emu import Box, EmuError  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).resolve().parent / "golden"
TOL = 1e-5


def _theta(wl):
    return np.concatenate([[wl.n_nu[0], wl.n_nubar[0]], wl.f_nu[0], wl.f_nubar[0]])


def _fields(t, nz):
    """Uniform per-cell fields from the 8 scalars (differentiable)."""
    return t[0].expand(nz), t[1].expand(nz), t[2:5].expand(nz, 3), t[5:8].expand(nz, 3)


def adjoint_gradient(sim, theta):
    """(values (2,), gradient (2, 8)) of the two objectives by the adjoint."""
    nz = sim.box.nz
    g = np.zeros((2, 8))
    vals = None
    for k in range(2):
        t = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
        L = objectives(Evolve.apply(*_fields(t, nz), sim))
        L[k].backward()
        g[k] = t.grad.cpu().numpy()
        vals = L.detach().cpu().numpy()
    return vals, g


def forward_values(sim, theta):
    nz = sim.box.nz
    with torch.no_grad():
        t = torch.tensor(theta, dtype=torch.float64, device="cuda")
        return objectives(Evolve.apply(*_fields(t, nz), sim)).cpu().numpy()


def fd_gradient(sim, theta, h=1e-6):
    s = h * max(abs(theta[0]), abs(theta[1]))
    g = np.zeros((2, 8))
    for i in range(8):
        e = np.zeros(8); e[i] = s
        g[:, i] = (forward_values(sim, theta + e) - forward_values(sim, theta - e)) / (2 * s)
    return g


def rel_rows(a, b):
    """Per objective: ||a - b|| / ||b|| over its gradient row, and, so that a
    component much smaller than the row's largest cannot hide inside the norm,
    the worst component error relative to that component's own size (floored
    at 1e-3 of the row norm: |a_i - b_i| / (|b_i| + 1e-3 ||b||)).  The larger
    of the two is compared with the 1e-5 bar."""
    out = []
    for k in range(2):
        nb = np.linalg.norm(b[k])
        row = np.linalg.norm(a[k] - b[k]) / nb
        comp = np.max(np.abs(a[k] - b[k]) / (np.abs(b[k]) + 1e-3 * nb))
        out.append(float(max(row, comp)))
    return out


def _kw(wl):
    return dict(nz=wl.nz, ndir=wl.ndir, Lz=wl.Lz, kappa=wl.kappa, c_light=wl.c_light)


def test_small_box_vs_finite_differences_and_oracle():
    wl = W.adjoint_box(nz=32, ndir=16, steps=60)
    box = Box.from_workload(wl, init=False)
    sim = Simulation(box, wl.steps, 3.4e-12, every=7, alpha=wl.alpha, seed=wl.seed)
    th = _theta(wl)
    vals, g = adjoint_gradient(sim, th)
    g_fd = fd_gradient(sim, th)
    g_or = og.fd_gradient(_kw(wl), th, wl.alpha, wl.seed, 3.4e-12, wl.steps)
    v_or = og.evaluate(_kw(wl), th, wl.alpha, wl.seed, 3.4e-12, wl.steps)
    assert np.allclose(vals, v_or, rtol=1e-12, atol=0)
    assert max(rel_rows(g, g_fd)) < TOL, (g, g_fd)
    assert max(rel_rows(g, g_or)) < TOL, (g, g_or)


def test_per_cell_gradient_directional_derivative():
    """Per-cell species (random densities, 3D fluxes): <grad, v> equals the
    central difference of the objective along a random direction v."""
    wl = W.random_box(40, 12, seed=5)
    wl.alpha = 1e-8
    box = Box.from_workload(wl, init=False)
    sim = Simulation(box, 25, 8.0e-13, every=6, alpha=wl.alpha, seed=wl.seed)
    base = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar)]
    rng = np.random.Generator(np.random.PCG64(9))
    v = [torch.tensor(rng.normal(size=a.shape) * 1e31, dtype=torch.float64, device="cuda") for a in base]
    for k in range(2):
        leaves = [a.clone().requires_grad_(True) for a in base]
        L = objectives(Evolve.apply(*leaves, sim))[k]
        L.backward()
        dirderiv = sum(float((l.grad * vi).sum()) for l, vi in zip(leaves, v))
        eps = 1e-6 * 1e33 / 1e31
        with torch.no_grad():
            lp = objectives(Evolve.apply(*[a + eps * vi for a, vi in zip(base, v)], sim))[k]
            lm = objectives(Evolve.apply(*[a - eps * vi for a, vi in zip(base, v)], sim))[k]
        fd = float(lp - lm) / (2 * eps)
        assert abs(dirderiv - fd) <= TOL * abs(fd), (k, dirderiv, fd)


def test_with_vacuum_and_matter_terms():
    """POT kernels: the constant H_vac + H_mat enters the transposed commutators."""
    wl = W.adjoint_box(nz=32, ndir=16, steps=40)
    osc = W.oscillation(mass_eV=(0.0, 8.6e-3, 5.0e-2), theta12=0.59, theta13=0.15, theta23=0.84, delta_cp=1.2,
                        energy_MeV=5e-5, rho_g_cm3=1e9, Ye=0.4)
    box = Box.from_workload(wl, init=False)
    box.set_oscillation(osc)
    sim = Simulation(box, wl.steps, 3.0e-12, every=9, alpha=1e-10, seed=wl.seed)
    th = _theta(wl)
    _, g = adjoint_gradient(sim, th)
    g_fd = fd_gradient(sim, th)
    kw = _kw(wl); kw["osc"] = osc
    g_or = og.fd_gradient(kw, th, 1e-10, wl.seed, 3.0e-12, wl.steps)
    assert max(rel_rows(g, g_fd)) < TOL, (g, g_fd)
    assert max(rel_rows(g, g_or)) < TOL, (g, g_or)


def test_checkpoint_interval_does_not_change_the_gradient():
    wl = W.adjoint_box(nz=32, ndir=16, steps=24)
    box = Box.from_workload(wl, init=False)
    th = _theta(wl)
    ref = None
    for every in (1, 5, 24, 100):
        _, g = adjoint_gradient(Simulation(box, wl.steps, 3.4e-12, every=every, alpha=wl.alpha, seed=wl.seed), th)
        if ref is None:
            ref = g
        assert np.array_equal(g, ref), every


def test_zero_steps_seed_only():
    """nsteps = 0: the gradient is the seed's direct term through Eq. 8 alone."""
    wl = W.adjoint_box(nz=30, ndir=8, steps=0)
    box = Box.from_workload(wl, init=False)
    sim = Simulation(box, 0, 3.4e-12, alpha=1e-6, seed=1)
    th = _theta(wl)
    _, g = adjoint_gradient(sim, th)
    g_or = og.fd_gradient(_kw(wl), th, 1e-6, 1, 3.4e-12, 0)
    assert max(rel_rows(g, g_or)) < TOL


def test_adjoint_box_full_size_vs_oracle_reference_gradient():
    """256 cells x 96 directions, 400 steps, checkpoints every 20 steps: the
    adjoint against the oracle's stored central-difference gradient and against
    central differences of the GPU forward path; backward cost reported."""
    ref = json.loads((GOLDEN / "adjoint_256x96.json").read_text())
    wl = W.adjoint_box()
    assert (wl.nz, wl.ndir, wl.steps) == (ref["config"]["nz"], ref["config"]["ndir"], ref["nsteps"])
    box = Box.from_workload(wl, init=False)
    sim = Simulation(box, wl.steps, ref["dt"], every=20, alpha=ref["alpha"], seed=ref["seed"])
    th = np.array(ref["theta"])
    nz = box.nz
    t = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = objectives(Evolve.apply(*_fields(t, nz), sim))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L[1].backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g1 = t.grad.cpu().numpy()
    vals, g = adjoint_gradient(sim, th)
    assert np.array_equal(g[1], g1)
    assert np.allclose(vals, ref["values"], rtol=1e-10, atol=0)
    g_ref = np.array(ref["gradient"])
    assert max(rel_rows(g, g_ref)) < TOL, (g, g_ref)
    g_fd = fd_gradient(sim, th)
    assert max(rel_rows(g, g_fd)) < TOL, (g, g_fd)
    print(f"\nadjoint {wl.name}: forward {1e3 * (t1 - t0):.1f} ms, backward {1e3 * (t2 - t1):.1f} ms "
          f"({(t2 - t1) / (t1 - t0):.2f}x), rel err vs oracle {rel_rows(g, g_ref)}, vs GPU FD {rel_rows(g, g_fd)}")


def test_batch_adjoint_matches_single_boxes():
    """One backward pass over a batch of two uneven boxes (different sizes,
    step sizes, per-cell species) gives each box the gradient its own
    single-box run gives (the boxes are independent; summation orders differ)."""
    wl1 = W.adjoint_box(nz=32, ndir=16, steps=18)
    wl2 = W.random_box(41, 10, seed=3)
    wl2.alpha = 1e-8
    wls, dts = [wl1, wl2], [3.4e-12, 1.1e-12]
    ins = [[torch.tensor(a, dtype=torch.float64, device="cuda") for a in (w.n_nu, w.n_nubar, w.f_nu, w.f_nubar)]
           for w in wls]

    def run(box, sim, parts, slices):
        leaves = [p.clone().requires_grad_(True) for p in parts]
        mom = Evolve.apply(*leaves, sim)
        L = sum(objectives(mom[:, sl])[1] for sl in slices)
        L.backward()
        return [l.grad.cpu().numpy() for l in leaves]

    batch = Box.from_workloads(wls, init=False)
    simb = Simulation(batch, 18, dts, every=5, alpha=[w.alpha for w in wls], seed=[w.seed for w in wls])
    cat = [torch.cat([ins[0][i], ins[1][i]]) for i in range(4)]
    gb = run(batch, simb, cat, [slice(0, 32), slice(32, 73)])
    off = 0
    for w, dt, parts in zip(wls, dts, ins):
        box = Box.from_workload(w, init=False)
        g = run(box, Simulation(box, 18, dt, every=5, alpha=w.alpha, seed=w.seed), parts, [slice(0, w.nz)])
        for a, b in zip(gb, g):
            part = a[off:off + w.nz]
            assert np.abs(part - b).max() <= 1e-9 * np.abs(b).max(), (w.name, np.abs(part - b).max(), np.abs(b).max())
        off += w.nz


def test_adjoint_bad_calls():
    from paper_2101_02745_gb300 import emu as E

    wl = W.adjoint_box(nz=32, ndir=4, steps=1)
    box = Box.from_workload(wl)
    P = box.P
    lam = box._f64(18, P); gN = box._f64(P); gNb = box._f64(P)
    n = E.emu_adjoint_workspace_bytes(box.cfg)
    assert n == 8 * (90 * P + 3 * (3 * P + 32 * box.nz))   # quadratic shape: 3 kept weights, 32-row potentials
    ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
    p = (ws.data_ptr() + 255) & ~255
    with pytest.raises(EmuError):
        E.emu_adjoint_step(box.box, 3e-12, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), p, n - 8)
    with pytest.raises(EmuError):
        E.emu_adjoint_step(box.box, -1.0, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), p, n)
    with pytest.raises(EmuError):
        E.emu_adjoint_step(box.box, 3e-12, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), p + 8, n)
    box.rk_stage(1, 3e-12)   # a step in progress
    with pytest.raises(EmuError):
        E.emu_adjoint_step(box.box, 3e-12, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), p, n)
    with pytest.raises(EmuError):
        box.adjoint_seed(box._f64(72, box.nz), lam, gN, gNb)
    for s in (2, 3, 4):
        box.rk_stage(s, 3e-12)
    E.emu_adjoint_step(box.box, 3e-12, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), p, n)
    box.sync()
    batch = Box.from_workloads([wl, wl])
    blam = batch._f64(18, batch.P)
    with pytest.raises(EmuError):     # a batch takes dt = 0 (its boxes' own step sizes)
        batch.adjoint_step(3e-12, blam, batch._f64(batch.P), batch._f64(batch.P))


def _grads(sim, parts):
    leaves = [p.clone().requires_grad_(True) for p in parts]
    mom = Evolve.apply(*leaves, sim)
    objectives(mom)[1].backward()
    return [l.grad.cpu().numpy() for l in leaves]


@pytest.mark.parametrize("case", ["quadratic", "cubic_osc", "ngp", "batch", "batch_osc_linear"])
def test_recorded_adjoint_equals_recomputed(case):
    """The recorded backward (each step's stage states, weights and potentials
    kept from one forward pass) runs the same kernels on the same data as the
    recomputing one: the gradients agree bit for bit."""
    if case.startswith("batch"):
        order = 1 if case == "batch_osc_linear" else 2
        wl2 = W.with_shape(W.random_box(41, 10, seed=3), order)
        wl2.alpha = 1e-8
        wls, dts = [W.with_shape(W.adjoint_box(nz=32, ndir=16, steps=13), order), wl2], [3.4e-12, 1.1e-12]
        box = Box.from_workloads(wls, init=False)
        if case == "batch_osc_linear":   # vacuum and matter terms on the second box only
            box.set_oscillation(W.oscillation(mass_eV=(0.0, 8.6e-3, 5.0e-2), theta12=0.59, theta13=0.15,
                                              theta23=0.84, delta_cp=1.2, energy_MeV=5e-5, rho_g_cm3=1e9, Ye=0.4),
                                box=1)
        mk = lambda rec: Simulation(box, 13, dts, every=5, alpha=[w.alpha for w in wls],
                                    seed=[w.seed for w in wls], record=rec)
        parts = [torch.cat([torch.tensor(getattr(w, a), dtype=torch.float64, device="cuda") for w in wls])
                 for a in ("n_nu", "n_nubar", "f_nu", "f_nubar")]
    else:
        order = {"quadratic": 2, "cubic_osc": 3, "ngp": 0}[case]
        wl = W.with_shape(W.adjoint_box(nz=33, ndir=16, steps=17), order)
        box = Box.from_workload(wl, init=False)
        if case == "cubic_osc":
            box.set_oscillation(W.oscillation(mass_eV=(0.0, 8.6e-3, 5.0e-2), theta12=0.59, theta13=0.15,
                                              theta23=0.84, delta_cp=1.2, energy_MeV=5e-5, rho_g_cm3=1e9, Ye=0.4))
        mk = lambda rec: Simulation(box, wl.steps, 3.1e-12, every=6, alpha=wl.alpha, seed=wl.seed, record=rec)
        parts = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (wl.n_nu, wl.n_nubar, wl.f_nu,
                                                                              wl.f_nubar)]
    ga = _grads(mk(False), parts)
    gb = _grads(mk(True), parts)
    for a, b in zip(ga, gb):
        assert np.array_equal(a, b), np.abs(a - b).max()


def test_recorded_adjoint_cost_large_box():
    """1024 cells x 1000 directions (above the recording threshold), 24 steps
    in segments of 8: the recorded backward matches the recomputing one bit for
    bit and runs in less time (best of two passes each); the forward/backward
    costs are reported."""
    wl = W.adjoint_box(nz=1024, ndir=1000, steps=24)
    box = Box.from_workload(wl, init=False)
    parts = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar)]
    times, grads = {}, {}
    for rec in (False, True, False, True):
        sim = Simulation(box, wl.steps, 3.4e-12, every=8, alpha=wl.alpha, seed=wl.seed, record=rec)
        leaves = [p.clone().requires_grad_(True) for p in parts]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = objectives(Evolve.apply(*leaves, sim))[1]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        prev = times.get(rec)
        times[rec] = (t1 - t0, t2 - t1) if prev is None else (min(prev[0], t1 - t0), min(prev[1], t2 - t1))
        grads[rec] = [l.grad.cpu().numpy() for l in leaves]
    assert Simulation(box, wl.steps, 3.4e-12, every=8).use_record()
    for a, b in zip(grads[False], grads[True]):
        assert np.array_equal(a, b)
    (f0, b0), (f1, b1) = times[False], times[True]
    print(f"\nadjoint 1024x1000, 24 steps: forward {1e3 * f0:.1f} ms, backward recomputing {1e3 * b0:.1f} ms "
          f"({b0 / f0:.2f}x), recorded {1e3 * b1:.1f} ms ({b1 / f1:.2f}x)")
    assert b1 < b0


def test_record_bad_calls():
    from paper_2101_02745_gb300 import emu as E

    wl = W.adjoint_box(nz=32, ndir=4, steps=1)
    box = Box.from_workload(wl)
    P = box.P
    n = E.emu_batch_adjoint_record_bytes([box.cfg])
    assert n == 8 * (54 * P + 4 * (3 * P + 32 * box.nz))
    raw, base, stride = box.record_buffer(1)
    with pytest.raises(EmuError):
        E.emu_adjoint_record_step(box.box, 3e-12, base, n - 8)
    with pytest.raises(EmuError):
        E.emu_adjoint_record_step(box.box, 3e-12, base + 8, n)
    with pytest.raises(EmuError):
        E.emu_adjoint_record_step(box.box, 0.0, base, n)   # no step size set on the box
    lam = box._f64(18, P); gN = box._f64(P); gNb = box._f64(P)
    ptr, m = box._adjoint_ws()
    box.rk_stage(1, 3e-12)   # a step in progress
    with pytest.raises(EmuError):
        E.emu_adjoint_record_step(box.box, 3e-12, base, n)
    with pytest.raises(EmuError):
        E.emu_adjoint_step_recorded(box.box, 3e-12, base, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), ptr, m)
    for s in (2, 3, 4):
        box.rk_stage(s, 3e-12)
    with pytest.raises(EmuError):     # workspace below 54 doubles per particle
        E.emu_adjoint_step_recorded(box.box, 3e-12, base, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), ptr,
                                    8 * 54 * P - 8)
    E.emu_adjoint_record_step(box.box, 3e-12, base, n)
    E.emu_adjoint_step_recorded(box.box, 3e-12, base, lam.data_ptr(), gN.data_ptr(), gNb.data_ptr(), ptr, m)
    box.sync()


def test_recorded_adjoint_graph_cache_eviction():
    """One segment of 140 recorded steps needs 280 step graphs, more than the
    256 a box keeps: the oldest are dropped and recaptured, and the gradient
    still equals the recomputing backward's bit for bit (twice, so the second
    pass replays the cache the first one left)."""
    wl = W.adjoint_box(nz=16, ndir=8, steps=140)
    box = Box.from_workload(wl, init=False)
    parts = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar)]
    mk = lambda rec: Simulation(box, wl.steps, 3.4e-12, every=140, alpha=wl.alpha, seed=wl.seed, record=rec)
    ref = _grads(mk(False), parts)
    for _ in range(2):
        got = _grads(mk(True), parts)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), np.abs(a - b).max()
