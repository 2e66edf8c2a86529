"""Shape orders 0, 1 and 3 (Sec. 2.2.1: from the delta function to the cubic
B-spline; the quadratic order 2 is covered by test_gpu_parity.py): parity of
the CUDA path with the oracle run at the same order, through the C ABI.

Bars as for the quadratic shape: deposit, moments and interpolation of one
state 1e-12 (family-wise, density-scaled), every one of the first 50 steps
1e-10."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_02745_gb300 import workloads as W
from tests.compare import density_scales, family_err, moment_families, oracle_moments, oracle_potential, pack

pytestmark = pytest.mark.gpu
ORDERS = [0, 1, 3]


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_02745_gb300 import build
    build.build()
    return torch


def _cfg(wl):
    return O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area,
                    shape_order=wl.shape_order)


def _oracle_init(wl):
    return O.init(_cfg(wl), wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)


def _box(wl):
    from paper_2101_02745_gb300.emu import Box
    return Box.from_workload(wl)


def _moment_errs(box, cfg, parts):
    got = box.moments().cpu().numpy()
    grid = O.deposit(cfg, parts)
    ref = oracle_moments(grid)
    sn, snb, _ = density_scales(grid)
    scales = [sn] * 4 + [snb] * 4
    return [family_err(g, r, s) for g, r, s in zip(moment_families(got), moment_families(ref), scales)]


def _advect(wl, parts, frac_dt):
    """Oracle particles moved by frac_dt * c * Omega_z (off the cell centres)."""
    q = parts.copy()
    cfg = _cfg(wl)
    for i in range(len(q)):
        q["z"][i] = O.wrap(cfg, q["z"][i] + frac_dt * wl.c_light * q["omega"][i][2])
    return q


# ragged sizes: several tiles with a partial last one, fewer cells than the stencil, one cell
SIZES = [(67, 11), (29, 5), (3, 4), (1, 3)]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("nz,ndir", SIZES)
def test_deposit_moments_interpolation(torch, order, nz, ndir):
    wl = W.with_shape(W.random_box(nz, ndir, seed=nz + order), order)
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    assert max(_moment_errs(box, cfg, parts)) < 1e-12
    # off the cell centres: deposit and interpolate at positions z + pos_dt c Omega_z
    pos_dt = 0.37 * wl.dz / wl.c_light
    A = box.deposit(0, pos_dt).cpu().numpy()
    moved = _advect(wl, parts, pos_dt)
    grid = O.deposit(cfg, moved)
    s = wl.kappa * density_scales(grid)[2]
    Aref = oracle_potential(grid, wl.kappa)
    for f in range(4):
        assert family_err(A[9 * f:9 * (f + 1)], Aref[9 * f:9 * (f + 1)], s) < 1e-12
    H = box.interpolate_H(pos_dt).cpu().numpy()
    Href = pack(O.hamiltonian(cfg, grid, moved))
    assert family_err(H, Href, s) < 1e-12


@pytest.mark.parametrize("order", ORDERS)
def test_fifty_steps(torch, order):
    wl = W.with_shape(W.tiny_fiducial(), order)
    box = _box(wl)
    cfg = _cfg(wl)
    parts = _oracle_init(wl)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    assert abs(box.timestep() / dt - 1) < 1e-14
    worst = 0.0
    for step in range(50):
        box.step(1, dt)
        O.rk4_step(cfg, parts, dt)
        h = box.get_host()
        e = max(family_err(h["rho"], pack(parts["rho"])), family_err(h["rhobar"], pack(parts["rhobar"])))
        worst = max(worst, e)
        assert e < 1e-10, (step, e)
        assert np.abs(h["z"] - parts["z"]).max() < 1e-12 * wl.Lz
    assert max(_moment_errs(box, cfg, parts)) < 1e-10
    print(f"\norder {order}: worst 50-step state error {worst:.2e}")


@pytest.mark.parametrize("order", ORDERS)
def test_random_box_steps_and_batch(torch, order):
    """Two uneven boxes advanced as one batch agree with the oracle run of each.
    The steps are 0.917 x those of Eq. 7: at Eq. 7's advective limit
    (0.4 dz/c) the 6-direction box moves its mu = 1/2 particles exactly onto a
    cell face at a stage position, where the order-0 shape is discontinuous
    and either cell is a correct choice that rounding decides."""
    from paper_2101_02745_gb300.emu import Box
    wls = [W.with_shape(W.random_box(45, 13, seed=7), order), W.with_shape(W.random_box(20, 6, seed=8), order)]
    batch = Box.from_workloads(wls)
    dts = batch.batch_timestep() * 0.917
    batch.batch_set_dt(dts)
    batch.batch_step(20)
    h = batch.get_host()
    off = 0
    for wl, dt in zip(wls, dts):
        cfg = _cfg(wl)
        parts = _oracle_init(wl)
        assert abs(dt / (0.917 * O.timestep(cfg, O.deposit(cfg, parts))) - 1) < 1e-14
        O.run(cfg, parts, dt, 20)
        sl = slice(off, off + wl.P)
        assert family_err(h["rho"][:, sl], pack(parts["rho"])) < 1e-10
        assert family_err(h["rhobar"][:, sl], pack(parts["rhobar"])) < 1e-10
        off += wl.P


def test_mixed_orders_rejected(torch):
    from paper_2101_02745_gb300 import emu as E
    wls = [W.with_shape(W.random_box(20, 4, seed=1), 1), W.with_shape(W.random_box(20, 4, seed=2), 3)]
    with pytest.raises(E.EmuError):
        E.Box.from_workloads(wls)


@pytest.mark.parametrize("order", [1, 3])
def test_adjoint_at_other_orders(torch, order):
    """The adjoint through the order's stencil, against central differences."""
    from paper_2101_02745_gb300.adjoint import Evolve, Simulation, objectives
    from paper_2101_02745_gb300.emu import Box
    wl = W.with_shape(W.adjoint_box(nz=32, ndir=16, steps=30), order)
    box = Box.from_workload(wl, init=False)
    sim = Simulation(box, wl.steps, 3.4e-12, every=8, alpha=wl.alpha, seed=wl.seed)
    th = np.concatenate([[wl.n_nu[0], wl.n_nubar[0]], wl.f_nu[0], wl.f_nubar[0]])
    nz = box.nz

    def fields(t):
        return t[0].expand(nz), t[1].expand(nz), t[2:5].expand(nz, 3), t[5:8].expand(nz, 3)

    t = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    L = objectives(Evolve.apply(*fields(t), sim))
    L[1].backward()
    g = t.grad.cpu().numpy()
    s = 1e-6 * th[1]
    fd = np.zeros(8)
    for i in range(8):
        e = np.zeros(8); e[i] = s
        with torch.no_grad():
            lp = objectives(Evolve.apply(*fields(torch.tensor(th + e, dtype=torch.float64, device="cuda")), sim))
            lm = objectives(Evolve.apply(*fields(torch.tensor(th - e, dtype=torch.float64, device="cuda")), sim))
        fd[i] = float(lp[1] - lm[1]) / (2 * s)
    assert np.linalg.norm(g - fd) < 1e-5 * np.linalg.norm(fd), (g, fd)
