"""Pins of the oracle's reference gradient (oracle/gradient.py) against results
fixed by the method's definitions, not by the oracle itself."""
import json
from pathlib import Path

import numpy as np
import pytest

from oracle import gradient, oracle
from paper_2101_02745_gb300 import workloads

GOLDEN = Path(__file__).resolve().parent / "golden"


def _kw(wl):
    return dict(nz=wl.nz, ndir=wl.ndir, Lz=wl.Lz, kappa=wl.kappa, c_light=wl.c_light)


def test_unperturbed_abundance_gradient_closed_form():
    """With no perturbation (alpha = 0) every rho stays diag(1, 0, 0): H is
    diagonal and commutes with it.  Then <n_ee> = sum_p N_p / (nz dV) (the
    shape weights of a particle sum to 1), and with Eq. 8 its gradient is
    exactly (1, 0, 3<Omega_x>, 3<Omega_y>, 3<Omega_z>, 0, 0, 0), <.> the mean
    over the Fibonacci directions (Sec. 3.1), for any number of steps."""
    wl = workloads.random_box(12, 10, seed=3)
    kw = _kw(wl)
    theta = np.array([4.0e32, 5.0e32, 0.3e32, -0.2e32, 0.5e32, -0.4e32, 0.1e32, -0.9e32])
    g = gradient.fd_gradient(kw, theta, 0.0, 0, 2e-12, 6)
    assert np.all(np.isnan(g[1]))                      # L1 = log <|n_emu|> is undefined without a perturbation
    M = wl.ndir
    mu = 1.0 - (2.0 * np.arange(M) + 1.0) / M          # Fibonacci midpoint directions
    phi = np.arange(M) * np.pi * (3.0 - np.sqrt(5.0))
    s = np.sqrt(1.0 - mu * mu)
    om = np.stack([s * np.cos(phi), s * np.sin(phi), mu], 1).mean(0)
    want = np.array([1.0, 0.0, 3 * om[0], 3 * om[1], 3 * om[2], 0.0, 0.0, 0.0])
    assert np.max(np.abs(g[0] - want)) < 1e-8


def test_difference_quotient_converges():
    """Central differences are second order: halving h changes the gradient of a
    smooth growth-phase objective by far less than the gradient itself."""
    wl = workloads.adjoint_box(nz=16, ndir=8, steps=12)
    kw = _kw(wl)
    theta = np.concatenate([[wl.n_nu[0], wl.n_nubar[0]], wl.f_nu[0], wl.f_nubar[0]])
    g1 = gradient.fd_gradient(kw, theta, wl.alpha, wl.seed, 3.4e-12, wl.steps, h=1e-5)
    g2 = gradient.fd_gradient(kw, theta, wl.alpha, wl.seed, 3.4e-12, wl.steps, h=5e-6)
    for k in range(2):
        assert np.linalg.norm(g1[k] - g2[k]) <= 1e-6 * np.linalg.norm(g2[k])


def test_growth_phase_gradient_matches_dispersion_relation():
    """In the linear phase log <|n_emu|> = C(theta) + gamma(theta) t plus decaying
    slower modes, so the gradient's change between two times t1 < t2 is
    (t2 - t1) dgamma/dtheta, where gamma is the largest growth rate of the
    linearised equations over the box's wavenumbers k = 2 pi m / Lz: the
    discrete-direction dispersion relation (Sec. 3.2) with the quadratic shape's
    transfer factor, solved as an eigenvalue problem by oracle/dispersion.py
    (pinned to the paper's growth rates).  32 cells over four fastest
    wavelengths, 16 directions, steps 200 and 300 (amplitude still ~1e-4)."""
    from oracle import dispersion

    wl = workloads.adjoint_box(nz=32, ndir=16, steps=300)
    kw = _kw(wl)
    theta = np.concatenate([[wl.n_nu[0], wl.n_nubar[0]], wl.f_nu[0], wl.f_nubar[0]])
    dt, t1, t2 = 3.4e-12, 200, 300
    g1 = gradient.fd_gradient(kw, theta, wl.alpha, wl.seed, dt, t1)
    g2 = gradient.fd_gradient(kw, theta, wl.alpha, wl.seed, dt, t2)
    rate = (g2[1] - g1[1]) / ((t2 - t1) * dt)

    M, nz, Lz = wl.ndir, wl.nz, wl.Lz
    dirs = np.array([oracle.fibonacci_direction(d, M) for d in range(M)])

    def gamma_max(th):
        g = (th[0] + 3.0 * dirs @ th[2:5]) / M       # Eq. 8 per direction, per unit volume
        gb = (th[1] + 3.0 * dirs @ th[5:8]) / M
        ks = 2.0 * np.pi * np.arange(-nz // 2, nz // 2 + 1) / Lz
        return max(dispersion.discrete_growth(k, dirs, g, gb, wl.kappa, wl.c_light,
                                              dispersion.shape_transfer(k, Lz / nz)) for k in ks)

    s = 1e-6 * theta[1]
    dgam = np.array([(gamma_max(theta + s * e) - gamma_max(theta - s * e)) / (2 * s) for e in np.eye(8)])
    assert np.linalg.norm(rate - dgam) <= 0.06 * np.linalg.norm(dgam)
    for i in (0, 1, 4, 7):   # n_nu, n_nubar, f_nu z, f_nubar z
        assert abs(rate[i] - dgam[i]) <= 0.05 * abs(dgam[i])


def test_golden_file_shape():
    p = GOLDEN / "adjoint_256x96.json"
    if not p.exists():
        pytest.skip("reference gradient not generated")
    d = json.loads(p.read_text())
    g = np.array(d["gradient"])
    assert g.shape == (2, 8) and np.all(np.isfinite(g))
    assert d["params"] == list(gradient.PARAMS)
    assert d["nsteps"] == 400 and d["config"]["nz"] == 256 and d["config"]["ndir"] == 96
