"""Reference gradients of two objectives of the particle step, by central
finite differences of the oracle.

TEST INFRASTRUCTURE ONLY, under the same rule as oracle.py: only the test
suite and the scripts under tests/golden/ may use it.

The paper computes no gradients.  What is differentiated here is the discrete
method itself: the particle weights of Eq. 8 built from uniform densities and
fluxes, then `nsteps` classic RK4 steps (Sec. 2.3) at a FIXED time step, then
the deposit of Eq. 5.  The objectives are functions of the final neutrino
number-density matrices n_j:

    L0 = <n_ee>          = (1/nz) sum_j Re n_ee,j        (final nu_e abundance)
    L1 = log <|n_emu|>   = log((1/nz) sum_j |n_emu,j|)    (growth measure, Eq. 10)

The parameters are theta = (n_nu, n_nubar, f_nu x, y, z, f_nubar x, y, z) in
cm^-3.  The derivative along parameter i is the symmetric difference quotient
(L(theta + s e_i) - L(theta - s e_i)) / (2 s) with one step s = h * max(n_nu,
n_nubar) for all eight (they share the unit cm^-3, and the fluxes may be 0).
"""
from __future__ import annotations

from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np

from . import oracle

PARAMS = ("n_nu", "n_nubar", "f_nu_x", "f_nu_y", "f_nu_z", "f_nubar_x", "f_nubar_y", "f_nubar_z")


def objectives(cfg, parts) -> np.ndarray:
    """(L0, L1) of the current particles (deposit of Eq. 5)."""
    grid = oracle.deposit(cfg, parts)
    nee = grid["n"][:, 0, 0].real
    nem = np.abs(grid["n"][:, 0, 1])
    with np.errstate(divide="ignore"):
        return np.array([nee.mean(), np.log(nem.mean())])


def evaluate(cfg_kw: dict, theta, alpha: float, seed: int, dt: float, nsteps: int, dirs=None) -> np.ndarray:
    """Objectives after nsteps steps from the uniform species theta."""
    cfg = oracle.config(**cfg_kw)
    theta = np.asarray(theta, float)
    parts = oracle.init(cfg, theta[0], theta[1], theta[2:5], theta[5:8], alpha, seed, dirs)
    if nsteps:
        oracle.run(cfg, parts, dt, nsteps)
    return objectives(cfg, parts)


def _eval_args(args):
    return evaluate(*args)


def fd_gradient(cfg_kw: dict, theta, alpha: float, seed: int, dt: float, nsteps: int, h: float = 1e-6,
                dirs=None, processes: int = 1) -> np.ndarray:
    """Central-difference gradient, shape (2, 8): row k is dL_k/dtheta (row 1
    is NaN where L1 is undefined: alpha = 0 leaves n_emu = 0).
    processes > 1 evaluates the 16 runs in a spawned process pool."""
    theta = np.asarray(theta, float)
    s = h * max(abs(theta[0]), abs(theta[1]))
    jobs = []
    for i in range(8):
        for sign in (1.0, -1.0):
            t = theta.copy()
            t[i] += sign * s
            jobs.append((cfg_kw, t, alpha, seed, dt, nsteps, dirs))
    if processes > 1:
        with ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
            vals = list(ex.map(_eval_args, jobs))
    else:
        vals = [evaluate(*j) for j in jobs]
    g = np.zeros((2, 8))
    for i in range(8):
        lo, hi = vals[2 * i], vals[2 * i + 1]
        for k in range(2):
            # L1 = log <|n_emu|> is undefined when n_emu stays 0 (no perturbation,
            # alpha = 0): its row is then NaN by definition, not by arithmetic
            g[k, i] = (lo[k] - hi[k]) / (2.0 * s) if np.isfinite(lo[k]) and np.isfinite(hi[k]) else np.nan
    return g
