"""Numerical linear-stability (dispersion) solve for the fast flavour instability.

TEST INFRASTRUCTURE ONLY (see oracle.py).

The paper (Sec. 3.2) computes the growth rate Im(omega) of perturbations
N_ex ~ exp(-i(omega t - k z)) of an initially pure electron-flavour state by a
linear stability analysis, and prints the peaks of the two branches of its
fiducial setup: 6.50e10 /s at 2.20 cm (axially symmetric) and 1.06e10 /s at
4.45 cm (axially asymmetric), with unstable modes for k c/(sqrt(2) G_F n/hbar)
below about 2.66.  This module restates that analysis as a matrix eigenvalue
problem so the oracle's simulated growth can be checked against it.

Linearisation (two flavours e, x; H in units of hbar, kappa = sqrt(2) G_F/hbar),
written from Eq. 2 and Eq. 4 of the paper:
  background rho = rhobar = diag(1, 0); perturbations x(Omega) = delta rho_ex and
  y(Omega) = (delta rhobar_ex)^*, with neutrino and antineutrino number
  densities per direction g(Omega), gbar(Omega).  With
      eps(Omega) = kappa [ (n - nbar) - Omega . (f - fbar) ]        (H_ee - H_xx)
      dH(Omega)  = kappa sum_j (1 - Omega . Omega_j) (g_j x_j - gbar_j y_j)
  the commutator of Eq. 4 gives, for a plane wave exp(i(k z - omega t)),
      omega x_i = (k c Omega_z,i + eps_i) x_i - S(k) dH_i
      omega y_i = (k c Omega_z,i + eps_i) y_i - S(k) dH_i
  (the antineutrino Hamiltonian -H^* of Sec. 2.1 makes the y equation
  identical after complex conjugation).  S(k) = 1 in the continuum; on the PIC
  grid the deposit followed by the interpolation with the quadratic shape
  multiplies a mode by W(k)^2, W(k) = 3/4 + 1/4 cos(k dz), for particles at
  cell centres.

Continuum (the paper's "cosine" distributions g = n/(4 pi) (1 + 3 (f/n) mu)):
directions are Gauss-Legendre nodes in mu; the azimuthal integral is done
analytically, which leaves the kernel 1 - mu mu' for axially symmetric modes
(m = 0) and -1/2 sin(theta) sin(theta') for modes ~ exp(i phi) (m = 1).
"""
from __future__ import annotations

import numpy as np


def _growth(kc, eps, mu_z, K, g, gbar, kappa, S):
    Q = len(g)
    D = np.diag(kc * mu_z + eps)
    A = kappa * S * K * g[None, :]
    B = kappa * S * K * gbar[None, :]
    M = np.block([[D - A, B], [-A, D + B]])
    w = np.linalg.eigvals(M)
    return float(np.max(w.imag))


def continuum_growth(k, n, nbar, fz, fbarz, kappa, c_light, m=0, nodes=192):
    """Max Im(omega) [1/s] at wavenumber k [1/cm] for axially symmetric
    backgrounds with fluxes along z (m = 0 or 1 azimuthal mode number)."""
    mu, w = np.polynomial.legendre.leggauss(nodes)
    g = 2.0 * np.pi * w * (n + 3.0 * fz * mu) / (4.0 * np.pi)
    gb = 2.0 * np.pi * w * (nbar + 3.0 * fbarz * mu) / (4.0 * np.pi)
    eps = kappa * ((n - nbar) - mu * (fz - fbarz))
    if m == 0:
        K = 1.0 - np.outer(mu, mu)
    elif m == 1:
        s = np.sqrt(1.0 - mu * mu)
        K = -0.5 * np.outer(s, s)
    else:
        raise ValueError("m must be 0 or 1")
    return _growth(k * c_light, eps, mu, K, g, gb, kappa, 1.0)


def discrete_growth(k, dirs, g, gbar, kappa, c_light, S=1.0):
    """Max Im(omega) [1/s] for a finite set of directions dirs (M x 3) with
    number densities per direction g, gbar [cm^-3] (homogeneous background)."""
    dirs = np.asarray(dirs, float)
    g = np.asarray(g, float); gbar = np.asarray(gbar, float)
    ntot = g.sum() - gbar.sum()
    ftot = (dirs * (g - gbar)[:, None]).sum(axis=0)
    eps = kappa * (ntot - dirs @ ftot)
    K = 1.0 - dirs @ dirs.T
    return _growth(k * c_light, eps, dirs[:, 2], K, g, gbar, kappa, S)


def shape_transfer(k, dz, order=2, spread=False):
    """W(k)^2, the deposit-then-interpolate factor of a Fourier mode.
    spread=False: particles at cell centres, W(k) = sum_m M(m) cos(k m dz)
    with M the B-spline shape of the given order sampled at the integers
    (order 0 and 1: W = 1; 2: 3/4 + cos(k dz)/4; 3: 2/3 + cos(k dz)/3).
    spread=True: particle offsets spread evenly over the cell (moving
    particles of many directions), W(k) = the B-spline's Fourier transform
    sinc(k dz / 2)^(order + 1)."""
    if spread:
        x = 0.5 * k * dz
        return (np.sin(x) / x if x != 0 else 1.0) ** (2 * (order + 1))
    from scipy.interpolate import BSpline

    knots = np.arange(order + 2) - 0.5 * (order + 1)
    B = BSpline.basis_element(knots, extrapolate=False)
    W = 0.0
    for m in range(-(order // 2) - 1, order // 2 + 2):
        v = B(float(m)) if knots[0] <= m < knots[-1] else 0.0
        v = 0.0 if np.isnan(v) else float(v)
        W = W + v * np.cos(k * m * dz)
    return W * W


def peak(growth_of_k, kmin, kmax, ngrid=200):
    """(k at the maximum, maximum) of a growth-rate function on [kmin, kmax]:
    a grid scan followed by golden-section refinement."""
    ks = np.linspace(kmin, kmax, ngrid)
    vals = np.array([growth_of_k(k) for k in ks])
    i = int(np.argmax(vals))
    a = ks[max(i - 1, 0)]
    b = ks[min(i + 1, ngrid - 1)]
    gr = (np.sqrt(5.0) - 1.0) / 2.0
    c = b - gr * (b - a)
    d = a + gr * (b - a)
    fc, fd = growth_of_k(c), growth_of_k(d)
    for _ in range(60):
        if fc > fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = growth_of_k(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = growth_of_k(d)
    kbest = 0.5 * (a + b)
    return kbest, growth_of_k(kbest)


def unstable_edge(growth_of_k, kpeak, kmax, tol=1e-6, floor=1e-4):
    """Smallest k > kpeak at which the growth rate falls below floor * peak."""
    g0 = growth_of_k(kpeak)
    lo, hi = kpeak, kmax
    assert growth_of_k(hi) < floor * g0
    while hi - lo > tol * kpeak:
        mid = 0.5 * (lo + hi)
        if growth_of_k(mid) > floor * g0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
