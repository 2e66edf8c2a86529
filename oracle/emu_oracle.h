/*
 * emu_oracle.h -- types and routines of the plain FP64 CPU oracle shared by
 * its 1D (emu_oracle.c) and 3D (emu_oracle3d.c) parts.
 *
 * TEST INFRASTRUCTURE ONLY: nothing in the product path includes, loads or
 * links the oracle, and the oracle includes nothing of the CUDA library.
 */
#ifndef EMU_ORACLE_H
#define EMU_ORACLE_H

#include <complex.h>
#include <stdint.h>

typedef double complex cplx;

/* Simulation parameters.  Layout mirrored by a ctypes Structure. */
typedef struct {
  int32_t nz;         /* number of cells on the periodic grid */
  int32_t ndir;       /* particles (directions) per cell, N_ppz of Eq. 8 */
  double Lz;          /* domain length [cm] */
  double area;        /* transverse cell area [cm^2] */
  double kappa;       /* sqrt(2) G_F / hbar [cm^3 / s] */
  double c_light;     /* speed of light [cm / s] */
  double cfl_adv;     /* C of Eq. 7 */
  double cfl_flavor;  /* C_F of Eq. 7 */
  /* Vacuum and matter terms of Eq. 2 (off when osc_on == 0):
   * masses m_i c^2 [eV], mixing angles theta12, theta13, theta23 and the
   * phase delta [rad] of the standard three-angle mixing matrix, neutrino
   * energy [erg], net electron density n_e [cm^-3], hbar [erg s], erg per eV. */
  int32_t osc_on;
  int32_t shape_order; /* 0..3: degree of the B-spline shape (Sec. 2.2.1), 2 = quadratic */
  double mass_eV[3];
  double theta12, theta13, theta23, delta_cp;
  double energy_erg;
  double n_e;
  double hbar;
  double erg_per_eV;
} or_config;

/* One computational particle (Sec. 2.2): position, direction, weights and
 * the two full 3x3 density matrices.  Flavour index order e, mu, tau. */
typedef struct {
  double z;
  double omega[3];
  double N, Nbar;
  cplx rho[3][3];
  cplx rhobar[3][3];
} or_particle;

/* One grid cell: the direction-integrated quantities of Eq. 5. */
typedef struct {
  cplx n[3][3];
  cplx nbar[3][3];
  cplx f[3][3][3];    /* f[i][a][b]: spatial component i of f_ab */
  cplx fbar[3][3][3];
} or_cell;

/* 1D routines the 3D part reuses. */
double or_bspline(int n, double x);
double or_uniform(uint64_t seed, int64_t p, int k);
void or_fibonacci_direction(int d, int M, double out[3]);
void or_vacuum_matter(const or_config* cfg, cplx Hvac[3][3], cplx Hmat[3][3]);
void or_hamiltonian_bar(cplx H[3][3], cplx Hbar[3][3]);
void or_commutator_rhs(cplx H[3][3], cplx rho[3][3], cplx out[3][3]);

#endif /* EMU_ORACLE_H */
