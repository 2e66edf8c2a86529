/*
 * emu_oracle.c -- plain, slow, FP64 CPU oracle for the particle-in-cell step of
 * Richers, Willcox, Ford & Myers, "Particle-in-cell Simulation of the Neutrino
 * Fast Flavor Instability" (arXiv:2101.02745).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, link or
 * call this file.  Only the test suite, the smoke check of the package entry
 * point, and the CPU-baseline leg of the benchmark use it.  It shares no code,
 * header, table or constant with the CUDA library: it is written directly from
 * the paper, in the paper's order and notation, with full complex 3x3 matrices
 * and sequential loops over particles in id order.
 *
 * What it computes (one explicit RK4 step of the 1D periodic PIC scheme):
 *   - particle -> grid deposit of n_ab, f_ab (neutrinos) and nbar_ab, fbar_ab
 *     (antineutrinos) with a shape function of order 0-3
 *     (quadratic by default)                                   (Eq. 5, Sec. 2.2.1)
 *   - grid -> particle interpolation                          (Eq. 6, Sec. 2.2.2)
 *   - the self-interaction Hamiltonian and its antineutrino
 *     counterpart Hbar = -H*                                   (Eq. 2, Sec. 2.1)
 *   - d rho/dt = -i[H, rho], d rhobar/dt = -i[Hbar, rhobar],
 *     dz/dt = c Omega_z                                        (Eq. 4, Sec. 2.2)
 *   - the classic fourth-order Runge-Kutta step with positions advanced
 *     together with the density matrices                       (Sec. 2.3)
 *   - the time step choice                                     (Eq. 7)
 *   - particle initialisation: weights (Eq. 8), initial flavour state (Eq. 9)
 *
 * Readings of points the paper leaves open:
 *   - H is carried as an angular frequency H/hbar [1/s]; kappa = sqrt(2) G_F/hbar
 *     [cm^3/s] is an input.
 *   - Cell volume dV = dz * area (area is an input, 1 cm^2 by default); it
 *     cancels between the weights of Eq. 8 and the deposit of Eq. 5.
 *   - Shape of order n (the paper offers orders 0 to 3 and uses 2): the
 *     cardinal B-spline of degree n, w_pj = M_{n+1}(z_p/dz - (j + 1/2)), on
 *     the n+1 cells it reaches, indices taken modulo nz (periodic, Sec. 2.3).
 *     Order 0 puts a particle on z = j dz in cell j (the cell containing it).
 *   - "Fourth-order explicit Runge-Kutta" is the classic tableau
 *     (0, 1/2, 1/2, 1; weights 1/6, 1/3, 1/3, 1/6).  No renormalisation of rho.
 *   - Eq. 9: eps_mu = |rho_emu|^2, eps_tau = |rho_etau|^2, rho_mutau = 0.
 *   - The random numbers U of Eq. 9 come from SplitMix64 (Steele, Lea & Flood,
 *     OOPSLA 2014): U(seed, p, k) = 2 * (out_{8p+k+1} >> 11) * 2^-53 - 1, where
 *     out_n is the n-th output of the generator whose state starts at `seed`.
 *     Draws k = 0..3 are Re/Im rho_emu, Re/Im rho_etau; k = 4..7 the same for rhobar.
 *   - Default directions: the midpoint Fibonacci sphere,
 *     mu_d = 1 - (2d+1)/M, phi_d = d * pi * (3 - sqrt 5).
 *   - Particle numbering: particle p = d * nz + j0 starts at the centre of cell j0
 *     with direction d (one particle per direction per cell, Sec. 3.1).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "emu_oracle.h"

static const double OR_PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- RNG --- */

/* n-th output (n >= 1) of SplitMix64 started from state `seed`. */
uint64_t or_splitmix64(uint64_t seed, uint64_t n) {
  uint64_t x = seed + n * 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

double or_uniform(uint64_t seed, int64_t p, int k) {
  uint64_t h = or_splitmix64(seed, (uint64_t)p * 8u + (uint64_t)k + 1u);
  double u01 = (double)(h >> 11) * 0x1.0p-53;
  return 2.0 * u01 - 1.0;
}

/* ---------------------------------------------------------- geometry --- */

double or_dz(const or_config* cfg) { return cfg->Lz / cfg->nz; }

void or_fibonacci_direction(int d, int M, double out[3]) {
  double mu = 1.0 - (2.0 * d + 1.0) / M;
  double phi = d * OR_PI * (3.0 - sqrt(5.0));
  double s = sqrt(1.0 - mu * mu);
  out[0] = s * cos(phi);
  out[1] = s * sin(phi);
  out[2] = mu;
}

/* z mapped into [0, Lz) (periodic domain, Sec. 2.3). */
double or_wrap(const or_config* cfg, double z) {
  double w = z - cfg->Lz * floor(z / cfg->Lz);
  if (w >= cfg->Lz) w -= cfg->Lz;
  if (w < 0.0) w = 0.0;
  return w;
}

/* Cardinal B-spline of degree n (support (-(n+1)/2, (n+1)/2), unit integral)
 * from its truncated-power form
 *   M_{n+1}(x) = (1/n!) sum_{k=0}^{n+1} (-1)^k C(n+1, k) (x + (n+1)/2 - k)_+^n,
 * with t_+^0 = 1 for t >= 0 (so that M_1 is 1 on [-1/2, 1/2)). */
double or_bspline(int n, double x) {
  double sum = 0.0, binom = 1.0, fact = 1.0;
  for (int k = 2; k <= n; ++k) fact *= k;
  for (int k = 0; k <= n + 1; ++k) {
    double t = x + 0.5 * (n + 1) - k;
    double tp = 0.0;
    if (n == 0) tp = t >= 0.0 ? 1.0 : 0.0;
    else if (t > 0.0) tp = pow(t, n);
    sum += (k % 2 ? -binom : binom) * tp;
    binom = binom * (n + 1 - k) / (k + 1);
  }
  return sum / fact;
}

/* Shape function of order n = cfg->shape_order (Sec. 2.2.1): the n+1 cells
 * j with |x_j| < (n+1)/2, x_j = z/dz - (j + 1/2) the particle's offset from
 * the centre of cell j in cell units, and the fraction w_pj = M_{n+1}(x_j)
 * of the particle in each (the w_pj of Eq. 5).  Returns the count n+1. */
int or_shape(const or_config* cfg, double z, int32_t cells[4], double w[4]) {
  int n = cfg->shape_order;
  double xi = z / or_dz(cfg) - 0.5;                 /* offset from the centre of cell 0 */
  long long j0 = (long long)floor(xi - 0.5 * (n + 1)) + 1;   /* first cell inside the support */
  for (int s = 0; s <= n; ++s) {
    long long j = j0 + s;
    w[s] = or_bspline(n, xi - (double)j);
    long long c = j % cfg->nz;
    if (c < 0) c += cfg->nz;
    cells[s] = (int32_t)c;
  }
  return n + 1;
}

/* ------------------------------------------------------- initialisation --- */

/* Eq. 8 weights and Eq. 9 initial flavour states.
 *   dirs:   M x 3 unit vectors, or NULL for the Fibonacci set
 *   n_nu, n_nubar:   per-cell input number densities [cm^-3] (length nz)
 *   f_nu, f_nubar:   per-cell input number-flux vectors [cm^-3] (nz x 3)
 * Returns 0, or -1 if a weight comes out negative (|f| > n/3). */
int or_init(const or_config* cfg, const double* dirs, const double* n_nu,
            const double* n_nubar, const double* f_nu, const double* f_nubar,
            double alpha, uint64_t seed, or_particle* parts) {
  int nz = cfg->nz, M = cfg->ndir;
  double dz = or_dz(cfg), dV = dz * cfg->area;
  int bad = 0;
  for (int d = 0; d < M; ++d) {
    double om[3];
    if (dirs) { om[0] = dirs[3 * d]; om[1] = dirs[3 * d + 1]; om[2] = dirs[3 * d + 2]; }
    else or_fibonacci_direction(d, M, om);
    for (int j0 = 0; j0 < nz; ++j0) {
      int64_t p = (int64_t)d * nz + j0;
      or_particle* q = &parts[p];
      memset(q, 0, sizeof(*q));
      q->z = (j0 + 0.5) * dz;
      q->omega[0] = om[0]; q->omega[1] = om[1]; q->omega[2] = om[2];
      double fdo = f_nu[3 * j0] * om[0] + f_nu[3 * j0 + 1] * om[1] + f_nu[3 * j0 + 2] * om[2];
      double fbdo = f_nubar[3 * j0] * om[0] + f_nubar[3 * j0 + 1] * om[1] + f_nubar[3 * j0 + 2] * om[2];
      q->N = (n_nu[j0] + 3.0 * fdo) * dV / M;
      q->Nbar = (n_nubar[j0] + 3.0 * fbdo) * dV / M;
      /* A flux factor of exactly 1/3 along a particle's own direction gives a
       * weight that is zero in exact arithmetic; rounding may leave it a few
       * ulp below zero.  Such weights become 0; clearly negative ones are an error. */
      double tol_nu = 1e-12 * (fabs(n_nu[j0]) + 3.0 * fabs(fdo)) * dV / M;
      double tol_nb = 1e-12 * (fabs(n_nubar[j0]) + 3.0 * fabs(fbdo)) * dV / M;
      if (q->N < 0.0 && q->N >= -tol_nu) q->N = 0.0;
      if (q->Nbar < 0.0 && q->Nbar >= -tol_nb) q->Nbar = 0.0;
      if (q->N < 0.0 || q->Nbar < 0.0) bad = 1;
      /* Eq. 9 for rho (draws 0..3) and rhobar (draws 4..7) */
      for (int which = 0; which < 2; ++which) {
        cplx (*r)[3] = which == 0 ? q->rho : q->rhobar;
        double u0 = or_uniform(seed, p, 4 * which + 0);
        double u1 = or_uniform(seed, p, 4 * which + 1);
        double u2 = or_uniform(seed, p, 4 * which + 2);
        double u3 = or_uniform(seed, p, 4 * which + 3);
        cplx em = alpha * u0 + I * (alpha * u1);
        cplx et = alpha * u2 + I * (alpha * u3);
        double eps_mu = creal(em) * creal(em) + cimag(em) * cimag(em);
        double eps_tau = creal(et) * creal(et) + cimag(et) * cimag(et);
        r[0][0] = 1.0 - eps_mu - eps_tau;
        r[1][1] = eps_mu;
        r[2][2] = eps_tau;
        r[0][1] = em; r[1][0] = conj(em);
        r[0][2] = et; r[2][0] = conj(et);
        r[1][2] = 0.0; r[2][1] = 0.0;
      }
    }
  }
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------- deposit --- */

/* Eq. 5: n_ab,j = (1/dV) sum_p N_p w_pj rho_ab,p and f_ab,j = (1/dV) sum_p
 * N_p w_pj rho_ab,p Omega_p; the same with Nbar, rhobar for antineutrinos.
 * Every particle adds into all three cells it touches; periodic wrap. */
void or_deposit(const or_config* cfg, const or_particle* parts, int64_t P, or_cell* grid) {
  double dV = or_dz(cfg) * cfg->area;
  memset(grid, 0, sizeof(or_cell) * (size_t)cfg->nz);
  for (int64_t p = 0; p < P; ++p) {
    const or_particle* q = &parts[p];
    int32_t cells[4]; double w[4];
    int ns = or_shape(cfg, q->z, cells, w);
    for (int s = 0; s < ns; ++s) {
      or_cell* g = &grid[cells[s]];
      double cn = q->N * w[s] / dV, cb = q->Nbar * w[s] / dV;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          g->n[a][b] += cn * q->rho[a][b];
          g->nbar[a][b] += cb * q->rhobar[a][b];
          for (int i = 0; i < 3; ++i) {
            g->f[i][a][b] += cn * q->rho[a][b] * q->omega[i];
            g->fbar[i][a][b] += cb * q->rhobar[a][b] * q->omega[i];
          }
        }
    }
  }
}

/* ------------------------------------------------- interpolation and H --- */

/* Eq. 6 (interpolate n, nbar, f, fbar to the particle with its own shape
 * weights) followed by the self-interaction term of Eq. 2 divided by hbar:
 *   H = kappa [ (n - nbar^*) - Omega . (f - fbar^*) ].
 * Vacuum and matter terms are not part of this path. */
void or_hamiltonian(const or_config* cfg, const or_cell* grid, const or_particle* q, cplx H[3][3]) {
  int32_t cells[4]; double w[4];
  int ns = or_shape(cfg, q->z, cells, w);
  cplx n[3][3] = {{0}}, nb[3][3] = {{0}}, f[3][3][3] = {{{0}}}, fb[3][3][3] = {{{0}}};
  for (int s = 0; s < ns; ++s) {
    const or_cell* g = &grid[cells[s]];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        n[a][b] += w[s] * g->n[a][b];
        nb[a][b] += w[s] * g->nbar[a][b];
        for (int i = 0; i < 3; ++i) {
          f[i][a][b] += w[s] * g->f[i][a][b];
          fb[i][a][b] += w[s] * g->fbar[i][a][b];
        }
      }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx v = n[a][b] - conj(nb[a][b]);
      for (int i = 0; i < 3; ++i) v -= q->omega[i] * (f[i][a][b] - conj(fb[i][a][b]));
      H[a][b] = cfg->kappa * v;
    }
}

/* Mixing matrix U (flavour <- mass basis) in the standard three-angle form:
 * U = R23 U13(delta) R12 with c_ij = cos theta_ij, s_ij = sin theta_ij. */
void or_mixing_matrix(const or_config* cfg, cplx U[3][3]) {
  double c12 = cos(cfg->theta12), s12 = sin(cfg->theta12);
  double c13 = cos(cfg->theta13), s13 = sin(cfg->theta13);
  double c23 = cos(cfg->theta23), s23 = sin(cfg->theta23);
  cplx ep = cexp(I * cfg->delta_cp), em = cexp(-I * cfg->delta_cp);
  U[0][0] = c12 * c13;
  U[0][1] = s12 * c13;
  U[0][2] = s13 * em;
  U[1][0] = -s12 * c23 - c12 * s23 * s13 * ep;
  U[1][1] = c12 * c23 - s12 * s23 * s13 * ep;
  U[1][2] = s23 * c13;
  U[2][0] = s12 * s23 - c12 * c23 * s13 * ep;
  U[2][1] = -c12 * s23 - s12 * c23 * s13 * ep;
  U[2][2] = c23 * c13;
}

/* Vacuum term of Eq. 2 divided by hbar: U diag(m_i^2 c^4 / (2 E)) U^dagger / hbar
 * (the flavour-blind |p| c part cancels in the commutator), and the matter
 * term kappa n_e diag(1, 0, 0) (comoving frame: no lepton flux). */
void or_vacuum_matter(const or_config* cfg, cplx Hvac[3][3], cplx Hmat[3][3]) {
  cplx U[3][3];
  or_mixing_matrix(cfg, U);
  double w[3];
  for (int i = 0; i < 3; ++i) {
    double mc2 = cfg->mass_eV[i] * cfg->erg_per_eV;
    w[i] = mc2 * mc2 / (2.0 * cfg->energy_erg) / cfg->hbar;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx v = 0.0;
      for (int i = 0; i < 3; ++i) v += U[a][i] * w[i] * conj(U[b][i]);
      Hvac[a][b] = v;
      Hmat[a][b] = 0.0;
    }
  Hmat[0][0] = cfg->kappa * cfg->n_e;
}

/* Sec. 2.1: for antineutrinos the self-interaction Hamiltonian is -H^*. */
void or_hamiltonian_bar(cplx H[3][3], cplx Hbar[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Hbar[a][b] = -conj(H[a][b]);
}

/* Eq. 4: d rho/dt = -i [H, rho] (H in units of hbar). */
void or_commutator_rhs(cplx H[3][3], cplx rho[3][3], cplx out[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx c = 0.0;
      for (int k = 0; k < 3; ++k) c += H[a][k] * rho[k][b] - rho[a][k] * H[k][b];
      out[a][b] = -I * c;
    }
}

/* Right-hand side of Eq. 4 for every particle at the given state:
 * deposit, then per particle interpolate, build H and Hbar, commutators. */
void or_rhs(const or_config* cfg, const or_particle* parts, int64_t P, or_cell* grid,
            cplx (*drho)[3][3], cplx (*drhobar)[3][3]) {
  or_deposit(cfg, parts, P, grid);
  cplx Hvac[3][3] = {{0}}, Hmat[3][3] = {{0}};
  if (cfg->osc_on) or_vacuum_matter(cfg, Hvac, Hmat);
  for (int64_t p = 0; p < P; ++p) {
    cplx H[3][3], Hb[3][3];
    or_hamiltonian(cfg, grid, &parts[p], H);
    or_hamiltonian_bar(H, Hb);
    /* Sec. 2.1: Hbar_vacuum = H_vacuum^*, Hbar_matter = -H_matter^* */
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        H[a][b] += Hvac[a][b] + Hmat[a][b];
        Hb[a][b] += conj(Hvac[a][b]) - conj(Hmat[a][b]);
      }
    cplx r[3][3], rb[3][3];
    memcpy(r, parts[p].rho, sizeof(r));
    memcpy(rb, parts[p].rhobar, sizeof(rb));
    or_commutator_rhs(H, r, drho[p]);
    or_commutator_rhs(Hb, rb, drhobar[p]);
  }
}

/* ---------------------------------------------------------------- RK4 --- */

/* One classic RK4 step of Eq. 4 for all particles together (Sec. 2.3).
 * Stage s (c_s = 0, 1/2, 1/2, 1) evaluates the right-hand side at
 * rho + c_s dt k_{s-1} and at the position z + c_s dt c Omega_z (wrapped), so
 * positions and density matrices advance together without operator
 * splitting.  The step ends at rho + dt/6 (k1 + 2 k2 + 2 k3 + k4) and
 * z + dt c Omega_z.  Returns 0, or -1 if scratch allocation fails. */
int or_rk4_step(const or_config* cfg, or_particle* parts, int64_t P, double dt) {
  static const double cstage[4] = {0.0, 0.5, 0.5, 1.0};
  or_particle* ystage = malloc(sizeof(or_particle) * (size_t)P);
  or_cell* grid = malloc(sizeof(or_cell) * (size_t)cfg->nz);
  cplx (*kr)[3][3] = malloc(sizeof(cplx) * 9 * 4 * (size_t)P);   /* k_s for rho,    [s*P + p] */
  cplx (*kb)[3][3] = malloc(sizeof(cplx) * 9 * 4 * (size_t)P);   /* k_s for rhobar, [s*P + p] */
  if (!ystage || !grid || !kr || !kb) {
    free(ystage); free(grid); free(kr); free(kb);
    return -1;
  }
  for (int s = 0; s < 4; ++s) {
    for (int64_t p = 0; p < P; ++p) {
      ystage[p] = parts[p];
      if (s > 0) {
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            ystage[p].rho[a][b] = parts[p].rho[a][b] + cstage[s] * dt * kr[(s - 1) * P + p][a][b];
            ystage[p].rhobar[a][b] = parts[p].rhobar[a][b] + cstage[s] * dt * kb[(s - 1) * P + p][a][b];
          }
        ystage[p].z = or_wrap(cfg, parts[p].z + cstage[s] * dt * cfg->c_light * parts[p].omega[2]);
      }
    }
    or_rhs(cfg, ystage, P, grid, kr + s * P, kb + s * P);
  }
  for (int64_t p = 0; p < P; ++p) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        parts[p].rho[a][b] += dt / 6.0 * (kr[p][a][b] + 2.0 * kr[P + p][a][b] +
                                          2.0 * kr[2 * P + p][a][b] + kr[3 * P + p][a][b]);
        parts[p].rhobar[a][b] += dt / 6.0 * (kb[p][a][b] + 2.0 * kb[P + p][a][b] +
                                             2.0 * kb[2 * P + p][a][b] + kb[3 * P + p][a][b]);
      }
    parts[p].z = or_wrap(cfg, parts[p].z + dt * cfg->c_light * parts[p].omega[2]);
  }
  free(ystage); free(grid); free(kr); free(kb);
  return 0;
}

/* nsteps RK4 steps with a fixed dt. */
int or_run(const or_config* cfg, or_particle* parts, int64_t P, double dt, int64_t nsteps) {
  for (int64_t n = 0; n < nsteps; ++n)
    if (or_rk4_step(cfg, parts, P, dt) != 0) return -1;
  return 0;
}

/* ------------------------------------------------------------ time step --- */

/* Eq. 7 with the maximum over grid cells and diagonal components of n and
 * nbar, and the lepton density n_a (the net electron density when the
 * matter term is on). */
double or_timestep(const or_config* cfg, const or_cell* grid) {
  double nmax = cfg->osc_on ? cfg->n_e : 0.0;
  for (int j = 0; j < cfg->nz; ++j)
    for (int a = 0; a < 3; ++a) {
      if (creal(grid[j].n[a][a]) > nmax) nmax = creal(grid[j].n[a][a]);
      if (creal(grid[j].nbar[a][a]) > nmax) nmax = creal(grid[j].nbar[a][a]);
    }
  double dt_adv = cfg->cfl_adv * or_dz(cfg) / cfg->c_light;
  double dt_flav = nmax > 0.0 ? cfg->cfl_flavor / (cfg->kappa * nmax) : dt_adv;
  return dt_adv < dt_flav ? dt_adv : dt_flav;
}

/* -------------------------------------------------------- diagnostics --- */

/* Domain-integrated lepton matrix E = sum_p (N_p rho_p - Nbar_p rhobar_p^*),
 * which Eq. 4 with the self-interaction Hamiltonian conserves exactly
 * (its change is a sum of commutators of a cell's potential with itself). */
void or_eln_matrix(const or_particle* parts, int64_t P, cplx E[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) E[a][b] = 0.0;
  for (int64_t p = 0; p < P; ++p)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        E[a][b] += parts[p].N * parts[p].rho[a][b] - parts[p].Nbar * conj(parts[p].rhobar[a][b]);
}

/* Eq. 10: domain averages <|n_ab|> and <|f^(x)_ab|> for neutrinos and
 * antineutrinos, plus the plain domain average <n_ab> (one snapshot of Eq. B1).
 * out_abs[4][3][3] = {|n|, |nbar|, |f_x|, |fbar_x|}; out_avg[2][3][3] complex. */
void or_domain_averages(const or_config* cfg, const or_cell* grid, double out_abs[4][3][3],
                        cplx out_avg[2][3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      cplx m0 = 0, m1 = 0;
      for (int j = 0; j < cfg->nz; ++j) {
        s0 += cabs(grid[j].n[a][b]);
        s1 += cabs(grid[j].nbar[a][b]);
        s2 += cabs(grid[j].f[0][a][b]);
        s3 += cabs(grid[j].fbar[0][a][b]);
        m0 += grid[j].n[a][b];
        m1 += grid[j].nbar[a][b];
      }
      out_abs[0][a][b] = s0 / cfg->nz;
      out_abs[1][a][b] = s1 / cfg->nz;
      out_abs[2][a][b] = s2 / cfg->nz;
      out_abs[3][a][b] = s3 / cfg->nz;
      out_avg[0][a][b] = m0 / cfg->nz;
      out_avg[1][a][b] = m1 / cfg->nz;
    }
}

/* Sizes of the structures, so the Python binding can check its mirror. */
int32_t or_sizeof_particle(void) { return (int32_t)sizeof(or_particle); }
int32_t or_sizeof_cell(void) { return (int32_t)sizeof(or_cell); }
int32_t or_sizeof_config(void) { return (int32_t)sizeof(or_config); }
