/*
 * emu_oracle3d.c -- plain, slow, FP64 CPU oracle of the particle-in-cell step
 * of Richers, Willcox, Ford & Myers (arXiv:2101.02745) on a 3D periodic grid.
 *
 * TEST INFRASTRUCTURE ONLY, under the same rule as emu_oracle.c (which this
 * file extends and is compiled with): nothing in the product path may load,
 * link or call it.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * The paper's runs are 1D; it names 3D runs as future work (Sec. 5) and
 * states the method for a general grid: the deposit of Eq. 5 and the
 * interpolation of Eq. 6 over grid cells j with the particle's shape weights
 * w_pj, and particles moving at c Omega (Eq. 4).  Readings for 3D:
 *   - box [0, Lx) x [0, Ly) x [0, Lz) with nx x ny x nz cells, periodic in
 *     every axis; cell volume dV = dx dy dz; cell (jx, jy, jz) has index
 *     c = (jx * ny + jy) * nz + jz;
 *   - shape: the tensor product of the 1D shape of order n on each axis,
 *     w_pj = M_{n+1}(x/dx - (jx + 1/2)) M_{n+1}(y/dy - (jy + 1/2)) M_{n+1}(z/dz - (jz + 1/2))
 *     (the 1D B-spline M_{n+1} of or_bspline);
 *   - one particle per direction per cell at the cell centre (Sec. 3.1),
 *     numbered p = d * (nx ny nz) + c0 with c0 the index of its first cell;
 *     Eq. 8 weights N_p = (n + 3 f . Omega) dV / M from that cell's inputs;
 *     Eq. 9 states with the random draws keyed by p (as in 1D);
 *   - Eq. 7 with the smallest cell edge: dt = min(C min(dx, dy, dz) / c,
 *     C_F / (kappa max n)).
 * With nx = ny = 1 (and area = Lx Ly) every function here reduces to its 1D
 * counterpart in emu_oracle.c.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "emu_oracle.h"

/* 3D box: the 1D config's physics fields (kappa, c, CFL factors, shape order,
 * vacuum and matter terms; its nz, ndir, Lz are those of the z axis) plus
 * the x and y axes.  Its area field is not used (dV = dx dy dz). */
typedef struct {
  or_config c;
  int32_t nx, ny;
  double Lx, Ly;
} or3_config;

/* One computational particle: position (x, y, z), direction, weights, and
 * the two full 3x3 density matrices. */
typedef struct {
  double x[3];
  double omega[3];
  double N, Nbar;
  cplx rho[3][3];
  cplx rhobar[3][3];
} or3_particle;

static int or3_cells(const or3_config* g) { return g->nx * g->ny * g->c.nz; }

static void or3_dims(const or3_config* g, int32_t n[3], double L[3]) {
  n[0] = g->nx; n[1] = g->ny; n[2] = g->c.nz;
  L[0] = g->Lx; L[1] = g->Ly; L[2] = g->c.Lz;
}

double or3_cell_volume(const or3_config* g) {
  return (g->Lx / g->nx) * (g->Ly / g->ny) * (g->c.Lz / g->c.nz);
}

/* Position mapped into [0, L) on one axis. */
static double or3_wrap_axis(double x, double L) {
  double w = x - L * floor(x / L);
  if (w >= L) w -= L;
  if (w < 0.0) w = 0.0;
  return w;
}

/* 1D shape of order n on an axis of ncell cells of width h (as or_shape):
 * the n+1 cells within the support and their weights.  Returns n+1. */
static int or3_shape_axis(int order, double x, double h, int32_t ncell, int32_t cells[4], double w[4]) {
  double xi = x / h - 0.5;
  long long j0 = (long long)floor(xi - 0.5 * (order + 1)) + 1;
  for (int s = 0; s <= order; ++s) {
    long long j = j0 + s;
    w[s] = or_bspline(order, xi - (double)j);
    long long c = j % ncell;
    if (c < 0) c += ncell;
    cells[s] = (int32_t)c;
  }
  return order + 1;
}

/* Tensor-product shape: up to 64 (cell index, weight) pairs.  Returns the count. */
int or3_shape(const or3_config* g, const double x[3], int32_t cells[64], double w[64]) {
  int32_t n[3]; double L[3];
  or3_dims(g, n, L);
  int32_t c[3][4]; double wa[3][4]; int ns[3];
  for (int a = 0; a < 3; ++a) ns[a] = or3_shape_axis(g->c.shape_order, x[a], L[a] / n[a], n[a], c[a], wa[a]);
  int k = 0;
  for (int i = 0; i < ns[0]; ++i)
    for (int j = 0; j < ns[1]; ++j)
      for (int l = 0; l < ns[2]; ++l) {
        cells[k] = (c[0][i] * g->ny + c[1][j]) * g->c.nz + c[2][l];
        w[k] = wa[0][i] * wa[1][j] * wa[2][l];
        ++k;
      }
  return k;
}

/* Eq. 8 weights and Eq. 9 states, one particle per direction per cell at the
 * cell centre.  Per-cell inputs (length nx ny nz, and x 3 for the fluxes) in
 * cell-index order; dirs M x 3 or NULL (Fibonacci set).  Returns 0, or -1 if
 * a weight is clearly negative (|f| > n/3). */
int or3_init(const or3_config* g, const double* dirs, const double* n_nu, const double* n_nubar,
             const double* f_nu, const double* f_nubar, double alpha, uint64_t seed, or3_particle* parts) {
  const int C = or3_cells(g), M = g->c.ndir;
  const double dx = g->Lx / g->nx, dy = g->Ly / g->ny, dz = g->c.Lz / g->c.nz;
  const double dV = or3_cell_volume(g);
  int bad = 0;
  for (int d = 0; d < M; ++d) {
    double om[3];
    if (dirs) { om[0] = dirs[3 * d]; om[1] = dirs[3 * d + 1]; om[2] = dirs[3 * d + 2]; }
    else or_fibonacci_direction(d, M, om);
    for (int c0 = 0; c0 < C; ++c0) {
      const int jz = c0 % g->c.nz, jy = (c0 / g->c.nz) % g->ny, jx = c0 / (g->c.nz * g->ny);
      const int64_t p = (int64_t)d * C + c0;
      or3_particle* q = &parts[p];
      memset(q, 0, sizeof(*q));
      q->x[0] = (jx + 0.5) * dx;
      q->x[1] = (jy + 0.5) * dy;
      q->x[2] = (jz + 0.5) * dz;
      q->omega[0] = om[0]; q->omega[1] = om[1]; q->omega[2] = om[2];
      double fdo = f_nu[3 * c0] * om[0] + f_nu[3 * c0 + 1] * om[1] + f_nu[3 * c0 + 2] * om[2];
      double fbdo = f_nubar[3 * c0] * om[0] + f_nubar[3 * c0 + 1] * om[1] + f_nubar[3 * c0 + 2] * om[2];
      q->N = (n_nu[c0] + 3.0 * fdo) * dV / M;
      q->Nbar = (n_nubar[c0] + 3.0 * fbdo) * dV / M;
      double tol_nu = 1e-12 * (fabs(n_nu[c0]) + 3.0 * fabs(fdo)) * dV / M;
      double tol_nb = 1e-12 * (fabs(n_nubar[c0]) + 3.0 * fabs(fbdo)) * dV / M;
      if (q->N < 0.0 && q->N >= -tol_nu) q->N = 0.0;
      if (q->Nbar < 0.0 && q->Nbar >= -tol_nb) q->Nbar = 0.0;
      if (q->N < 0.0 || q->Nbar < 0.0) bad = 1;
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

/* Eq. 5 on the 3D grid: every particle adds N w_pj rho (and times Omega) into
 * each cell of its support, divided by dV; the same for antineutrinos. */
void or3_deposit(const or3_config* g, const or3_particle* parts, int64_t P, or_cell* grid) {
  const double dV = or3_cell_volume(g);
  memset(grid, 0, sizeof(or_cell) * (size_t)or3_cells(g));
  for (int64_t p = 0; p < P; ++p) {
    const or3_particle* q = &parts[p];
    int32_t cells[64]; double w[64];
    int ns = or3_shape(g, q->x, cells, w);
    for (int s = 0; s < ns; ++s) {
      or_cell* cell = &grid[cells[s]];
      double cn = q->N * w[s] / dV, cb = q->Nbar * w[s] / dV;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cell->n[a][b] += cn * q->rho[a][b];
          cell->nbar[a][b] += cb * q->rhobar[a][b];
          for (int i = 0; i < 3; ++i) {
            cell->f[i][a][b] += cn * q->rho[a][b] * q->omega[i];
            cell->fbar[i][a][b] += cb * q->rhobar[a][b] * q->omega[i];
          }
        }
    }
  }
}

/* Eq. 6 with the particle's tensor-product weights, then the
 * self-interaction term of Eq. 2 over hbar:
 * H = kappa [(n - nbar^*) - Omega . (f - fbar^*)]. */
void or3_hamiltonian(const or3_config* g, const or_cell* grid, const or3_particle* q, cplx H[3][3]) {
  int32_t cells[64]; double w[64];
  int ns = or3_shape(g, q->x, cells, w);
  cplx n[3][3] = {{0}}, nb[3][3] = {{0}}, f[3][3][3] = {{{0}}}, fb[3][3][3] = {{{0}}};
  for (int s = 0; s < ns; ++s) {
    const or_cell* cell = &grid[cells[s]];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        n[a][b] += w[s] * cell->n[a][b];
        nb[a][b] += w[s] * cell->nbar[a][b];
        for (int i = 0; i < 3; ++i) {
          f[i][a][b] += w[s] * cell->f[i][a][b];
          fb[i][a][b] += w[s] * cell->fbar[i][a][b];
        }
      }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx v = n[a][b] - conj(nb[a][b]);
      for (int i = 0; i < 3; ++i) v -= q->omega[i] * (f[i][a][b] - conj(fb[i][a][b]));
      H[a][b] = g->c.kappa * v;
    }
}

/* Right-hand side of Eq. 4 for every particle at the given state. */
void or3_rhs(const or3_config* g, const or3_particle* parts, int64_t P, or_cell* grid, cplx (*drho)[3][3],
             cplx (*drhobar)[3][3]) {
  or3_deposit(g, parts, P, grid);
  cplx Hvac[3][3] = {{0}}, Hmat[3][3] = {{0}};
  if (g->c.osc_on) or_vacuum_matter(&g->c, Hvac, Hmat);
  for (int64_t p = 0; p < P; ++p) {
    cplx H[3][3], Hb[3][3];
    or3_hamiltonian(g, grid, &parts[p], H);
    or_hamiltonian_bar(H, Hb);
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

/* One classic RK4 step (Sec. 2.3), positions advancing with the stages on
 * every axis (x_i + c_s dt c Omega_i, wrapped).  Returns 0, or -1 if scratch
 * allocation fails. */
int or3_rk4_step(const or3_config* g, or3_particle* parts, int64_t P, double dt) {
  static const double cstage[4] = {0.0, 0.5, 0.5, 1.0};
  int32_t n[3]; double L[3];
  or3_dims(g, n, L);
  or3_particle* ystage = malloc(sizeof(or3_particle) * (size_t)P);
  or_cell* grid = malloc(sizeof(or_cell) * (size_t)or3_cells(g));
  cplx (*kr)[3][3] = malloc(sizeof(cplx) * 9 * 4 * (size_t)P);
  cplx (*kb)[3][3] = malloc(sizeof(cplx) * 9 * 4 * (size_t)P);
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
        for (int i = 0; i < 3; ++i)
          ystage[p].x[i] = or3_wrap_axis(parts[p].x[i] + cstage[s] * dt * g->c.c_light * parts[p].omega[i], L[i]);
      }
    }
    or3_rhs(g, ystage, P, grid, kr + s * P, kb + s * P);
  }
  for (int64_t p = 0; p < P; ++p) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        parts[p].rho[a][b] += dt / 6.0 * (kr[p][a][b] + 2.0 * kr[P + p][a][b] + 2.0 * kr[2 * P + p][a][b] +
                                          kr[3 * P + p][a][b]);
        parts[p].rhobar[a][b] += dt / 6.0 * (kb[p][a][b] + 2.0 * kb[P + p][a][b] + 2.0 * kb[2 * P + p][a][b] +
                                             kb[3 * P + p][a][b]);
      }
    for (int i = 0; i < 3; ++i)
      parts[p].x[i] = or3_wrap_axis(parts[p].x[i] + dt * g->c.c_light * parts[p].omega[i], L[i]);
  }
  free(ystage); free(grid); free(kr); free(kb);
  return 0;
}

int or3_run(const or3_config* g, or3_particle* parts, int64_t P, double dt, int64_t nsteps) {
  for (int64_t n = 0; n < nsteps; ++n)
    if (or3_rk4_step(g, parts, P, dt) != 0) return -1;
  return 0;
}

/* Eq. 7 with the smallest cell edge and the maximum over cells and diagonal
 * components of n, nbar (and the lepton density with the matter term). */
double or3_timestep(const or3_config* g, const or_cell* grid) {
  double nmax = g->c.osc_on ? g->c.n_e : 0.0;
  for (int j = 0; j < or3_cells(g); ++j)
    for (int a = 0; a < 3; ++a) {
      if (creal(grid[j].n[a][a]) > nmax) nmax = creal(grid[j].n[a][a]);
      if (creal(grid[j].nbar[a][a]) > nmax) nmax = creal(grid[j].nbar[a][a]);
    }
  double h = g->Lx / g->nx;
  if (g->Ly / g->ny < h) h = g->Ly / g->ny;
  if (g->c.Lz / g->c.nz < h) h = g->c.Lz / g->c.nz;
  double dt_adv = g->c.cfl_adv * h / g->c.c_light;
  double dt_flav = nmax > 0.0 ? g->c.cfl_flavor / (g->c.kappa * nmax) : dt_adv;
  return dt_adv < dt_flav ? dt_adv : dt_flav;
}

int32_t or3_sizeof_particle(void) { return (int32_t)sizeof(or3_particle); }
int32_t or3_sizeof_config(void) { return (int32_t)sizeof(or3_config); }
