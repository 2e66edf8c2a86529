// kernels3d.cuh -- GB300 (sm_103a) FP64 device code of the particle-in-cell step
// on a 3D periodic grid (the paper's method, Eq. 2, 4-6 and Sec. 2.3, on the 3D
// grid it names as future work in Sec. 5).  Included once, by emu.cu, after
// kernels.cuh, whose helpers (shape weights, Spread, gather, commutator,
// rk_particle, k_combine) it reuses.
//
// A 3D box has nx x ny x nz cells (index c = (jx ny + jy) nz + jz; a *row* is
// the nz cells of one (jx, jy)) and M directions; particle p = d C + site,
// C = nx ny nz, starts at the centre of cell `site` (one particle per direction
// per cell, Sec. 3.1).  The particles of one direction translate rigidly
// (constant velocity c Omega, Eq. 4), so they stay a lattice: the particle on
// cell (jx, jy, jz) is the one of site (jx - sx_d, jy - sy_d, jz - sz_d) (mod
// the cell counts), with one shift per axis, direction and RK stage.  The
// generic kernels (k3_deposit, k3_interpolate) use each particle's own position
// for its weights, checked against the cell its site assigns (ERR_LATTICE
// otherwise).
//
// Shape: the tensor product of the 1D shape of order ORDER on each axis, so
// a particle reaches (2H+1)^3 cells.  Work units are (row, z tile of T cells,
// direction), rows outer, directions inner; a warp's lanes are the cells of
// its tile (with H halo lanes a side, as in 1D).
//   deposit (Eq. 5): for each of the (2H+1)^2 rows next to its own, the warp
//     loads the particles of that row (its lanes' z cells), forms x-weight x
//     y-weight toward its own row times B_p, and spreads that along z with the
//     particles' z-weights through shuffles; the sum over neighbour rows and
//     directions stays in registers and goes out as one partial per (warp,
//     row tile), added in warp order by k_combine (each row is one "box" of
//     that kernel's batch view);
//   interpolation (Eq. 6): the same gather transposed.
// The step itself is separable: all particles of a direction sit at the same
// offset inside their cells (up to rounding), so their weights on each axis
// are the direction's (k3_shifts computes them from the site-0 particle), and
// the deposit of one direction is a 3-tap convolution along z, then y, then x
// of its B field (k3_spread), summed over directions with (1, Omega) into the
// potential (k3_spread_x_sum); the interpolation of G = A0 - Omega . A is the
// transposed convolution (k3_gather along x and y, then z by shuffles in
// k3_rk_stage).  Three 3-tap passes per direction and cell instead of a
// (2H+1)^2-row gather per particle.
#pragma once

namespace emu_dev {

struct Box3 {
  int n[3];            // cells per axis (x, y, z)
  int M, C, R;         // directions, cells, rows (nx ny)
  int ntz, T;          // z tiles per row, cells per tile
  int nw;              // warps that split the units
  int ntz32, nw32;     // the RK stage's 32-cell z tiles per row, warps that split its units
  int64_t U32;         // its units (R ntz32 M)
  int use_dirs;
  int64_t U, P;        // units (R ntz M), particles (M C)
  double L[3], inv_h[3], n_d[3], h[3];
  double kappa_dV, inv_dV, c_light;
  double alpha;
  uint64_t seed;
  const double* dt;    // the box's step size (device)
  const BoxGeo* g;     // device copy: vacuum and matter terms (vnu, vnubar) and Lz, for rk_particle
};

__device__ __forceinline__ int64_t unit3_begin(int64_t w, const Box3& b) { return w >= b.nw ? b.U : w * b.U / b.nw; }

__device__ __forceinline__ int wrapn(int j, int n) {
  int r = j % n;
  return r < 0 ? r + n : r;
}

// w[i] for a run-time i, by selects (no indexed access to a register array).
template <int NW>
__device__ __forceinline__ double pick(const double (&w)[NW], int i) {
  double v = w[0];
#pragma unroll
  for (int k = 1; k < NW; ++k) v = i == k ? w[k] : v;
  return v;
}

// Direction table ([6][M]: Omega, then c Omega) from each direction's site-0
// particle; every particle of a direction must carry its direction.
__global__ void k3_dirtable(Box3 b, Parts pt, double* __restrict__ dirtab, int* __restrict__ err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= b.P) return;
  const int d = (int)(p / b.C);
  const int64_t p0 = (int64_t)d * b.C;
  const double ox = pt.ox[p0], oy = pt.oy[p0], oz = pt.oz[p0];
  if (pt.ox[p] != ox || pt.oy[p] != oy || pt.oz[p] != oz) atomicOr(err, ERR_RING);
  if (p == p0) {
    dirtab[d] = ox;
    dirtab[b.M + d] = oy;
    dirtab[2 * b.M + d] = oz;
    dirtab[3 * b.M + d] = b.c_light * ox;
    dirtab[4 * b.M + d] = b.c_light * oy;
    dirtab[5 * b.M + d] = b.c_light * oz;
  }
}

// Lattice shifts of every direction for up to 4 position offsets frac[s] dt:
// the cell, on each axis, of the direction's site-0 particle at x + frac dt c
// Omega; shift[(s * 3 + axis) * M + d].  With wtab, also that particle's
// shape weights there, the direction's weights on each axis (all its
// particles share the offset inside their cells): wtab[((s * 3 + axis) * 5 +
// q) * M + d], q < NW.
template <int ORDER>
__global__ void k3_shifts(Box3 b, const double* __restrict__ x, const double* __restrict__ y,
                          const double* __restrict__ z, const double* __restrict__ dirtab, Fracs fr, int nrows,
                          int* __restrict__ shift, double* __restrict__ wtab) {
  griddep_wait();
  constexpr int NW = Sten<ORDER>::NW;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= b.M) return;
  const int64_t p0 = (int64_t)d * b.C;
  const double pos[3] = {x[p0], y[p0], z[p0]};
  const double dt = *b.dt;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s >= nrows) break;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double xs = fma(fr.v[s] * dt, dirtab[(3 + a) * b.M + d], pos[a]);
      const int cell = wrapn((int)floor(xs * b.inv_h[a]), b.n[a]);
      shift[(s * 3 + a) * b.M + d] = cell;
      if (wtab != nullptr) {
        double w[NW];
        (void)shape_weights<ORDER>(xs, (double)cell + 0.5, b.inv_h[a], b.n_d[a], w);
#pragma unroll
        for (int q = 0; q < NW; ++q) wtab[((s * 3 + a) * 5 + q) * b.M + d] = w[q];
      }
    }
  }
}

// Site of the particle of direction d on cell (jx, jy, jz) for shifts (sx, sy, sz).
__device__ __forceinline__ int64_t site3(const Box3& b, int d, int jx, int jy, int jz, int sx, int sy, int sz) {
  const int ix = wrapn(jx - sx, b.n[0]), iy = wrapn(jy - sy, b.n[1]), iz = wrapn(jz - sz, b.n[2]);
  return (int64_t)d * b.C + ((int64_t)ix * b.n[1] + iy) * b.n[2] + iz;
}

// Deposit (Eq. 5) on the 3D grid, first phase.  MODE as k_deposit: 0 the
// potential's B = N rho - Nbar rhobar^* (36 rows), 1 N rho, 2 Nbar rhobar,
// 4 the diagnostics' n, f_x, nbar, fbar_x.
// Positions x + frac dt c Omega.  srow: the shift rows (3 x M) of these positions.
template <int MODE, int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k3_deposit(Box3 b, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
           const double* __restrict__ N, const double* __restrict__ Nbar, const double* __restrict__ r_nu,
           const double* __restrict__ r_nb, const double* __restrict__ dirtab, const int* __restrict__ srow,
           double frac, double* __restrict__ partial, int* __restrict__ err) {
  griddep_wait();
  constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T, NW = Sten<ORDER>::NW;
  constexpr int NA = kNA;
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int64_t u0 = unit3_begin(w, b), u1 = unit3_begin(w + 1, b);
  if (u0 >= u1) return;
  const int64_t P = b.P;
  const int M = b.M, nx = b.n[0], ny = b.n[1], nz = b.n[2];
  const double pos_dt = frac * *b.dt;
  int bad = 0;
  for (int64_t u = u0; u < u1;) {          // one segment per (row, tile)
    const int64_t gtile = u / M;
    const int row = (int)(gtile / b.ntz), tile = (int)(gtile - (int64_t)row * b.ntz);
    const int jx = row / ny, jy = row - jx * ny;
    const int dfirst = (int)(u - gtile * M);
    const int64_t uend = min(u1, (gtile + 1) * M);
    const int dlast = (int)(uend - gtile * M);
    u = uend;
    const int craw = tile * T - H + lane;
    const int jz = wrapc(craw, nz);
    double acc[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) acc[c] = 0.0;
    for (int d = dfirst; d < dlast; ++d) {
      const double ox = __ldg(dirtab + d), oy = __ldg(dirtab + M + d), oz = __ldg(dirtab + 2 * M + d);
      const double vx = __ldg(dirtab + 3 * M + d), vy = __ldg(dirtab + 4 * M + d), vz = __ldg(dirtab + 5 * M + d);
      const int sx = __ldg(srow + d), sy = __ldg(srow + M + d), sz = __ldg(srow + 2 * M + d);
      constexpr int NS = MODE == 4 ? 18 : 9;   // components summed over neighbour rows
      double S[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) S[c] = 0.0;
#pragma unroll 1
      for (int a = -H; a <= H; ++a) {
#pragma unroll 1
        for (int bb = -H; bb <= H; ++bb) {
          if (ORDER == 0 && (a != 0 || bb != 0)) continue;
          const int sjx = wrapn(jx + a, nx), sjy = wrapn(jy + bb, ny);   // the source row's cell
          const int64_t p = site3(b, d, sjx, sjy, jz, sx, sy, sz);
          double wx[NW], wy[NW], wz[NW];
          bad |= shape_weights<ORDER>(fma(pos_dt, vx, __ldg(x + p)), (double)sjx + 0.5, b.inv_h[0], b.n_d[0], wx);
          bad |= shape_weights<ORDER>(fma(pos_dt, vy, __ldg(y + p)), (double)sjy + 0.5, b.inv_h[1], b.n_d[1], wy);
          bad |= shape_weights<ORDER>(fma(pos_dt, vz, __ldg(z + p)), (double)jz + 0.5, b.inv_h[2], b.n_d[2], wz);
          const double f = pick(wx, H - a) * pick(wy, H - bb);   // this particle's share of the warp's row
          Spread<ORDER> spread;
          spread.init(wz);
          if constexpr (MODE == 4) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              S[k] += spread.apply(f * __ldg(N + p) * __ldg(r_nu + k * P + p));
              S[9 + k] += spread.apply(f * __ldg(Nbar + p) * __ldg(r_nb + k * P + p));
            }
          } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              const double n1 = (MODE == 0 || MODE == 1) ? f * __ldg(N + p) : 0.0;
              const double n2 = (MODE == 0 || MODE == 2) ? f * __ldg(Nbar + p) : 0.0;
              double bv;
              if (MODE == 0) {
                const double xv = __ldg(r_nu + k * P + p), yv = __ldg(r_nb + k * P + p);
                bv = (k == 4 || k == 6 || k == 8) ? fma(n2, yv, n1 * xv) : fma(-n2, yv, n1 * xv);
              } else if (MODE == 1) {
                bv = n1 * __ldg(r_nu + k * P + p);
              } else {
                bv = n2 * __ldg(r_nb + k * P + p);
              }
              S[k] += spread.apply(bv);
            }
          }
        }
      }
      // moments of this direction: (1, Omega) x S (Omega is the direction's)
      if constexpr (MODE == 4) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          acc[k] += S[k];
          acc[9 + k] = fma(ox, S[k], acc[9 + k]);
          acc[18 + k] += S[9 + k];
          acc[27 + k] = fma(ox, S[9 + k], acc[27 + k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          acc[k] += S[k];
          acc[9 + k] = fma(ox, S[k], acc[9 + k]);
          acc[18 + k] = fma(oy, S[k], acc[18 + k]);
          acc[27 + k] = fma(oz, S[k], acc[27 + k]);
        }
      }
    }
    flush_tile<ORDER>(acc, gtile, craw, nz, w, lane, partial);
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// The step's deposit (MODE 5 of k3_deposit), separable.  k3_prep: one thread
// per particle; checks its position against the cell its site assigns at the
// stage (ERR_LATTICE) and writes the 8 traceless components of
// B = N rho - Nbar rhobar^* (Eq. 5) at that cell of its direction's field:
// Bf[c * P + d * C + cell].
__global__ void __launch_bounds__(kThreads)
k3_prep(Box3 b, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
        const double* __restrict__ N, const double* __restrict__ Nbar, const double* __restrict__ r_nu,
        const double* __restrict__ r_nb, const double* __restrict__ dirtab, const int* __restrict__ srow,
        double frac, double* __restrict__ Bf, int* __restrict__ err) {
  griddep_wait();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= b.P) return;
  const int64_t P = b.P;
  const int M = b.M;
  const int d = (int)(p / b.C);
  const int c0 = (int)(p - (int64_t)d * b.C);
  const int iz = c0 % b.n[2], iy = (c0 / b.n[2]) % b.n[1], ix = c0 / (b.n[2] * b.n[1]);
  const int jx = wrapn(ix + __ldg(srow + d), b.n[0]);
  const int jy = wrapn(iy + __ldg(srow + M + d), b.n[1]);
  const int jz = wrapn(iz + __ldg(srow + 2 * M + d), b.n[2]);
  const double pos_dt = frac * *b.dt;
  int bad = off_site(fma(pos_dt, __ldg(dirtab + 3 * M + d), x[p]), (double)jx + 0.5, b.inv_h[0], b.n_d[0]);
  bad |= off_site(fma(pos_dt, __ldg(dirtab + 4 * M + d), y[p]), (double)jy + 0.5, b.inv_h[1], b.n_d[1]);
  bad |= off_site(fma(pos_dt, __ldg(dirtab + 5 * M + d), z[p]), (double)jz + 0.5, b.inv_h[2], b.n_d[2]);
  const int64_t out = (int64_t)d * b.C + ((int64_t)jx * b.n[1] + jy) * b.n[2] + jz;
  const double n1 = N[p], n2 = Nbar[p];
  double bprev = 0.0;
#pragma unroll
  for (int c = 0; c < kNC; ++c) {
    double bv;
    if (c < 2) {
      if (c == 0) bprev = fma(-n2, r_nb[p], n1 * r_nu[p]);
      const double bn = fma(-n2, r_nb[(c + 1) * P + p], n1 * r_nu[(c + 1) * P + p]);
      bv = bprev - bn;
      bprev = bn;
    } else {
      const int k = c + 1;
      const double xv = r_nu[k * P + p], yv = r_nb[k * P + p];
      bv = (k == 4 || k == 6 || k == 8) ? fma(n2, yv, n1 * xv) : fma(-n2, yv, n1 * xv);
    }
    Bf[c * P + out] = bv;
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// Neighbour of cell (jx, jy, jz) at offset o along AXIS (periodic).
template <int AXIS>
__device__ __forceinline__ int64_t cell_along(const Box3& b, int jx, int jy, int jz, int o) {
  if (AXIS == 0) jx = wrapn(jx + o, b.n[0]);
  else if (AXIS == 1) jy = wrapn(jy + o, b.n[1]);
  else jz = wrapn(jz + o, b.n[2]);
  return ((int64_t)jx * b.n[1] + jy) * b.n[2] + jz;
}

// One 3-tap (NW-tap) pass along AXIS of the 8-component field of every
// direction, thread per (direction, cell) i = d C + cell:
//   SPREAD (deposit, Eq. 5): out(cell) = sum_q w_d[q] in(cell - (q - H))
//     (a particle's weight q goes to the cell q - H away from its own);
//   otherwise (interpolation, Eq. 6): out(cell) = sum_q w_d[q] in(cell + q - H).
// w_d: the direction's weights on AXIS at the stage (wrow = wtab + stage rows).
template <int ORDER, int AXIS, bool SPREAD>
__global__ void __launch_bounds__(kThreads)
k3_pass(Box3 b, const double* __restrict__ in, const double* __restrict__ wrow, double* __restrict__ out) {
  griddep_wait();
  constexpr int H = Sten<ORDER>::H, NW = Sten<ORDER>::NW;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t P = b.P;
  if (i >= P) return;
  const int d = (int)(i / b.C);
  const int cell = (int)(i - (int64_t)d * b.C);
  const int jz = cell % b.n[2], jy = (cell / b.n[2]) % b.n[1], jx = cell / (b.n[2] * b.n[1]);
  const double* src = in + (int64_t)d * b.C;
  double w[NW];
  int64_t nb[NW];
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    w[q] = __ldg(wrow + ((AXIS * 5) + q) * b.M + d);
    nb[q] = cell_along<AXIS>(b, jx, jy, jz, SPREAD ? H - q : q - H);
  }
#pragma unroll
  for (int c = 0; c < kNC; ++c) {
    const double* sc = src + c * P;
    double v = w[0] * __ldg(sc + nb[0]);
#pragma unroll
    for (int q = 1; q < NW; ++q) v = fma(w[q], __ldg(sc + nb[q]), v);
    out[c * P + i] = v;
  }
}

// The last deposit pass: along x, summed over directions in order with
// (1, Omega_x, Omega_y, Omega_z) into the traceless potential (thread per
// cell): At[(m * 8 + c) * C + cell] = kappa / dV sum_d Omega~_m,d (the
// direction's x-spread of its y- and z-spread B field).  No partial sums.
template <int ORDER>
__global__ void __launch_bounds__(kThreads)
k3_spread_x_sum(Box3 b, const double* __restrict__ in, const double* __restrict__ wrow,
                const double* __restrict__ dirtab, double* __restrict__ At, int* __restrict__ err) {
  griddep_wait();
  constexpr int H = Sten<ORDER>::H, NW = Sten<ORDER>::NW;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= b.C) return;
  const int64_t P = b.P;
  const int M = b.M;
  const int jz = cell % b.n[2], jy = (cell / b.n[2]) % b.n[1], jx = cell / (b.n[2] * b.n[1]);
  int64_t nb[NW];
#pragma unroll
  for (int q = 0; q < NW; ++q) nb[q] = cell_along<0>(b, jx, jy, jz, H - q);
  double acc[kNT];
#pragma unroll
  for (int c = 0; c < kNT; ++c) acc[c] = 0.0;
  for (int d = 0; d < M; ++d) {
    const double ox = __ldg(dirtab + d), oy = __ldg(dirtab + M + d), oz = __ldg(dirtab + 2 * M + d);
    double w[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) w[q] = __ldg(wrow + q * M + d);
    const double* src = in + (int64_t)d * b.C;
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const double* sc = src + c * P;
      double v = w[0] * __ldg(sc + nb[0]);
#pragma unroll
      for (int q = 1; q < NW; ++q) v = fma(w[q], __ldg(sc + nb[q]), v);
      acc[c] += v;
      acc[kNC + c] = fma(ox, v, acc[kNC + c]);
      acc[2 * kNC + c] = fma(oy, v, acc[2 * kNC + c]);
      acc[3 * kNC + c] = fma(oz, v, acc[3 * kNC + c]);
    }
  }
  int bad = 0;
#pragma unroll
  for (int c = 0; c < kNT; ++c) {
    const double v = acc[c] * b.kappa_dV;
    bad |= !isfinite(v);
    At[(int64_t)c * b.C + cell] = v;
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

// G = A0 - Omega_d . A of every (direction, cell) from the traceless
// potential, once per stage: Gf[c][d][cell] (component c, M C values each).
// The RK stage's interpolation reads the G of its neighbour rows instead of
// forming it for each of the (2H+1)^2 rows that need it.
__global__ void __launch_bounds__(kThreads)
k3_gfield(Box3 b, const double* __restrict__ At, const double* __restrict__ dirtab, double* __restrict__ Gf) {
  griddep_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t MC = (int64_t)b.M * b.C;
  if (i >= MC) return;
  const int d = (int)(i / b.C);
  const int64_t cell = i - (int64_t)d * b.C;
  const double ox = __ldg(dirtab + d), oy = __ldg(dirtab + b.M + d), oz = __ldg(dirtab + 2 * b.M + d);
  const double* Aj = At + cell;
  const int64_t Cn = b.C;
#pragma unroll
  for (int c = 0; c < kNC; ++c)
    Gf[c * MC + i] = fma(-oz, Aj[(3 * kNC + c) * Cn],
                         fma(-oy, Aj[(2 * kNC + c) * Cn], fma(-ox, Aj[(kNC + c) * Cn], Aj[c * Cn])));
}

// H of the lane's particle (traceless components, Eq. 6 then Eq. 2): its
// x- and y-weights over the neighbour rows times the z-interpolation of
// G = A0 - Omega . A along each row.  Every lane must call it.
template <int ORDER, int NCOMP>
__device__ __forceinline__ void interp3(const Box3& b, const double* A, int jx, int jy, int jz, double ox, double oy,
                                        double oz, const double (&wx)[Sten<ORDER>::NW],
                                        const double (&wy)[Sten<ORDER>::NW], const double (&wz)[Sten<ORDER>::NW],
                                        double (&Hm)[NCOMP]) {
  constexpr int H = Sten<ORDER>::H;
  const int64_t Cn = b.C;
#pragma unroll
  for (int c = 0; c < NCOMP; ++c) Hm[c] = 0.0;
#pragma unroll 1
  for (int a = -H; a <= H; ++a) {
#pragma unroll 1
    for (int bb = -H; bb <= H; ++bb) {
      if (ORDER == 0 && (a != 0 || bb != 0)) continue;
      const int row = wrapn(jx + a, b.n[0]) * b.n[1] + wrapn(jy + bb, b.n[1]);
      const double* Aj = A + (int64_t)row * b.n[2] + jz;
      const double wab = pick(wx, H + a) * pick(wy, H + bb);
#pragma unroll
      for (int c = 0; c < NCOMP; ++c) {
        const double G = fma(-oz, __ldg(Aj + (3 * NCOMP + c) * Cn),
                             fma(-oy, __ldg(Aj + (2 * NCOMP + c) * Cn),
                                 fma(-ox, __ldg(Aj + (NCOMP + c) * Cn), __ldg(Aj + c * Cn))));
        Hm[c] = fma(wab, gather<ORDER>(wz, G), Hm[c]);
      }
    }
  }
}

// One RK4 stage s (1..4) on the 3D grid after the deposit of the stage state
// (as k_rk_stage): H from Gxy (G = A0 - Omega . A interpolated along x and y
// by k3_pass) interpolated along z with the direction's z-weights, H and Hbar,
// commutators, RK update; stage 4 also moves the particle on every axis (dry:
// the results of stage 4 go to the RK scratch, for the autotuner's timing).
// Units are (row, 32-cell z tile, direction), every lane on its own cell: the
// z neighbours' G come from the field in memory (L1), not from halo lanes, so
// no lane idles except past the end of a row.
template <bool POT, int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k3_rk_stage(Box3 b, Parts pt, double* __restrict__ x, double* __restrict__ y, const double* __restrict__ dirtab,
            const int* __restrict__ srow, const double* __restrict__ Gxy, const double* __restrict__ wrow, int s,
            int dry) {
  griddep_wait();
  constexpr int H = Sten<ORDER>::H, NW = Sten<ORDER>::NW;
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int64_t u0 = w >= b.nw32 ? b.U32 : w * b.U32 / b.nw32, u1 = w + 1 >= b.nw32 ? b.U32 : (w + 1) * b.U32 / b.nw32;
  if (u0 >= u1) return;
  const int64_t P = b.P;
  const int M = b.M, ny = b.n[1], nz = b.n[2];
  const double dt = *b.dt;
  const double bdt = (s == 1 || s == 4) ? dt / 6.0 : dt / 3.0;
  const double cdt = (s == 3) ? dt : 0.5 * dt;
  const double* src_b = (s == 1) ? pt.rhobar : pt.stage + 9 * P;
  const double* src_r = (s == 1) ? pt.rho : pt.stage;
  for (int64_t u = u0; u < u1; ++u) {
    const int64_t gtile = u / M;
    const int d = (int)(u - gtile * M);
    const int row = (int)(gtile / b.ntz32), tile = (int)(gtile - (int64_t)row * b.ntz32);
    const int jx = row / ny, jy = row - jx * ny;
    const int jz = tile * kLanes + lane;
    if (jz >= nz) continue;
    const double vx = __ldg(dirtab + 3 * M + d), vy = __ldg(dirtab + 4 * M + d);
    const int64_t p = site3(b, d, jx, jy, jz, __ldg(srow + d), __ldg(srow + M + d), __ldg(srow + 2 * M + d));
    double wz[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) wz[q] = __ldg(wrow + (2 * 5 + q) * M + d);
    const double* G = Gxy + (int64_t)d * b.C + (int64_t)row * nz;
    int cz[NW];   // the stencil's z cells, cell jz + q - H (periodic)
#pragma unroll
    for (int q = 0; q < NW; ++q) cz[q] = wrapn(jz + q - H, nz);
    double Hm[kNC];
#pragma unroll
    for (int c = 0; c < kNC; ++c) {   // (the taps in gather's order)
      const double* Gc = G + c * P;
      double h = wz[NW - 1] * __ldg(Gc + cz[NW - 1]);
#pragma unroll
      for (int q = NW - 2; q >= 0; --q) h = fma(wz[q], __ldg(Gc + cz[q]), h);
      Hm[c] = h;
    }
    double r[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) r[k] = src_r[k * P + p];
    rk_particle<POT, false>(*b.g, pt, src_b, P, p, s, dry, bdt, cdt, dt, dirtab + 5 * M + d, Hm, r);
    if (s == 4) {   // x and y move as z does (rk_particle moved z; dry: into the RK scratch)
      const double xn = wrap_z(fma(dt, vx, x[p]), b.L[0]), yn = wrap_z(fma(dt, vy, y[p]), b.L[1]);
      if (dry) { pt.acc[p] = xn; pt.acc[P + p] = yn; }
      else { x[p] = xn; y[p] = yn; }
    }
  }
}

// Interpolation only (Eq. 6 then Eq. 2) of the full 36-row potential A at the
// particles' positions x + frac dt c Omega: H[k * P + p], 9 packed components.
template <int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k3_interpolate(Box3 b, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
               const double* __restrict__ dirtab, const int* __restrict__ srow, const double* __restrict__ A,
               double frac, double* __restrict__ Hout, int* __restrict__ err) {
  constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T, NW = Sten<ORDER>::NW;
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int64_t u0 = unit3_begin(w, b), u1 = unit3_begin(w + 1, b);
  if (u0 >= u1) return;
  const int64_t P = b.P;
  const int M = b.M, ny = b.n[1], nz = b.n[2];
  const double pos_dt = frac * *b.dt;
  int bad = 0;
  for (int64_t u = u0; u < u1; ++u) {
    const int64_t gtile = u / M;
    const int d = (int)(u - gtile * M);
    const int row = (int)(gtile / b.ntz), tile = (int)(gtile - (int64_t)row * b.ntz);
    const int jx = row / ny, jy = row - jx * ny;
    const int craw = tile * T - H + lane, jz = wrapc(craw, nz);
    const bool active = lane >= H && lane < H + T && craw < nz;
    const double ox = __ldg(dirtab + d), oy = __ldg(dirtab + M + d), oz = __ldg(dirtab + 2 * M + d);
    const int64_t p = site3(b, d, jx, jy, jz, __ldg(srow + d), __ldg(srow + M + d), __ldg(srow + 2 * M + d));
    double wx[NW], wy[NW], wz[NW];
    bad |= shape_weights<ORDER>(fma(pos_dt, __ldg(dirtab + 3 * M + d), x[p]), (double)jx + 0.5, b.inv_h[0],
                                b.n_d[0], wx);
    bad |= shape_weights<ORDER>(fma(pos_dt, __ldg(dirtab + 4 * M + d), y[p]), (double)jy + 0.5, b.inv_h[1],
                                b.n_d[1], wy);
    bad |= shape_weights<ORDER>(fma(pos_dt, __ldg(dirtab + 5 * M + d), z[p]), (double)jz + 0.5, b.inv_h[2],
                                b.n_d[2], wz);
    double Hf[9];
    interp3<ORDER, 9>(b, A, jx, jy, jz, ox, oy, oz, wx, wy, wz, Hf);
    if (active) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Hout[k * P + p] = Hf[k];
    }
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// Initial particles on the 3D lattice (Sec. 3.1, Eq. 8, 9; as k_init):
// particle p = d C + c0 at the centre of cell c0.  species: n_nu[C],
// n_nubar[C], f_nu[3C], f_nubar[3C]; dirs[3M] (with use_dirs).
__global__ void k3_init(Box3 b, Parts pt, double* __restrict__ x, double* __restrict__ y,
                        const double* __restrict__ species, const double* __restrict__ dirs, int* __restrict__ err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= b.P) return;
  const int d = (int)(p / b.C), c0 = (int)(p % b.C);
  const int jz = c0 % b.n[2], jy = (c0 / b.n[2]) % b.n[1], jx = c0 / (b.n[2] * b.n[1]);
  double o[3];
  if (b.use_dirs) {
    o[0] = dirs[3 * d]; o[1] = dirs[3 * d + 1]; o[2] = dirs[3 * d + 2];
  } else {
    const double mu = __dsub_rn(1.0, __ddiv_rn(__dadd_rn(__dmul_rn(2.0, (double)d), 1.0), (double)b.M));
    const double phi = __dmul_rn(__dmul_rn((double)d, 3.14159265358979323846), __dsub_rn(3.0, sqrt(5.0)));
    const double sn = sqrt(__dsub_rn(1.0, __dmul_rn(mu, mu)));
    o[0] = __dmul_rn(sn, cos(phi));
    o[1] = __dmul_rn(sn, sin(phi));
    o[2] = mu;
  }
  x[p] = __dmul_rn(__dadd_rn((double)jx, 0.5), b.h[0]);
  y[p] = __dmul_rn(__dadd_rn((double)jy, 0.5), b.h[1]);
  pt.z[p] = __dmul_rn(__dadd_rn((double)jz, 0.5), b.h[2]);
  pt.ox[p] = o[0]; pt.oy[p] = o[1]; pt.oz[p] = o[2];
  const int64_t C = b.C;
  const double dV = __dmul_rn(__dmul_rn(b.h[0], b.h[1]), b.h[2]);
  double wgt[2];
  for (int sp = 0; sp < 2; ++sp) {
    const double n = species[sp * C + c0];
    const double* f = species + 2 * C + sp * 3 * C + 3 * (int64_t)c0;
    const double fdo = __dadd_rn(__dadd_rn(__dmul_rn(f[0], o[0]), __dmul_rn(f[1], o[1])), __dmul_rn(f[2], o[2]));
    double wt = __ddiv_rn(__dmul_rn(__dadd_rn(n, __dmul_rn(3.0, fdo)), dV), (double)b.M);
    const double tol = 1e-12 * (fabs(n) + 3.0 * fabs(fdo)) * dV / b.M;
    if (wt < 0.0 && wt >= -tol) wt = 0.0;
    if (wt < 0.0) atomicOr(err, ERR_WEIGHT);
    wgt[sp] = wt;
  }
  pt.N[p] = wgt[0];
  pt.Nbar[p] = wgt[1];
  const int64_t P = b.P;
  for (int sp = 0; sp < 2; ++sp) {
    double* r = sp ? pt.rhobar : pt.rho;
    const double emr = __dmul_rn(b.alpha, uniform_pm1(b.seed, p, 4 * sp + 0));
    const double emi = __dmul_rn(b.alpha, uniform_pm1(b.seed, p, 4 * sp + 1));
    const double etr = __dmul_rn(b.alpha, uniform_pm1(b.seed, p, 4 * sp + 2));
    const double eti = __dmul_rn(b.alpha, uniform_pm1(b.seed, p, 4 * sp + 3));
    const double eps_mu = __dadd_rn(__dmul_rn(emr, emr), __dmul_rn(emi, emi));
    const double eps_tau = __dadd_rn(__dmul_rn(etr, etr), __dmul_rn(eti, eti));
    r[0 * P + p] = __dsub_rn(__dsub_rn(1.0, eps_mu), eps_tau);
    r[1 * P + p] = eps_mu;
    r[2 * P + p] = eps_tau;
    r[3 * P + p] = emr;
    r[4 * P + p] = emi;
    r[5 * P + p] = etr;
    r[6 * P + p] = eti;
    r[7 * P + p] = 0.0;
    r[8 * P + p] = 0.0;
  }
}

}  // namespace emu_dev
