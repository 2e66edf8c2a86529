// emu.cu -- GB300 (sm_103a) FP64 kernels and C ABI of the particle-in-cell step
// for the neutrino fast flavour instability (Richers, Willcox, Ford & Myers,
// arXiv:2101.02745).  Declarations and conventions: include/emu.h.
//
// Data layout (structure of arrays, FP64):
//   particle p = d * nz + i  (direction d, ring index i); matrix component k at [k * P + p]
//   grid potential A[c * nz + j], c = 0..35 (A0, A_x, A_y, A_z; 9 packed components each)
//
// Parallel layout.  A block covers a tile of kTile = 30 consecutive cells and a
// chunk of directions; each of its 8 warps walks its directions one at a time
// with lane l on cell (tile * 30 - 1 + l).  Lanes 1..30 own the tile's cells;
// lanes 0 and 31 are halo lanes that supply the neighbour values every
// three-cell stencil needs.  Because the particles of one direction form a
// rigidly translating lattice (one per cell at a common offset, Sec. 3.1 and
// Eq. 4), the particle whose lattice site is cell j sits at ring index
// (j - shift_d) mod nz, and its two stencil neighbours are the particles of the
// adjacent lanes: both the deposit (Eq. 5) and the interpolation (Eq. 6) become
// warp-shuffle gathers, with no atomics and a fixed summation order.
//
// The deposit sums over directions in registers (fixed order per lane), then
// across the block's warps in shared memory (fixed order), then across
// direction chunks (fixed order, done by the last block of each tile to
// finish, found with an integer atomic ticket).  Results are therefore
// bitwise reproducible from run to run for a given (nz, ndir).
#include "emu.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <mutex>
#include <vector>

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kLanes = 32;
constexpr int kTile = 30;         // cells owned by a warp row (lanes 1..30)
constexpr int kNA = 36;           // components of the grid potential
constexpr int kNM = 72;           // components of the per-species moments
constexpr int kTargetBlocks = 4 * 152;  // 4 resident blocks on each of GB300's 152 SMs
constexpr double kLatticeTol = 1e-6;    // allowed distance from the lattice site, in cells
constexpr unsigned kFull = 0xffffffffu;
// Persistent schedule of the step kernels: a fixed grid of 2 blocks per SM
// (the kernels use up to 128 registers per thread), whose warps split the
// U = ntiles * ndir warp-units (one cell tile x one direction) into equal
// contiguous ranges.  The split depends only on (nz, ndir), never on the
// device, so the deposit's summation order is fixed.
constexpr int kPersistBlocks = 2 * 152;
constexpr int kPersistWarps = kPersistBlocks * kWarps;

enum : int { ERR_LATTICE = 1, ERR_NONFINITE = 2, ERR_WEIGHT = 4, ERR_RING = 8 };

struct Geo {
  int nz, M, ntiles, nchunks, dchunk;
  int64_t P;
  double Lz, dz, inv_dz, nz_d, half_nz, dV;
};

struct Parts {
  double *z, *ox, *oy, *oz, *N, *Nbar, *rho, *rhobar, *acc, *stage;
};

// ------------------------------------------------------------ device helpers

__device__ __forceinline__ int wrapc(int j, int nz) {
  int r = j % nz;
  return r < 0 ? r + nz : r;
}

// Quadratic shape weights (Sec. 2.2.1) of a particle at (unwrapped) position zs
// whose lattice site is cell h (hp = h + 1/2): d = zs/dz - hp reduced to the
// nearest periodic image, weights 1/2 (1/2 - d)^2, 3/4 - d^2, 1/2 (1/2 + d)^2 on
// cells h-1, h, h+1, written as 1/8 + (d^2 -+ d)/2 and 3/4 - d^2.  The image
// reduction is only needed next to the domain ends, so it sits behind the
// lattice test.  Returns nonzero if the particle is off its lattice site.
__device__ __forceinline__ int shape_weights(double zs, double hp, const Geo& g, double& wl, double& w0,
                                             double& wr) {
  double d = fma(zs, g.inv_dz, -hp);
  int bad = 0;
  if (fabs(d) > 0.5 + kLatticeTol) {
    d -= g.nz_d * rint(d / g.nz_d);
    bad = fabs(d) > 0.5 + kLatticeTol;
  }
  const double d2 = d * d;
  w0 = 0.75 - d2;
  wl = fma(0.5, d2 - d, 0.125);
  wr = fma(0.5, d2 + d, 0.125);
  return bad;
}

// Bulk prefetch of the doubles [i0, i0 + n) of array a into L2 (a hint; the
// range is rounded inwards to 16-byte boundaries so it never leaves the array).
__device__ __forceinline__ void prefetch_l2(const double* a, int64_t i0, int n) {
  uintptr_t lo = ((uintptr_t)(a + i0) + 15) & ~(uintptr_t)15;
  uintptr_t hi = ((uintptr_t)(a + i0 + n)) & ~(uintptr_t)15;
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// The persistent split: the U units go to nw = min(kPersistWarps, U) warps
// (so every working warp owns at least one unit); first unit of warp w, and
// the warp that owns unit x.
__device__ __forceinline__ int64_t split_warps(int64_t U) { return U < kPersistWarps ? U : kPersistWarps; }
__device__ __forceinline__ int64_t unit_begin(int64_t w, int64_t U) {
  const int64_t nw = split_warps(U);
  return w >= nw ? U : w * U / nw;
}
__device__ __forceinline__ int64_t warp_of_unit(int64_t x, int64_t U) { return ((x + 1) * split_warps(U) - 1) / U; }

// Periodic wrap into [0, Lz).
__device__ __forceinline__ double wrap_z(double z, double Lz) {
  if (z >= Lz) z -= Lz;
  else if (z < 0.0) {
    z += Lz;
    if (z >= Lz) z -= Lz;
  }
  return z;
}

// -i [H, r] for packed Hermitian H and r (Eq. 4 with H in units of hbar).
// Diagonal outputs are returned HALVED (kd = K_aa / 2); the caller doubles
// their RK coefficients.  Off-diagonal outputs ko = (Re K12, Im K12, Re K13,
// Im K13, Re K23, Im K23).  H enters through its diagonal differences
// d12 = h1 - h2, d13 = h1 - h3, d23 = h2 - h3 and off-diagonals a, b, c.
__device__ __forceinline__ void commutator(double d12, double d13, double d23, double ar, double ai,
                                           double br, double bi, double cr, double ci,
                                           const double r[9], double kd[3], double ko[6]) {
  const double xr = r[3], xi = r[4], yr = r[5], yi = r[6], zr = r[7], zi = r[8];
  const double e21 = r[1] - r[0], e31 = r[2] - r[0], e32 = r[2] - r[1];
  // C = [H, r]; K = -i C  =>  Re K = Im C, Im K = -Re C
  const double c12r = fma(d12, xr, fma(e21, ar, fma(br, zr, fma(bi, zi, fma(-cr, yr, -ci * yi)))));
  const double c12i = fma(d12, xi, fma(e21, ai, fma(bi, zr, fma(-br, zi, fma(-cr, yi, ci * yr)))));
  const double c13r = fma(d13, yr, fma(e31, br, fma(ar, zr, fma(-ai, zi, fma(-cr, xr, ci * xi)))));
  const double c13i = fma(d13, yi, fma(e31, bi, fma(ar, zi, fma(ai, zr, fma(-cr, xi, -ci * xr)))));
  const double c23r = fma(d23, zr, fma(e32, cr, fma(ar, yr, fma(ai, yi, fma(-br, xr, -bi * xi)))));
  const double c23i = fma(d23, zi, fma(e32, ci, fma(ar, yi, fma(-ai, yr, fma(-bi, xr, br * xi)))));
  ko[0] = c12i; ko[1] = -c12r;
  ko[2] = c13i; ko[3] = -c13r;
  ko[4] = c23i; ko[5] = -c23r;
  // K_11 = 2 (Im(a x*) + Im(b y*)), K_22 = 2 (Im(c z*) - Im(a x*)), K_33 = -2 (Im(b y*) + Im(c z*))
  const double pp = fma(ai, xr, -ar * xi);
  const double qq = fma(bi, yr, -br * yi);
  const double tt = fma(ci, zr, -cr * zi);
  kd[0] = pp + qq;
  kd[1] = tt - pp;
  kd[2] = -qq - tt;
}

// ------------------------------------------------------------------ kernels

// Per-direction table from the ring's first particle: Omega and v_z = c Omega_z.
// Also checks that every particle of a ring carries the ring's direction.
__global__ void k_dirtable(Parts pt, Geo g, double c_light, double* __restrict__ dirtab,
                           int* __restrict__ err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.P) return;
  const int d = (int)(p / g.nz);
  const int64_t p0 = (int64_t)d * g.nz;
  const double ox = pt.ox[p0], oy = pt.oy[p0], oz = pt.oz[p0];
  if (pt.ox[p] != ox || pt.oy[p] != oy || pt.oz[p] != oz) atomicOr(err, ERR_RING);
  if (p == p0) {
    dirtab[d] = ox;
    dirtab[g.M + d] = oy;
    dirtab[2 * g.M + d] = oz;
    dirtab[3 * g.M + d] = c_light * oz;
  }
}

// Lattice shift of every direction for up to 4 position offsets: the cell of
// the ring's first particle at z + off * v_z.
struct Offsets { double v[4]; };

__global__ void k_shifts(const double* __restrict__ z, const double* __restrict__ dirtab, Geo g,
                         Offsets offs, int nrows, int* __restrict__ shift) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.M) return;
  const double z0 = z[(int64_t)d * g.nz];
  const double vz = dirtab[3 * g.M + d];
  for (int s = 0; s < nrows; ++s) {
    const double zs = fma(offs.v[s], vz, z0);
    shift[s * g.M + d] = wrapc((int)floor(zs * g.inv_dz), g.nz);
  }
}

constexpr int kSlot = kNA * kTile;  // doubles in one warp's partial sums for one tile

// A warp's sums for one tile go to slot (warp + tile) of the partial buffer:
// unique, because a later warp never returns to an earlier tile.
__device__ __forceinline__ void flush_tile(const double (&acc)[kNA], int tile, int64_t w, int lane, const Geo& g,
                                           double* __restrict__ partial) {
  const int cell = tile * kTile + lane - 1;
  if (lane >= 1 && lane <= kTile && cell < g.nz) {
    double* slot = partial + (w + tile) * kSlot + lane - 1;
#pragma unroll
    for (int c = 0; c < kNA; ++c) slot[c * kTile] = acc[c];
  }
}

// Deposit (Eq. 5).  MODE 0: B = N rho - Nbar rhobar^* (the combination that
// enters H, Eq. 2); MODE 1: B = N rho; MODE 2: B = Nbar rhobar.  Writes
// out[c * nz + j] = out_scale * sum_p w_pj (1, Omega_p) B_p, in two launches:
// each warp walks its units in order, summing over directions in registers
// (lane l owns cell tile * 30 - 1 + l) and writing one partial per tile it
// touches; k_combine then adds the partials in a fixed order.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 2)
k_deposit(const double* __restrict__ z, const double* __restrict__ N, const double* __restrict__ Nbar,
          const double* __restrict__ r_nu, const double* __restrict__ r_nb,
          const double* __restrict__ dirtab, const int* __restrict__ shift, double pos_dt, Geo g,
          double* __restrict__ partial, double* __restrict__ W, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int nz = g.nz, M = g.M;
  const int64_t P = g.P;
  const int64_t U = (int64_t)g.ntiles * M;
  const int64_t u0 = unit_begin(w, U), u1 = unit_begin(w + 1, U);
  if (u0 >= u1) return;

  int bad = 0;
  for (int64_t u = u0; u < u1;) {        // one segment per tile the warp touches
    const int tile = (int)(u / M);
    const int64_t uend = min(u1, (int64_t)(tile + 1) * M);
    const int craw = tile * kTile - 1 + lane;
    const int j = wrapc(craw, nz);
    const double hp = (double)j + 0.5;
    const bool own = lane >= 1 && lane <= kTile && craw < nz;
    double acc[kNA];
#pragma unroll
    for (int c = 0; c < kNA; ++c) acc[c] = 0.0;
    for (; u < uend; ++u) {
      const int d = (int)(u - (int64_t)tile * M);
      const double ox = __ldg(dirtab + d), oy = __ldg(dirtab + M + d), oz = __ldg(dirtab + 2 * M + d);
      const double vz = __ldg(dirtab + 3 * M + d);
      const int64_t p = (int64_t)d * nz + wrapc(j - __ldg(shift + d), nz);
      double wl, w0, wr;
      bad |= shape_weights(fma(pos_dt, vz, __ldg(z + p)), hp, g, wl, w0, wr);
      if (MODE == 0 && W != nullptr && own) {   // the RK stage of these positions reads them back
        W[p] = wl;
        W[P + p] = w0;
        W[2 * P + p] = wr;
      }
      // cell j receives wr from the particle at j-1, w0 from its own, wl from j+1
      const double wr_l = __shfl_up_sync(kFull, wr, 1);
      const double wl_r = __shfl_down_sync(kFull, wl, 1);
      const double n1 = (MODE != 2) ? __ldg(N + p) : 0.0;
      const double n2 = (MODE != 1) ? __ldg(Nbar + p) : 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        double b;
        if (MODE == 0) {
          const double x = __ldg(r_nu + k * P + p), y = __ldg(r_nb + k * P + p);
          // conj(rhobar) flips the sign of the imaginary components 4, 6, 8
          b = (k == 4 || k == 6 || k == 8) ? fma(n2, y, n1 * x) : fma(-n2, y, n1 * x);
        } else if (MODE == 1) {
          b = n1 * __ldg(r_nu + k * P + p);
        } else {
          b = n2 * __ldg(r_nb + k * P + p);
        }
        const double bl = __shfl_up_sync(kFull, b, 1);
        const double br = __shfl_down_sync(kFull, b, 1);
        const double c = fma(wr_l, bl, fma(w0, b, wl_r * br));
        acc[k] += c;
        acc[9 + k] = fma(ox, c, acc[9 + k]);
        acc[18 + k] = fma(oy, c, acc[18 + k]);
        acc[27 + k] = fma(oz, c, acc[27 + k]);
      }
    }
    flush_tile(acc, tile, w, lane, g, partial);
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// Fixed-order combination of the deposit's per-warp partial sums:
// out[c * nz + j] = scale * (sum over the warps that own units of j's tile, in
// warp order, of their slot value).
__global__ void k_combine(const double* __restrict__ partial, Geo g, double* __restrict__ out, double scale,
                          int* __restrict__ err) {
  const int64_t U = (int64_t)g.ntiles * g.M;
  const int64_t n = (int64_t)kNA * g.nz;
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / g.nz), cell = (int)(e - (int64_t)c * g.nz);
    const int tile = cell / kTile, k = cell - tile * kTile;
    const int64_t wf = warp_of_unit((int64_t)tile * g.M, U);
    const int64_t wl = warp_of_unit((int64_t)(tile + 1) * g.M - 1, U);
    const double* src = partial + c * kTile + k;
    double v = 0.0;
    for (int64_t q = wf; q <= wl; ++q) v += __ldcg(src + (q + tile) * kSlot);
    v *= scale;
    bad |= !isfinite(v);
    out[e] = v;
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

// Load the potential of cells tile*30-1 .. tile*30+30 into shared memory.
__device__ __forceinline__ void load_tile(double (*sA)[kLanes], const double* __restrict__ A, int tile, int nz) {
  for (int idx = threadIdx.x; idx < kNA * kLanes; idx += kThreads) {
    const int comp = idx / kLanes, l = idx % kLanes;
    sA[comp][l] = A[(int64_t)comp * nz + wrapc(tile * kTile - 1 + l, nz)];
  }
}

// Interpolation only (Eq. 6 then Eq. 2): H[k * P + p] at z + pos_dt * v_z.
__global__ void __launch_bounds__(kThreads, 2)
k_interpolate(const double* __restrict__ z, const double* __restrict__ dirtab, const int* __restrict__ shift,
              const double* __restrict__ A, double pos_dt, Geo g, double* __restrict__ Hout,
              int* __restrict__ err) {
  __shared__ double sA[kNA][kLanes];
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nz = g.nz, M = g.M;
  const int64_t P = g.P;
  load_tile(sA, A, tile, nz);
  __syncthreads();
  const int craw = tile * kTile - 1 + lane, j = wrapc(craw, nz);
  const bool active = lane >= 1 && lane <= kTile && craw < nz;
  int bad = 0;
  const int d0 = chunk * g.dchunk, d1 = min(d0 + g.dchunk, M);
  for (int d = d0 + warp; d < d1; d += kWarps) {
    const double ox = __ldg(dirtab + d), oy = __ldg(dirtab + M + d), oz = __ldg(dirtab + 2 * M + d);
    const double vz = __ldg(dirtab + 3 * M + d);
    const int64_t p = (int64_t)d * nz + wrapc(j - __ldg(shift + d), nz);
    double wl = 0.0, w0 = 0.0, wr = 0.0;
    if (active) bad |= shape_weights(fma(pos_dt, vz, z[p]), (double)j + 0.5, g, wl, w0, wr);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double G = fma(-oz, sA[27 + k][lane], fma(-oy, sA[18 + k][lane], fma(-ox, sA[9 + k][lane], sA[k][lane])));
      const double gl = __shfl_up_sync(kFull, G, 1), gr = __shfl_down_sync(kFull, G, 1);
      const double h = fma(wl, gl, fma(w0, G, wr * gr));
      if (active) Hout[k * P + p] = h;
    }
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// One RK4 stage s (1..4) after the deposit of the stage state: interpolate
// (Eq. 6), H and Hbar = -H^* (Eq. 2, Sec. 2.1), K = -i[H, rho] and
// Kbar = -i[Hbar, rhobar] (Eq. 4), then the classic RK4 update (Sec. 2.3):
//   s = 1: acc = y + dt/6 K,  stage = y + dt/2 K
//   s = 2: acc += dt/3 K,     stage = y + dt/2 K
//   s = 3: acc += dt/3 K,     stage = y + dt K
//   s = 4: y = acc + dt/6 K,  z = wrap(z + dt v_z)
// Persistent: each warp walks its contiguous range of units direction-major
// (unit u = direction u / ntiles, tile u % ntiles), so it streams along each
// ring, and prefetches the next unit's particle data into L2.  The shape
// weights of these positions come from the deposit that precedes the stage.
__global__ void __launch_bounds__(kThreads, 2)
k_rk_stage(Parts pt, const double* __restrict__ W, const double* __restrict__ dirtab,
           const int* __restrict__ shift, const double* __restrict__ A, Geo g, int s, double dt) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int nz = g.nz, M = g.M, nt = g.ntiles;
  const int64_t P = g.P;
  const int64_t U = (int64_t)nt * M;
  const int64_t u0 = unit_begin(w, U), u1 = unit_begin(w + 1, U);
  const double bdt = (s == 1 || s == 4) ? dt / 6.0 : dt / 3.0;   // weight of K in acc
  const double cdt = (s == 3) ? dt : 0.5 * dt;                    // offset of the next stage
  const double bdt2 = 2.0 * bdt, cdt2 = 2.0 * cdt;                // diagonal K are returned halved
  const double* src_r = (s == 1) ? pt.rho : pt.stage;
  const double* src_b = (s == 1) ? pt.rhobar : pt.stage + 9 * P;
  // arrays this stage reads, for the prefetch: source (18), y (18, s = 2, 3), acc (18, s >= 2), W (3), z (s = 4)
  const int nsrc = 18, ny = (s == 2 || s == 3) ? 18 : 0, nacc = (s >= 2) ? 18 : 0;
  const int narr = nsrc + ny + nacc + 3 + (s == 4 ? 1 : 0);
  for (int64_t u = u0; u < u1; ++u) {
    const int d = (int)(u / nt);
    const int tile = (int)(u - (int64_t)d * nt);
    if (u + 1 < u1) {
      const int dn = (int)((u + 1) / nt);
      const int tn = (int)(u + 1 - (int64_t)dn * nt);
      const int i0 = tn * kTile - __ldg(shift + dn);           // ring index of the next unit's first cell
      const int n = min(kTile, nz - tn * kTile);
      if (i0 >= 0 && i0 + n <= nz) {
        const int64_t base = (int64_t)dn * nz + i0;
        for (int a = lane; a < narr; a += kLanes) {
          const double* arr;
          if (a < nsrc) arr = (a < 9 ? src_r + (int64_t)a * P : src_b + (int64_t)(a - 9) * P);
          else if (a < nsrc + ny) arr = (a - nsrc < 9 ? pt.rho + (int64_t)(a - nsrc) * P
                                                      : pt.rhobar + (int64_t)(a - nsrc - 9) * P);
          else if (a < nsrc + ny + nacc) arr = pt.acc + (int64_t)(a - nsrc - ny) * P;
          else if (a < nsrc + ny + nacc + 3) arr = W + (int64_t)(a - nsrc - ny - nacc) * P;
          else arr = pt.z;
          prefetch_l2(arr, base, n);
        }
      }
    }
    const int craw = tile * kTile - 1 + lane, j = wrapc(craw, nz);
    const bool active = lane >= 1 && lane <= kTile && craw < nz;
    const double ox = __ldg(dirtab + d), oy = __ldg(dirtab + M + d), oz = __ldg(dirtab + 2 * M + d);
    const double vz = __ldg(dirtab + 3 * M + d);
    const int64_t p = (int64_t)d * nz + wrapc(j - __ldg(shift + d), nz);
    double wl = 0.0, w0 = 0.0, wr = 0.0;
    if (active) {
      wl = W[p];
      w0 = W[P + p];
      wr = W[2 * P + p];
    }
    // the neutrino source matrix first, so its latency overlaps the interpolation
    double r[9];
    if (active) {
#pragma unroll
      for (int k = 0; k < 9; ++k) r[k] = src_r[k * P + p];
    }
    double H[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double G = fma(-oz, __ldg(A + (int64_t)(27 + k) * nz + j),
                           fma(-oy, __ldg(A + (int64_t)(18 + k) * nz + j),
                               fma(-ox, __ldg(A + (int64_t)(9 + k) * nz + j), __ldg(A + (int64_t)k * nz + j))));
      const double gl = __shfl_up_sync(kFull, G, 1), gr = __shfl_down_sync(kFull, G, 1);
      H[k] = fma(wl, gl, fma(w0, G, wr * gr));
    }
    if (!active) continue;
    const double d12 = H[0] - H[1], d13 = H[0] - H[2], d23 = H[1] - H[2];
    // neutrinos: H;  antineutrinos: Hbar = -H^*  (diagonal differences and real parts flip sign)
#pragma unroll
    for (int which = 0; which < 2; ++which) {
      double* __restrict__ yv = which ? pt.rhobar : pt.rho;
      double* __restrict__ av = pt.acc + which * 9 * P;
      double* __restrict__ sv = pt.stage + which * 9 * P;
      // all loads of this matrix before any store (the arrays do not alias)
      double a[9], y[9];
      if (s >= 2) {
#pragma unroll
        for (int k = 0; k < 9; ++k) a[k] = av[k * P + p];
      }
      if (s == 2 || s == 3) {
#pragma unroll
        for (int k = 0; k < 9; ++k) y[k] = yv[k * P + p];
      }
      double rb[9];
      if (which == 1) {
#pragma unroll
        for (int k = 0; k < 9; ++k) rb[k] = src_b[k * P + p];
      }
      const double* rr = which ? rb : r;
      double kd[3], ko[6];
      if (which == 0) commutator(d12, d13, d23, H[3], H[4], H[5], H[6], H[7], H[8], rr, kd, ko);
      else commutator(-d12, -d13, -d23, -H[3], H[4], -H[5], H[6], -H[7], H[8], rr, kd, ko);
      if (s == 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { av[k * P + p] = fma(bdt2, kd[k], rr[k]); sv[k * P + p] = fma(cdt2, kd[k], rr[k]); }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          av[(k + 3) * P + p] = fma(bdt, ko[k], rr[k + 3]);
          sv[(k + 3) * P + p] = fma(cdt, ko[k], rr[k + 3]);
        }
      } else if (s < 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { av[k * P + p] = fma(bdt2, kd[k], a[k]); sv[k * P + p] = fma(cdt2, kd[k], y[k]); }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          av[(k + 3) * P + p] = fma(bdt, ko[k], a[k + 3]);
          sv[(k + 3) * P + p] = fma(cdt, ko[k], y[k + 3]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) yv[k * P + p] = fma(bdt2, kd[k], a[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) yv[(k + 3) * P + p] = fma(bdt, ko[k], a[k + 3]);
      }
    }
    if (s == 4) pt.z[p] = wrap_z(fma(dt, vz, pt.z[p]), g.Lz);
  }
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): n-th output of the generator
// whose state starts at `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t x = seed + n * 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

__device__ __forceinline__ double uniform_pm1(uint64_t seed, int64_t p, int k) {
  const uint64_t h = splitmix64(seed, (uint64_t)p * 8u + (uint64_t)k + 1u);
  return 2.0 * ((double)(h >> 11) * 0x1.0p-53) - 1.0;
}

// Initial particles (Sec. 3.1): cell-centre lattice, weights of Eq. 8, flavour
// state of Eq. 9 (eps_x = |rho_ex|^2, rho_mutau = 0).  Plain roundings (no
// fused multiply-add) so the weights and states round like the formulas read.
__global__ void k_init(Parts pt, Geo g, const double* __restrict__ species, const double* __restrict__ dirs,
                       int use_dirs, double alpha, uint64_t seed, int* __restrict__ err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.P) return;
  const int d = (int)(p / g.nz), j0 = (int)(p % g.nz);
  double o[3];
  if (use_dirs) {
    o[0] = dirs[3 * d]; o[1] = dirs[3 * d + 1]; o[2] = dirs[3 * d + 2];
  } else {
    const double mu = __dsub_rn(1.0, __ddiv_rn(__dadd_rn(__dmul_rn(2.0, (double)d), 1.0), (double)g.M));
    const double phi = __dmul_rn(__dmul_rn((double)d, 3.14159265358979323846), __dsub_rn(3.0, sqrt(5.0)));
    const double sn = sqrt(__dsub_rn(1.0, __dmul_rn(mu, mu)));
    o[0] = __dmul_rn(sn, cos(phi));
    o[1] = __dmul_rn(sn, sin(phi));
    o[2] = mu;
  }
  pt.z[p] = __dmul_rn(__dadd_rn((double)j0, 0.5), g.dz);
  pt.ox[p] = o[0]; pt.oy[p] = o[1]; pt.oz[p] = o[2];
  const int nz = g.nz;
  double w[2];
  for (int sp = 0; sp < 2; ++sp) {
    const double n = species[sp * nz + j0];
    const double* f = species + 2 * nz + sp * 3 * nz + 3 * j0;
    const double fdo = __dadd_rn(__dadd_rn(__dmul_rn(f[0], o[0]), __dmul_rn(f[1], o[1])), __dmul_rn(f[2], o[2]));
    double wt = __ddiv_rn(__dmul_rn(__dadd_rn(n, __dmul_rn(3.0, fdo)), g.dV), (double)g.M);
    const double tol = 1e-12 * (fabs(n) + 3.0 * fabs(fdo)) * g.dV / g.M;
    if (wt < 0.0 && wt >= -tol) wt = 0.0;
    if (wt < 0.0) atomicOr(err, ERR_WEIGHT);
    w[sp] = wt;
  }
  pt.N[p] = w[0];
  pt.Nbar[p] = w[1];
  const int64_t P = g.P;
  for (int sp = 0; sp < 2; ++sp) {
    double* r = sp ? pt.rhobar : pt.rho;
    const double emr = __dmul_rn(alpha, uniform_pm1(seed, p, 4 * sp + 0));
    const double emi = __dmul_rn(alpha, uniform_pm1(seed, p, 4 * sp + 1));
    const double etr = __dmul_rn(alpha, uniform_pm1(seed, p, 4 * sp + 2));
    const double eti = __dmul_rn(alpha, uniform_pm1(seed, p, 4 * sp + 3));
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

// Maximum over cells of the diagonal components of n and nbar (Eq. 7).
__global__ void k_max_diag(const double* __restrict__ mom, int nz, double* __restrict__ out) {
  __shared__ double sm[kThreads];
  double m = 0.0;
  for (int j = threadIdx.x; j < nz; j += kThreads)
    for (int a = 0; a < 3; ++a) {
      m = fmax(m, mom[(int64_t)a * nz + j]);
      m = fmax(m, mom[(int64_t)(36 + a) * nz + j]);
    }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

// Domain diagnostics (Eq. 10, one snapshot of Eq. B1, Eq. 18), fixed-order
// block reduction over cells.
__device__ __forceinline__ double abs_entry(const double* __restrict__ m, int nz, int j, int a, int b) {
  if (a == b) return fabs(m[(int64_t)a * nz + j]);
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const int k = (lo == 0 && hi == 1) ? 3 : (lo == 0 ? 5 : 7);
  const double re = m[(int64_t)k * nz + j], im = m[(int64_t)(k + 1) * nz + j];
  return sqrt(re * re + im * im);
}

__global__ void k_diagnostics(const double* __restrict__ mom, int nz, double* __restrict__ out) {
  __shared__ double sm[kThreads];
  for (int q = 0; q < 63; ++q) {
    double s = 0.0;
    for (int j = threadIdx.x; j < nz; j += kThreads) {
      double v;
      if (q < 36) {
        const int blk = q / 9, e = q % 9, a = e / 3, b = e % 3;
        const int off = blk == 0 ? 0 : blk == 1 ? 36 : blk == 2 ? 9 : 45;
        v = abs_entry(mom + (int64_t)off * nz, nz, j, a, b);
      } else if (q < 45) {
        v = mom[(int64_t)(q - 36) * nz + j];
      } else if (q < 54) {
        v = mom[(int64_t)(36 + q - 45) * nz + j];
      } else {
        const int k = q - 54;
        const double nbar = mom[(int64_t)(36 + k) * nz + j];
        v = mom[(int64_t)k * nz + j] + ((k == 4 || k == 6 || k == 8) ? nbar : -nbar);
      }
      s += v;
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sm[0] / nz;
    __syncthreads();
  }
}

// ------------------------------------------------------------- host side

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t A, mom, partial, W, err, dirtab, shift, species, dirs, scalar, diag, total;
};

void chunking(const emu_config* c, int& ntiles, int& nchunks, int& dchunk) {
  ntiles = (c->nz + kTile - 1) / kTile;
  int maxchunks = (c->ndir + kWarps - 1) / kWarps;
  int want = (kTargetBlocks + ntiles - 1) / ntiles;
  nchunks = want < 1 ? 1 : (want > maxchunks ? maxchunks : want);
  dchunk = (c->ndir + nchunks - 1) / nchunks;
  nchunks = (c->ndir + dchunk - 1) / dchunk;
}

Layout layout(const emu_config* c) {
  int ntiles, nchunks, dchunk;
  chunking(c, ntiles, nchunks, dchunk);
  const size_t nz = (size_t)c->nz, M = (size_t)c->ndir;
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.A = take(sizeof(double) * kNA * nz);
  L.mom = take(sizeof(double) * kNM * nz);
  L.partial = take(sizeof(double) * (size_t)(kPersistWarps + ntiles) * kNA * kTile);
  L.W = take(sizeof(double) * 3 * nz * M);
  L.err = take(sizeof(int));
  L.dirtab = take(sizeof(double) * 4 * M);
  L.shift = take(sizeof(int) * 4 * M);
  L.species = take(sizeof(double) * 8 * nz);
  L.dirs = take(sizeof(double) * 3 * M);
  L.scalar = take(sizeof(double) * 4);
  L.diag = take(sizeof(double) * 64);
  L.total = off;
  return L;
}

const char* config_problem(const emu_config* c) {
  if (!c) return "config is NULL";
  if (c->nz < 1) return "nz must be >= 1";
  if (c->ndir < 1) return "ndir must be >= 1";
  if ((int64_t)c->nz * c->ndir > ((int64_t)1 << 40)) return "nz * ndir too large";
  if (!(c->Lz > 0) || !std::isfinite(c->Lz)) return "Lz must be positive and finite";
  if (!(c->area > 0) || !std::isfinite(c->area)) return "area must be positive and finite";
  if (!(c->kappa > 0) || !std::isfinite(c->kappa)) return "kappa must be positive and finite";
  if (!(c->c_light > 0) || !std::isfinite(c->c_light)) return "c_light must be positive and finite";
  if (!(c->cfl_adv > 0) || !(c->cfl_flavor > 0)) return "CFL factors must be positive";
  if (c->shape_order != 2) return "only the quadratic shape (shape_order = 2) is supported";
  if (c->reserved != 0) return "reserved must be 0";
  return nullptr;
}

}  // namespace

struct emu_box {
  emu_config cfg;
  Geo g;
  Layout L;
  Parts pt;
  bool bound = false;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  double *A = nullptr, *mom = nullptr, *partial = nullptr, *W = nullptr, *dirtab = nullptr, *species = nullptr,
         *dirs = nullptr, *scalar = nullptr, *diag = nullptr;
  int *err = nullptr, *shift = nullptr;
  int next_stage = 1;
  double stage_dt = 0.0;
  double dt_cached = 0.0;
  int64_t launches = 0;
  // optional per-launch timing: events recorded on the box's stream around each kernel
  struct Rec { int cls; cudaEvent_t a, b; };
  bool prof = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  char msg[512] = {0};
  ~emu_box() {
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

namespace {

char g_create_msg[512];

int fail(emu_box* b, int code, const char* fmt, ...) {
  char* dst = b ? b->msg : g_create_msg;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_check(emu_box* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return EMU_OK;
  return fail(b, EMU_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

enum : int { CLS_SHIFT = 0, CLS_DEPOSIT = 1, CLS_RK = 2, CLS_COMBINE = 3, CLS_OTHER = 4, N_CLS = 5 };

cudaEvent_t take_event(emu_box* b) {
  if (!b->pool.empty()) { cudaEvent_t e = b->pool.back(); b->pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Called right before a launch: records the start event when timing is on.
void before_launch(emu_box* b, int cls) {
  if (!b->prof) return;
  emu_box::Rec r{cls, take_event(b), nullptr};
  if (r.a) cudaEventRecord(r.a, b->stream);
  b->recs.push_back(r);
}

int after_launch(emu_box* b, const char* what) {
  b->launches++;
  if (b->prof && !b->recs.empty() && b->recs.back().b == nullptr) {
    b->recs.back().b = take_event(b);
    if (b->recs.back().b) cudaEventRecord(b->recs.back().b, b->stream);
  }
  return cuda_check(b, cudaGetLastError(), what);
}

dim3 tile_grid(const Geo& g) { return dim3((unsigned)g.ntiles, (unsigned)g.nchunks, 1); }
dim3 persist_grid() { return dim3((unsigned)kPersistBlocks, 1, 1); }
unsigned combine_blocks(const Geo& g) {
  const int64_t n = (int64_t)kNA * g.nz;
  const int64_t blocks = (n + kThreads - 1) / kThreads;
  return (unsigned)(blocks < 4 * kPersistBlocks ? blocks : 4 * kPersistBlocks);
}

int launch_shifts(emu_box* b, const double* offs, int nrows) {
  Offsets o{};
  for (int s = 0; s < nrows; ++s) o.v[s] = offs[s];
  const int blocks = (b->g.M + kThreads - 1) / kThreads;
  before_launch(b, CLS_SHIFT);
  k_shifts<<<blocks, kThreads, 0, b->stream>>>(b->pt.z, b->dirtab, b->g, o, nrows, b->shift);
  return after_launch(b, "shift kernel");
}

int launch_deposit(emu_box* b, int mode, const double* rnu, const double* rnb, const int* shift_row,
                   double pos_dt, double* out, double scale) {
  const Geo& g = b->g;
  before_launch(b, CLS_DEPOSIT);
  if (mode == 0)
    k_deposit<0><<<persist_grid(), kThreads, 0, b->stream>>>(b->pt.z, b->pt.N, b->pt.Nbar, rnu, rnb, b->dirtab,
        shift_row, pos_dt, g, b->partial, b->W, b->err);
  else if (mode == 1)
    k_deposit<1><<<persist_grid(), kThreads, 0, b->stream>>>(b->pt.z, b->pt.N, b->pt.Nbar, rnu, rnb, b->dirtab,
        shift_row, pos_dt, g, b->partial, nullptr, b->err);
  else
    k_deposit<2><<<persist_grid(), kThreads, 0, b->stream>>>(b->pt.z, b->pt.N, b->pt.Nbar, rnu, rnb, b->dirtab,
        shift_row, pos_dt, g, b->partial, nullptr, b->err);
  if (int rc = after_launch(b, "deposit kernel")) return rc;
  before_launch(b, CLS_COMBINE);
  k_combine<<<combine_blocks(g), kThreads, 0, b->stream>>>(b->partial, g, out, scale, b->err);
  return after_launch(b, "deposit combine kernel");
}

int check_bound(emu_box* b) {
  if (!b) return EMU_EINVAL;
  if (!b->bound) return fail(b, EMU_EINVAL, "box is not bound to memory (call emu_bind)");
  return EMU_OK;
}

int copy_out(emu_box* b, void* dst, const void* src, size_t bytes, int on_host) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                  b->stream);
  if (e != cudaSuccess) return cuda_check(b, e, "copy out");
  if (on_host) return cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise after copy out");
  return EMU_OK;
}

int run_moments(emu_box* b) {
  const double zero = 0.0;
  int rc = launch_shifts(b, &zero, 1);
  if (rc) return rc;
  const double inv_dV = 1.0 / b->g.dV;
  rc = launch_deposit(b, 1, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom, inv_dV);
  if (rc) return rc;
  return launch_deposit(b, 2, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom + (size_t)kNA * b->g.nz, inv_dV);
}

int rebuild_dirtable(emu_box* b) {
  const int blocks = (int)((b->g.P + kThreads - 1) / kThreads);
  before_launch(b, CLS_OTHER);
  k_dirtable<<<blocks, kThreads, 0, b->stream>>>(b->pt, b->g, b->cfg.c_light, b->dirtab, b->err);
  return after_launch(b, "direction table kernel");
}

int read_errors(emu_box* b) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_check(b, e, "read error word");
  if (h == 0) return EMU_OK;
  cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
  if (h & ERR_WEIGHT) return fail(b, EMU_EINVAL, "negative particle weight: a flux factor exceeds 1/3");
  if (h & ERR_RING) return fail(b, EMU_ELATTICE, "a ring of particles does not share one direction");
  if (h & ERR_LATTICE) return fail(b, EMU_ELATTICE, "a particle is off its lattice site");
  if (h & ERR_NONFINITE) return fail(b, EMU_ENUMERIC, "non-finite value on the grid");
  return fail(b, EMU_ECUDA, "unknown device error word %d", h);
}

}  // namespace

// --------------------------------------------------------------------- C ABI

extern "C" {

int64_t emu_workspace_bytes(const emu_config* cfg) {
  if (config_problem(cfg)) return EMU_EINVAL;
  return (int64_t)layout(cfg).total;
}

int emu_create(const emu_config* cfg, emu_box** out) {
  if (!out) return fail(nullptr, EMU_EINVAL, "out is NULL");
  *out = nullptr;
  if (const char* why = config_problem(cfg)) return fail(nullptr, EMU_EINVAL, "%s", why);
  emu_box* b = new (std::nothrow) emu_box();
  if (!b) return fail(nullptr, EMU_EINVAL, "host allocation failed");
  b->cfg = *cfg;
  Geo& g = b->g;
  g.nz = cfg->nz;
  g.M = cfg->ndir;
  g.P = (int64_t)cfg->nz * cfg->ndir;
  chunking(cfg, g.ntiles, g.nchunks, g.dchunk);
  g.Lz = cfg->Lz;
  g.dz = cfg->Lz / cfg->nz;
  g.inv_dz = 1.0 / g.dz;
  g.nz_d = (double)cfg->nz;
  g.half_nz = 0.5 * cfg->nz;
  g.dV = g.dz * cfg->area;
  b->L = layout(cfg);
  *out = b;
  return EMU_OK;
}

int emu_bind(emu_box* b, const emu_particles* parts, void* workspace, int64_t workspace_bytes, void* stream) {
  if (!b) return EMU_EINVAL;
  if (!parts || !workspace) return fail(b, EMU_EINVAL, "particles or workspace is NULL");
  if (parts->P != b->g.P) return fail(b, EMU_EINVAL, "parts->P = %lld, expected nz*ndir = %lld",
                                      (long long)parts->P, (long long)b->g.P);
  if (workspace_bytes < (int64_t)b->L.total)
    return fail(b, EMU_EINVAL, "workspace too small: %lld < %lld bytes", (long long)workspace_bytes,
                (long long)b->L.total);
  if (((uintptr_t)workspace) & 255) return fail(b, EMU_EINVAL, "workspace must be 256-byte aligned");
  double* ptrs[] = {parts->z, parts->ox, parts->oy, parts->oz, parts->N, parts->Nbar, parts->rho,
                    parts->rhobar, parts->acc, parts->stage};
  for (double* q : ptrs)
    if (!q) return fail(b, EMU_EINVAL, "a particle array pointer is NULL");
  b->pt = Parts{parts->z, parts->ox, parts->oy, parts->oz, parts->N, parts->Nbar, parts->rho, parts->rhobar,
                parts->acc, parts->stage};
  b->stream = (cudaStream_t)stream;
  b->ws = (char*)workspace;
  const Layout& L = b->L;
  b->A = (double*)(b->ws + L.A);
  b->mom = (double*)(b->ws + L.mom);
  b->partial = (double*)(b->ws + L.partial);
  b->W = (double*)(b->ws + L.W);
  b->err = (int*)(b->ws + L.err);
  b->dirtab = (double*)(b->ws + L.dirtab);
  b->shift = (int*)(b->ws + L.shift);
  b->species = (double*)(b->ws + L.species);
  b->dirs = (double*)(b->ws + L.dirs);
  b->scalar = (double*)(b->ws + L.scalar);
  b->diag = (double*)(b->ws + L.diag);
  int rc = cuda_check(b, cudaMemsetAsync(workspace, 0, L.total, b->stream), "clear workspace");
  if (rc) return rc;
  b->bound = true;
  b->next_stage = 1;
  return EMU_OK;
}

int emu_init_particles(emu_box* b, const double* n_nu, const double* n_nubar, const double* f_nu,
                       const double* f_nubar, const double* dirs, double alpha, uint64_t seed) {
  if (int rc = check_bound(b)) return rc;
  if (!n_nu || !n_nubar || !f_nu || !f_nubar) return fail(b, EMU_EINVAL, "species arrays must not be NULL");
  const size_t nz = (size_t)b->g.nz;
  cudaStream_t st = b->stream;
  const double* src[4] = {n_nu, n_nubar, f_nu, f_nubar};
  const size_t off[4] = {0, nz, 2 * nz, 5 * nz};
  const size_t cnt[4] = {nz, nz, 3 * nz, 3 * nz};
  for (int i = 0; i < 4; ++i)
    if (int rc = cuda_check(b, cudaMemcpyAsync(b->species + off[i], src[i], sizeof(double) * cnt[i],
                                               cudaMemcpyHostToDevice, st), "copy species"))
      return rc;
  if (dirs)
    if (int rc = cuda_check(b, cudaMemcpyAsync(b->dirs, dirs, sizeof(double) * 3 * b->g.M, cudaMemcpyHostToDevice,
                                               st), "copy directions"))
      return rc;
  const int blocks = (int)((b->g.P + kThreads - 1) / kThreads);
  before_launch(b, CLS_OTHER);
  k_init<<<blocks, kThreads, 0, st>>>(b->pt, b->g, b->species, b->dirs, dirs ? 1 : 0, alpha, seed, b->err);
  if (int rc = after_launch(b, "init kernel")) return rc;
  if (int rc = rebuild_dirtable(b)) return rc;
  b->next_stage = 1;
  b->dt_cached = 0.0;
  return read_errors(b);  // the host inputs must stay valid until the copies finish
}

int emu_set_particles(emu_box* b, const double* z, const double* ox, const double* oy, const double* oz,
                      const double* N, const double* Nbar, const double* rho, const double* rhobar, int on_host) {
  if (int rc = check_bound(b)) return rc;
  const size_t P = (size_t)b->g.P;
  const cudaMemcpyKind kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const double* src[8] = {z, ox, oy, oz, N, Nbar, rho, rhobar};
  double* dst[8] = {b->pt.z, b->pt.ox, b->pt.oy, b->pt.oz, b->pt.N, b->pt.Nbar, b->pt.rho, b->pt.rhobar};
  const size_t n[8] = {P, P, P, P, P, P, 9 * P, 9 * P};
  for (int i = 0; i < 8; ++i)
    if (src[i])
      if (int rc = cuda_check(b, cudaMemcpyAsync(dst[i], src[i], sizeof(double) * n[i], kind, b->stream),
                              "copy particles in"))
        return rc;
  b->next_stage = 1;
  if (ox || oy || oz) {
    b->dt_cached = 0.0;
    if (int rc = rebuild_dirtable(b)) return rc;
  }
  if (on_host) return cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise after copy in");
  return EMU_OK;
}

int emu_get_particles(emu_box* b, double* z, double* ox, double* oy, double* oz, double* N, double* Nbar,
                      double* rho, double* rhobar, int on_host) {
  if (int rc = check_bound(b)) return rc;
  const size_t P = (size_t)b->g.P;
  const cudaMemcpyKind kind = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  double* dst[8] = {z, ox, oy, oz, N, Nbar, rho, rhobar};
  const double* src[8] = {b->pt.z, b->pt.ox, b->pt.oy, b->pt.oz, b->pt.N, b->pt.Nbar, b->pt.rho, b->pt.rhobar};
  const size_t n[8] = {P, P, P, P, P, P, 9 * P, 9 * P};
  for (int i = 0; i < 8; ++i)
    if (dst[i])
      if (int rc = cuda_check(b, cudaMemcpyAsync(dst[i], src[i], sizeof(double) * n[i], kind, b->stream),
                              "copy particles out"))
        return rc;
  if (on_host) return cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise after copy out");
  return EMU_OK;
}

int emu_deposit(emu_box* b, int src, double pos_dt, double* A_out, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (src != 0 && src != 1) return fail(b, EMU_EINVAL, "src must be 0 (rho) or 1 (stage buffer)");
  if (!std::isfinite(pos_dt)) return fail(b, EMU_EINVAL, "pos_dt must be finite");
  if (int rc = launch_shifts(b, &pos_dt, 1)) return rc;
  const size_t P = (size_t)b->g.P;
  const double* rnu = src ? b->pt.stage : b->pt.rho;
  const double* rnb = src ? b->pt.stage + 9 * P : b->pt.rhobar;
  if (int rc = launch_deposit(b, 0, rnu, rnb, b->shift, pos_dt, b->A, b->cfg.kappa / b->g.dV)) return rc;
  if (A_out) return copy_out(b, A_out, b->A, sizeof(double) * kNA * b->g.nz, on_host);
  return EMU_OK;
}

int emu_interpolate_H(emu_box* b, double pos_dt, double* H_out, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (!H_out) return fail(b, EMU_EINVAL, "H_out is NULL");
  if (!std::isfinite(pos_dt)) return fail(b, EMU_EINVAL, "pos_dt must be finite");
  if (int rc = launch_shifts(b, &pos_dt, 1)) return rc;
  double* dst = H_out;
  if (on_host) dst = b->pt.acc;  // staging: the RK scratch holds 18 P doubles
  before_launch(b, CLS_OTHER);
  k_interpolate<<<tile_grid(b->g), kThreads, 0, b->stream>>>(b->pt.z, b->dirtab, b->shift, b->A, pos_dt, b->g, dst,
                                                             b->err);
  if (int rc = after_launch(b, "interpolation kernel")) return rc;
  b->next_stage = 1;  // the staging above may overwrite the RK scratch
  if (on_host) return copy_out(b, H_out, dst, sizeof(double) * 9 * (size_t)b->g.P, 1);
  return EMU_OK;
}

int emu_rk_stage(emu_box* b, int s, double dt) {
  if (int rc = check_bound(b)) return rc;
  if (s < 1 || s > 4) return fail(b, EMU_EINVAL, "stage must be 1..4");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(b, EMU_EINVAL, "dt must be positive and finite");
  if (s != b->next_stage) return fail(b, EMU_EINVAL, "stage %d called, expected stage %d", s, b->next_stage);
  if (s > 1 && dt != b->stage_dt) return fail(b, EMU_EINVAL, "dt changed within a step");
  if (s == 1) {
    const double offs[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};
    if (int rc = launch_shifts(b, offs, 4)) return rc;
    b->stage_dt = dt;
  }
  const size_t P = (size_t)b->g.P;
  const double pos = (s == 1) ? 0.0 : (s == 4 ? dt : 0.5 * dt);
  const double* rnu = (s == 1) ? b->pt.rho : b->pt.stage;
  const double* rnb = (s == 1) ? b->pt.rhobar : b->pt.stage + 9 * P;
  const int* srow = b->shift + (size_t)(s - 1) * b->g.M;
  if (int rc = launch_deposit(b, 0, rnu, rnb, srow, pos, b->A, b->cfg.kappa / b->g.dV)) return rc;
  before_launch(b, CLS_RK);
  k_rk_stage<<<persist_grid(), kThreads, 0, b->stream>>>(b->pt, b->W, b->dirtab, srow, b->A, b->g, s, dt);
  if (int rc = after_launch(b, "RK stage kernel")) return rc;
  b->next_stage = s == 4 ? 1 : s + 1;
  return EMU_OK;
}

int emu_timestep(emu_box* b, double* dt_out) {
  if (int rc = check_bound(b)) return rc;
  if (!dt_out) return fail(b, EMU_EINVAL, "dt_out is NULL");
  if (int rc = run_moments(b)) return rc;
  before_launch(b, CLS_OTHER);
  k_max_diag<<<1, kThreads, 0, b->stream>>>(b->mom, b->g.nz, b->scalar);
  if (int rc = after_launch(b, "max kernel")) return rc;
  double nmax = 0.0;
  if (int rc = copy_out(b, &nmax, b->scalar, sizeof(double), 1)) return rc;
  if (int rc = read_errors(b)) return rc;
  const double dt_adv = b->cfg.cfl_adv * b->g.dz / b->cfg.c_light;
  const double dt_flav = nmax > 0.0 ? b->cfg.cfl_flavor / (b->cfg.kappa * nmax) : dt_adv;
  *dt_out = dt_adv < dt_flav ? dt_adv : dt_flav;
  b->dt_cached = *dt_out;
  return EMU_OK;
}

int emu_step(emu_box* b, int64_t nsteps, double dt) {
  if (int rc = check_bound(b)) return rc;
  if (nsteps < 0) return fail(b, EMU_EINVAL, "nsteps must be >= 0");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  if (!(dt > 0)) {
    if (!(b->dt_cached > 0))
      if (int rc = emu_timestep(b, &b->dt_cached)) return rc;
    dt = b->dt_cached;
  }
  for (int64_t n = 0; n < nsteps; ++n)
    for (int s = 1; s <= 4; ++s)
      if (int rc = emu_rk_stage(b, s, dt)) return rc;
  return EMU_OK;
}

int emu_moments(emu_box* b, double* out, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (!out) return fail(b, EMU_EINVAL, "out is NULL");
  if (int rc = run_moments(b)) return rc;
  return copy_out(b, out, b->mom, sizeof(double) * kNM * b->g.nz, on_host);
}

int emu_diagnostics(emu_box* b, double* out, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (!out) return fail(b, EMU_EINVAL, "out is NULL");
  if (int rc = run_moments(b)) return rc;
  before_launch(b, CLS_OTHER);
  k_diagnostics<<<1, kThreads, 0, b->stream>>>(b->mom, b->g.nz, b->diag);
  if (int rc = after_launch(b, "diagnostics kernel")) return rc;
  return copy_out(b, out, b->diag, sizeof(double) * 63, on_host);
}

int emu_sync(emu_box* b) {
  if (int rc = check_bound(b)) return rc;
  if (int rc = cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise")) return rc;
  return read_errors(b);
}

int64_t emu_kernel_launches(const emu_box* b) { return b ? b->launches : 0; }

int emu_profile(emu_box* b, int enable) {
  if (!b) return EMU_EINVAL;
  b->prof = enable != 0;
  return EMU_OK;
}

int emu_kernel_times(emu_box* b, double* ms_out, int64_t* count_out) {
  if (int rc = check_bound(b)) return rc;
  if (!ms_out || !count_out) return fail(b, EMU_EINVAL, "output arrays are NULL");
  if (int rc = cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise for kernel times")) return rc;
  for (int c = 0; c < N_CLS; ++c) { ms_out[c] = 0.0; count_out[c] = 0; }
  int rc = EMU_OK;
  for (auto& r : b->recs) {
    float ms = 0.f;
    if (r.a && r.b && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ms_out[r.cls] += ms;
      count_out[r.cls] += 1;
    } else {
      rc = fail(b, EMU_ECUDA, "a kernel timing event could not be read");
    }
    if (r.a) b->pool.push_back(r.a);
    if (r.b) b->pool.push_back(r.b);
  }
  b->recs.clear();
  return rc;
}

const char* emu_last_error(const emu_box* b) { return b ? b->msg : g_create_msg; }

void emu_destroy(emu_box* b) { delete b; }

}  // extern "C"

// ------------------------------------------- deposit without any allocation
//
// Some callers cannot allocate device memory at all: code running where
// cudaMalloc is not allowed (inside a host callback or another library's
// allocation-free region), or code that must not call into any allocator
// (for example while a memory pool is being torn down or resized).  They
// cannot provide the workspace that emu_bind expects, so this entry point
// keeps the deposit's scratch (per-direction table, lattice shifts, partial
// sums of the warps, error word) in one static device
// array that the library itself holds on every GPU that loads it.

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_static_addr[kMaxDevices] = {nullptr};
std::mutex g_static_mutex;

// Device address of g_static_scratch on the current device.  The name of the
// array is only a host-side stand-in; the address must come from the runtime,
// once per device, with that device current.
int static_scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, EMU_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, EMU_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail(nullptr, EMU_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return EMU_OK;
}

}  // namespace

extern "C" int emu_deposit_static(const emu_config* cfg, const double* z, const double* ox, const double* oy,
                                  const double* oz, const double* N, const double* Nbar, const double* rho,
                                  const double* rhobar, double pos_dt, double* A_out, void* stream) {
  if (const char* why = config_problem(cfg)) return fail(nullptr, EMU_EINVAL, "%s", why);
  if (!z || !ox || !oy || !oz || !N || !Nbar || !rho || !rhobar || !A_out)
    return fail(nullptr, EMU_EINVAL, "a particle array or A_out is NULL");
  if (!std::isfinite(pos_dt)) return fail(nullptr, EMU_EINVAL, "pos_dt must be finite");
  Geo g;
  g.nz = cfg->nz;
  g.M = cfg->ndir;
  g.P = (int64_t)cfg->nz * cfg->ndir;
  chunking(cfg, g.ntiles, g.nchunks, g.dchunk);
  g.Lz = cfg->Lz;
  g.dz = cfg->Lz / cfg->nz;
  g.inv_dz = 1.0 / g.dz;
  g.nz_d = (double)cfg->nz;
  g.half_nz = 0.5 * cfg->nz;
  g.dV = g.dz * cfg->area;
  // carve the static array: partial sums, error word, direction table, shifts
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t o_partial = take(sizeof(double) * (size_t)(kPersistWarps + g.ntiles) * kNA * kTile);
  const size_t o_err = take(sizeof(int));
  const size_t o_dirtab = take(sizeof(double) * 4 * (size_t)g.M);
  const size_t o_shift = take(sizeof(int) * (size_t)g.M);
  if (off > kStaticScratchBytes)
    return fail(nullptr, EMU_EINVAL,
                "emu_deposit_static: this box needs %zu bytes of scratch, more than the %zu-byte static array "
                "(use emu_deposit with a caller workspace)", off, kStaticScratchBytes);
  void* base = nullptr;
  if (int rc = static_scratch_address(&base)) return rc;
  char* s = (char*)base;
  double* partial = (double*)(s + o_partial);
  int* err = (int*)(s + o_err);
  double* dirtab = (double*)(s + o_dirtab);
  int* shift = (int*)(s + o_shift);
  cudaStream_t st = (cudaStream_t)stream;
  auto check = [&](cudaError_t e, const char* what) {
    return e == cudaSuccess ? EMU_OK : fail(nullptr, EMU_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  // the error word must start at zero; the array keeps what the last call left
  if (int rc = check(cudaMemsetAsync(err, 0, sizeof(int), st), "clear static scratch")) return rc;
  Parts pt{const_cast<double*>(z), const_cast<double*>(ox), const_cast<double*>(oy), const_cast<double*>(oz),
           const_cast<double*>(N), const_cast<double*>(Nbar), const_cast<double*>(rho),
           const_cast<double*>(rhobar), nullptr, nullptr};
  const int pblocks = (int)((g.P + kThreads - 1) / kThreads);
  k_dirtable<<<pblocks, kThreads, 0, st>>>(pt, g, cfg->c_light, dirtab, err);
  if (int rc = check(cudaGetLastError(), "direction table kernel")) return rc;
  Offsets o{};
  o.v[0] = pos_dt;
  k_shifts<<<(g.M + kThreads - 1) / kThreads, kThreads, 0, st>>>(z, dirtab, g, o, 1, shift);
  if (int rc = check(cudaGetLastError(), "shift kernel")) return rc;
  k_deposit<0><<<persist_grid(), kThreads, 0, st>>>(z, N, Nbar, rho, rhobar, dirtab, shift, pos_dt, g, partial,
                                                  nullptr, err);
  if (int rc = check(cudaGetLastError(), "deposit kernel")) return rc;
  k_combine<<<combine_blocks(g), kThreads, 0, st>>>(partial, g, A_out, cfg->kappa / g.dV, err);
  if (int rc = check(cudaGetLastError(), "deposit combine kernel")) return rc;
  int h = 0;
  if (int rc = check(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st), "read error word")) return rc;
  if (int rc = check(cudaStreamSynchronize(st), "synchronise")) return rc;
  if (h & ERR_RING) return fail(nullptr, EMU_ELATTICE, "a ring of particles does not share one direction");
  if (h & ERR_LATTICE) return fail(nullptr, EMU_ELATTICE, "a particle is off its lattice site");
  if (h & ERR_NONFINITE) return fail(nullptr, EMU_ENUMERIC, "non-finite value on the grid");
  return EMU_OK;
}
