// kernels.cuh -- GB300 (sm_103a) FP64 device code of the particle-in-cell step
// for the neutrino fast flavour instability (Richers, Willcox, Ford & Myers,
// arXiv:2101.02745).  Included once, by emu.cu.
//
// A *batch* is a set of independent 1D periodic boxes advanced together; one
// box is a batch of one.  All arrays of a batch are concatenated:
//   particles: box b occupies [poff_b, poff_b + nz_b * ndir_b) of every SoA array;
//              particle (d, i) of box b is poff_b + d * nz_b + i; component k of a
//              matrix array at [k * Ptot + particle]
//   grid:      cell j of box b is column coff_b + j of A[36][NZ] (the full
//              potential), At[32][NZ] (the step's traceless potential) and mom[72][NZ]
//   tables:    direction d of box b is entry doff_b + d of the per-direction tables
//
// Parallel layout.  Work is split into *units* = (one tile of T cells, one
// direction) of one box: box b has ntiles_b * ndir_b units, numbered box after
// box.  A warp works on one unit at a time with lane l on cell
// (tile * T - H + l): lanes H..H+T-1 own the tile's cells, the H lanes on each
// side are halo lanes that supply the neighbour values of the stencil.  The
// shape orders 0-2 (Sec. 2.2.1) reach one cell on each side (H = 1, T = 30),
// the cubic shape two (H = 2, T = 28).  Because
// the particles of one direction (a ring) translate rigidly (one per cell at a
// common offset, Sec. 3.1 and Eq. 4), the particle on cell j is ring entry
// (j - shift_d) mod nz and its stencil neighbours sit on the adjacent lanes:
// deposit (Eq. 5) and interpolation (Eq. 6) are warp-shuffle gathers.  The
// RK stage also has a form without halo lanes (k_rk_stage32: 32-cell tiles,
// the tile ends through shared memory).
//
// Persistent schedule.  The step kernels run a fixed grid (2 blocks of 8 warps
// per SM); the first nw warps split the U units of the batch into equal
// contiguous ranges.  The deposit's summation order (registers over a warp's
// directions, one partial per (warp, tile), partials added in warp order by
// k_combine) depends only on the batch and nw: no atomics, bitwise reproducible.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace emu_dev {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kLanes = 32;
constexpr int kTileMax = 30;       // most cells a warp owns (shape orders 0-2)
constexpr int kNA = 36;            // components of the grid potential (and of a deposit's partial sums)
// Components of the traceless grid potential the step reads: per moment (n,
// f_x, f_y, f_z) the diagonal differences B_11 - B_22, B_22 - B_33 and the
// six off-diagonal reals.  The trace of H commutes with every rho, so
// -i[H, rho] (Eq. 4) depends on H only through these 8 (per moment: 32).
constexpr int kNT = 32;
constexpr int kNC = 8;             // components of one traceless matrix
constexpr int kNM = 72;            // components of the per-species moments
constexpr int kWSlots = 5;         // weight slots per stage row of the direction weight table (the cubic shape's 5)
constexpr int kSlot = kNA * kTileMax; // doubles in one warp's partial sums for one tile
constexpr double kLatticeTol = 1e-6;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kPersistBlocks = 2 * 152;  // default grid: 2 resident blocks on each of GB300's 152 SMs
constexpr int kMaxBlocks = 4 * 152;      // largest grid the autotuner tries
constexpr int kMaxWarps = kMaxBlocks * kWarps;

enum : int { ERR_LATTICE = 1, ERR_NONFINITE = 2, ERR_WEIGHT = 4, ERR_RING = 8, ERR_STEP = 32 };

// Stencil of the shape of order ORDER (Sec. 2.2.1, orders 0-3): a particle on
// lattice site h (the cell containing it) reaches cells h-H .. h+H, weight
// slots 0 .. NW-1; NWS weight arrays are kept from the deposit for the RK stage
// (none for order 0, whose only weight is 1).
template <int ORDER>
struct Sten {
  static_assert(ORDER >= 0 && ORDER <= 3, "shape orders 0..3");
  static constexpr int H = ORDER == 3 ? 2 : 1;
  static constexpr int T = kLanes - 2 * H;
  static constexpr int NW = 2 * H + 1;
  static constexpr int NWS = ORDER == 0 ? 0 : NW;
  static_assert(T <= kTileMax, "a tile's partial sums must fit a slot");
};

// One box of a batch (device copy lives in the workspace).
struct BoxGeo {
  int nz, M, ntiles, use_dirs;
  int coff, toff, doff, ntiles32;  // ntiles32: 32-cell tiles of the RK stage
  int toff32, reserved_;           // toff32: first 32-cell tile of the box among all boxes'
  int64_t P, poff, uoff, uoff32;   // uoff32: first 32-cell unit of the box
  double Lz, dz, inv_dz, nz_d, dV, c_light;
  double kappa_dV;   // kappa / dV: scale of the grid potential
  double inv_dV;     // 1 / dV: scale of the moments
  double alpha;      // Eq. 9 perturbation strength (init)
  uint64_t seed;     // Eq. 9 random stream (init)
  double cfl_adv, cfl_flavor, kappa;  // Eq. 7
  double n_e;        // net electron density (matter term of Eq. 2, lepton density of Eq. 7)
  // constant parts of the Hamiltonians in the traceless components (H_11 - H_22,
  // H_22 - H_33, off-diagonal reals): (H_vacuum + H_matter) / hbar for neutrinos,
  // (H_vacuum^* - H_matter^*) / hbar for antineutrinos
  double vnu[kNC];
  double vnubar[kNC];
};

// Kernel view of a batch (passed by value).
struct Batch {
  const BoxGeo* box;   // [nbox]
  const double* dt;    // [nbox] step size of every box
  int nbox;
  int nw;              // warps that split the units
  int NZ, MT, NT;      // total cells, directions, tiles
  int T;               // cells per tile (the shape order's Sten<>::T)
  int64_t U, Ptot;     // total units, particles
  int64_t U32;         // total 32-cell units of the RK stage (shape orders 0-2)
  int nw32;            // warps that split them
};

struct Parts {
  double *z, *ox, *oy, *oz, *N, *Nbar, *rho, *rhobar, *acc, *stage;
};

// ------------------------------------------------------------ device helpers

// The step kernels are launched with programmatic dependent launch: their
// blocks may be scheduled while the previous kernel of the stream drains.  Each
// calls this first, before any memory access: it returns once the previous
// kernel has completed and its writes are visible (at once without one).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int wrapc(int j, int nz) {
  int r = j % nz;
  return r < 0 ? r + nz : r;
}

__device__ __forceinline__ int64_t unit_begin(int64_t w, const Batch& B) {
  return w >= B.nw ? B.U : w * B.U / B.nw;
}
__device__ __forceinline__ int64_t warp_of_unit(int64_t x, const Batch& B) { return ((x + 1) * B.nw - 1) / B.U; }
__device__ __forceinline__ int64_t unit32_begin(int64_t w, const Batch& B) {
  return w >= B.nw32 ? B.U32 : w * B.U32 / B.nw32;
}

// Index of the box containing unit u / cell c / particle p / direction d
// (binary search over the boxes' offsets; all arguments are warp-uniform in
// the step kernels).
__device__ __forceinline__ int box_of_unit(const Batch& B, int64_t u) {
  int lo = 0, hi = B.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.box[mid].uoff <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int box_of_unit32(const Batch& B, int64_t u) {
  int lo = 0, hi = B.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.box[mid].uoff32 <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int box_of_cell(const Batch& B, int c) {
  int lo = 0, hi = B.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.box[mid].coff <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int box_of_particle(const Batch& B, int64_t p) {
  int lo = 0, hi = B.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.box[mid].poff <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int box_of_direction(const Batch& B, int d) {
  int lo = 0, hi = B.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.box[mid].doff <= d) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Shape weights (Sec. 2.2.1) of order ORDER of a particle at (unwrapped)
// position zs whose lattice site is cell h (hp = h + 1/2): the offset
// d = zs/dz - hp, reduced to the nearest periodic image, lies in [-1/2, 1/2),
// and w[s] is the weight of cell h + s - H, the cardinal B-spline of degree
// ORDER at the cell centre's distance:
//   order 0: 1 on cell h;   order 1: -d_+ , 1 - |d|, d_+ on h-1, h, h+1;
//   order 2: 1/2 (1/2 - d)^2, 3/4 - d^2, 1/2 (1/2 + d)^2, written as
//            1/8 + (d^2 -+ d)/2 and 3/4 - d^2;
//   order 3: from the base cell j0 = h (d >= 0) or h - 1 (d < 0) and
//            f = d - (j0 - h) in [0, 1): (1-f)^3/6, 2/3 - f^2 + f^3/2,
//            2/3 - (1-f)^2 + (1-f)^3/2, f^3/6 on cells j0-1 .. j0+2.
// The image reduction is only needed next to the domain ends, so it sits
// behind the lattice test.  Returns nonzero if the particle is off its site.
template <int ORDER>
__device__ __forceinline__ int shape_weights(double zs, double hp, double inv_dz, double nz_d,
                                             double (&w)[Sten<ORDER>::NW]) {
  double d = fma(zs, inv_dz, -hp);
  int bad = 0;
  if (fabs(d) > 0.5 + kLatticeTol) {
    d -= nz_d * rint(d / nz_d);
    bad = fabs(d) > 0.5 + kLatticeTol;
  }
  if constexpr (ORDER == 0) {
    w[0] = 0.0; w[1] = 1.0; w[2] = 0.0;
  } else if constexpr (ORDER == 1) {
    w[0] = fmax(-d, 0.0);
    w[1] = 1.0 - fabs(d);
    w[2] = fmax(d, 0.0);
  } else if constexpr (ORDER == 2) {
    const double d2 = d * d;
    w[1] = 0.75 - d2;
    w[0] = fma(0.5, d2 - d, 0.125);
    w[2] = fma(0.5, d2 + d, 0.125);
  } else {
    const bool up = d >= 0.0;
    const double f = up ? d : 1.0 + d, g = 1.0 - f;
    const double a = g * g * g * (1.0 / 6.0);
    const double bb = fma(f * f, fma(0.5, f, -1.0), 2.0 / 3.0);
    const double c = fma(g * g, fma(0.5, g, -1.0), 2.0 / 3.0);
    const double e = f * f * f * (1.0 / 6.0);
    w[0] = up ? 0.0 : a;
    w[1] = up ? a : bb;
    w[2] = up ? bb : c;
    w[3] = up ? c : e;
    w[4] = up ? e : 0.0;
  }
  return bad;
}

// The lattice test of shape_weights alone: nonzero if the particle at zs is
// off the cell whose centre is hp (in cells), up to the periodic image.
__device__ __forceinline__ int off_site(double zs, double hp, double inv_dz, double nz_d) {
  double d = fma(zs, inv_dz, -hp);
  if (fabs(d) > 0.5 + kLatticeTol) {
    d -= nz_d * rint(d / nz_d);
    return fabs(d) > 0.5 + kLatticeTol;
  }
  return 0;
}

// Loads of data that a fused step launch (k_step) writes before it reads
// them (positions, stage states, shape weights, grid potential, lattice
// shifts) must not take the read-only (non-coherent) path, which is only
// valid across launches.  COH = true selects a weak global load instead: it
// may hit in L1, which the acquire fence of every grid barrier invalidates,
// so after a barrier it sees what other blocks wrote before it.  The
// separate kernels keep the read-only path (ldd, ldi) or a plain load (ldp).
__device__ __forceinline__ double ld_weak(const double* p) {
  double v;
  asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int ld_weak(const int* p) {
  int v;
  asm volatile("ld.global.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
template <bool COH>
__device__ __forceinline__ double ldd(const double* p) {
  if constexpr (COH) return ld_weak(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ int ldi(const int* p) {
  if constexpr (COH) return ld_weak(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ double ldp(const double* p) {
  if constexpr (COH) return ld_weak(p);
  else return *p;
}

// Index of this warp among the warps of a persistent grid: warp i of every
// block comes before warp i + 1 of any block.  Units are split into
// contiguous ranges in this order, so when a batch has fewer units than the
// grid has warps the busy warps spread over all blocks, and so over all SMs
// (GB300's FP64 pipe is shared by the four sub-partitions of an SM), instead
// of filling the first blocks.  The split itself, and so every sum, does not
// depend on this numbering.
__device__ __forceinline__ int64_t logical_warp() {
  return (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
}

// The weights kept by the deposit for the RK stage (order 0: 1 on the own cell).
template <int ORDER, bool COH = false>
__device__ __forceinline__ void load_weights(const double* W, int64_t P, int64_t p, double (&w)[Sten<ORDER>::NW]) {
  if constexpr (ORDER == 0) {
    w[0] = 0.0; w[1] = 1.0; w[2] = 0.0;
  } else {
#pragma unroll
    for (int s = 0; s < Sten<ORDER>::NW; ++s) w[s] = ldp<COH>(W + s * P + p);
  }
}

template <int ORDER>
__device__ __forceinline__ void zero_weights(double (&w)[Sten<ORDER>::NW]) {
#pragma unroll
  for (int s = 0; s < Sten<ORDER>::NW; ++s) w[s] = 0.0;
}

// Interpolation through the stencil (Eq. 6): sum over s of w[s] times the
// value v on the lane of cell h + s - H.  Every lane must call it.
template <int ORDER>
__device__ __forceinline__ double gather(const double (&w)[Sten<ORDER>::NW], double v) {
  if constexpr (ORDER == 0) {
    return v;
  } else {
    constexpr int H = Sten<ORDER>::H, NW = Sten<ORDER>::NW;
    double h = w[NW - 1] * __shfl_down_sync(kFull, v, H);
#pragma unroll
    for (int s = NW - 2; s >= 0; --s) {
      const int o = s - H;
      const double x = o > 0 ? __shfl_down_sync(kFull, v, o) : o < 0 ? __shfl_up_sync(kFull, v, -o) : v;
      h = fma(w[s], x, h);
    }
    return h;
  }
}

// Deposit through the stencil (Eq. 5): a lane's cell receives from the
// particle o lanes to its left the weight that particle gives to cell
// (its site + o), and likewise from the right.  init() shuffles the weights
// once per unit; apply(v) returns the sum over those particles of weight x v.
// Every lane must call both.
template <int ORDER>
struct Spread {
  static constexpr int H = Sten<ORDER>::H;
  double w0, fl[H], fr[H];
  __device__ __forceinline__ void init(const double (&w)[Sten<ORDER>::NW]) {
    w0 = w[H];
#pragma unroll
    for (int o = 1; o <= H; ++o) {
      fl[o - 1] = __shfl_up_sync(kFull, w[H + o], o);
      fr[o - 1] = __shfl_down_sync(kFull, w[H - o], o);
    }
  }
  __device__ __forceinline__ double apply(double v) const {
    if constexpr (ORDER == 0) {
      return v;
    } else {
      double c = fr[H - 1] * __shfl_down_sync(kFull, v, H);
#pragma unroll
      for (int o = H - 1; o >= 1; --o) c = fma(fr[o - 1], __shfl_down_sync(kFull, v, o), c);
      c = fma(w0, v, c);
#pragma unroll
      for (int o = 1; o <= H; ++o) c = fma(fl[o - 1], __shfl_up_sync(kFull, v, o), c);
      return c;
    }
  }
};

// Bulk prefetch of the doubles [i0, i0 + n) of array a into L2 (a hint; the
// range is rounded inwards to 16-byte boundaries so it never leaves the array).
__device__ __forceinline__ void prefetch_l2(const double* a, int64_t i0, int n) {
  uintptr_t lo = ((uintptr_t)(a + i0) + 15) & ~(uintptr_t)15;
  uintptr_t hi = ((uintptr_t)(a + i0 + n)) & ~(uintptr_t)15;
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

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
//
// Every step kernel is a thin wrapper around a *phase*: the work of one warp
// (deposit, RK stage) or of one block (deposit combination, lattice shifts) in
// a persistent grid.  The separate kernels run one phase per launch; the fused
// step kernel (k_step) runs all phases of a step in one cooperative launch
// with grid barriers between them.  COH = true marks the fused form, whose
// loads of data written earlier in the same launch take the coherent path.

// Per-direction table from each ring's first particle: Omega and v_z = c Omega_z
// ([4][MT]); also checks that every particle of a ring carries its direction.
__global__ void k_dirtable(Batch B, Parts pt, double* __restrict__ dirtab, int* __restrict__ err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B.Ptot) return;
  const BoxGeo& g = B.box[box_of_particle(B, p)];
  const int d = (int)((p - g.poff) / g.nz);
  const int64_t p0 = g.poff + (int64_t)d * g.nz;
  const double ox = pt.ox[p0], oy = pt.oy[p0], oz = pt.oz[p0];
  if (pt.ox[p] != ox || pt.oy[p] != oy || pt.oz[p] != oz) atomicOr(err, ERR_RING);
  if (p == p0) {
    const int gd = g.doff + d;
    dirtab[gd] = ox;
    dirtab[B.MT + gd] = oy;
    dirtab[2 * B.MT + gd] = oz;
    dirtab[3 * B.MT + gd] = g.c_light * oz;
  }
}

// Lattice shift of every direction for up to 4 position offsets frac[s] * dt_b:
// the cell of the ring's first particle at z + frac[s] dt_b v_z ([nrows][MT]).
// A fifth row (nrows = 5) holds the shift of the next step's first stage: the
// cell of wrap(z + dt_b v_z), the position stage 4 writes, computed exactly as
// the RK stage computes it.  Beside each shift row the ring's shape weights
// (the direction weight table, kWSlots per row): a ring translates rigidly, so
// all its particles sit at its first particle's offset inside their cells.
struct Fracs { double v[4]; };

// Position offset of RK stage s (0-based), in units of dt (Sec. 2.3, classic tableau).
__device__ __forceinline__ double stage_frac(int s) { return s == 0 ? 0.0 : s == 3 ? 1.0 : 0.5; }

__device__ __forceinline__ int lattice_cell(double z0, double frac_dt, double vz, const BoxGeo& g) {
  const double zs = fma(frac_dt, vz, z0);
  return wrapc((int)floor(zs * g.inv_dz), g.nz);
}

// Row `row` of the tables for direction gd: the shift (the cell of the ring's
// first particle at its row position) and, with wtab, that particle's shape
// weights there.  Rows 0-3: z + frac[row] dt_b v_z; row 4: wrap(z + dt_b v_z).
template <bool COH, int ORDER>
__device__ __forceinline__ void shifts_row(const Batch& B, int gd, const double* z, const double* __restrict__ dirtab,
                                           const Fracs& fr, int row, int* shift, double* wtab) {
  const int b = box_of_direction(B, gd);
  const BoxGeo& g = B.box[b];
  const double z0 = ldp<COH>(z + g.poff + (int64_t)(gd - g.doff) * g.nz);
  const double vz = dirtab[3 * B.MT + gd];
  const double dt = B.dt[b];
  const double zs = row < 4 ? fma(fr.v[row] * dt, vz, z0) : wrap_z(fma(dt, vz, z0), g.Lz);
  const int cell = lattice_cell(zs, 0.0, vz, g);
  shift[row * B.MT + gd] = cell;
  if (wtab != nullptr) {   // the ring's weights: its first particle's, at the cell the shift assigns it
    double w[Sten<ORDER>::NW];
    (void)shape_weights<ORDER>(zs, (double)cell + 0.5, g.inv_dz, g.nz_d, w);
#pragma unroll
    for (int q = 0; q < Sten<ORDER>::NWS; ++q) wtab[(row * kWSlots + q) * B.MT + gd] = w[q];
  }
}

template <bool COH, int ORDER>
__device__ __forceinline__ void shifts_phase(const Batch& B, int gd, const double* z, const double* __restrict__ dirtab,
                                             const Fracs& fr, int nrows, int* shift, double* wtab) {
  if (gd >= B.MT) return;
  for (int row = 0; row < nrows && row < 5; ++row) shifts_row<COH, ORDER>(B, gd, z, dirtab, fr, row, shift, wtab);
}

// One thread per (direction, row): the rows' chains run side by side.
template <int ORDER>
__global__ void k_shifts(Batch B, const double* __restrict__ z, const double* __restrict__ dirtab, Fracs fr,
                         int nrows, int* __restrict__ shift, double* __restrict__ wtab) {
  griddep_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / B.MT, gd = t - row * B.MT;
  if (row >= nrows) return;
  shifts_row<false, ORDER>(B, gd, z, dirtab, fr, row, shift, wtab);
}

// A warp's sums for one tile go to slot (warp + global tile) of the partial
// buffer: unique, because a later warp never returns to an earlier tile.
template <int ORDER, int NA>
__device__ __forceinline__ void flush_tile(const double (&acc)[NA], int64_t gtile, int local_cell, int nz,
                                           int64_t w, int lane, double* __restrict__ partial) {
  constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T;
  if (lane >= H && lane < H + T && local_cell < nz) {
    double* slot = partial + (w + gtile) * kSlot + lane - H;
#pragma unroll
    for (int c = 0; c < NA; ++c) slot[c * T] = acc[c];
  }
}

// The direction loop of the deposit for one tile: warp lane `lane` of a tile
// of box b (lane l owns cell tile * T - H + l) adds the rings dfirst..dlast-1
// of the tile, in order, to acc (MODES as deposit_phase).  Shared by the
// per-warp deposit and the cluster deposit.
template <int MODE, int ORDER, bool COH, int NA>
__device__ __forceinline__ void deposit_tile_dirs(const Batch& B, int b, int tile, int dfirst, int dlast, int lane,
                                                  const double* z, const double* __restrict__ N,
                                                  const double* __restrict__ Nbar, const double* r_nu,
                                                  const double* r_nb, const double* __restrict__ dirtab,
                                                  const int* shift, const double* wrow, double frac, double* W,
                                                  double (&acc)[NA], int& bad) {
  const BoxGeo& g = B.box[b];
  const int nz = g.nz;
  const int64_t P = B.Ptot;
  const int MT = B.MT;
  constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T;
  const int craw = tile * T - H + lane;
  const int j = wrapc(craw, nz);
  const double hp = (double)j + 0.5;
  const bool own = lane >= H && lane < H + T && craw < nz;
  const double pos_dt = frac * B.dt[b];
  const int64_t pbase = g.poff;
  const int dbase = g.doff;
  for (int d = dfirst; d < dlast; ++d) {
    const int gd = dbase + d;
    const double ox = __ldg(dirtab + gd), oy = __ldg(dirtab + MT + gd), oz = __ldg(dirtab + 2 * MT + gd);
    const double vz = __ldg(dirtab + 3 * MT + gd);
    const int64_t p = pbase + (int64_t)d * nz + wrapc(j - ldi<COH>(shift + gd), nz);
    double wt[Sten<ORDER>::NW];
    const double zs = fma(pos_dt, vz, ldd<COH>(z + p));
    if (wrow != nullptr) {
      bad |= off_site(zs, hp, __ldg(&g.inv_dz), __ldg(&g.nz_d));
      if constexpr (ORDER == 0) {
        wt[0] = 0.0; wt[1] = 1.0; wt[2] = 0.0;
      } else {
#pragma unroll
        for (int q = 0; q < Sten<ORDER>::NW; ++q) wt[q] = ldp<COH>(wrow + q * B.MT + gd);
      }
    } else {
      bad |= shape_weights<ORDER>(zs, hp, __ldg(&g.inv_dz), __ldg(&g.nz_d), wt);
    }
    if ((MODE == 0 || MODE == 5) && W != nullptr && own) {   // the RK stage of these positions reads them back
#pragma unroll
      for (int q = 0; q < Sten<ORDER>::NWS; ++q) W[q * P + p] = wt[q];
    }
    Spread<ORDER> spread;
    spread.init(wt);
    if constexpr (MODE == 5) {
      const double n1 = __ldg(N + p), n2 = __ldg(Nbar + p);
      double bprev = 0.0;   // B of the previous diagonal entry
#pragma unroll
      for (int c = 0; c < kNC; ++c) {
        double bv;
        if (c < 2) {
          if (c == 0) bprev = fma(-n2, ldd<COH>(r_nb + p), n1 * ldd<COH>(r_nu + p));
          const double bn =
              fma(-n2, ldd<COH>(r_nb + (c + 1) * P + p), n1 * ldd<COH>(r_nu + (c + 1) * P + p));
          bv = bprev - bn;
          bprev = bn;
        } else {
          const int k = c + 1;
          const double x = ldd<COH>(r_nu + k * P + p), y = ldd<COH>(r_nb + k * P + p);
          bv = (k == 4 || k == 6 || k == 8) ? fma(n2, y, n1 * x) : fma(-n2, y, n1 * x);
        }
        const double cc = spread.apply(bv);
        acc[c] += cc;
        acc[kNC + c] = fma(ox, cc, acc[kNC + c]);
        acc[2 * kNC + c] = fma(oy, cc, acc[2 * kNC + c]);
        acc[3 * kNC + c] = fma(oz, cc, acc[3 * kNC + c]);
      }
    } else if constexpr (MODE == 4) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const double c1 = spread.apply(__ldg(N + p) * ldd<COH>(r_nu + k * P + p));
        const double c2 = spread.apply(__ldg(Nbar + p) * ldd<COH>(r_nb + k * P + p));
        acc[k] += c1;
        acc[9 + k] = fma(ox, c1, acc[9 + k]);
        acc[18 + k] += c2;
        acc[27 + k] = fma(ox, c2, acc[27 + k]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        // (the weights are read inside the loop: fewer live registers across it)
        const double n1 = (MODE == 0 || MODE == 1) ? __ldg(N + p) : 0.0;
        const double n2 = (MODE == 0 || MODE == 2) ? __ldg(Nbar + p) : 0.0;
        double bv;
        if (MODE == 0) {
          const double x = ldd<COH>(r_nu + k * P + p), y = ldd<COH>(r_nb + k * P + p);
          // conj(rhobar) flips the sign of the imaginary components 4, 6, 8
          bv = (k == 4 || k == 6 || k == 8) ? fma(n2, y, n1 * x) : fma(-n2, y, n1 * x);
        } else if (MODE == 1) {
          bv = n1 * ldd<COH>(r_nu + k * P + p);
        } else if (MODE == 2) {
          bv = n2 * ldd<COH>(r_nb + k * P + p);
        } else {
          bv = ldd<COH>(r_nu + k * P + p);
        }
        const double c = spread.apply(bv);
        acc[k] += c;
        acc[9 + k] = fma(ox, c, acc[9 + k]);
        acc[18 + k] = fma(oy, c, acc[18 + k]);
        acc[27 + k] = fma(oz, c, acc[27 + k]);
      }
    }
  }
}

// Deposit (Eq. 5), first phase.  MODE 0: B = N rho - Nbar rhobar^* (the
// combination that enters H, Eq. 2); MODE 1: B = N rho; MODE 2: B = Nbar rhobar;
// MODE 3: B = r_nu (packed matrices given per particle: the adjoint's Gamma);
// MODE 4: the moments the diagnostics read (Eq. 10), both species in one
// pass: rows 0-8 n, 9-17 f_x (from N rho), 18-26 nbar, 27-35 fbar_x (Nbar rhobar);
// MODE 5: MODE 0's B in the traceless components the step reads (kNT rows:
// moment m, component c at row m * kNC + c; c = 0, 1 the diagonal differences
// B_11 - B_22 and B_22 - B_33, c = 2..7 the off-diagonal reals 3..8).
// Warp w walks its units in order (box, tile, direction), summing
// w_pj (1, Omega_p) B_p over directions in registers (lane l owns cell
// tile * T - H + l) and writing one partial per tile it touches; MODES 0 and 5
// also store every particle's weights for the RK stage.  Positions: z + frac dt_b v_z.
// With wrow (the stage's row of the direction weight table k_shifts writes)
// every particle of a ring takes the ring's weights: the ring translates
// rigidly, so its particles share their offset inside the cells (to
// rounding); each particle's position is still checked against its cell.
template <int MODE, int ORDER, bool COH>
__device__ __forceinline__ void deposit_phase(const Batch& B, int64_t w, int lane, const double* z,
                                              const double* __restrict__ N, const double* __restrict__ Nbar,
                                              const double* r_nu, const double* r_nb,
                                              const double* __restrict__ dirtab, const int* shift,
                                              const double* wrow, double frac, double* __restrict__ partial,
                                              double* W, int* err) {
  const int64_t u0 = unit_begin(w, B), u1 = unit_begin(w + 1, B);
  if (u0 >= u1) return;
  int bad = 0;
  int b = box_of_unit(B, u0);
  for (int64_t u = u0; u < u1;) {        // one segment per (box, tile) the warp touches
    while (u >= B.box[b].uoff + (int64_t)B.box[b].ntiles * B.box[b].M) ++b;
    const BoxGeo& g = B.box[b];
    const int M = g.M;
    const int tile = (int)((u - g.uoff) / M);
    const int64_t uend = min(u1, g.uoff + (int64_t)(tile + 1) * M);
    const int64_t ubase = g.uoff + (int64_t)tile * M;
    const int dfirst = (int)(u - ubase), dlast = (int)(uend - ubase);
    u = uend;
    constexpr int NA = MODE == 5 ? kNT : kNA;
    double acc[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) acc[c] = 0.0;
    deposit_tile_dirs<MODE, ORDER, COH>(B, b, tile, dfirst, dlast, lane, z, N, Nbar, r_nu, r_nb, dirtab, shift, wrow,
                                        frac, W, acc, bad);
    constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T;
    flush_tile<ORDER>(acc, g.toff + tile, tile * T - H + lane, g.nz, w, lane, partial);
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// TAB: the rings' weights from the weight row wrow; otherwise each
// particle's own (wrow unused, and the table's code compiled out).
template <int MODE, int ORDER, bool TAB = false>
__global__ void __launch_bounds__(kThreads, 2)
k_deposit(Batch B, const double* __restrict__ z, const double* __restrict__ N, const double* __restrict__ Nbar,
          const double* __restrict__ r_nu, const double* __restrict__ r_nb, const double* __restrict__ dirtab,
          const int* __restrict__ shift, const double* __restrict__ wrow, double frac, double* __restrict__ partial,
          double* __restrict__ W, int* __restrict__ err) {
  griddep_wait();
  deposit_phase<MODE, ORDER, false>(B, logical_warp(), threadIdx.x & 31, z, N, Nbar, r_nu, r_nb, dirtab, shift,
                                    TAB ? wrow : nullptr, frac, partial, W, err);
}

// ------------------------------------------------------- cluster deposit
//
// The step's deposit (MODE 5) by thread-block clusters of CL blocks (8 or 16),
// with no separate combination: cluster c takes the tiles c, c + clusters,
// ... (all boxes' tiles in order).  For each tile the cluster's W =
// CL x kWarps warps split its rings (warp i: rings [i M / W,
// (i + 1) M / W), summed in order in registers as in deposit_phase); the
// warps of each block are added in warp order through shared memory, then the
// blocks in rank order through distributed shared memory, and the potential
// of the tile's cells is written.  The summation order depends only on the
// box and the cluster size, not on the grid: results are bitwise reproducible.
// All blocks of a cluster walk the same tiles, so every block reaches every
// cluster barrier (hardware barriers, as __syncthreads: no spin on memory).
constexpr int kDepClusterSmem = kWarps * kNT * kLanes * (int)sizeof(double);   // 64 KB

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Barrier of all threads of the cluster; shared-memory writes before it are
// visible to every block of the cluster after it.  (The non-.aligned form:
// correct whether or not the threads of a warp arrive together.)
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// The double at this block's shared address a, read from block `rank` of the cluster.
__device__ __forceinline__ double ld_cluster(const double* a, unsigned rank) {
  const unsigned local = (unsigned)__cvta_generic_to_shared(a);
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
  return v;
}

__device__ __forceinline__ int box_of_tile(const Batch& B, int64_t t) {
  int lo = 0, hi = B.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.box[mid].toff <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// out: the potential ([kNT][NZ], scale kappa / dV of each box); W as k_deposit.
template <int ORDER, bool TAB, int CL>
__global__ void __launch_bounds__(kThreads, 2)
k_deposit_cluster(Batch B, const double* __restrict__ z, const double* __restrict__ N,
                  const double* __restrict__ Nbar, const double* __restrict__ r_nu, const double* __restrict__ r_nb,
                  const double* __restrict__ dirtab, const int* __restrict__ shift, const double* __restrict__ wrow,
                  double frac, double* __restrict__ out, double* __restrict__ W, int* __restrict__ err) {
  griddep_wait();
  extern __shared__ double red[];   // [kWarps][kNT][kLanes]: each warp's sums of the tile
  constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T;
  constexpr int NE = kNT * kLanes, per = NE / CL, nwc = CL * kWarps;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned rank = cluster_rank();
  const int gw = (int)rank * kWarps + wib;
  int bad = 0, nonfinite = 0;
  for (int64_t gt = cluster_index(); gt < B.NT; gt += cluster_count()) {
    const int b = box_of_tile(B, gt);
    const BoxGeo& g = B.box[b];
    const int tile = (int)(gt - g.toff);
    const int d0 = (int)((int64_t)gw * g.M / nwc), d1 = (int)((int64_t)(gw + 1) * g.M / nwc);
    double acc[kNT];
#pragma unroll
    for (int c = 0; c < kNT; ++c) acc[c] = 0.0;
    if (d0 < d1)
      deposit_tile_dirs<5, ORDER, false>(B, b, tile, d0, d1, lane, z, N, Nbar, r_nu, r_nb, dirtab, shift,
                                         TAB ? wrow : nullptr, frac, W, acc, bad);
#pragma unroll
    for (int c = 0; c < kNT; ++c) red[(wib * kNT + c) * kLanes + lane] = acc[c];
    __syncthreads();
    for (int e = threadIdx.x; e < NE; e += kThreads) {   // the block's warps, in warp order
      double v = red[e];
#pragma unroll
      for (int i = 1; i < kWarps; ++i) v += red[i * NE + e];
      red[e] = v;
    }
    cluster_sync();
    if (threadIdx.x < per) {   // the cluster's blocks, in rank order; this block's share of the outputs
      const int e = (int)rank * per + threadIdx.x;
      double v = ld_cluster(red + e, 0);
#pragma unroll
      for (unsigned q = 1; q < CL; ++q) v += ld_cluster(red + e, q);
      const int c = e / kLanes, l = e - c * kLanes, craw = tile * T - H + l;
      if (l >= H && l < H + T && craw < g.nz) {
        v *= g.kappa_dV;
        nonfinite |= !isfinite(v);
        out[(int64_t)c * B.NZ + g.coff + craw] = v;
      }
    }
    cluster_sync();   // the slots are free for the next tile, and no block leaves while read
  }
  if (bad) atomicOr(err, ERR_LATTICE);
  if (nonfinite) atomicOr(err, ERR_NONFINITE);
}

// Deposit, second phase: fixed-order sum of the per-warp partials.
// out[c * NZ + coff_b + j] (c < rows) = scale_b * (sum over the warps that own
// units of j's tile), scale_b = kappa_b / dV_b (potential) or 1 / dV_b.  Lane l of a warp
// takes output e0 + l (consecutive cells: coalesced reads of the partials).
// With `split` > 1 (a power of two <= 8), `split` warps of a block take the
// same 32 outputs: warp i adds the partials of warps wf + i, wf + i + split,
// ..., and the first adds the split sums in warp order through shared
// memory.  A warp keeps kCombineILP running sums (its partials taken
// round-robin, then added pairwise) so that many loads are in flight.  The
// order depends only on the batch, the number of warps that split the units
// and `split`, not on the grid of this phase: results are bitwise reproducible.
// The partials are read through L2 (coherent within a fused launch too).
constexpr int kCombineILP = 8;
__device__ __forceinline__ void combine_phase(const Batch& B, const double* partial, double* out, int rows,
                                              int potential, int split, int* err) {
  __shared__ double sums[kWarps][kLanes];
  const int64_t n = (int64_t)rows * B.NZ;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int grp = wib / split, wi = wib - grp * split;       // output group of this warp, rank within it
  const int groups = kWarps / split;
  int bad = 0;
  // every block runs the same number of rounds (it synchronises inside)
  for (int64_t base = (int64_t)blockIdx.x * groups * kLanes; base < n; base += (int64_t)gridDim.x * groups * kLanes) {
    const int64_t e = base + (int64_t)grp * kLanes + lane;
    double v = 0.0;
    const BoxGeo* g = nullptr;
    if (e < n) {
      const int c = (int)(e / B.NZ), gc = (int)(e - (int64_t)c * B.NZ);
      g = &B.box[box_of_cell(B, gc)];
      const int lc = gc - g->coff;
      const int tile = lc / B.T, k = lc - tile * B.T;
      const int64_t gtile = g->toff + tile;
      const int64_t wf = warp_of_unit(g->uoff + (int64_t)tile * g->M, B);
      const int64_t wl = warp_of_unit(g->uoff + (int64_t)(tile + 1) * g->M - 1, B);
      const double* src = partial + c * B.T + k;
      double a[kCombineILP] = {};
      int64_t q = wf + wi;
      for (; q + (kCombineILP - 1) * split <= wl; q += kCombineILP * split) {
#pragma unroll
        for (int i = 0; i < kCombineILP; ++i) a[i] += __ldcg(src + (q + i * split + gtile) * kSlot);
      }
      for (; q <= wl; q += split) a[0] += __ldcg(src + (q + gtile) * kSlot);
#pragma unroll
      for (int h = kCombineILP / 2; h >= 1; h /= 2) {   // pairwise: ((a0 + a4) + (a2 + a6)) + ...
#pragma unroll
        for (int i = 0; i < h; ++i) a[i] += a[i + h];
      }
      v = a[0];
    }
    if (split > 1) {
      sums[wib][lane] = v;
      __syncthreads();
      if (wi == 0)
        for (int i = 1; i < split; ++i) v += sums[wib + i][lane];
      __syncthreads();
    }
    if (e < n && wi == 0) {
      v *= potential ? g->kappa_dV : g->inv_dV;
      bad |= !isfinite(v);
      out[e] = v;
    }
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

__global__ void k_combine(Batch B, const double* __restrict__ partial, double* __restrict__ out, int rows,
                          int potential, int split, int* __restrict__ err) {
  griddep_wait();
  combine_phase(B, partial, out, rows, potential, split, err);
}

// Interpolation only (Eq. 6 then Eq. 2): H[k * Ptot + p] at z + frac dt_b v_z.
template <int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k_interpolate(Batch B, const double* __restrict__ z, const double* __restrict__ dirtab,
              const int* __restrict__ shift, const double* __restrict__ A, double frac, double* __restrict__ Hout,
              int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int64_t u0 = unit_begin(w, B), u1 = unit_begin(w + 1, B);
  const int64_t P = B.Ptot;
  const int MT = B.MT, NZ = B.NZ;
  int bad = 0;
  if (u0 >= u1) return;
  int b = box_of_unit(B, u0);
  for (int64_t u = u0; u < u1; ++u) {
    while (u >= B.box[b].uoff + (int64_t)B.box[b].ntiles * B.box[b].M) ++b;
    const BoxGeo& g = B.box[b];
    const int nz = g.nz, M = g.M;
    const int tile = (int)((u - g.uoff) / M), d = (int)(u - g.uoff - (int64_t)tile * M);
    constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T;
    const int craw = tile * T - H + lane, j = wrapc(craw, nz);
    const bool active = lane >= H && lane < H + T && craw < nz;
    const int gd = g.doff + d;
    const double ox = __ldg(dirtab + gd), oy = __ldg(dirtab + MT + gd), oz = __ldg(dirtab + 2 * MT + gd);
    const double vz = __ldg(dirtab + 3 * MT + gd);
    const int64_t p = g.poff + (int64_t)d * nz + wrapc(j - __ldg(shift + gd), nz);
    double wt[Sten<ORDER>::NW];
    zero_weights<ORDER>(wt);
    if (active) bad |= shape_weights<ORDER>(fma(frac * B.dt[b], vz, z[p]), (double)j + 0.5, g.inv_dz, g.nz_d, wt);
    const double* Aj = A + g.coff + j;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double G = fma(-oz, __ldg(Aj + (int64_t)(27 + k) * NZ),
                           fma(-oy, __ldg(Aj + (int64_t)(18 + k) * NZ),
                               fma(-ox, __ldg(Aj + (int64_t)(9 + k) * NZ), __ldg(Aj + (int64_t)k * NZ))));
      const double h = gather<ORDER>(wt, G);
      if (active) Hout[k * P + p] = h;
    }
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// The RK4 update (Sec. 2.3) of particle p (ring direction gd) of box g at
// stage s, given its interpolated self-interaction Hamiltonian Hm (Eq. 6,
// Eq. 2) and its neutrino source matrix r (already loaded): K = -i[H, rho],
// Kbar = -i[Hbar, rhobar] (Eq. 4) with Hbar = -H^* (plus the vacuum and
// matter terms with POT), then the accumulator and next stage state (stage 4:
// the new state and position).  vz points at the particle's v_z in the
// direction table.  With KEEP
// the state it stores (the next stage's, or at stage 4 the new one), rho and
// rhobar, is also combined as B = n1 rho - n2 rhobar^* into keep[9] (the
// arithmetic of the deposit, Eq. 5) and the new position returned in *zkeep.
template <bool POT, bool COH, bool KEEP = false>
__device__ __forceinline__ void rk_particle(const BoxGeo& g, const Parts& pt, const double* src_b, int64_t P,
                                            int64_t p, int s, int dry, double bdt, double cdt, double dtb,
                                            const double* __restrict__ vz, double (&Hm)[kNC], const double (&r)[9],
                                            double* keep = nullptr, double* zkeep = nullptr, double n1 = 0.0,
                                            double n2 = 0.0) {
  const double bdt2 = 2.0 * bdt, cdt2 = 2.0 * cdt;   // diagonal K are returned halved
  // Hm: H in the traceless components.  Antineutrinos: Hbar = -H^* (diagonal
  // differences and real parts flip sign, imaginary parts stay)
  double Hb[kNC];
  if (POT) {
    const double* vn = g.vnu;
    const double* vb = g.vnubar;
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const bool im = (c == 3 || c == 5 || c == 7);
      Hb[c] = (im ? Hm[c] : -Hm[c]) + __ldg(vb + c);
      Hm[c] += __ldg(vn + c);
    }
  }
  const double d12 = Hm[0], d23 = Hm[1], d13 = d12 + d23;
#pragma unroll
  for (int which = 0; which < 2; ++which) {
    double* __restrict__ yv = which ? pt.rhobar : pt.rho;
    double* __restrict__ av = pt.acc + which * 9 * P;
    double* __restrict__ sv = pt.stage + which * 9 * P;
    // all loads of this matrix before any store (the arrays do not alias)
    double a[9], y[9], rb[9];
    if (which == 1) {
#pragma unroll
      for (int k = 0; k < 9; ++k) rb[k] = ldp<COH>(src_b + k * P + p);
    }
    if (s >= 2) {
#pragma unroll
      for (int k = 0; k < 9; ++k) a[k] = ldp<COH>(av + k * P + p);
    }
    if (s == 2 || s == 3) {
#pragma unroll
      for (int k = 0; k < 9; ++k) y[k] = ldp<COH>(yv + k * P + p);
    }
    const double* rr = which ? rb : r;
    double kd[3], ko[6];
    if (which == 0) commutator(d12, d13, d23, Hm[2], Hm[3], Hm[4], Hm[5], Hm[6], Hm[7], rr, kd, ko);
    else if (POT) commutator(Hb[0], Hb[0] + Hb[1], Hb[1], Hb[2], Hb[3], Hb[4], Hb[5], Hb[6], Hb[7], rr, kd, ko);
    else commutator(-d12, -d13, -d23, -Hm[2], Hm[3], -Hm[4], Hm[5], -Hm[6], Hm[7], rr, kd, ko);
    if constexpr (!KEEP) {
      if (s == 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          av[k * P + p] = fma(bdt2, kd[k], rr[k]);
          sv[k * P + p] = fma(cdt2, kd[k], rr[k]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          av[(k + 3) * P + p] = fma(bdt, ko[k], rr[k + 3]);
          sv[(k + 3) * P + p] = fma(cdt, ko[k], rr[k + 3]);
        }
      } else if (s < 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          av[k * P + p] = fma(bdt2, kd[k], a[k]);
          sv[k * P + p] = fma(cdt2, kd[k], y[k]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          av[(k + 3) * P + p] = fma(bdt, ko[k], a[k + 3]);
          sv[(k + 3) * P + p] = fma(cdt, ko[k], y[k + 3]);
        }
      } else {
        double* __restrict__ dst = dry ? sv : yv;
#pragma unroll
        for (int k = 0; k < 3; ++k) dst[k * P + p] = fma(bdt2, kd[k], a[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) dst[(k + 3) * P + p] = fma(bdt, ko[k], a[k + 3]);
      }
    } else {
      double nv[9];   // the state stored as the next stage's (stage 4: the new state)
      if (s == 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { av[k * P + p] = fma(bdt2, kd[k], rr[k]); nv[k] = fma(cdt2, kd[k], rr[k]); }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          av[(k + 3) * P + p] = fma(bdt, ko[k], rr[k + 3]);
          nv[k + 3] = fma(cdt, ko[k], rr[k + 3]);
        }
      } else if (s < 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { av[k * P + p] = fma(bdt2, kd[k], a[k]); nv[k] = fma(cdt2, kd[k], y[k]); }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          av[(k + 3) * P + p] = fma(bdt, ko[k], a[k + 3]);
          nv[k + 3] = fma(cdt, ko[k], y[k + 3]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) nv[k] = fma(bdt2, kd[k], a[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) nv[k + 3] = fma(bdt, ko[k], a[k + 3]);
      }
      double* __restrict__ dst = (s < 4 || dry) ? sv : yv;
#pragma unroll
      for (int k = 0; k < 9; ++k) dst[k * P + p] = nv[k];
      // B = n1 rho - n2 rhobar^*: conj(rhobar) flips the sign of the imaginary components 4, 6, 8
      if (which == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) keep[k] = n1 * nv[k];
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) keep[k] = fma((k == 4 || k == 6 || k == 8) ? n2 : -n2, nv[k], keep[k]);
      }
    }
  }
  if (s == 4) {
    const double vzv = *vz;   // (a plain load: vz may point at a caller's local value)
    const double zn = wrap_z(fma(dtb, vzv, ldp<COH>(pt.z + p)), g.Lz);
    if (dry) pt.stage[p] = zn;  // (only to keep the work of the real stage)
    else pt.z[p] = zn;
    if constexpr (KEEP) *zkeep = zn;
  }
}

// One RK4 stage s (1..4) after the deposit of the stage state: interpolate
// (Eq. 6), H and Hbar = -H^* (Eq. 2, Sec. 2.1), K = -i[H, rho] and
// Kbar = -i[Hbar, rhobar] (Eq. 4), then the classic RK4 update (Sec. 2.3):
//   s = 1: acc = y + dt/6 K,  stage = y + dt/2 K
//   s = 2: acc += dt/3 K,     stage = y + dt/2 K
//   s = 3: acc += dt/3 K,     stage = y + dt K
//   s = 4: y = acc + dt/6 K,  z = wrap(z + dt v_z)   (dry: into the stage buffer instead)
// With POT the constant vacuum and matter terms of the box are added:
// H = H_self + V, Hbar = -H_self^* + Vbar (Eq. 2, Sec. 2.1).
// Persistent: each warp walks its contiguous range of units, direction-major
// within a box (unit = direction * ntiles + tile) so it streams along each
// ring, and prefetches the next unit's particle data into L2.  The shape
// weights come from the deposit.  Stages 2-4 read their state from stage_src
// (normally the stage buffer itself, updated in place; a separate buffer when
// the stage states are kept for the adjoint).
template <bool POT, int ORDER, bool COH>
__device__ __forceinline__ void rk_phase(const Batch& B, int64_t w, int lane, const Parts& pt, const double* W,
                                         const double* __restrict__ dirtab, const int* shift, const double* A,
                                         const double* stage_src, int s, int dry) {
  const int64_t u0 = unit_begin(w, B), u1 = unit_begin(w + 1, B);
  if (u0 >= u1) return;
  const int64_t P = B.Ptot;
  const int MT = B.MT, NZ = B.NZ;
  const double* src_r = (s == 1) ? pt.rho : stage_src;
  const double* src_b = (s == 1) ? pt.rhobar : stage_src + 9 * P;
  // arrays this stage reads, for the prefetch: source (18), y (18, s = 2, 3), acc (18, s >= 2), W (NWS), z (s = 4)
  constexpr int H = Sten<ORDER>::H, T = Sten<ORDER>::T, NWS = Sten<ORDER>::NWS;
  const int nsrc = 18, ny = (s == 2 || s == 3) ? 18 : 0, nacc = (s >= 2) ? 18 : 0;
  const int narr = nsrc + ny + nacc + NWS + (s == 4 ? 1 : 0);
  int b = box_of_unit(B, u0);
  double bdt = 0.0, cdt = 0.0;
  int bcur = -1;
  for (int64_t u = u0; u < u1; ++u) {
    while (u >= B.box[b].uoff + (int64_t)B.box[b].ntiles * B.box[b].M) ++b;
    const BoxGeo& g = B.box[b];
    const int nz = g.nz, nt = g.ntiles;
    if (b != bcur) {
      bcur = b;
      const double dt = B.dt[b];
      bdt = (s == 1 || s == 4) ? dt / 6.0 : dt / 3.0;   // weight of K in acc
      cdt = (s == 3) ? dt : 0.5 * dt;                   // offset of the next stage
    }
    const int lu = (int)(u - g.uoff);        // unit within the box: direction-major
    const int d = lu / nt, tile = lu - d * nt;
    if (u + 1 < u1 && lu + 1 < nt * g.M) {   // prefetch the next unit of the same box
      const int dn = (lu + 1) / nt, tn = lu + 1 - dn * nt;
      const int i0 = tn * T - ldi<COH>(shift + g.doff + dn);   // ring index of the next unit's first cell
      const int n = min(T, nz - tn * T);
      if (i0 >= 0 && i0 + n <= nz) {
        const int64_t base = g.poff + (int64_t)dn * nz + i0;
        for (int a = lane; a < narr; a += kLanes) {
          const double* arr;
          if (a < nsrc) arr = (a < 9 ? src_r + (int64_t)a * P : src_b + (int64_t)(a - 9) * P);
          else if (a < nsrc + ny) arr = (a - nsrc < 9 ? pt.rho + (int64_t)(a - nsrc) * P
                                                      : pt.rhobar + (int64_t)(a - nsrc - 9) * P);
          else if (a < nsrc + ny + nacc) arr = pt.acc + (int64_t)(a - nsrc - ny) * P;
          else if (a < nsrc + ny + nacc + NWS) arr = W + (int64_t)(a - nsrc - ny - nacc) * P;
          else arr = pt.z;
          prefetch_l2(arr, base, n);
        }
      }
    }
    const int craw = tile * T - H + lane, j = wrapc(craw, nz);
    const bool active = lane >= H && lane < H + T && craw < nz;
    const int gd = g.doff + d;
    const double ox = __ldg(dirtab + gd), oy = __ldg(dirtab + MT + gd), oz = __ldg(dirtab + 2 * MT + gd);
    const int64_t p = g.poff + (int64_t)d * nz + wrapc(j - ldi<COH>(shift + gd), nz);
    double wt[Sten<ORDER>::NW];
    zero_weights<ORDER>(wt);
    // the neutrino source matrix first, so its latency overlaps the interpolation
    double r[9];
    if (active) {
      load_weights<ORDER, COH>(W, P, p, wt);
#pragma unroll
      for (int k = 0; k < 9; ++k) r[k] = ldp<COH>(src_r + k * P + p);
    }
    double Hm[kNC];
    const double* Aj = A + g.coff + j;
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const double G = fma(-oz, ldd<COH>(Aj + (int64_t)(3 * kNC + c) * NZ),
                           fma(-oy, ldd<COH>(Aj + (int64_t)(2 * kNC + c) * NZ),
                               fma(-ox, ldd<COH>(Aj + (int64_t)(kNC + c) * NZ), ldd<COH>(Aj + (int64_t)c * NZ))));
      Hm[c] = gather<ORDER>(wt, G);
    }
    if (!active) continue;
    rk_particle<POT, COH>(g, pt, src_b, P, p, s, dry, bdt, cdt, B.dt[b], dirtab + 3 * MT + gd, Hm, r);
  }
}

template <bool POT, int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k_rk_stage(Batch B, Parts pt, const double* __restrict__ W, const double* __restrict__ dirtab,
           const int* __restrict__ shift, const double* __restrict__ A, const double* stage_src, int s, int dry) {
  griddep_wait();
  rk_phase<POT, ORDER, false>(B, logical_warp(), threadIdx.x & 31, pt, W, dirtab, shift, A, stage_src, s, dry);
}

// The RK stage with 32 cells per warp: the same arithmetic as k_rk_stage,
// without its halo lanes (two for shape orders 0-2, four for the cubic
// shape).  Units are (32-cell tile, direction), direction-major, split evenly
// over the warps.  A warp writes G = A0 - Omega . A of a unit's cells into
// shared memory and finishes that unit one iteration later, when the next
// tile's first cells are known: the stencil neighbours of its end cells (H on
// each side) come from the adjacent tiles of the same ring when the warp
// handles them in order, and are computed directly (one cell at a time, by the
// whole warp) at ring and range boundaries.
template <bool COH>
__device__ __forceinline__ void ring_cell_G(const double* A, int NZ, int coff, int cell, double ox, double oy,
                                            double oz, double (&G)[kNC]) {
  const double* Aj = A + coff + cell;
#pragma unroll
  for (int c = 0; c < kNC; ++c)
    G[c] = fma(-oz, ldd<COH>(Aj + (int64_t)(3 * kNC + c) * NZ),
               fma(-oy, ldd<COH>(Aj + (int64_t)(2 * kNC + c) * NZ),
                   fma(-ox, ldd<COH>(Aj + (int64_t)(kNC + c) * NZ), ldd<COH>(Aj + (int64_t)c * NZ))));
}

// Component c of G at one cell, the arithmetic of ring_cell_G (for one lane
// per component).
template <bool COH>
__device__ __forceinline__ double cell_G_component(const double* A, int NZ, int coff, int cell, int c, double ox,
                                                   double oy, double oz) {
  const double* Aj = A + coff + cell;
  return fma(-oz, ldd<COH>(Aj + (int64_t)(3 * kNC + c) * NZ),
             fma(-oy, ldd<COH>(Aj + (int64_t)(2 * kNC + c) * NZ),
                 fma(-ox, ldd<COH>(Aj + (int64_t)(kNC + c) * NZ), ldd<COH>(Aj + (int64_t)c * NZ))));
}

// Cell index on a ring of nz cells for cells within two rings of it (the
// stencil reaches at most two cells past a tile; rings may be shorter).
__device__ __forceinline__ int ring_wrap(int cell, int nz) {
  while (cell < 0) cell += nz;
  while (cell >= nz) cell -= nz;
  return cell;
}

template <bool POT, int ORDER, bool COH>
__device__ __forceinline__ void rk32_phase(const Batch& B, int64_t w, const Parts& pt, const double* W,
                                           const double* __restrict__ dirtab, const int* shift, const double* A,
                                           const double* stage_src, int s, int dry) {
  constexpr int H = Sten<ORDER>::H, NW = Sten<ORDER>::NW;
  __shared__ double gsm[kWarps][2][kNC][kLanes];   // G of the last two units, per warp
  __shared__ double edge[kWarps][2][H][kNC];       // the H cells left / right of the unit being finished
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t u0 = unit32_begin(w, B), u1 = unit32_begin(w + 1, B);
  if (u0 >= u1) return;
  const int64_t P = B.Ptot;
  const int MT = B.MT, NZ = B.NZ;
  const double* src_r = (s == 1) ? pt.rho : stage_src;
  const double* src_b = (s == 1) ? pt.rhobar : stage_src + 9 * P;
  constexpr int NWS = Sten<ORDER>::NWS;
  const int nsrc = 18, ny = (s == 2 || s == 3) ? 18 : 0, nacc = (s >= 2) ? 18 : 0;
  const int narr = nsrc + ny + nacc + NWS + (s == 4 ? 1 : 0);
  // the unit being finished (previous iteration's)
  int pb = -1, pd = 0, pt_ = 0, pn = 0, pgd = 0;
  int bcur = -1;                    // box of the RK coefficients below (divisions once per box)
  double dtb = 0.0, bdt = 0.0, cdt = 0.0;
  int b = box_of_unit32(B, u0);
  for (int64_t u = u0; u <= u1; ++u) {
    const int slot = (int)((u - u0) & 1);
    int cb = -1, cd = 0, ct = 0, cn = 0, cgd = 0;   // this iteration's unit (none at u == u1)
    if (u < u1) {
      while (u >= B.box[b].uoff32 + (int64_t)B.box[b].ntiles32 * B.box[b].M) ++b;
      const BoxGeo& g = B.box[b];
      const int lu = (int)(u - g.uoff32);
      cb = b;
      cd = lu / g.ntiles32;
      ct = lu - cd * g.ntiles32;
      cn = min(kLanes, g.nz - ct * kLanes);
      cgd = g.doff + cd;
      // prefetch this unit's particle data into L2 (it is finished next iteration)
      const int i0 = ct * kLanes - ldi<COH>(shift + cgd);
      if (i0 >= 0 && i0 + cn <= g.nz) {
        const int64_t base = g.poff + (int64_t)cd * g.nz + i0;
        for (int a = lane; a < narr; a += kLanes) {
          const double* arr;
          if (a < nsrc) arr = (a < 9 ? src_r + (int64_t)a * P : src_b + (int64_t)(a - 9) * P);
          else if (a < nsrc + ny) arr = (a - nsrc < 9 ? pt.rho + (int64_t)(a - nsrc) * P
                                                      : pt.rhobar + (int64_t)(a - nsrc - 9) * P);
          else if (a < nsrc + ny + nacc) arr = pt.acc + (int64_t)(a - nsrc - ny) * P;
          else if (a < nsrc + ny + nacc + NWS) arr = W + (int64_t)(a - nsrc - ny - nacc) * P;
          else arr = pt.z;
          prefetch_l2(arr, base, cn);
        }
      }
      // G of this unit's cells
      if (lane < cn) {
        double G[kNC];
        ring_cell_G<COH>(A, NZ, g.coff, ct * kLanes + lane, __ldg(dirtab + cgd), __ldg(dirtab + MT + cgd),
                         __ldg(dirtab + 2 * MT + cgd), G);
#pragma unroll
        for (int k = 0; k < kNC; ++k) gsm[wib][slot][k][lane] = G[k];
      }
    }
    // does this unit continue the ring of the one being finished?
    const bool next_in_ring = pb >= 0 && cb == pb && cd == pd && ct == pt_ + 1;
    if (pb >= 0) {
      const BoxGeo& g = B.box[pb];
      const double ox = __ldg(dirtab + pgd), oy = __ldg(dirtab + MT + pgd), oz = __ldg(dirtab + 2 * MT + pgd);
      // the H cells right of the finished unit's last cell: from this unit's
      // first cells when it continues the ring and has them, else computed
      // (lane k < 8 forms component k, in ring_cell_G's order)
#pragma unroll
      for (int o = 0; o < H; ++o) {
        if (!(next_in_ring && (H == 1 || o < cn))) {   // (a unit that continues a ring has a first cell)
          const int cell = pt_ * kLanes + pn + o;
          if (lane < kNC)
            edge[wib][1][o][lane] = cell_G_component<COH>(
                A, NZ, g.coff, H == 1 ? (cell >= g.nz ? cell - g.nz : cell) : ring_wrap(cell, g.nz), lane, ox, oy, oz);
        }
      }
      __syncwarp();
      if (next_in_ring && lane == 0) {
#pragma unroll
        for (int o = 0; o < H; ++o)
          if (H == 1 || o < cn) {
#pragma unroll
            for (int k = 0; k < kNC; ++k) edge[wib][1][o][k] = gsm[wib][slot][k][o];
          }
      }
      __syncwarp();
      // finish the previous unit: interpolation (the taps in k_rk_stage's
      // order), commutators, RK update
      const int psl = slot ^ 1;
      if (lane < pn) {
        const int64_t p =
            g.poff + (int64_t)pd * g.nz + wrapc(pt_ * kLanes + lane - ldi<COH>(shift + pgd), g.nz);
        double wt[NW];
        double r[9];
        load_weights<ORDER, COH>(W, P, p, wt);
#pragma unroll
        for (int k = 0; k < 9; ++k) r[k] = ldp<COH>(src_r + k * P + p);
        double Hm[kNC];
#pragma unroll
        for (int k = 0; k < kNC; ++k) {
          if (ORDER == 0) {
            Hm[k] = gsm[wib][psl][k][lane];
          } else if (H == 1) {
            const double gl = lane == 0 ? edge[wib][0][0][k] : gsm[wib][psl][k][lane - 1];
            const double gr = lane == pn - 1 ? edge[wib][1][0][k] : gsm[wib][psl][k][lane + 1];
            Hm[k] = fma(wt[0], gl, fma(wt[1], gsm[wib][psl][k][lane], wt[2] * gr));
          } else {
            // value of G at tap offset o: this unit's cells, or the edges
            auto gv = [&](int o) {
              const int i = lane + o;
              return i < 0 ? edge[wib][0][-i - 1][k] : i >= pn ? edge[wib][1][i - pn][k] : gsm[wib][psl][k][i];
            };
            double h = wt[NW - 1] * gv(H);
#pragma unroll
            for (int t = NW - 2; t >= 0; --t) h = fma(wt[t], gv(t - H), h);
            Hm[k] = h;
          }
        }
        if (pb != bcur) {
          bcur = pb;
          dtb = B.dt[pb];
          bdt = (s == 1 || s == 4) ? dtb / 6.0 : dtb / 3.0;   // weight of K in acc
          cdt = (s == 3) ? dtb : 0.5 * dtb;                   // offset of the next stage
        }
        rk_particle<POT, COH>(g, pt, src_b, P, p, s, dry, bdt, cdt, dtb, dirtab + 3 * MT + pgd, Hm, r);
      }
      __syncwarp();
    }
    // the H cells left of this unit's first cell, for when it is finished:
    // the previous unit's last cells when this one continues its ring (that
    // unit then has all 32 cells), else computed
    if (cb >= 0) {
      if (next_in_ring) {
        if (lane == 0) {
#pragma unroll
          for (int o = 1; o <= H; ++o) {
#pragma unroll
            for (int k = 0; k < kNC; ++k) edge[wib][0][o - 1][k] = gsm[wib][slot ^ 1][k][kLanes - o];
          }
        }
      } else {
        const BoxGeo& g = B.box[cb];
#pragma unroll
        for (int o = 1; o <= H; ++o) {
          const int cell = ct * kLanes - o;
          if (lane < kNC)
            edge[wib][0][o - 1][lane] = cell_G_component<COH>(
                A, NZ, g.coff, H == 1 ? (cell < 0 ? cell + g.nz : cell) : ring_wrap(cell, g.nz), lane,
                __ldg(dirtab + cgd), __ldg(dirtab + MT + cgd), __ldg(dirtab + 2 * MT + cgd));
        }
      }
      __syncwarp();
    }
    pb = cb; pd = cd; pt_ = ct; pn = cn; pgd = cgd;
  }
}

template <bool POT, int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k_rk_stage32(Batch B, Parts pt, const double* __restrict__ W, const double* __restrict__ dirtab,
             const int* __restrict__ shift, const double* __restrict__ A, const double* stage_src, int s, int dry) {
  griddep_wait();
  rk32_phase<POT, ORDER, false>(B, logical_warp(), pt, W, dirtab, shift, A, stage_src, s, dry);
}

// ------------------------------------------- RK stage with the next deposit
//
// Step form 2: every RK stage also deposits (Eq. 5) the state it has just
// computed, at the positions of the next stage (at stage 4: the first stage of
// the next step), so a step is four (combination, RK stage) launch pairs and
// the separate deposit kernel with its re-read of the state is gone.  Units
// are (32-cell tile, direction), TILE-major: a warp walks directions of one
// tile and sums their deposits in shared memory.  Lane l holds the particle on
// cell tile * 32 + l at the stage's positions; every lane owns its particle
// (the G values left of lane 0 and right of the last lane are formed by 16
// lanes, one component each).  Between two stages a ring moves rigidly by
// delta cells, |delta| <= 1 when dt c < 2 dz (the host runs this form only
// then), so the particles of one unit deposit onto cells
// tile * 32 + delta - 1 .. tile * 32 + n + delta: a warp's sums for one tile
// cover the frame of kFrame cells tile * 32 - 2 .. tile * 32 + 33 and go to
// slot (warp + global 32-cell tile) of the partial buffer (unique, as for
// k_deposit).  k_frame_sum adds the slots of each tile in warp order (the
// tile's frame sums), and the next RK stage adds, for each cell, the frame
// entries of the tiles that reach it in a fixed order: bitwise reproducible
// for a fixed grid.  For the shapes of one cell of reach (orders 0-2).
constexpr int kFrame = kLanes + 4;
constexpr int kSlotF = kNT * kFrame;   // doubles in one warp's frame sums for one tile
constexpr int kFrameSmem = (int)sizeof(double) * kWarps * kSlotF;   // dynamic shared memory of k_rk_deposit

__device__ __forceinline__ int64_t warp_of_unit32(int64_t x, const Batch& B) {
  return ((x + 1) * B.nw32 - 1) / B.U32;
}

// Writes a warp's frame sums to its slot and clears them.
__device__ __forceinline__ void flush_frame(double* acc, double* __restrict__ dst, int lane) {
  __syncwarp();
  for (int k = lane; k < kSlotF; k += kLanes) {
    dst[k] = acc[k];
    acc[k] = 0.0;
  }
  __syncwarp();
}

// The frame entries that add up to the potential at cell x of box g: Fr
// offsets of component row 0 in o[0..4] (-1: none).  A tile's frame covers
// cell tile * 32 - 2 + k for k < (its cells) + 4, modulo nz.  When the box has
// at least three tiles and its last tile at least two cells, only the tile of
// x (entry x - tile * 32 + 2) and, for the two cells at either end of a tile,
// the adjacent tile reach x.  Otherwise (rings of few tiles) the tiles of
// cells x - 2 .. x + 2 are taken in that order, once each, with every entry
// of theirs that covers x.
__device__ __forceinline__ bool frame_fast(const BoxGeo& g) {
  return g.ntiles32 >= 3 && g.nz - (g.ntiles32 - 1) * kLanes >= 2;
}
__device__ __forceinline__ void frame_sources(const BoxGeo& g, int x, int (&o)[5]) {
  const int nz = g.nz, nt = g.ntiles32;
#pragma unroll
  for (int q = 0; q < 5; ++q) o[q] = -1;
  if (frame_fast(g)) {
    const int t = x / kLanes, i = x - t * kLanes, n = min(kLanes, nz - t * kLanes);
    o[0] = (g.toff32 + t) * kSlotF + i + 2;
    if (i < 2) {
      const int tl = t == 0 ? nt - 1 : t - 1;
      o[1] = (g.toff32 + tl) * kSlotF + min(kLanes, nz - tl * kLanes) + 2 + i;
    }
    if (i >= n - 2) {
      const int tr = t == nt - 1 ? 0 : t + 1;
      o[2] = (g.toff32 + tr) * kSlotF + i - n + 2;
    }
    return;
  }
  int cnt = 0;
  int prev[4] = {-1, -1, -1, -1};
#pragma unroll
  for (int d = -2; d <= 2; ++d) {
    const int tau = wrapc(x + d, nz) / kLanes;
    bool seen = false;
#pragma unroll
    for (int q = 0; q < d + 2; ++q) seen |= prev[q] == tau;
    if (d < 2) prev[d + 2] = tau;
    if (seen) continue;
    const int ntau = min(kLanes, nz - tau * kLanes);
    const int base = (g.toff32 + tau) * kSlotF;
    for (int k = wrapc(x - tau * kLanes + 2, nz); k < ntau + 4; k += nz) {
#pragma unroll
      for (int q = 0; q < 5; ++q)
        if (q == cnt) o[q] = base + k;
      ++cnt;
    }
  }
}

// Value of component row r of the potential from its frame entries.
__device__ __forceinline__ double frame_value(const double* __restrict__ Fr, const int (&o)[5], int r) {
  double v = __ldg(Fr + o[0] + r * kFrame);
#pragma unroll
  for (int q = 1; q < 5; ++q)
    if (o[q] >= 0) v += __ldg(Fr + o[q] + r * kFrame);
  return v;
}

// Stage s (1..4) of every box: the RK4 update of k_rk_stage32 (same
// arithmetic; the potential of a cell is the sum of the frame entries of
// k_frame_sum that cover it, Fr), then the
// deposit of its result at the next stage's positions: the shape weights
// (kept in W for the next stage), B = N rho - Nbar rhobar^* in the traceless
// components (Eq. 5, Eq. 2) and w (1, Omega) B summed per frame cell.
// STAGE 0: no RK update; the deposit of the state in rho, rhobar at the first
// stage's positions (the first launch of a run of steps).  Shift rows: this
// stage's s - 1, the deposit's s (row 4: the next step's first stage).  The
// stage is a template parameter: each instance keeps only its own stage's
// loads live (fewer registers than one kernel for all four).
template <bool POT, int ORDER, int STAGE>
__global__ void __launch_bounds__(kThreads, 2)
k_rk_deposit(Batch B, Parts pt, double* __restrict__ W, const double* __restrict__ dirtab,
             const int* __restrict__ shift, const double* __restrict__ Fr, int dry,
             double* __restrict__ partial, int* __restrict__ err) {
  static_assert(Sten<ORDER>::H == 1, "the frame covers the shapes of one cell of reach");
  static_assert(STAGE >= 0 && STAGE <= 4, "stages 1-4, or 0 for the first deposit");
  constexpr bool DEP_ONLY = STAGE == 0;
  constexpr int s = STAGE;
  constexpr int NW = Sten<ORDER>::NW, NWS = Sten<ORDER>::NWS;
  extern __shared__ double frame_sm[];
  __shared__ double gsm[kWarps][kNC][kLanes];   // G of the unit's cells
  __shared__ double gedge[kWarps][2 * kNC];      // G left of lane 0, right of lane n - 1
  griddep_wait();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* acc = frame_sm + wib * kSlotF;
  const int64_t w = logical_warp();
  const int64_t u0 = unit32_begin(w, B), u1 = unit32_begin(w + 1, B);
  if (u0 >= u1) return;
  for (int k = lane; k < kSlotF; k += kLanes) acc[k] = 0.0;
  __syncwarp();
  const int64_t P = B.Ptot;
  const int MT = B.MT;
  const bool first = DEP_ONLY || s == 1;
  const double* src_r = first ? pt.rho : pt.stage;
  const double* src_b = first ? pt.rhobar : pt.stage + 9 * P;
  const int* sh_cur = shift + (DEP_ONLY ? 0 : s - 1) * MT;
  const int* sh_next = shift + (DEP_ONLY ? 0 : s) * MT;
  // arrays read per particle, for the L2 prefetch of the next unit: the state
  // (18), y (18, s = 2, 3), acc (18, s >= 2), W (NWS), z, N, Nbar
  const int ny = (!DEP_ONLY && (s == 2 || s == 3)) ? 18 : 0, nacc = (!DEP_ONLY && s >= 2) ? 18 : 0;
  const int nw_ = DEP_ONLY ? 0 : NWS;
  const int narr = 18 + ny + nacc + nw_ + 3;
  int lat = 0, far = 0;
  int b = box_of_unit32(B, u0);
  int bcur = -1;
  double dtb = 0.0, bdt = 0.0, cdt = 0.0;
  int64_t stile = -1;   // global tile whose sums acc holds
  for (int64_t u = u0; u < u1; ++u) {
    while (u >= B.box[b].uoff32 + (int64_t)B.box[b].ntiles32 * B.box[b].M) ++b;
    const BoxGeo& g = B.box[b];
    const int nz = g.nz, M = g.M;
    const int lu = (int)(u - g.uoff32);
    const int tile = lu / M, d = lu - tile * M;
    const int64_t gtile = g.toff32 + tile;
    if (gtile != stile) {
      if (stile >= 0) flush_frame(acc, partial + (w + stile) * kSlotF, lane);
      stile = gtile;
    }
    if (b != bcur) {
      bcur = b;
      dtb = B.dt[b];
      bdt = (s == 1 || s == 4) ? dtb / 6.0 : dtb / 3.0;   // weight of K in acc
      cdt = (s == 3) ? dtb : 0.5 * dtb;                   // offset of the next stage
    }
    if (u + 1 < u1 && lu + 1 < g.ntiles32 * M) {   // prefetch the next unit of the same box
      const int tn = (lu + 1) / M, dn = lu + 1 - tn * M;
      const int i0 = tn * kLanes - __ldg(sh_cur + g.doff + dn);
      const int cnt = min(kLanes, nz - tn * kLanes);
      if (i0 >= 0 && i0 + cnt <= nz) {
        const int64_t base = g.poff + (int64_t)dn * nz + i0;
        for (int a = lane; a < narr; a += kLanes) {
          const double* arr;
          if (a < 18) arr = a < 9 ? src_r + (int64_t)a * P : src_b + (int64_t)(a - 9) * P;
          else if (a < 18 + ny) arr = a - 18 < 9 ? pt.rho + (int64_t)(a - 18) * P : pt.rhobar + (int64_t)(a - 27) * P;
          else if (a < 18 + ny + nacc) arr = pt.acc + (int64_t)(a - 18 - ny) * P;
          else if (a < 18 + ny + nacc + nw_) arr = W + (int64_t)(a - 18 - ny - nacc) * P;
          else {
            const int k = a - 18 - ny - nacc - nw_;
            arr = k == 0 ? pt.z : k == 1 ? pt.N : pt.Nbar;
          }
          prefetch_l2(arr, base, cnt);
        }
      }
    }
    const int n = min(kLanes, nz - tile * kLanes);
    const bool active = lane < n;
    const int j = tile * kLanes + lane;   // this lane's cell at the stage's positions
    const int gd = g.doff + d;
    const double ox = __ldg(dirtab + gd), oy = __ldg(dirtab + MT + gd), oz = __ldg(dirtab + 2 * MT + gd);
    const double vz = __ldg(dirtab + 3 * MT + gd);
    const int sc = __ldg(sh_cur + gd);
    const int64_t p = g.poff + (int64_t)d * nz + wrapc(j - sc, nz);
    double bm[9];       // B = N rho - Nbar rhobar^* of the state deposited (Eq. 5)
    double zs = 0.0;    // and its position
    double n1 = 0.0, n2 = 0.0;
    if (active) {
      n1 = __ldg(pt.N + p);
      n2 = __ldg(pt.Nbar + p);
    }
    if constexpr (DEP_ONLY) {
      if (active) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const double x = __ldg(src_r + k * P + p), y = __ldg(src_b + k * P + p);
          bm[k] = (k == 4 || k == 6 || k == 8) ? fma(n2, y, n1 * x) : fma(-n2, y, n1 * x);
        }
        zs = __ldg(pt.z + p);
      }
    } else {
      // G = A0 - Omega . A of this lane's cell into shared memory
      if (frame_fast(g)) {
        // its tile's frame entry lane + 2, then (one value per lane) the
        // adjacent tiles' entries for the two cells at each end of the tile:
        // lanes 0-15 cells 0, 1 from the tile before, lanes 16-31 cells
        // n - 2, n - 1 from the tile after, added in that order
        const double* f0 = Fr + (int64_t)(g.toff32 + tile) * kSlotF + lane + 2;
#pragma unroll
        for (int c = 0; c < kNC; ++c)
          gsm[wib][c][lane] = fma(-oz, __ldg(f0 + (3 * kNC + c) * kFrame),
                                  fma(-oy, __ldg(f0 + (2 * kNC + c) * kFrame),
                                      fma(-ox, __ldg(f0 + (kNC + c) * kFrame), __ldg(f0 + c * kFrame))));
        const int nt = g.ntiles32, c = lane & (kNC - 1), right = lane >> 4;
        const int ce = right ? n - 2 + ((lane >> 3) & 1) : (lane >> 3) & 1;
        const int tn = right ? (tile == nt - 1 ? 0 : tile + 1) : (tile == 0 ? nt - 1 : tile - 1);
        const int k = right ? ce - n + 2 : min(kLanes, nz - tn * kLanes) + 2 + ce;
        const double* f1 = Fr + (int64_t)(g.toff32 + tn) * kSlotF + k;
        const double gc = fma(-oz, __ldg(f1 + (3 * kNC + c) * kFrame),
                              fma(-oy, __ldg(f1 + (2 * kNC + c) * kFrame),
                                  fma(-ox, __ldg(f1 + (kNC + c) * kFrame), __ldg(f1 + c * kFrame))));
        __syncwarp();
        if (!right) gsm[wib][c][ce] += gc;
        __syncwarp();
        if (right) gsm[wib][c][ce] += gc;
      } else {
        int off[5];
        frame_sources(g, active ? j : wrapc(j, nz), off);
#pragma unroll
        for (int c = 0; c < kNC; ++c)
          gsm[wib][c][lane] = fma(-oz, frame_value(Fr, off, 3 * kNC + c),
                                  fma(-oy, frame_value(Fr, off, 2 * kNC + c),
                                      fma(-ox, frame_value(Fr, off, kNC + c), frame_value(Fr, off, c))));
      }
      // lanes 0-15 (component lane mod 8): G of the cell left of lane 0
      // (lanes 0-7) and right of lane n - 1 (lanes 8-15)
      if (ORDER > 0 && lane < 2 * kNC) {
        const int c = lane & (kNC - 1);
        const int right = tile * kLanes + n;
        const int cell = lane < kNC ? (tile == 0 ? nz - 1 : tile * kLanes - 1) : (right == nz ? 0 : right);
        int off[5];
        frame_sources(g, cell, off);
        gedge[wib][lane] = fma(-oz, frame_value(Fr, off, 3 * kNC + c),
                               fma(-oy, frame_value(Fr, off, 2 * kNC + c),
                                   fma(-ox, frame_value(Fr, off, kNC + c), frame_value(Fr, off, c))));
      }
      __syncwarp();
      if (active) {
        double wt[NW];
        double r[9];
        load_weights<ORDER>(W, P, p, wt);
#pragma unroll
        for (int k = 0; k < 9; ++k) r[k] = src_r[k * P + p];
        double Hm[kNC];
#pragma unroll
        for (int c = 0; c < kNC; ++c) {
          if constexpr (ORDER == 0) {
            Hm[c] = gsm[wib][c][lane];
          } else {
            const double gl = lane == 0 ? gedge[wib][c] : gsm[wib][c][lane - 1];
            const double gr = lane == n - 1 ? gedge[wib][kNC + c] : gsm[wib][c][lane + 1];
            Hm[c] = fma(wt[0], gl, fma(wt[1], gsm[wib][c][lane], wt[2] * gr));
          }
        }
        double zn = 0.0;
        rk_particle<POT, false, true>(g, pt, src_b, P, p, s, dry, bdt, cdt, dtb, dirtab + 3 * MT + gd, Hm, r,
                                      bm, &zn, n1, n2);
        zs = s < 4 ? fma(stage_frac(s) * dtb, vz, pt.z[p]) : zn;
      }
      __syncwarp();   // (gsm is rewritten by the next unit)
    }
    // the ring's move to the next stage's positions
    int delta = 0;
    if constexpr (!DEP_ONLY) {
      delta = wrapc(__ldg(sh_next + gd) - sc, nz);
      if (2 * delta > nz) delta -= nz;
      if (delta < -1 || delta > 1) {   // (excluded by the host; the unit's deposit is skipped)
        far = 1;
        continue;
      }
    }
    double wn[NW];
    zero_weights<ORDER>(wn);
    double bv[kNC];
#pragma unroll
    for (int c = 0; c < kNC; ++c) bv[c] = 0.0;
    if (active) {
      lat |= shape_weights<ORDER>(zs, (double)wrapc(j + delta, nz) + 0.5, g.inv_dz, g.nz_d, wn);
#pragma unroll
      for (int q = 0; q < NWS; ++q) W[q * P + p] = wn[q];
      bv[0] = bm[0] - bm[1];   // the traceless components
      bv[1] = bm[1] - bm[2];
#pragma unroll
      for (int k = 3; k < 9; ++k) bv[k - 1] = bm[k];
    }
    // this lane's cell tile * 32 + lane + delta receives from the particles on
    // lanes lane - 1, lane, lane + 1 of this unit
    const double wup = __shfl_up_sync(kFull, wn[2], 1), wdn = __shfl_down_sync(kFull, wn[0], 1);
    const double fl = lane == 0 ? 0.0 : wup;
    const double fr = lane == kLanes - 1 ? 0.0 : wdn;
    double* a = acc + lane + delta + 2;
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const double v = bv[c];
      double cc;
      if constexpr (ORDER == 0) {
        cc = wn[1] * v;
      } else {
        const double vl = __shfl_up_sync(kFull, v, 1), vr = __shfl_down_sync(kFull, v, 1);
        cc = fma(fr, vr, fma(wn[1], v, fl * vl));
      }
      if (active) {
        a[c * kFrame] += cc;
        a[(kNC + c) * kFrame] = fma(ox, cc, a[(kNC + c) * kFrame]);
        a[(2 * kNC + c) * kFrame] = fma(oy, cc, a[(2 * kNC + c) * kFrame]);
        a[(3 * kNC + c) * kFrame] = fma(oz, cc, a[(3 * kNC + c) * kFrame]);
      }
    }
    if constexpr (ORDER > 0) {
      // the cells left of lane 0's and right of lane n - 1's: only those two
      // particles' outer weights; lane f * 8 + c adds component c of moment f
      // (1, Omega_x, Omega_y, Omega_z) of both
      __syncwarp();
      const int c = lane & (kNC - 1), f = lane >> 3;
      double bl = 0.0, br = 0.0;
#pragma unroll
      for (int k = 0; k < kNC; ++k) {
        const double x0 = __shfl_sync(kFull, bv[k], 0), x1 = __shfl_sync(kFull, bv[k], n - 1);
        if (k == c) {
          bl = x0;
          br = x1;
        }
      }
      const double wl = __shfl_sync(kFull, wn[0], 0), wr = __shfl_sync(kFull, wn[2], n - 1);
      const double of = f == 0 ? 1.0 : f == 1 ? ox : f == 2 ? oy : oz;
      double* row = acc + lane * kFrame;
      row[delta + 1] = fma(of, wl * bl, row[delta + 1]);
      row[n + delta + 2] = fma(of, wr * br, row[n + delta + 2]);
    }
    __syncwarp();
  }
  flush_frame(acc, partial + (w + stile) * kSlotF, lane);
  if (lat) atomicOr(err, ERR_LATTICE);
  if (far) atomicOr(err, ERR_STEP);
}

__device__ __forceinline__ int box_of_tile32(const Batch& B, int64_t t) {
  int lo = 0, hi = B.nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.box[mid].toff32 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Deposit combination of step form 2: the frame sums of every 32-cell tile,
// Fr[gtile * kSlotF + e] = kappa_b / dV_b x (sum over the warps that own
// units of the tile of their slot's entry e), in warp order.  A group of 32
// lanes takes 32 consecutive entries of one tile (kSlotF = 36 x 32), so every
// lane of a warp walks the same warps.  Split over warps and running sums as
// in combine_phase.  The potential at a cell is the sum of the frame entries
// that cover it (frame_sources).
__global__ void k_frame_sum(Batch B, const double* __restrict__ partial, double* __restrict__ Fr, int64_t NT32,
                            int split, int* __restrict__ err) {
  __shared__ double sums[kWarps][kLanes];
  griddep_wait();
  const int64_t n = NT32 * kSlotF;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int grp = wib / split, wi = wib - grp * split;
  const int groups = kWarps / split;
  int bad = 0;
  for (int64_t base = (int64_t)blockIdx.x * groups * kLanes; base < n; base += (int64_t)gridDim.x * groups * kLanes) {
    const int64_t e0 = base + (int64_t)grp * kLanes;   // first entry of this group (one tile)
    double v = 0.0;
    const BoxGeo* g = nullptr;
    if (e0 < n) {
      const int64_t gtile = e0 / kSlotF;
      g = &B.box[box_of_tile32(B, gtile)];
      const int64_t tau = gtile - g->toff32;
      const int64_t wf = warp_of_unit32(g->uoff32 + tau * g->M, B);
      const int64_t wl = warp_of_unit32(g->uoff32 + (tau + 1) * g->M - 1, B);
      const double* src = partial + (e0 - gtile * kSlotF) + lane;
      double a[kCombineILP] = {};
      int64_t q = wf + wi;
      for (; q + (kCombineILP - 1) * split <= wl; q += kCombineILP * split) {
#pragma unroll
        for (int i = 0; i < kCombineILP; ++i) a[i] += __ldcg(src + (q + i * split + gtile) * kSlotF);
      }
      for (; q <= wl; q += split) a[0] += __ldcg(src + (q + gtile) * kSlotF);
#pragma unroll
      for (int h = kCombineILP / 2; h >= 1; h /= 2) {
#pragma unroll
        for (int i = 0; i < h; ++i) a[i] += a[i + h];
      }
      v = a[0];
    }
    if (split > 1) {
      sums[wib][lane] = v;
      __syncthreads();
      if (wi == 0)
        for (int i = 1; i < split; ++i) v += sums[wib + i][lane];
      __syncthreads();
    }
    if (e0 < n && wi == 0) {
      v *= g->kappa_dV;
      bad |= !isfinite(v);
      Fr[e0 + lane] = v;
    }
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

// ------------------------------------------------------- fused step kernel
//
// All phases of nsteps RK4 steps in one cooperative launch (every block
// resident): per step the lattice shifts and ring weights, then per stage the
// deposit, its combination and the RK stage, separated by grid barriers.  The
// arithmetic and the order of every sum are those of the separate kernels with
// the same grid: results are bitwise the same.
//
// Grid barrier: each block's thread 0 adds to an arrival word (block 0 adds
// 2^31 - (blocks - 1), the others 1, so the top bit flips when the last block
// arrives and the word is ready for the next barrier) and waits for the flip.
// The wait is bounded: after limit_ns nanoseconds (device global timer), or as
// soon as another block has given up, the block sets the abort word and
// ERR_TIMEOUT and the kernel returns.  A launch that finds the abort word set
// returns at once; the host clears it (and the arrival word) when it reports
// the error.
enum : int { ERR_TIMEOUT = 16 };

struct StepArgs {
  const double* dirtab;
  int* shift;          // [4][MT] shift rows of the step
  double* wtab;        // [4 x kWSlots][MT] the rings' weights at those rows (nullptr: each particle's own)
  double* W;           // kept shape weights
  double* At;          // traceless grid potential
  double* partial;     // per-warp deposit partials
  int* err;
  unsigned* bar;       // [0] arrival word, [1] abort word
  unsigned long long limit_ns;
  int64_t nsteps;
  int split;           // combine split (as the separate deposit uses)
  int dry;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns true if the launch must stop (a wait gave up here or elsewhere).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned long long limit_ns, int* err) {
  __shared__ int stop;
  __syncthreads();
  if (threadIdx.x == 0) {
    int give_up = 0;
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();                         // this block's writes before its arrival
    const unsigned old = atomicAdd(bar, inc);
    const unsigned long long t0 = global_ns();
    while (((old ^ ld_acquire_u32(bar)) & 0x80000000u) == 0) {
      if (ld_acquire_u32(bar + 1) != 0u || global_ns() - t0 > limit_ns) {
        atomicExch(bar + 1, 1u);
        atomicOr(err, ERR_TIMEOUT);
        give_up = 1;
        break;
      }
    }
    __threadfence();                         // the other blocks' writes after the barrier
    stop = give_up;
  }
  __syncthreads();
  return stop != 0;
}

// The phases of the fused kernel, inlined (measured on GB300: calling them as
// separate functions, which keeps each phase's register allocation but saves
// and restores registers around every call, was 4-5% slower per step).
template <int ORDER>
__device__ __forceinline__ void fused_deposit(const Batch& B, int64_t w, int lane, const Parts& pt, const double* rnu,
                                           const double* rnb, const StepArgs& a, const int* srow,
                                           const double* wrow, double frac) {
  deposit_phase<5, ORDER, true>(B, w, lane, pt.z, pt.N, pt.Nbar, rnu, rnb, a.dirtab, srow, wrow, frac, a.partial,
                                a.W, a.err);
}

__device__ __forceinline__ void fused_combine(const Batch& B, const StepArgs& a) {
  combine_phase(B, a.partial, a.At, kNT, 1, a.split, a.err);
}

template <bool POT, int ORDER, bool RK32>
__device__ __forceinline__ void fused_rk(const Batch& B, int64_t w, int lane, const Parts& pt, const StepArgs& a,
                                     const int* srow, int s) {
  if constexpr (RK32) rk32_phase<POT, ORDER, true>(B, w, pt, a.W, a.dirtab, srow, a.At, pt.stage, s, a.dry);
  else rk_phase<POT, ORDER, true>(B, w, lane, pt, a.W, a.dirtab, srow, a.At, pt.stage, s, a.dry);
}

template <bool POT, int ORDER, bool RK32>
__global__ void __launch_bounds__(kThreads, 2) k_step(Batch B, Parts pt, StepArgs a) {
  __shared__ int aborted;
  if (threadIdx.x == 0) aborted = ld_acquire_u32(a.bar + 1) != 0u;
  __syncthreads();
  if (aborted) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int MT = B.MT;
  Fracs fr;
#pragma unroll
  for (int q = 0; q < 4; ++q) fr.v[q] = stage_frac(q);
  const int64_t P = B.Ptot;
  for (int64_t n = 0; n < a.nsteps; ++n) {
    for (int gd = blockIdx.x * blockDim.x + threadIdx.x; gd < MT; gd += gridDim.x * blockDim.x)
      shifts_phase<true, ORDER>(B, gd, pt.z, a.dirtab, fr, 4, a.shift, a.wtab);
    if (grid_barrier(a.bar, a.limit_ns, a.err)) return;
    for (int s = 1; s <= 4; ++s) {
      const int* srow = a.shift + (s - 1) * MT;
      const double* wrow = a.wtab != nullptr ? a.wtab + (s - 1) * kWSlots * MT : nullptr;
      const double* rnu = s == 1 ? pt.rho : pt.stage;
      const double* rnb = s == 1 ? pt.rhobar : pt.stage + 9 * P;
      fused_deposit<ORDER>(B, w, lane, pt, rnu, rnb, a, srow, wrow, stage_frac(s - 1));
      if (grid_barrier(a.bar, a.limit_ns, a.err)) return;
      fused_combine(B, a);
      if (grid_barrier(a.bar, a.limit_ns, a.err)) return;
      fused_rk<POT, ORDER, RK32>(B, w, lane, pt, a, srow, s);
      if (grid_barrier(a.bar, a.limit_ns, a.err)) return;
    }
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
// Box-local particle numbers key the random draws.  species: per box, at
// 8 * coff_b: n_nu[nz], n_nubar[nz], f_nu[3 nz], f_nubar[3 nz]; dirs[3 * MT].
__global__ void k_init(Batch B, Parts pt, const double* __restrict__ species, const double* __restrict__ dirs,
                       int* __restrict__ err) {
  const int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= B.Ptot) return;
  const BoxGeo& g = B.box[box_of_particle(B, gp)];
  const int64_t p = gp - g.poff;
  const int d = (int)(p / g.nz), j0 = (int)(p % g.nz);
  double o[3];
  if (g.use_dirs) {
    const int gd = g.doff + d;
    o[0] = dirs[3 * gd]; o[1] = dirs[3 * gd + 1]; o[2] = dirs[3 * gd + 2];
  } else {
    const double mu = __dsub_rn(1.0, __ddiv_rn(__dadd_rn(__dmul_rn(2.0, (double)d), 1.0), (double)g.M));
    const double phi = __dmul_rn(__dmul_rn((double)d, 3.14159265358979323846), __dsub_rn(3.0, sqrt(5.0)));
    const double sn = sqrt(__dsub_rn(1.0, __dmul_rn(mu, mu)));
    o[0] = __dmul_rn(sn, cos(phi));
    o[1] = __dmul_rn(sn, sin(phi));
    o[2] = mu;
  }
  pt.z[gp] = __dmul_rn(__dadd_rn((double)j0, 0.5), g.dz);
  pt.ox[gp] = o[0]; pt.oy[gp] = o[1]; pt.oz[gp] = o[2];
  const int nz = g.nz;
  const double* sp_base = species + 8 * (int64_t)g.coff;
  double wgt[2];
  for (int sp = 0; sp < 2; ++sp) {
    const double n = sp_base[sp * nz + j0];
    const double* f = sp_base + 2 * nz + sp * 3 * nz + 3 * j0;
    const double fdo = __dadd_rn(__dadd_rn(__dmul_rn(f[0], o[0]), __dmul_rn(f[1], o[1])), __dmul_rn(f[2], o[2]));
    double wt = __ddiv_rn(__dmul_rn(__dadd_rn(n, __dmul_rn(3.0, fdo)), g.dV), (double)g.M);
    const double tol = 1e-12 * (fabs(n) + 3.0 * fabs(fdo)) * g.dV / g.M;
    if (wt < 0.0 && wt >= -tol) wt = 0.0;
    if (wt < 0.0) atomicOr(err, ERR_WEIGHT);
    wgt[sp] = wt;
  }
  pt.N[gp] = wgt[0];
  pt.Nbar[gp] = wgt[1];
  const int64_t P = B.Ptot;
  for (int sp = 0; sp < 2; ++sp) {
    double* r = sp ? pt.rhobar : pt.rho;
    const double emr = __dmul_rn(g.alpha, uniform_pm1(g.seed, p, 4 * sp + 0));
    const double emi = __dmul_rn(g.alpha, uniform_pm1(g.seed, p, 4 * sp + 1));
    const double etr = __dmul_rn(g.alpha, uniform_pm1(g.seed, p, 4 * sp + 2));
    const double eti = __dmul_rn(g.alpha, uniform_pm1(g.seed, p, 4 * sp + 3));
    const double eps_mu = __dadd_rn(__dmul_rn(emr, emr), __dmul_rn(emi, emi));
    const double eps_tau = __dadd_rn(__dmul_rn(etr, etr), __dmul_rn(eti, eti));
    r[0 * P + gp] = __dsub_rn(__dsub_rn(1.0, eps_mu), eps_tau);
    r[1 * P + gp] = eps_mu;
    r[2 * P + gp] = eps_tau;
    r[3 * P + gp] = emr;
    r[4 * P + gp] = emi;
    r[5 * P + gp] = etr;
    r[6 * P + gp] = eti;
    r[7 * P + gp] = 0.0;
    r[8 * P + gp] = 0.0;
  }
}

// Per box: maximum over cells of the diagonal components of n and nbar (Eq. 7).
// One block per box.
__global__ void k_max_diag(Batch B, const double* __restrict__ mom, double* __restrict__ out) {
  __shared__ double sm[kThreads];
  const BoxGeo& g = B.box[blockIdx.x];
  double m = 0.0;
  for (int j = threadIdx.x; j < g.nz; j += kThreads)
    for (int a = 0; a < 3; ++a) {
      m = fmax(m, mom[(int64_t)a * B.NZ + g.coff + j]);
      m = fmax(m, mom[(int64_t)(36 + a) * B.NZ + g.coff + j]);
    }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

// Eq. 7 per box from the maxima: dt_b = min(C dz / c, C_F / (kappa n_max)).
__global__ void k_dt_from_max(Batch B, const double* __restrict__ nmax, double* __restrict__ dt_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B.nbox) return;
  const BoxGeo& g = B.box[b];
  const double dt_adv = g.cfl_adv * g.dz / g.c_light;
  const double nm = nmax[b] > g.n_e ? nmax[b] : g.n_e;
  const double dt_flav = nm > 0.0 ? g.cfl_flavor / (g.kappa * nm) : dt_adv;
  dt_out[b] = dt_adv < dt_flav ? dt_adv : dt_flav;
}

// Writes one box descriptor and step size from kernel parameters (used where
// no host-to-device copy may be issued).
__global__ void k_write_geo(BoxGeo g, double dt, BoxGeo* __restrict__ dst, double* __restrict__ dt_dst) {
  *dst = g;
  *dt_dst = dt;
}

// Domain diagnostics per box (Eq. 10, one snapshot of Eq. B1, Eq. 18), fixed-
// order block reduction over the box's cells.  One block per (box, quantity):
// blockIdx.x = box, blockIdx.y = q; out[63 * b + q].  mom: the [36][NZ] moments
// of the diagnostic deposit (rows 0-8 n, 9-17 f_x, 18-26 nbar, 27-35 fbar_x).
__device__ __forceinline__ double abs_entry(const double* __restrict__ m, int64_t NZ, int64_t j, int a, int b) {
  if (a == b) return fabs(m[(int64_t)a * NZ + j]);
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const int k = (lo == 0 && hi == 1) ? 3 : (lo == 0 ? 5 : 7);
  const double re = m[(int64_t)k * NZ + j], im = m[(int64_t)(k + 1) * NZ + j];
  return sqrt(re * re + im * im);
}

__global__ void k_diagnostics(Batch B, const double* __restrict__ mom, double* __restrict__ out) {
  __shared__ double sm[kThreads];
  const BoxGeo& g = B.box[blockIdx.x];
  const int64_t NZ = B.NZ;
  const int q = blockIdx.y;
  double s = 0.0;
  for (int jj = threadIdx.x; jj < g.nz; jj += kThreads) {
    const int64_t j = g.coff + jj;
    double v;
    if (q < 36) {
      const int blk = q / 9, e = q % 9, a = e / 3, bb = e % 3;
      const int off = blk == 0 ? 0 : blk == 1 ? 18 : blk == 2 ? 9 : 27;
      v = abs_entry(mom + (int64_t)off * NZ, NZ, j, a, bb);
    } else if (q < 45) {
      v = mom[(int64_t)(q - 36) * NZ + j];
    } else if (q < 54) {
      v = mom[(int64_t)(18 + q - 45) * NZ + j];
    } else {
      const int k = q - 54;
      const double nbar = mom[(int64_t)(18 + k) * NZ + j];
      v = mom[(int64_t)k * NZ + j] + ((k == 4 || k == 6 || k == 8) ? nbar : -nbar);
    }
    s += v;
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[63 * blockIdx.x + q] = sm[0] / g.nz;
}

// ------------------------------------------------------------------ adjoint
//
// Discrete adjoint of the RK4 step in the packed 9-real representation.  With
// the packing metric D = diag(1, 1, 1, 2, ..., 2) (<X, Y>_Frobenius = x^T D y),
// K(H, r) = -i[H, r] and the sign pattern S of Hbar = -H^* (packed: S H):
//   transpose of r -> K(H, r):  m -> -D K(H, D^-1 m)   (the generator is anti-self-adjoint)
//   transpose of H -> K(H, r):  m -> D K(r, D^-1 m)
//   transpose of H -> K(S H + V, rbar):  m -> S D K(rbar, D^-1 m)
// The self-interaction operator B -> H (deposit, Eq. 5, then interpolation,
// Eq. 6, with the shared weights) is symmetric, so its transpose is the same
// deposit-and-interpolate applied to the adjoint Gamma = dL/dH.

// First adjoint launch of stage s.  m = a lam + c lamn, the adjoint of this
// stage's derivative k_s, with the box's step dt: a = dt/6 (s = 1, 4) or dt/3,
// c = dt/2 (s = 1, 2) or dt (s = 3), lamn the adjoint of stage s + 1 (NULL
// for s = 4); writes lam_out = J_rho^T m (direct terms) and Gam = dL/dH_self.
// pt.rho / pt.rhobar point at the stage state.  The metric D folds into the
// commutator: D K(X, D^-1 m) is the commutator's raw output (halved diagonal,
// off-diagonals) for X and m2 = m with its diagonal doubled, so
//   lam_out = -D K(H, D^-1 m) = raw(-H, m2),   Gamma += S D K(r, D^-1 m) = S raw(r, m2).
template <bool POT, int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k_adj_a(Batch B, Parts pt, const double* __restrict__ W, const double* __restrict__ dirtab,
        const int* __restrict__ shift, const double* __restrict__ A, const double* __restrict__ lam,
        const double* __restrict__ lamn, int s, double* __restrict__ lam_out, double* __restrict__ Gam) {
  griddep_wait();
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int64_t u0 = unit_begin(w, B), u1 = unit_begin(w + 1, B);
  if (u0 >= u1) return;
  const int64_t P = B.Ptot;
  const int MT = B.MT, NZ = B.NZ;
  int b = box_of_unit(B, u0);
  for (int64_t u = u0; u < u1; ++u) {
    while (u >= B.box[b].uoff + (int64_t)B.box[b].ntiles * B.box[b].M) ++b;
    const BoxGeo& g = B.box[b];
    const double dtb = B.dt[b];
    const double a = (s == 1 || s == 4) ? dtb / 6.0 : dtb / 3.0;
    const double bc = (s == 3) ? dtb : 0.5 * dtb;
    const int nz = g.nz, nt = g.ntiles;
    const int lu = (int)(u - g.uoff);
    const int d = lu / nt, tile = lu - d * nt;
    constexpr int Hh = Sten<ORDER>::H, T = Sten<ORDER>::T;
    const int craw = tile * T - Hh + lane, j = wrapc(craw, nz);
    const bool active = lane >= Hh && lane < Hh + T && craw < nz;
    const int gd = g.doff + d;
    const double ox = __ldg(dirtab + gd), oy = __ldg(dirtab + MT + gd), oz = __ldg(dirtab + 2 * MT + gd);
    const int64_t p = g.poff + (int64_t)d * nz + wrapc(j - __ldg(shift + gd), nz);
    double wt[Sten<ORDER>::NW];
    zero_weights<ORDER>(wt);
    if (active) load_weights<ORDER>(W, P, p, wt);
    double H[kNC];   // traceless components of the stage's H
    const double* Aj = A + g.coff + j;
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const double G = fma(-oz, __ldg(Aj + (int64_t)(3 * kNC + c) * NZ),
                           fma(-oy, __ldg(Aj + (int64_t)(2 * kNC + c) * NZ),
                               fma(-ox, __ldg(Aj + (int64_t)(kNC + c) * NZ), __ldg(Aj + (int64_t)c * NZ))));
      H[c] = gather<ORDER>(wt, G);
    }
    if (!active) continue;
    const double a2 = 2.0 * a, bc2 = 2.0 * bc;
    double Gm[9];
#pragma unroll
    for (int which = 0; which < 2; ++which) {
      double nH[kNC], r[9], m2[9], kd[3], ko[6];
#pragma unroll
      for (int c = 0; c < kNC; ++c) {                                       // -(S H + V), S for antineutrinos
        const bool im = (c == 3 || c == 5 || c == 7);
        const double nsgn = which ? (im ? -1.0 : 1.0) : -1.0;
        nH[c] = nsgn * H[c] - (POT ? __ldg((which ? g.vnubar : g.vnu) + c) : 0.0);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const double l = lam[(which * 9 + k) * P + p];
        const double ln = lamn ? lamn[(which * 9 + k) * P + p] : 0.0;
        m2[k] = k < 3 ? fma(a2, l, bc2 * ln) : fma(a, l, bc * ln);
        r[k] = (which ? pt.rhobar : pt.rho)[k * P + p];
      }
      commutator(nH[0], nH[0] + nH[1], nH[1], nH[2], nH[3], nH[4], nH[5], nH[6], nH[7], m2, kd, ko);
#pragma unroll
      for (int k = 0; k < 3; ++k) lam_out[(which * 9 + k) * P + p] = kd[k];
#pragma unroll
      for (int k = 0; k < 6; ++k) lam_out[(which * 9 + 3 + k) * P + p] = ko[k];
      commutator(r[0] - r[1], r[0] - r[2], r[1] - r[2], r[3], r[4], r[5], r[6], r[7], r[8], m2, kd, ko);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const bool im = (k == 4 || k == 6 || k == 8);
        const double v = k < 3 ? kd[k] : ko[k - 3];
        if (which == 0) Gm[k] = v;
        else Gm[k] += (im ? v : -v);
      }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) Gam[k * P + p] = Gm[k];
  }
}

// Second adjoint launch of one stage: GB = interpolation of the deposited
// Gamma grid E (= dL/dB), then lam_out += N GB (rho) and -Nbar conj(GB)
// (rhobar), gN += <GB, rho>, gNbar -= <conj(GB), rhobar>; finally
// lam_tot += lam_out.
template <int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k_adj_b(Batch B, Parts pt, const double* __restrict__ W, const double* __restrict__ dirtab,
        const int* __restrict__ shift, const double* __restrict__ E, double* __restrict__ lam_out,
        double* __restrict__ lam_tot, double* __restrict__ gN, double* __restrict__ gNbar) {
  griddep_wait();
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int64_t u0 = unit_begin(w, B), u1 = unit_begin(w + 1, B);
  if (u0 >= u1) return;
  const int64_t P = B.Ptot;
  const int MT = B.MT, NZ = B.NZ;
  constexpr int Hh = Sten<ORDER>::H, T = Sten<ORDER>::T, NWS = Sten<ORDER>::NWS;
  const double* __restrict__ rho = pt.rho;
  const double* __restrict__ rhobar = pt.rhobar;
  const double* __restrict__ Nw = pt.N;
  const double* __restrict__ Nbw = pt.Nbar;
  // arrays read per particle, for the L2 prefetch of the next unit: rho, rhobar (18),
  // lam_out, lam_tot (36), N, Nbar, gN, gNbar (4), weights (NWS)
  constexpr int narr = 18 + 36 + 4 + NWS;
  int b = box_of_unit(B, u0);
  for (int64_t u = u0; u < u1; ++u) {
    while (u >= B.box[b].uoff + (int64_t)B.box[b].ntiles * B.box[b].M) ++b;
    const BoxGeo& g = B.box[b];
    const int nz = g.nz, nt = g.ntiles;
    const int lu = (int)(u - g.uoff);
    const int d = lu / nt, tile = lu - d * nt;
    if (u + 1 < u1 && lu + 1 < nt * g.M) {   // prefetch the next unit of the same box (same ring or the next)
      const int dn = (lu + 1) / nt, tn = lu + 1 - dn * nt;
      const int i0 = tn * T - __ldg(shift + g.doff + dn);
      const int n = min(T, nz - tn * T);
      if (i0 >= 0 && i0 + n <= nz) {
        const int64_t base = g.poff + (int64_t)dn * nz + i0;
        for (int a = lane; a < narr; a += kLanes) {
          const double* arr;
          if (a < 9) arr = rho + (int64_t)a * P;
          else if (a < 18) arr = rhobar + (int64_t)(a - 9) * P;
          else if (a < 36) arr = lam_out + (int64_t)(a - 18) * P;
          else if (a < 54) arr = lam_tot + (int64_t)(a - 36) * P;
          else if (a == 54) arr = Nw;
          else if (a == 55) arr = Nbw;
          else if (a == 56) arr = gN;
          else if (a == 57) arr = gNbar;
          else arr = W + (int64_t)(a - 58) * P;
          prefetch_l2(arr, base, n);
        }
      }
    }
    const int craw = tile * T - Hh + lane, j = wrapc(craw, nz);
    const bool active = lane >= Hh && lane < Hh + T && craw < nz;
    const int gd = g.doff + d;
    const double ox = __ldg(dirtab + gd), oy = __ldg(dirtab + MT + gd), oz = __ldg(dirtab + 2 * MT + gd);
    const int64_t p = g.poff + (int64_t)d * nz + wrapc(j - __ldg(shift + gd), nz);
    double wt[Sten<ORDER>::NW];
    zero_weights<ORDER>(wt);
    double n1 = 0.0, n2 = 0.0;
    if (active) {
      load_weights<ORDER>(W, P, p, wt);
      n1 = Nw[p];
      n2 = Nbw[p];
    }
    double GB[9];
    const double* Ej = E + g.coff + j;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double G = fma(-oz, __ldg(Ej + (int64_t)(27 + k) * NZ),
                           fma(-oy, __ldg(Ej + (int64_t)(18 + k) * NZ),
                               fma(-ox, __ldg(Ej + (int64_t)(9 + k) * NZ), __ldg(Ej + (int64_t)k * NZ))));
      GB[k] = gather<ORDER>(wt, G);
    }
    if (!active) continue;
    // neutrinos, then antineutrinos: every load of a half before its stores
#pragma unroll
    for (int which = 0; which < 2; ++which) {
      const double* __restrict__ r = which ? rhobar : rho;
      double rv[9], lo[9], lt[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        rv[k] = r[k * P + p];
        lo[k] = lam_out[(which * 9 + k) * P + p];
        lt[k] = lam_tot[(which * 9 + k) * P + p];
      }
      double sum = 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        // B = N rho - Nbar conj(rhobar): dB/drhobar = -Nbar conj(.), conjugation
        // flipping the imaginary components 4, 6, 8
        const double sg = which ? ((k == 4 || k == 6 || k == 8) ? 1.0 : -1.0) : 1.0;
        const double l = fma((which ? n2 : n1) * sg, GB[k], lo[k]);
        lam_out[(which * 9 + k) * P + p] = l;
        lam_tot[(which * 9 + k) * P + p] = lt[k] + l;
        sum = fma(sg * GB[k], rv[k], sum);
      }
      if (which) gNbar[p] += sum;
      else gN[p] += sum;
    }
  }
}

// Adjoint seed from a loss on the moments at the current positions: with
// dmom = dL/d(mom) on the [72][NZ] layout of the moments (Eq. 5 per species),
//   lam_rho,p    = N_p    (1/dV) sum_j w_pj (dmom_n,j    + Omega_p . dmom_f,j)
//   lam_rhobar,p = Nbar_p (1/dV) sum_j w_pj (dmom_nbar,j + Omega_p . dmom_fbar,j)
// and gN_p += lam_rho,p . rho_p / N_p (likewise gNbar); lam is overwritten.
template <int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k_adj_seed(Batch B, Parts pt, const double* __restrict__ dirtab, const int* __restrict__ shift,
           const double* __restrict__ dmom, double* __restrict__ lam, double* __restrict__ gN,
           double* __restrict__ gNbar, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t w = logical_warp();
  const int64_t u0 = unit_begin(w, B), u1 = unit_begin(w + 1, B);
  if (u0 >= u1) return;
  const int64_t P = B.Ptot;
  const int MT = B.MT, NZ = B.NZ;
  int bad = 0;
  int b = box_of_unit(B, u0);
  for (int64_t u = u0; u < u1; ++u) {
    while (u >= B.box[b].uoff + (int64_t)B.box[b].ntiles * B.box[b].M) ++b;
    const BoxGeo& g = B.box[b];
    const int nz = g.nz, nt = g.ntiles;
    const int lu = (int)(u - g.uoff);
    const int d = lu / nt, tile = lu - d * nt;
    constexpr int Hh = Sten<ORDER>::H, T = Sten<ORDER>::T;
    const int craw = tile * T - Hh + lane, j = wrapc(craw, nz);
    const bool active = lane >= Hh && lane < Hh + T && craw < nz;
    const int gd = g.doff + d;
    const double ox = __ldg(dirtab + gd), oy = __ldg(dirtab + MT + gd), oz = __ldg(dirtab + 2 * MT + gd);
    const int64_t p = g.poff + (int64_t)d * nz + wrapc(j - __ldg(shift + gd), nz);
    double wt[Sten<ORDER>::NW];
    zero_weights<ORDER>(wt);
    if (active) bad |= shape_weights<ORDER>(pt.z[p], (double)j + 0.5, g.inv_dz, g.nz_d, wt);
    const double* Ej = dmom + g.coff + j;
#pragma unroll
    for (int which = 0; which < 2; ++which) {
      const int64_t base = which * kNA;
      double GB[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const double G = fma(oz, __ldg(Ej + (base + 27 + k) * NZ),
                             fma(oy, __ldg(Ej + (base + 18 + k) * NZ),
                                 fma(ox, __ldg(Ej + (base + 9 + k) * NZ), __ldg(Ej + (base + k) * NZ))));
        GB[k] = gather<ORDER>(wt, G) * g.inv_dV;
      }
      if (active) {
        const double Nw = which ? pt.Nbar[p] : pt.N[p];
        const double* r = which ? pt.rhobar : pt.rho;
        double sN = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          lam[(which * 9 + k) * P + p] = Nw * GB[k];
          sN = fma(GB[k], r[k * P + p], sN);
        }
        if (which) gNbar[p] += sN;
        else gN[p] += sN;
      }
    }
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// Chain rule through Eq. 8, N_p = (n_c + 3 f_c . Omega_p) dV / M with c the
// particle's initial cell: per cell (thread) and in direction order,
// out[0] dL/dn_nu, out[1] dL/dn_nubar, out[2..4] dL/df_nu, out[5..7] dL/df_nubar ([8][NZ]).
__global__ void k_weight_grad(Batch B, const double* __restrict__ gN, const double* __restrict__ gNbar,
                              const double* __restrict__ dirtab, double* __restrict__ out) {
  const int gc = blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= B.NZ) return;
  const BoxGeo& g = B.box[box_of_cell(B, gc)];
  const int c = gc - g.coff;
  const double f = g.dV / g.M;
  double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int d = 0; d < g.M; ++d) {
    const int64_t p = g.poff + (int64_t)d * g.nz + c;
    const int gd = g.doff + d;
    const double o[3] = {dirtab[gd], dirtab[B.MT + gd], dirtab[2 * B.MT + gd]};
    a[0] += gN[p];
    a[1] += gNbar[p];
    for (int i = 0; i < 3; ++i) {
      a[2 + i] += 3.0 * o[i] * gN[p];
      a[5 + i] += 3.0 * o[i] * gNbar[p];
    }
  }
  for (int k = 0; k < 8; ++k) out[(int64_t)k * B.NZ + gc] = a[k] * f;
}

}  // namespace emu_dev
