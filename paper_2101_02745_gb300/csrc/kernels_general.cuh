// kernels_general.cuh -- GB300 (sm_103a) FP64 device code of the particle step
// for particles at ANY positions and directions (1D boxes and batches).
// Included once, by emu.cu, after kernels.cuh.
//
// The lattice path (kernels.cuh) needs every particle on its ring's lattice
// site, which the paper's initial conditions and constant velocities keep
// (Sec. 3.1, Eq. 4).  The method itself (Eq. 5, 6) is defined for particles
// anywhere.  This path makes no assumption on positions or directions:
//   1. keys: every particle's containing cell at the stage positions (a
//      global cell index over the batch);
//   2. a stable least-significant-digit radix sort of (key, particle) with
//      4-bit digits: per block a digit histogram, one exclusive scan over
//      (digit, block), then a scatter in which each block ranks its items
//      stably (items in index order within a thread, threads in order);
//      particles of a cell end up in increasing index order;
//   3. cell starts from the sorted keys;
//   4. deposit (Eq. 5): one warp per cell sums, over the cells its stencil
//      reaches from (H on each side) and the particles of each in sorted
//      order, w_pj (1, Omega_p) B_p; lane l takes every 32nd particle, and
//      the lanes' sums are added by a fixed butterfly: no float atomics, the
//      same order on every run;
//   5. RK stage / interpolation: one thread per particle, its weights from
//      its own position and G = A0 - Omega_p . A at the cells it reaches.
#pragma once

namespace emu_dev {

constexpr int kRadixBits = 4;
constexpr int kRadixBuckets = 1 << kRadixBits;
constexpr int kRadixItems = 8;                       // items per thread
constexpr int kRadixTile = kThreads * kRadixItems;   // items per block

// Containing cell (global index) of every particle at z + frac dt_b c Omega_z;
// ids[p] = p.  Non-finite positions are an error (key 0).
__global__ void k_gkeys(Batch B, const double* __restrict__ z, const double* __restrict__ oz, double frac,
                        unsigned* __restrict__ keys, int* __restrict__ ids, int* __restrict__ err) {
  griddep_wait();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B.Ptot) return;
  const int b = box_of_particle(B, p);
  const BoxGeo& g = B.box[b];
  const double zs = fma(frac * B.dt[b], g.c_light * oz[p], z[p]);
  int h = 0;
  if (isfinite(zs)) h = wrapc((int)floor(zs * g.inv_dz), g.nz);
  else atomicOr(err, ERR_NONFINITE);
  keys[p] = (unsigned)(g.coff + h);
  ids[p] = (int)p;
}

// Radix sort, pass histogram: hist[d * nblk + block] = count of digit d in the block's tile.
__global__ void k_radix_hist(const unsigned* __restrict__ keys, int64_t n, int shift, int* __restrict__ hist,
                             int nblk) {
  __shared__ int cnt[kRadixBuckets];
  if (threadIdx.x < kRadixBuckets) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)threadIdx.x * kRadixItems;
#pragma unroll
  for (int i = 0; i < kRadixItems; ++i)
    if (base + i < n) atomicAdd(&cnt[(keys[base + i] >> shift) & (kRadixBuckets - 1)], 1);
  __syncthreads();
  if (threadIdx.x < kRadixBuckets) hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of v[0, n) in place by one block of kThreads threads (each
// takes a contiguous chunk; the chunk sums are scanned in shared memory).
__global__ void k_scan_exclusive(int* __restrict__ v, int64_t n) {
  __shared__ int64_t part[kThreads];
  const int64_t chunk = (n + kThreads - 1) / kThreads;
  const int64_t lo = min(n, (int64_t)threadIdx.x * chunk), hi = min(n, lo + chunk);
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < kThreads; off <<= 1) {   // inclusive Hillis-Steele scan of the chunk sums
    const int64_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t i = lo; i < hi; ++i) {
    const int x = v[i];
    v[i] = (int)run;
    run += x;
  }
}

// Radix sort, pass scatter: stable ranks within the block (a thread's items in
// index order, threads in order), offsets from the scanned histogram.
__global__ void k_radix_scatter(const unsigned* __restrict__ keys, const int* __restrict__ vals, int64_t n,
                                int shift, const int* __restrict__ offs, int nblk, unsigned* __restrict__ keys_out,
                                int* __restrict__ vals_out) {
  __shared__ int cnt[kRadixBuckets][kThreads];
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)t * kRadixItems;
  unsigned k[kRadixItems];
  int mine[kRadixBuckets];
#pragma unroll
  for (int d = 0; d < kRadixBuckets; ++d) mine[d] = 0;
#pragma unroll
  for (int i = 0; i < kRadixItems; ++i) {
    k[i] = base + i < n ? keys[base + i] : 0u;
    if (base + i < n) {
      const int d = (k[i] >> shift) & (kRadixBuckets - 1);
#pragma unroll
      for (int e = 0; e < kRadixBuckets; ++e) mine[e] += (e == d);
    }
  }
#pragma unroll
  for (int d = 0; d < kRadixBuckets; ++d) cnt[d][t] = mine[d];
  __syncthreads();
  // exclusive scan over the threads, per digit (warp shuffles, then warp totals)
  const int lane = t & 31, warp = t >> 5;
  __shared__ int wsum[kRadixBuckets][kWarps];
#pragma unroll 1
  for (int d = 0; d < kRadixBuckets; ++d) {
    int x = cnt[d][t];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[d][warp] = x;
    cnt[d][t] = x - cnt[d][t];       // exclusive within the warp
  }
  __syncthreads();
  int run[kRadixBuckets];
#pragma unroll
  for (int d = 0; d < kRadixBuckets; ++d) {
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[d][w];
    run[d] = offs[(int64_t)d * nblk + blockIdx.x] + before + cnt[d][t];
  }
#pragma unroll
  for (int i = 0; i < kRadixItems; ++i) {
    if (base + i < n) {
      const int d = (k[i] >> shift) & (kRadixBuckets - 1);
      int pos = 0;
#pragma unroll
      for (int e = 0; e < kRadixBuckets; ++e)
        if (e == d) pos = run[e]++;
      keys_out[pos] = k[i];
      vals_out[pos] = vals[base + i];
    }
  }
}

// start[c] = first index of sorted key c (start[NZ] = n): a cell without
// particles starts where the next non-empty one does.
__global__ void k_cell_start(const unsigned* __restrict__ keys, int64_t n, int NZ, int* __restrict__ start) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int lo = i == 0 ? -1 : (int)keys[i - 1];
  const int hi = i == n ? NZ : (int)keys[i];
  for (int c = lo + 1; c <= hi; ++c) start[c] = (int)i;
}

// Fixed-order sum of one value over the 32 lanes (butterfly); every lane gets it.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Deposit (Eq. 5) of particles anywhere: one warp per global cell (grid-
// stride), MODE as k_deposit (0, 1, 2, 4, 5); out as the lattice deposit's
// combination writes it (rows x NZ, scaled by kappa/dV or 1/dV).
template <int MODE, int ORDER>
__global__ void __launch_bounds__(kThreads)
k_gdeposit(Batch B, Parts pt, const double* __restrict__ r_nu, const double* __restrict__ r_nb, double frac,
           const int* __restrict__ ids, const int* __restrict__ start, double* __restrict__ out,
           int* __restrict__ err) {
  griddep_wait();
  constexpr int H = Sten<ORDER>::H, NW = Sten<ORDER>::NW;
  constexpr int NA = MODE == 5 ? kNT : kNA;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t P = B.Ptot;
  int bad = 0;
  for (int64_t gc = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); gc < B.NZ; gc += nwarps) {
    const int b = box_of_cell(B, (int)gc);
    const BoxGeo& g = B.box[b];
    const int j = (int)gc - g.coff;
    const double pos_dt = frac * B.dt[b];
    double acc[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) acc[c] = 0.0;
    for (int o = -H; o <= H; ++o) {             // source cells j - o: their particles' weight slot H + o
      if (ORDER == 0 && o != 0) continue;
      const int sc = g.coff + wrapc(j - o, g.nz);
      const int i0 = start[sc], i1 = start[sc + 1];
      for (int i = i0 + lane; i < i1; i += kLanes) {
        const int64_t p = ids[i];
        const double ox = pt.ox[p], oy = pt.oy[p], oz = pt.oz[p];
        const double zs = fma(pos_dt, g.c_light * oz, pt.z[p]);
        const int h = wrapc((int)floor(zs * g.inv_dz), g.nz);
        double wt[NW];
        bad |= shape_weights<ORDER>(zs, (double)h + 0.5, g.inv_dz, g.nz_d, wt);
        double w = wt[0];
#pragma unroll
        for (int s = 1; s < NW; ++s) w = (s == H + o) ? wt[s] : w;
        if constexpr (MODE == 5) {
          const double n1 = w * pt.N[p], n2 = w * pt.Nbar[p];
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
            acc[c] += bv;
            acc[kNC + c] = fma(ox, bv, acc[kNC + c]);
            acc[2 * kNC + c] = fma(oy, bv, acc[2 * kNC + c]);
            acc[3 * kNC + c] = fma(oz, bv, acc[3 * kNC + c]);
          }
        } else if constexpr (MODE == 4) {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const double c1 = w * pt.N[p] * r_nu[k * P + p];
            const double c2 = w * pt.Nbar[p] * r_nb[k * P + p];
            acc[k] += c1;
            acc[9 + k] = fma(ox, c1, acc[9 + k]);
            acc[18 + k] += c2;
            acc[27 + k] = fma(ox, c2, acc[27 + k]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const double n1 = (MODE == 0 || MODE == 1) ? w * pt.N[p] : 0.0;
            const double n2 = (MODE == 0 || MODE == 2) ? w * pt.Nbar[p] : 0.0;
            double bv;
            if (MODE == 0) {
              const double xv = r_nu[k * P + p], yv = r_nb[k * P + p];
              bv = (k == 4 || k == 6 || k == 8) ? fma(n2, yv, n1 * xv) : fma(-n2, yv, n1 * xv);
            } else if (MODE == 1) {
              bv = n1 * r_nu[k * P + p];
            } else {
              bv = n2 * r_nb[k * P + p];
            }
            acc[k] += bv;
            acc[9 + k] = fma(ox, bv, acc[9 + k]);
            acc[18 + k] = fma(oy, bv, acc[18 + k]);
            acc[27 + k] = fma(oz, bv, acc[27 + k]);
          }
        }
      }
    }
    const double scale = (MODE == 0 || MODE == 5) ? g.kappa_dV : g.inv_dV;
#pragma unroll
    for (int c = 0; c < NA; ++c) {
      const double v = warp_sum(acc[c]) * scale;
      if (lane == (c & 31)) {
        bad |= !isfinite(v) ? 2 : 0;
        out[(int64_t)c * B.NZ + gc] = v;
      }
    }
  }
  if (bad & 1) atomicOr(err, ERR_LATTICE);
  if (bad & 2) atomicOr(err, ERR_NONFINITE);
}

// The step's deposit (MODE 5) in two parts.  k_gprep: one thread per sorted
// position i (particle p = ids[i]): its weights at its stage position (as
// k_gdeposit forms them), the 8 traceless components of B = N rho - Nbar
// rhobar^* (Eq. 5) and its direction, stored in sorted order (Ws[q][i],
// Bs[c][i], Os[a][i]) so that the deposit reads each particle's data once per
// stage and contiguously instead of forming it for every cell that gathers it.
template <int ORDER>
__global__ void __launch_bounds__(kThreads)
k_gprep(Batch B, Parts pt, const double* __restrict__ r_nu, const double* __restrict__ r_nb, double frac,
        const int* __restrict__ ids, double* __restrict__ Ws, double* __restrict__ Bs, double* __restrict__ Os,
        int* __restrict__ err) {
  griddep_wait();
  constexpr int NW = Sten<ORDER>::NW, NWS = Sten<ORDER>::NWS;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t P = B.Ptot;
  if (i >= P) return;
  const int64_t p = ids[i];
  const int b = box_of_particle(B, p);
  const BoxGeo& g = B.box[b];
  const double ox = pt.ox[p], oy = pt.oy[p], oz = pt.oz[p];
  const double zs = fma(frac * B.dt[b], g.c_light * oz, pt.z[p]);
  const int h = wrapc((int)floor(zs * g.inv_dz), g.nz);
  double wt[NW];
  const int bad = shape_weights<ORDER>(zs, (double)h + 0.5, g.inv_dz, g.nz_d, wt);
#pragma unroll
  for (int q = 0; q < NWS; ++q) Ws[q * P + i] = wt[q];
  Os[i] = ox;
  Os[P + i] = oy;
  Os[2 * P + i] = oz;
  const double n1 = pt.N[p], n2 = pt.Nbar[p];
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
    Bs[c * P + i] = bv;
  }
  if (bad) atomicOr(err, ERR_LATTICE);
}

// The step's deposit from k_gprep's sorted data: kGSplit warps per global
// cell (one group of warps of a block), warp k of a group taking every
// kGSplit-th run of 32 particles of each source cell; each warp's sums are
// added over its lanes in a fixed order (a transpose through shared memory)
// and the group's warps in warp order: no float atomics, the same order on
// every run.
// out as k_gdeposit<5>: the traceless potential (kNT rows x NZ, kappa / dV).
constexpr int kGSplit = 4;
template <int ORDER>
__global__ void __launch_bounds__(kThreads)
k_gdeposit_sorted(Batch B, const double* __restrict__ Ws, const double* __restrict__ Bs,
                  const double* __restrict__ Os, const int* __restrict__ start, double* __restrict__ out,
                  int* __restrict__ err) {
  __shared__ double part[kWarps][kNT];
  __shared__ double tr[kWarps][kLanes][17];   // a warp's sums, 16 rows at a time (padded: no bank conflicts)
  griddep_wait();
  constexpr int H = Sten<ORDER>::H;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int grp = wib / kGSplit, k = wib - grp * kGSplit;
  constexpr int kGroups = kWarps / kGSplit;
  const int64_t P = B.Ptot;
  int bad = 0;
  // every block runs the same number of rounds (it synchronises inside)
  for (int64_t base = (int64_t)blockIdx.x * kGroups; base < B.NZ; base += (int64_t)gridDim.x * kGroups) {
    const int64_t gc = base + grp;
    double acc[kNT];
#pragma unroll
    for (int c = 0; c < kNT; ++c) acc[c] = 0.0;
    const BoxGeo* g = nullptr;
    if (gc < B.NZ) {
      g = &B.box[box_of_cell(B, (int)gc)];
      const int j = (int)gc - g->coff;
      for (int o = -H; o <= H; ++o) {           // source cells j - o: their particles' weight slot H + o
        if (ORDER == 0 && o != 0) continue;
        const int sc = g->coff + wrapc(j - o, g->nz);
        const int i0 = start[sc], i1 = start[sc + 1];
        for (int i = i0 + k * kLanes + lane; i < i1; i += kGSplit * kLanes) {
          const double w = ORDER == 0 ? 1.0 : __ldg(Ws + (int64_t)(H + o) * P + i);
          const double wx = w * __ldg(Os + i), wy = w * __ldg(Os + P + i), wz = w * __ldg(Os + 2 * P + i);
#pragma unroll
          for (int c = 0; c < kNC; ++c) {
            const double bv = __ldg(Bs + (int64_t)c * P + i);
            acc[c] = fma(w, bv, acc[c]);
            acc[kNC + c] = fma(wx, bv, acc[kNC + c]);
            acc[2 * kNC + c] = fma(wy, bv, acc[2 * kNC + c]);
            acc[3 * kNC + c] = fma(wz, bv, acc[3 * kNC + c]);
          }
        }
      }
    }
    // the sum over the lanes of each of the 32 rows, 16 rows at a time through
    // shared memory: lane l adds column l mod 16 over rows 16 (l / 16) .. +15,
    // then the two halves (lanes l and l + 16) are added
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int c = 0; c < 16; ++c) tr[wib][lane][c] = acc[half * 16 + c];
      __syncwarp();
      const int col = lane & 15, r0 = (lane >> 4) * 16;
      double v = tr[wib][r0][col];
#pragma unroll
      for (int r = 1; r < 16; ++r) v += tr[wib][r0 + r][col];
      v += __shfl_down_sync(kFull, v, 16);
      if (lane < 16) part[wib][half * 16 + lane] = v;
      __syncwarp();
    }
    __syncthreads();
    if (gc < B.NZ && k == 0) {
      const int c = lane;   // kNT = 32 rows, one per lane
      double v = part[wib][c];
      for (int q = 1; q < kGSplit; ++q) v += part[wib + q][c];
      v *= g->kappa_dV;
      bad |= !isfinite(v);
      out[(int64_t)c * B.NZ + gc] = v;
    }
    __syncthreads();
  }
  if (bad) atomicOr(err, ERR_NONFINITE);
}

// H (traceless components, or all 9 with NC = 9) of particle p at its stage
// position from the potential A (NC rows per moment): its weights and
// G = A0 - Omega_p . A at the cells it reaches.
template <int ORDER, int NC>
__device__ __forceinline__ void ginterp(const BoxGeo& g, int NZ, const double* __restrict__ A, double zs, double ox,
                                        double oy, double oz, double (&Hm)[NC]) {
  constexpr int H = Sten<ORDER>::H, NW = Sten<ORDER>::NW;
  const int h = wrapc((int)floor(zs * g.inv_dz), g.nz);
  double wt[NW];
  shape_weights<ORDER>(zs, (double)h + 0.5, g.inv_dz, g.nz_d, wt);
#pragma unroll
  for (int c = 0; c < NC; ++c) Hm[c] = 0.0;
#pragma unroll
  for (int s = 0; s < NW; ++s) {
    if (ORDER == 0 && s != H) continue;
    const double* Aj = A + g.coff + wrapc(h + s - H, g.nz);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double G = fma(-oz, Aj[(int64_t)(3 * NC + c) * NZ],
                           fma(-oy, Aj[(int64_t)(2 * NC + c) * NZ], fma(-ox, Aj[(int64_t)(NC + c) * NZ],
                                                                         Aj[(int64_t)c * NZ])));
      Hm[c] = fma(wt[s], G, Hm[c]);
    }
  }
}

// One RK4 stage of particles anywhere (as k_rk_stage): one thread per particle.
template <bool POT, int ORDER>
__global__ void __launch_bounds__(kThreads, 2)
k_grk_stage(Batch B, Parts pt, const double* __restrict__ At, int s, int dry) {
  griddep_wait();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B.Ptot) return;
  const int b = box_of_particle(B, p);
  const BoxGeo& g = B.box[b];
  const int64_t P = B.Ptot;
  const double dt = B.dt[b];
  const double bdt = (s == 1 || s == 4) ? dt / 6.0 : dt / 3.0;
  const double cdt = (s == 3) ? dt : 0.5 * dt;
  const double ox = pt.ox[p], oy = pt.oy[p], oz = pt.oz[p];
  const double vz = g.c_light * oz;
  const double zs = fma(stage_frac(s - 1) * dt, vz, pt.z[p]);
  double Hm[kNC];
  ginterp<ORDER, kNC>(g, B.NZ, At, zs, ox, oy, oz, Hm);
  const double* src_r = (s == 1) ? pt.rho : pt.stage;
  const double* src_b = (s == 1) ? pt.rhobar : pt.stage + 9 * P;
  double r[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) r[k] = src_r[k * P + p];
  rk_particle<POT, false>(g, pt, src_b, P, p, s, dry, bdt, cdt, dt, &vz, Hm, r);
}

// Interpolation only (Eq. 6 then Eq. 2) for particles anywhere: H[k * P + p].
template <int ORDER>
__global__ void k_ginterpolate(Batch B, Parts pt, const double* __restrict__ A, double frac, double* __restrict__ Hout) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B.Ptot) return;
  const int b = box_of_particle(B, p);
  const BoxGeo& g = B.box[b];
  const double ox = pt.ox[p], oy = pt.oy[p], oz = pt.oz[p];
  const double zs = fma(frac * B.dt[b], g.c_light * oz, pt.z[p]);
  double Hf[9];
  ginterp<ORDER, 9>(g, B.NZ, A, zs, ox, oy, oz, Hf);
#pragma unroll
  for (int k = 0; k < 9; ++k) Hout[k * B.Ptot + p] = Hf[k];
}

// Lattice contract check (the lattice path's precondition): every particle of
// a ring carries the ring's direction and sits in the cell its ring index
// assigns (within the lattice tolerance).  Sets *bad_out to 1 otherwise.
__global__ void k_lattice_check(Batch B, Parts pt, int* __restrict__ bad_out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B.Ptot) return;
  const BoxGeo& g = B.box[box_of_particle(B, p)];
  const int64_t lp = p - g.poff;
  const int d = (int)(lp / g.nz), i = (int)(lp - (int64_t)d * g.nz);
  const int64_t p0 = g.poff + (int64_t)d * g.nz;
  bool bad = pt.ox[p] != pt.ox[p0] || pt.oy[p] != pt.oy[p0] || pt.oz[p] != pt.oz[p0];
  const double z = pt.z[p], z0 = pt.z[p0];
  if (!isfinite(z) || !isfinite(z0)) {
    bad = true;
  } else {
    const int s0 = wrapc((int)floor(z0 * g.inv_dz), g.nz);
    const int j = wrapc(i + s0, g.nz);
    double dd = fma(z, g.inv_dz, -((double)j + 0.5));
    if (fabs(dd) > 0.5 + kLatticeTol) {
      dd -= g.nz_d * rint(dd / g.nz_d);
      bad = bad || fabs(dd) > 0.5 + kLatticeTol;
    }
  }
  if (bad) atomicOr(bad_out, 1);
}

}  // namespace emu_dev
