// emu.cu -- host side and C ABI of the GB300 (sm_103a) particle-in-cell step for
// the neutrino fast flavour instability (Richers, Willcox, Ford & Myers,
// arXiv:2101.02745).  Declarations and conventions: include/emu.h; device code
// and the data/parallel layout: kernels.cuh.
//
// One engine serves both the single-box entry points (a batch of one box) and
// the batch entry points (many independent boxes advanced by the same launches).
#include "emu.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "kernels3d.cuh"
#include "kernels_general.cuh"

using namespace emu_dev;

namespace {

constexpr int kMaxBoxes = 1 << 20;

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Geometry of a batch, from its configurations only (no device needed).
struct Shape {
  int nbox = 0;
  int64_t Ptot = 0, U = 0, U32 = 0;
  int NZ = 0, MT = 0, NT = 0;
  int NT32 = 0;    // 32-cell tiles of all boxes
  int order = 2;   // shape order of every box (Sec. 2.2.1)
  int Mmax = 0;    // most directions of a box
  int T = 30;      // cells per tile for that order
  std::vector<BoxGeo> geo;
};

// Cells per tile and kept weight arrays of a shape order (Sten<> on the host).
int tile_cells(int order) { return order == 3 ? Sten<3>::T : Sten<2>::T; }
int kept_weights(int order) {
  return order == 0 ? Sten<0>::NWS : order == 1 ? Sten<1>::NWS : order == 2 ? Sten<2>::NWS : Sten<3>::NWS;
}

// Calls f(std::integral_constant<int, ORDER>) for the runtime shape order.
template <typename F>
int by_order(int order, F&& f) {
  switch (order) {
    case 0: return f(std::integral_constant<int, 0>{});
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    default: return f(std::integral_constant<int, 3>{});
  }
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
  if (c->shape_order < 0 || c->shape_order > 3) return "shape_order must be 0, 1, 2 or 3";
  if (c->reserved != 0) return "reserved must be 0";
  return nullptr;
}

const char* make_shape(const emu_config* cfgs, int nbox, Shape& S) {
  if (!cfgs) return "config array is NULL";
  if (nbox < 1 || nbox > kMaxBoxes) return "nbox out of range";
  S = Shape();
  S.nbox = nbox;
  S.geo.resize(nbox);
  S.order = cfgs[0].shape_order;
  S.T = tile_cells(S.order);
  int64_t NZ = 0, MT = 0, NT = 0;
  for (int b = 0; b < nbox; ++b) {
    const emu_config* c = &cfgs[b];
    if (const char* why = config_problem(c)) return why;
    if (c->shape_order != S.order) return "all boxes of a batch must use the same shape order";
    BoxGeo& g = S.geo[b];
    std::memset(&g, 0, sizeof(g));
    g.nz = c->nz;
    g.M = c->ndir;
    g.ntiles = (c->nz + S.T - 1) / S.T;
    g.P = (int64_t)c->nz * c->ndir;
    g.poff = S.Ptot;
    g.uoff = S.U;
    g.ntiles32 = (c->nz + kLanes - 1) / kLanes;
    g.uoff32 = S.U32;
    g.toff32 = S.NT32;
    g.coff = (int)NZ;
    g.toff = (int)NT;
    g.doff = (int)MT;
    g.Lz = c->Lz;
    g.dz = c->Lz / c->nz;
    g.inv_dz = 1.0 / g.dz;
    g.nz_d = (double)c->nz;
    g.dV = g.dz * c->area;
    g.c_light = c->c_light;
    g.kappa_dV = c->kappa / g.dV;
    g.inv_dV = 1.0 / g.dV;
    g.cfl_adv = c->cfl_adv;
    g.cfl_flavor = c->cfl_flavor;
    g.kappa = c->kappa;
    // the kernels index a box's units with int (unit = direction * ntiles + tile)
    if ((int64_t)g.ntiles * g.M > INT32_MAX) return "box too large: its tiles x directions exceed 2^31";
    S.Ptot += g.P;
    S.U += (int64_t)g.ntiles * g.M;
    S.U32 += (int64_t)g.ntiles32 * g.M;
    S.Mmax = g.M > S.Mmax ? g.M : S.Mmax;
    NZ += c->nz;
    MT += c->ndir;
    NT += g.ntiles;
    S.NT32 += g.ntiles32;
    if (NZ > INT32_MAX / kNM || MT > INT32_MAX / 4 || S.Ptot > ((int64_t)1 << 40)) return "batch too large";
  }
  S.NZ = (int)NZ;
  S.MT = (int)MT;
  S.NT = (int)NT;
  return nullptr;
}

struct Layout {
  size_t geo, dts, nmax, A, At, mom, partial, W, err, dirtab, shift, wtab, bar, species, dirs, diag, scalar, total;
  size_t rowgeo = 0;   // 3D boxes: one descriptor per cell row (the deposit combination's batch view)
  // particles anywhere (kernels_general.cuh): sort keys and values (two of
  // each), digit histogram, cell starts, lattice-check flag
  size_t gkeys = 0, gkeys2 = 0, gids = 0, gids2 = 0, ghist = 0, gstart = 0, gflag = 0;
  size_t gprep = 0;  // particles anywhere: B (8) and Omega (3) of every particle in sorted order (k_gprep)
  size_t frame = 0; // step form 2: the frame sums of every 32-cell tile (k_frame_sum)
  size_t bw3 = 0;   // 3D boxes: 8-component field of every (direction, cell): B, its spread passes (k3_prep, k3_pass)
  size_t gf3 = 0;   // 3D boxes: a second such field: G = A0 - Omega . A and its gather passes (k3_gfield, k3_pass)
  size_t wdir3 = 0; // 3D boxes: every direction's shape weights per stage and axis (k3_shifts)
};

Layout layout(const Shape& S) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t nb = (size_t)S.nbox, NZ = (size_t)S.NZ, MT = (size_t)S.MT;
  L.geo = take(sizeof(BoxGeo) * nb);
  L.dts = take(sizeof(double) * nb);
  L.nmax = take(sizeof(double) * nb);
  L.A = take(sizeof(double) * kNA * NZ);
  L.At = take(sizeof(double) * kNT * NZ);
  L.mom = take(sizeof(double) * kNM * NZ);
  // per-warp partial sums of k_deposit, or of k_rk_deposit (step form 2)
  const size_t slots = (size_t)(kMaxWarps + S.NT) * kSlot, slots32 = (size_t)(kMaxWarps + S.NT32) * kSlotF;
  L.partial = take(sizeof(double) * (slots > slots32 ? slots : slots32));
  L.W = take(sizeof(double) * kept_weights(S.order) * (size_t)S.Ptot);
  L.err = take(sizeof(int));
  L.dirtab = take(sizeof(double) * 4 * MT);
  L.shift = take(sizeof(int) * 5 * MT);    // rows: the four stages, the next step's first (step form 2)
  L.frame = take(sizeof(double) * (size_t)S.NT32 * kSlotF);
  L.wtab = take(sizeof(double) * 5 * kWSlots * MT);   // the rings' shape weights at each shift row
  L.bar = take(sizeof(unsigned) * 2);       // the fused step's grid barrier: arrival word, abort word
  L.species = take(sizeof(double) * 8 * NZ);
  L.dirs = take(sizeof(double) * 3 * MT);
  L.diag = take(sizeof(double) * 63 * nb);
  L.scalar = take(sizeof(double) * 4);
  const size_t P = (size_t)S.Ptot, nblk = (P + kRadixTile - 1) / kRadixTile;
  L.gkeys = take(sizeof(unsigned) * P);
  L.gkeys2 = take(sizeof(unsigned) * P);
  L.gids = take(sizeof(int) * P);
  L.gids2 = take(sizeof(int) * P);
  L.ghist = take(sizeof(int) * kRadixBuckets * (nblk ? nblk : 1));
  L.gstart = take(sizeof(int) * ((size_t)NZ + 1));
  L.gflag = take(sizeof(int));
  L.gprep = take(sizeof(double) * (size_t)(kNC + 3) * P);
  L.total = off;
  return L;
}

enum : int {
  CLS_SHIFT = 0, CLS_DEPOSIT = 1, CLS_RK = 2, CLS_COMBINE = 3, CLS_OTHER = 4, CLS_STEP = 5, CLS_RKDEP = 6, N_CLS = 7
};

const double kStageFrac[4] = {0.0, 0.5, 0.5, 1.0};  // position offset of RK stage s, in units of dt

}  // namespace

struct emu_box {
  Shape S;
  Layout L;
  std::vector<emu_config> cfg;
  Parts pt{};
  bool bound = false;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  BoxGeo* geo_d = nullptr;
  // A: full grid potential of emu_deposit; At: the step's traceless potential
  double *dts = nullptr, *nmax = nullptr, *A = nullptr, *At = nullptr, *mom = nullptr, *partial = nullptr,
         *W = nullptr, *dirtab = nullptr, *species = nullptr, *dirs = nullptr, *diag = nullptr, *scalar = nullptr,
         *frame = nullptr;
  int *err = nullptr, *shift = nullptr;
  double* wtab = nullptr;   // the rings' shape weights at each shift row [5 x kWSlots][MT] (k_shifts)
  unsigned* bar = nullptr;
  int blocks = kPersistBlocks;  // grid of the step kernels (autotuned); its warps split the units
  int rk_form = -1;             // RK stage: 0 halo-lane, 1 32-cell, -1 by units per warp (autotuned)
  int dep_form = 0;             // the form-0 step's deposit: 0 per-warp partials and their combination,
                                // 1, 2 thread-block clusters of 8, 16 blocks writing the potential
  int dep_clusters[2] = {-1, -1};   // clusters of 8, 16 blocks resident at once (-1: not asked yet)
  int step_form = 0;            // 0: one launch per phase, 1: one cooperative launch per step (k_step),
                                // 2: RK stages that deposit the next stage (k_rk_deposit)
  unsigned long long limit_ns = 1000000000ull;   // bound of each grid-barrier wait of k_step
  // 3D boxes (emu3_create): the box is S's single box (cells in 3D index order),
  // positions x, y beside the particle arrays, and one descriptor per cell row
  int layout = -1;        // particle layout: 0 lattice, 1 anywhere, -1 checked when particles are installed
  bool general = false;   // the step runs the path for particles anywhere (kernels_general.cuh)
  bool is3d = false;
  emu3_config c3{};
  double *x3 = nullptr, *y3 = nullptr;
  std::vector<BoxGeo> rows;
  BoxGeo* rows_d = nullptr;
  int ntz = 0;
  bool pot = false;             // some box has vacuum or matter terms
  int next_stage = 1;
  std::vector<double> dt_h;  // step sizes currently on the device
  bool dt_set = false;
  std::vector<double> step_dt;  // the boxes' RK step sizes (Eq. 7 or set by the caller)
  bool step_valid = false;
  int64_t launches = 0;
  // optional per-launch timing: events recorded on the box's stream around each kernel
  struct Rec { int cls; cudaEvent_t a, b; };
  bool prof = false;
  bool capturing = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaGraphExec_t graph = nullptr;   // one step of every box
  int64_t graph_launches = 0;
  cudaGraphExec_t graph1 = nullptr;  // step form 2: the first step of a call (with the first deposit)
  int64_t graph1_launches = 0;
  bool graph_rd = false;             // the step graphs run step form 2
  // one adjoint step, for the buffers and step size it was captured with
  cudaGraphExec_t adj_graph = nullptr;
  int64_t adj_launches = 0;
  const void* adj_key[4] = {nullptr, nullptr, nullptr, nullptr};
  // recorded-adjoint steps (record / backward), one graph per set of buffers
  struct KeyedGraph { const void* key[6]; cudaGraphExec_t exec; int64_t launches; };
  std::vector<KeyedGraph> rec_graphs;
  // graphs of a box bound to the legacy default stream run on this blocking
  // stream, which the legacy stream orders implicitly with its own work
  cudaStream_t cap = nullptr;
  char msg[512] = {0};
  ~emu_box() {
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
    if (graph) cudaGraphExecDestroy(graph);
    if (graph1) cudaGraphExecDestroy(graph1);
    if (adj_graph) cudaGraphExecDestroy(adj_graph);
    for (auto& g : rec_graphs) cudaGraphExecDestroy(g.exec);
    if (cap) cudaStreamDestroy(cap);
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

Batch batch_view(const emu_box* b) {
  Batch B;
  B.box = b->geo_d;
  B.dt = b->dts;
  B.nbox = b->S.nbox;
  const int64_t nw = (int64_t)b->blocks * kWarps;
  B.nw = (int)(b->S.U < nw ? b->S.U : nw);
  B.NZ = b->S.NZ;
  B.MT = b->S.MT;
  B.NT = b->S.NT;
  B.T = b->S.T;
  B.U = b->S.U;
  B.U32 = b->S.U32;
  B.nw32 = (int)(b->S.U32 < nw ? b->S.U32 : nw);
  B.Ptot = b->S.Ptot;
  return B;
}

cudaEvent_t take_event(emu_box* b) {
  if (!b->pool.empty()) { cudaEvent_t e = b->pool.back(); b->pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Called right before a launch: records the start event when timing is on.
void before_launch(emu_box* b, int cls) {
  if (!b->prof || b->capturing) return;
  emu_box::Rec r{cls, take_event(b), nullptr};
  if (r.a) cudaEventRecord(r.a, b->stream);
  b->recs.push_back(r);
}

int after_launch(emu_box* b, const char* what) {
  b->launches++;
  if (b->prof && !b->capturing && !b->recs.empty() && b->recs.back().b == nullptr) {
    b->recs.back().b = take_event(b);
    if (b->recs.back().b) cudaEventRecord(b->recs.back().b, b->stream);
  }
  return cuda_check(b, cudaGetLastError(), what);
}

dim3 persist_grid(const emu_box* b) { return dim3((unsigned)b->blocks, 1, 1); }

// Warps per group of 32 outputs in k_combine.  Long sums (more than 8
// partials per tile: small boxes, whose warps own one unit or few) are split
// over more warps, as far as needed to fill about one wave of the persistent
// grid (304 blocks x 8 warps); short sums keep one warp (coalesced, latency
// hidden by the other warps).
int combine_split(const Shape& S, int64_t nw, bool frame = false) {
  const int64_t U = frame ? S.U32 : S.U;
  const int64_t per_warp = nw > 0 && U / nw > 0 ? U / nw : 1;       // fewest units a warp takes
  const int64_t most = (S.Mmax + per_warp - 1) / per_warp + 1;        // most warps over one tile
  if (most <= 8) return 1;
  const int64_t out_warps = ((int64_t)(frame ? kNT : kNA) * S.NZ + kLanes - 1) / kLanes;
  int split = 1;
  while (split < kWarps && out_warps * split * 2 <= (int64_t)kPersistBlocks * kWarps && split * 8 < most)
    split <<= 1;
  return split;
}

unsigned combine_blocks(int rows, int NZ, int split) {
  const int64_t groups = (int64_t)(kWarps / split);
  const int64_t blocks = ((int64_t)rows * NZ + groups * kLanes - 1) / (groups * kLanes);
  return (unsigned)(blocks < 8 * kPersistBlocks ? blocks : 8 * kPersistBlocks);
}

int check_bound(emu_box* b) {
  if (!b) return EMU_EINVAL;
  if (!b->bound) return fail(b, EMU_EINVAL, "box is not bound to memory (call emu_bind)");
  return EMU_OK;
}

int check_single(emu_box* b) {
  if (int rc = check_bound(b)) return rc;
  if (b->S.nbox != 1) return fail(b, EMU_EINVAL, "this call takes a single box; use the emu_batch_* calls");
  return EMU_OK;
}

void invalidate_graph(emu_box* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (b->graph1) {
    cudaGraphExecDestroy(b->graph1);
    b->graph1 = nullptr;
  }
  if (b->adj_graph) {
    cudaGraphExecDestroy(b->adj_graph);
    b->adj_graph = nullptr;
  }
  for (auto& g : b->rec_graphs) cudaGraphExecDestroy(g.exec);
  b->rec_graphs.clear();
}

// Stream the box's graphs are captured on and replayed on: its own stream, or
// for the legacy default stream (which cannot be captured) a blocking stream
// of the box, implicitly ordered with the legacy stream in both directions.
int graph_stream(emu_box* b, cudaStream_t* out) {
  if (b->stream) { *out = b->stream; return EMU_OK; }
  if (!b->cap)
    if (int rc = cuda_check(b, cudaStreamCreate(&b->cap), "create graph stream")) return rc;
  *out = b->cap;
  return EMU_OK;
}

// Captures the launches of body() into *exec (their count into *count).
template <typename F>
int capture(emu_box* b, cudaGraphExec_t* exec, int64_t* count, F&& body) {
  cudaStream_t gs = nullptr;
  if (int rc = graph_stream(b, &gs)) return rc;
  const int64_t before = b->launches;
  if (int rc = cuda_check(b, cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal), "begin capture"))
    return rc;
  cudaStream_t saved = b->stream;
  b->stream = gs;
  b->capturing = true;
  int rc = body();
  b->capturing = false;
  b->stream = saved;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(gs, &g);
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return cuda_check(b, e, "end capture");
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { *exec = nullptr; return cuda_check(b, e, "instantiate graph"); }
  *count = b->launches - before;
  b->launches = before;
  return EMU_OK;
}

int launch_graph(emu_box* b, cudaGraphExec_t exec, int64_t count) {
  cudaStream_t gs = nullptr;
  if (int rc = graph_stream(b, &gs)) return rc;
  if (int rc = cuda_check(b, cudaGraphLaunch(exec, gs), "graph launch")) return rc;
  b->launches += count;
  return EMU_OK;
}

// Replays the graph captured from body() for these buffers (key), capturing
// it on first use; at most kKeyedGraphs are kept (the oldest is dropped).
constexpr size_t kKeyedGraphs = 256;
template <class F>
int keyed_graph(emu_box* b, const void* const (&key)[6], F&& body) {
  for (auto& g : b->rec_graphs)
    if (std::memcmp(g.key, key, sizeof(g.key)) == 0) return launch_graph(b, g.exec, g.launches);
  if (b->rec_graphs.size() >= kKeyedGraphs) {
    cudaGraphExecDestroy(b->rec_graphs.front().exec);
    b->rec_graphs.erase(b->rec_graphs.begin());
  }
  emu_box::KeyedGraph g{};
  std::memcpy(g.key, key, sizeof(g.key));
  if (int rc = capture(b, &g.exec, &g.launches, body)) return rc;
  b->rec_graphs.push_back(g);
  return launch_graph(b, g.exec, g.launches);
}

int copy_out(emu_box* b, void* dst, const void* src, size_t bytes, int on_host) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                  b->stream);
  if (e != cudaSuccess) return cuda_check(b, e, "copy out");
  if (on_host) return cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise after copy out");
  return EMU_OK;
}

// Upload per-box step sizes (host values) if they differ from what the device holds.
int set_dts(emu_box* b, const double* dt) {
  bool same = b->dt_set;
  for (int i = 0; same && i < b->S.nbox; ++i) same = b->dt_h[i] == dt[i];
  if (same) return EMU_OK;
  b->dt_h.assign(dt, dt + b->S.nbox);
  b->dt_set = true;
  return cuda_check(b, cudaMemcpyAsync(b->dts, b->dt_h.data(), sizeof(double) * b->S.nbox,
                                       cudaMemcpyHostToDevice, b->stream), "upload step sizes");
}

// Launch with programmatic dependent launch: the kernel's blocks may be
// scheduled while the previous kernel of the stream drains; the step kernels
// begin with griddepcontrol.wait, so they touch memory only once it is done.
// A failed launch is left for after_launch's cudaGetLastError.
template <typename... KArgs, typename... Args>
void pdl(cudaStream_t st, void (*kernel)(KArgs...), dim3 grid, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
void pdl_smem(cudaStream_t st, void (*kernel)(KArgs...), dim3 grid, int smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Whether the deposit takes the rings' weights from the weight table: when
// every warp walks at least 4 units (on boxes whose warps take one or two
// units the table's loads lengthen each warp's chain more than the weights'
// arithmetic they replace: 256 x 96 +4%, 2048 x 1000 -1.5% per step).  The
// rule depends only on the batch and the grid, as the summation order does.
bool use_wtab(const emu_box* b) {
  const Batch B = batch_view(b);
  return B.U >= 4 * (int64_t)B.nw;
}

// nrows = 5: the four stages' rows and the next step's first (k_shifts); the
// rings' shape weights at every row go to the weight table.
int launch_shifts(emu_box* b, const double* fracs, int nrows) {
  Fracs f{};
  for (int s = 0; s < nrows && s < 4; ++s) f.v[s] = fracs[s];
  const int blocks = (int)(((int64_t)b->S.MT * nrows + kThreads - 1) / kThreads);
  before_launch(b, CLS_SHIFT);
  by_order(b->S.order, [&](auto O) {
    pdl(b->stream, k_shifts<decltype(O)::value>, dim3(blocks), batch_view(b), b->pt.z, b->dirtab, f, nrows, b->shift,
        use_wtab(b) ? b->wtab : nullptr);
    return 0;
  });
  return after_launch(b, "shift kernel");
}

// The weight-table row matching a shift row of the box's table (nullptr for
// other shift rows, or when the table is not used: the deposit then forms
// each particle's weights).
const double* weight_row(const emu_box* b, const int* shift_row) {
  if (!use_wtab(b)) return nullptr;
  const int64_t MT = b->S.MT;
  const int64_t off = shift_row - b->shift;
  if (MT <= 0 || off < 0 || off >= 5 * MT || off % MT != 0) return nullptr;
  return b->wtab + (off / MT) * kWSlots * MT;
}

// Launch of a cluster kernel (clusters of `cl` blocks along x) with
// programmatic dependent launch and `smem` bytes of dynamic shared memory.
template <typename... KArgs, typename... Args>
cudaError_t cluster_pdl(cudaStream_t st, void (*kernel)(KArgs...), int clusters, int cl, int smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * cl));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

using DepClusterKernel = void (*)(Batch, const double*, const double*, const double*, const double*, const double*,
                                  const double*, const int*, const double*, double, double*, double*, int*);

int dep_cluster_size(int form) { return form == 2 ? 16 : 8; }

// The cluster deposit's instance for the box's shape order, the weight table
// and the cluster size of deposit form `form` (1: 8 blocks, 2: 16), with its
// attributes set for the current device (64 KB of shared memory; 16-block
// clusters are beyond the portable size).
DepClusterKernel dep_cluster_kernel(const emu_box* b, int form, bool tab, cudaError_t* e) {
  DepClusterKernel k = nullptr;
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    if (form == 2) k = tab ? k_deposit_cluster<R, true, 16> : k_deposit_cluster<R, false, 16>;
    else k = tab ? k_deposit_cluster<R, true, 8> : k_deposit_cluster<R, false, 8>;
    return 0;
  });
  *e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kDepClusterSmem);
  if (*e == cudaSuccess && form == 2) *e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return k;
}

// Clusters of the cluster deposit of form 1 or 2 that fit on the device at
// once (0: it cannot run here).  Asked once per box.
int dep_cluster_capacity(emu_box* b, int form) {
  int& cached = b->dep_clusters[form == 2 ? 1 : 0];
  if (cached >= 0) return cached;
  int n = 0;
  cudaError_t e;
  DepClusterKernel k = dep_cluster_kernel(b, form, false, &e);
  if (e == cudaSuccess) {
    const int cl = dep_cluster_size(form);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(64 * cl));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kDepClusterSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) n = 0;
  }
  (void)cudaGetLastError();   // a refusal above is an answer, not a pending error
  cached = n;
  return n;
}

// The step's deposit (mode 5) by clusters: one launch, the potential written
// directly (no combination).  The clusters stay resident: as many as fit, at
// most one per tile.
int launch_deposit_cluster(emu_box* b, const double* rnu, const double* rnb, const int* shift_row, double frac,
                           double* out, double* W) {
  const int form = b->dep_form;
  const int cap = dep_cluster_capacity(b, form);
  if (cap <= 0) return fail(b, EMU_EINVAL, "the device cannot run the cluster deposit");
  const Batch B = batch_view(b);
  const int clusters = (int)std::min<int64_t>(B.NT, cap);
  const double* wrow = weight_row(b, shift_row);
  cudaError_t e;
  DepClusterKernel k = dep_cluster_kernel(b, form, wrow != nullptr, &e);
  if (e != cudaSuccess) return cuda_check(b, e, "cluster deposit attributes");
  before_launch(b, CLS_DEPOSIT);
  e = cluster_pdl(b->stream, k, clusters, dep_cluster_size(form), kDepClusterSmem, B, b->pt.z, b->pt.N, b->pt.Nbar,
                  rnu, rnb, b->dirtab, shift_row, wrow, frac, out, W, b->err);
  const int rc = after_launch(b, "cluster deposit kernel");   // (closes the timing record either way)
  return e != cudaSuccess ? cuda_check(b, e, "cluster deposit launch") : rc;
}

// Deposit (two launches) of the state (rnu, rnb) at positions z + frac dt_b v_z
// with the shift row shift_row, into out ([36][NZ]; mode 5: [32][NZ]).  Modes as k_deposit; the
// potential scale kappa/dV for modes 0 and 3, 1/dV for the moments.
int launch_deposit(emu_box* b, int mode, const double* rnu, const double* rnb, const int* shift_row, double frac,
                   double* out, double* W = nullptr) {
  if (!W) W = b->W;   // where modes 0 and 5 keep the shape weights
  if (mode == 5 && b->dep_form != 0) return launch_deposit_cluster(b, rnu, rnb, shift_row, frac, out, W);
  const Batch B = batch_view(b);
  before_launch(b, CLS_DEPOSIT);
  const dim3 grid = persist_grid(b);
  cudaStream_t st = b->stream;
  const double* z = b->pt.z;
  const double* N = b->pt.N;
  const double* Nb = b->pt.Nbar;
  const double* wrow = weight_row(b, shift_row);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    if (mode == 0)
      pdl(st, k_deposit<0, R>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial, W, b->err);
    else if (mode == 1)
      pdl(st, k_deposit<1, R>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial, nullptr,
          b->err);
    else if (mode == 2)
      pdl(st, k_deposit<2, R>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial, nullptr,
          b->err);
    else if (mode == 3 && wrow != nullptr)   // (the adjoint's deposit: the weights its forward step used)
      pdl(st, k_deposit<3, R, true>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial,
          nullptr, b->err);
    else if (mode == 3)
      pdl(st, k_deposit<3, R>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial, nullptr,
          b->err);
    else if (mode == 4)
      pdl(st, k_deposit<4, R>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial, nullptr,
          b->err);
    else if (wrow != nullptr)
      pdl(st, k_deposit<5, R, true>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial, W,
          b->err);
    else
      pdl(st, k_deposit<5, R>, grid, B, z, N, Nb, rnu, rnb, b->dirtab, shift_row, wrow, frac, b->partial, W, b->err);
    return 0;
  });
  if (int rc = after_launch(b, "deposit kernel")) return rc;
  before_launch(b, CLS_COMBINE);
  const int split = combine_split(b->S, B.nw);
  const int rows = mode == 5 ? kNT : kNA;
  const int potential = (mode == 0 || mode == 3 || mode == 5) ? 1 : 0;
  pdl(b->stream, k_combine, dim3(combine_blocks(rows, B.NZ, split)), B, b->partial, out, rows, potential,
      split, b->err);
  return after_launch(b, "deposit combine kernel");
}

// One RK stage of every box with its device step size (the shift rows of the
// step must have been computed by stage 1's caller).
int launch_rk(emu_box* b, int s, const int* srow, int dry);

// The 3D box's launches (defined with the other 3D helpers below).
int launch3_step(emu_box* b, int dry);
int launch3_stage(emu_box* b, int s, int dry);
int launch3_shifts(emu_box* b, const double* fracs, int nrows);
int launch3_deposit(emu_box* b, int mode, const double* rnu, const double* rnb, const int* srow, double frac,
                    double* out);
int run3_moments(emu_box* b);
int rebuild_dirtable3(emu_box* b);
// The launches for particles anywhere (defined below).
int launch_gstep(emu_box* b, int dry);
int launch_gstage(emu_box* b, int s, int dry);
int launch_gdeposit(emu_box* b, int mode, const double* rnu, const double* rnb, double frac, double* out);

int launch_stage(emu_box* b, int s, int dry) {
  const size_t P = (size_t)b->S.Ptot;
  const double* rnu = (s == 1) ? b->pt.rho : b->pt.stage;
  const double* rnb = (s == 1) ? b->pt.rhobar : b->pt.stage + 9 * P;
  const int* srow = b->shift + (size_t)(s - 1) * b->S.MT;
  if (int rc = launch_deposit(b, 5, rnu, rnb, srow, kStageFrac[s - 1], b->At)) return rc;
  return launch_rk(b, s, srow, dry);
}

// Whether the RK stage runs with 32 cells per warp (no halo lanes): when every
// warp walks at least 8 units (the tile ends at ring and range boundaries are
// computed directly), unless a form was chosen; otherwise the halo-lane form,
// which gives bitwise the same results.
bool use_rk32(const emu_box* b, const Batch& Bv) {
  return b->rk_form >= 0 ? b->rk_form == 1 : Bv.U32 >= 8 * (int64_t)Bv.nw32;
}

// Most blocks of the fused step kernel that can be resident at once (its
// cooperative launch needs every block resident).
int fused_max_blocks(const emu_box* b) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  // every instantiation has the same launch bounds; the largest (cubic shape,
  // vacuum terms, 32-cell RK stage) stands for all
  (void)b;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<true, 3, true>, kThreads, 0) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

// nsteps RK4 steps of every box in one cooperative launch of k_step (dry: the
// results of stage 4 go to the stage buffer, as in launch_step).
int launch_fused(emu_box* b, int dry, int64_t nsteps) {
  const int maxb = fused_max_blocks(b);
  if (b->blocks > maxb)
    return fail(b, EMU_EINVAL, "the fused step needs all %d blocks resident at once; at most %d fit", b->blocks, maxb);
  const Batch B = batch_view(b);
  StepArgs a{};
  a.dirtab = b->dirtab;
  a.shift = b->shift;
  a.wtab = use_wtab(b) ? b->wtab : nullptr;
  a.W = b->W;
  a.At = b->At;
  a.partial = b->partial;
  a.err = b->err;
  a.bar = b->bar;
  a.limit_ns = b->limit_ns;
  a.nsteps = nsteps;
  a.split = combine_split(b->S, B.nw);
  a.dry = dry;
  const bool r32 = use_rk32(b, B);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = persist_grid(b);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  before_launch(b, CLS_STEP);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    if (b->pot) {
      if (r32) (void)cudaLaunchKernelEx(&cfg, k_step<true, R, true>, B, b->pt, a);
      else (void)cudaLaunchKernelEx(&cfg, k_step<true, R, false>, B, b->pt, a);
    } else {
      if (r32) (void)cudaLaunchKernelEx(&cfg, k_step<false, R, true>, B, b->pt, a);
      else (void)cudaLaunchKernelEx(&cfg, k_step<false, R, false>, B, b->pt, a);
    }
    return 0;
  });
  return after_launch(b, "fused step kernel");
}

// The RK-stage kernel of stage s from the shape weights W and the traceless
// potential At of its deposit; stages 2-4 read their state from stage_src and
// write the next one to pt.stage.
int launch_rk_on(emu_box* b, int s, const int* srow, int dry, const Parts& pt, const double* W, const double* At,
                 const double* stage_src) {
  before_launch(b, CLS_RK);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    // 32 cells per warp, no halo lanes, when every warp walks at least 8 units (the
    // tile ends at ring and range boundaries are computed directly); otherwise
    // the halo-lane kernel, which gives bitwise the same results
    const Batch Bv = batch_view(b);
    const dim3 grid = persist_grid(b);
    const bool use32 = use_rk32(b, Bv);
    if (!use32) {
      if (b->pot)
        pdl(b->stream, k_rk_stage<true, R>, grid, Bv, pt, W, b->dirtab, srow, At, stage_src, s, dry);
      else
        pdl(b->stream, k_rk_stage<false, R>, grid, Bv, pt, W, b->dirtab, srow, At, stage_src, s, dry);
      return 0;
    }
    if (b->pot)
      pdl(b->stream, k_rk_stage32<true, R>, grid, Bv, pt, W, b->dirtab, srow, At, stage_src, s, dry);
    else
      pdl(b->stream, k_rk_stage32<false, R>, grid, Bv, pt, W, b->dirtab, srow, At, stage_src, s, dry);
    return 0;
  });
  return after_launch(b, "RK stage kernel");
}

int launch_rk(emu_box* b, int s, const int* srow, int dry) {
  return launch_rk_on(b, s, srow, dry, b->pt, b->W, b->At, b->pt.stage);
}

// Step form 2 (k_rk_deposit, k_combine_frame) covers 1D boxes on the lattice
// path with shape orders 0-2 ...
bool rd_possible(const emu_box* b) { return !b->is3d && !b->general && b->S.order <= 2; }

// ... and step sizes with dt c < 1.9 dz in every box: a ring then moves at
// most one cell between two stages (half a step).
bool rd_step_sizes_ok(const emu_box* b) {
  if (!b->dt_set) return false;
  for (int i = 0; i < b->S.nbox; ++i) {
    const BoxGeo& g = b->S.geo[i];
    if (!(b->dt_h[i] * g.c_light < 1.9 * g.dz)) return false;
  }
  return true;
}

// Whether the steps run form 2: chosen, and possible for these boxes and step
// sizes (otherwise form 0 runs, with the same results to rounding).
bool use_rd(const emu_box* b) { return b->step_form == 2 && rd_possible(b) && rd_step_sizes_ok(b); }

// Raises the dynamic shared memory limit of k_rk_deposit (its frame sums)
// once per device; outside any stream capture.
template <bool POT, int R, int STAGE>
int rd_attr(emu_box* b) {
  static std::atomic<unsigned> done{0};
  int dev = 0;
  if (int rc = cuda_check(b, cudaGetDevice(&dev), "get device")) return rc;
  if (dev < 32 && ((done.load() >> dev) & 1u)) return EMU_OK;
  if (int rc = cuda_check(b, cudaFuncSetAttribute(k_rk_deposit<POT, R, STAGE>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kFrameSmem),
                          "set shared memory of the RK-deposit kernel"))
    return rc;
  if (dev < 32) done.fetch_or(1u << dev);
  return EMU_OK;
}

template <bool POT, int R>
int rd_attr_stages(emu_box* b) {
  if (int rc = rd_attr<POT, R, 1>(b)) return rc;
  if (int rc = rd_attr<POT, R, 2>(b)) return rc;
  if (int rc = rd_attr<POT, R, 3>(b)) return rc;
  return rd_attr<POT, R, 4>(b);
}

int rd_prepare(emu_box* b) {
  return by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    if constexpr (R <= 2) {
      if (int rc = rd_attr<false, R, 0>(b)) return rc;
      return b->pot ? rd_attr_stages<true, R>(b) : rd_attr_stages<false, R>(b);
    }
    return fail(b, EMU_EINVAL, "step form 2 covers the shape orders 0-2");
  });
}

template <bool POT, int R>
void launch_rd_stage(emu_box* b, const Batch& Bv, dim3 grid, int s, int dry) {
  auto go = [&](auto kernel) {
    pdl_smem(b->stream, kernel, grid, kFrameSmem, Bv, b->pt, b->W, b->dirtab, b->shift, b->frame, dry, b->partial,
             b->err);
  };
  switch (s) {
    case 1: go(k_rk_deposit<POT, R, 1>); break;
    case 2: go(k_rk_deposit<POT, R, 2>); break;
    case 3: go(k_rk_deposit<POT, R, 3>); break;
    default: go(k_rk_deposit<POT, R, 4>); break;
  }
}

// Stage s (1..4) of form 2 with the deposit of the next stage, or (s = 0)
// the first deposit of a run of steps.
int launch_rd(emu_box* b, int s, int dry) {
  before_launch(b, s == 0 ? CLS_DEPOSIT : CLS_RKDEP);
  const Batch Bv = batch_view(b);
  const dim3 grid = persist_grid(b);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    if constexpr (R <= 2) {
      if (s == 0)
        pdl_smem(b->stream, k_rk_deposit<false, R, 0>, grid, kFrameSmem, Bv, b->pt, b->W, b->dirtab, b->shift,
                 b->frame, 0, b->partial, b->err);
      else if (b->pot)
        launch_rd_stage<true, R>(b, Bv, grid, s, dry);
      else
        launch_rd_stage<false, R>(b, Bv, grid, s, dry);
    }
    return 0;
  });
  return after_launch(b, s == 0 ? "first deposit kernel" : "RK stage and deposit kernel");
}

// The frame sums of every tile (k_frame_sum) from k_rk_deposit's partials.
int launch_combine_frame(emu_box* b) {
  const Batch B = batch_view(b);
  before_launch(b, CLS_COMBINE);
  const int split = combine_split(b->S, B.nw32, true);
  const int64_t n = (int64_t)b->S.NT32 * kSlotF, per_block = (int64_t)(kWarps / split) * kLanes;
  const int64_t blocks = (n + per_block - 1) / per_block;
  pdl(b->stream, k_frame_sum, dim3((unsigned)(blocks < 8 * kPersistBlocks ? blocks : 8 * kPersistBlocks)), B,
      b->partial, b->frame, (int64_t)b->S.NT32, split, b->err);
  return after_launch(b, "frame sum kernel");
}

// One step of form 2: the shift rows (with the next step's first), then four
// (combination, RK stage with the next deposit) pairs; the first step of a
// run deposits its state first.
int launch_step_rd(emu_box* b, int dry, bool first) {
  if (int rc = launch_shifts(b, kStageFrac, 5)) return rc;
  if (first)
    if (int rc = launch_rd(b, 0, 0)) return rc;
  for (int s = 1; s <= 4; ++s) {
    if (int rc = launch_combine_frame(b)) return rc;
    if (int rc = launch_rd(b, s, dry)) return rc;
  }
  return EMU_OK;
}

// One step of every box (first: the first of a run of steps, which form 2
// needs to know).
int launch_step(emu_box* b, int dry, bool first = true) {
  if (b->is3d) return launch3_step(b, dry);
  if (b->general) return launch_gstep(b, dry);
  if (b->step_form == 1) return launch_fused(b, dry, 1);
  if (use_rd(b)) return launch_step_rd(b, dry, first);
  if (int rc = launch_shifts(b, kStageFrac, 4)) return rc;
  for (int s = 1; s <= 4; ++s)
    if (int rc = launch_stage(b, s, dry)) return rc;
  return EMU_OK;
}

// nsteps steps of every box with the step sizes on the device: one step is
// captured as a CUDA graph and replayed (kernels launched directly while
// per-kernel timing is on).  Form 2 replays a graph of its first step (which
// deposits the state first) and then one of the later steps.
int run_steps(emu_box* b, int64_t nsteps) {
  if (nsteps == 0) return EMU_OK;
  const bool rd = use_rd(b);
  if (rd)
    if (int rc = rd_prepare(b)) return rc;
  if (b->prof) {
    for (int64_t n = 0; n < nsteps; ++n)
      if (int rc = launch_step(b, 0, n == 0)) return rc;
    return EMU_OK;
  }
  if (rd != b->graph_rd) {   // the step sizes moved the steps into or out of form 2
    invalidate_graph(b);
    b->graph_rd = rd;
  }
  if (rd) {
    if (!b->graph1)
      if (int rc = capture(b, &b->graph1, &b->graph1_launches, [&] { return launch_step(b, 0, true); })) return rc;
    if (int rc = launch_graph(b, b->graph1, b->graph1_launches)) return rc;
    if (nsteps > 1 && !b->graph)
      if (int rc = capture(b, &b->graph, &b->graph_launches, [&] { return launch_step(b, 0, false); })) return rc;
    for (int64_t n = 1; n < nsteps; ++n)
      if (int rc = launch_graph(b, b->graph, b->graph_launches)) return rc;
    return EMU_OK;
  }
  if (!b->graph)
    if (int rc = capture(b, &b->graph, &b->graph_launches, [&] { return launch_step(b, 0); })) return rc;
  for (int64_t n = 0; n < nsteps; ++n)
    if (int rc = launch_graph(b, b->graph, b->graph_launches)) return rc;
  return EMU_OK;
}

int run_moments(emu_box* b) {
  if (b->is3d) return run3_moments(b);
  if (b->general) {
    if (int rc = launch_gdeposit(b, 1, b->pt.rho, b->pt.rhobar, 0.0, b->mom)) return rc;
    return launch_gdeposit(b, 2, b->pt.rho, b->pt.rhobar, 0.0, b->mom + (size_t)kNA * b->S.NZ);
  }
  const double zero = 0.0;
  if (int rc = launch_shifts(b, &zero, 1)) return rc;
  if (int rc = launch_deposit(b, 1, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom)) return rc;
  return launch_deposit(b, 2, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom + (size_t)kNA * b->S.NZ);
}

int rebuild_dirtable(emu_box* b) {
  if (b->is3d) return rebuild_dirtable3(b);
  const int blocks = (int)((b->S.Ptot + kThreads - 1) / kThreads);
  before_launch(b, CLS_OTHER);
  k_dirtable<<<blocks, kThreads, 0, b->stream>>>(batch_view(b), b->pt, b->dirtab, b->err);
  return after_launch(b, "direction table kernel");
}

int upload_geo(emu_box* b) {
  return cuda_check(b, cudaMemcpyAsync(b->geo_d, b->S.geo.data(), sizeof(BoxGeo) * b->S.nbox,
                                       cudaMemcpyHostToDevice, b->stream), "upload box descriptors");
}

int read_errors(emu_box* b) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_check(b, e, "read error word");
  if (h == 0) return EMU_OK;
  cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
  if (h & ERR_TIMEOUT) {
    // a fused step gave up at a grid barrier: its arrival word is left mid-count
    // and its abort word set; clear both so that the next fused launch runs
    cudaMemsetAsync(b->bar, 0, sizeof(unsigned) * 2, b->stream);
    return fail(b, EMU_ETIMEOUT, "a grid-barrier wait of the fused step gave up after %llu ns; the particle state "
                "is that of an unfinished step", b->limit_ns);
  }
  if (h & ERR_WEIGHT) return fail(b, EMU_EINVAL, "negative particle weight: a flux factor exceeds 1/3");
  if (h & ERR_STEP) return fail(b, EMU_EINVAL, "a ring moved more than one cell between two stages of step form 2");
  if (h & ERR_RING) return fail(b, EMU_ELATTICE, "a ring of particles does not share one direction");
  if (h & ERR_LATTICE) return fail(b, EMU_ELATTICE, "a particle is off its lattice site");
  if (h & ERR_NONFINITE) return fail(b, EMU_ENUMERIC, "non-finite value on the grid");
  return fail(b, EMU_ECUDA, "unknown device error word %d", h);
}

// Eq. 7 for every box from the moments of the current state; leaves the
// results in b->dts (device) and dt_out (host).
int run_timestep(emu_box* b, double* dt_out) {
  if (int rc = run_moments(b)) return rc;
  const Batch B = batch_view(b);
  before_launch(b, CLS_OTHER);
  k_max_diag<<<B.nbox, kThreads, 0, b->stream>>>(B, b->mom, b->nmax);
  if (int rc = after_launch(b, "max kernel")) return rc;
  before_launch(b, CLS_OTHER);
  k_dt_from_max<<<(B.nbox + kThreads - 1) / kThreads, kThreads, 0, b->stream>>>(B, b->nmax, b->dts);
  if (int rc = after_launch(b, "time step kernel")) return rc;
  b->dt_h.assign(b->S.nbox, 0.0);
  if (int rc = copy_out(b, b->dt_h.data(), b->dts, sizeof(double) * b->S.nbox, 1)) return rc;
  b->dt_set = true;
  b->step_dt = b->dt_h;
  b->step_valid = true;
  if (int rc = read_errors(b)) return rc;
  if (dt_out) std::memcpy(dt_out, b->dt_h.data(), sizeof(double) * b->S.nbox);
  return EMU_OK;
}


// ------------------------------------------------------------------ 3D boxes
//
// A 3D box is S's single box with its cells in 3D index order (the time
// step, the diagnostics and the vacuum and matter terms read that
// descriptor), plus one descriptor per cell row, which the deposit
// combination (k_combine) takes as its batch: row r holds cells
// [r nz, (r + 1) nz) and the units of its z tiles.

const char* config3_problem(const emu3_config* c) {
  if (!c) return "config is NULL";
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return "nx, ny and nz must be >= 1";
  if (c->ndir < 1) return "ndir must be >= 1";
  for (double L : {c->Lx, c->Ly, c->Lz})
    if (!(L > 0) || !std::isfinite(L)) return "Lx, Ly and Lz must be positive and finite";
  if (!(c->kappa > 0) || !std::isfinite(c->kappa)) return "kappa must be positive and finite";
  if (!(c->c_light > 0) || !std::isfinite(c->c_light)) return "c_light must be positive and finite";
  if (!(c->cfl_adv > 0) || !(c->cfl_flavor > 0)) return "CFL factors must be positive";
  if (c->shape_order < 0 || c->shape_order > 3) return "shape_order must be 0, 1, 2 or 3";
  if (c->reserved != 0) return "reserved must be 0";
  return nullptr;
}

const char* make_shape3(const emu3_config* c, Shape& S, std::vector<BoxGeo>& rows, int& ntz) {
  if (const char* why = config3_problem(c)) return why;
  const int64_t R = (int64_t)c->nx * c->ny, C = R * c->nz;
  if (R > kMaxBoxes) return "too many cell rows (nx * ny)";
  if (C > INT32_MAX / kNM) return "too many cells";
  if (C * c->ndir > ((int64_t)1 << 40)) return "too many particles";
  S = Shape();
  S.nbox = 1;
  S.order = c->shape_order;
  S.T = tile_cells(S.order);
  ntz = (c->nz + S.T - 1) / S.T;
  const double dx = c->Lx / c->nx, dy = c->Ly / c->ny, dz = c->Lz / c->nz;
  const double dV = dx * dy * dz;
  double hmin = dx;
  if (dy < hmin) hmin = dy;
  if (dz < hmin) hmin = dz;
  BoxGeo g;
  std::memset(&g, 0, sizeof(g));
  g.nz = (int)C;            // the whole box as one list of cells (time step, diagnostics)
  g.M = c->ndir;
  g.ntiles = (int)(R * ntz);
  g.P = C * c->ndir;
  g.Lz = c->Lz;             // rk_particle wraps z with it
  g.dz = hmin;              // Eq. 7 with the smallest cell edge
  g.inv_dz = 1.0 / dz;
  g.nz_d = (double)c->nz;
  g.dV = dV;
  g.c_light = c->c_light;
  g.kappa_dV = c->kappa / dV;
  g.inv_dV = 1.0 / dV;
  g.cfl_adv = c->cfl_adv;
  g.cfl_flavor = c->cfl_flavor;
  g.kappa = c->kappa;
  S.geo.assign(1, g);
  rows.assign((size_t)R, BoxGeo{});
  for (int64_t r = 0; r < R; ++r) {
    BoxGeo& q = rows[(size_t)r];
    std::memset(&q, 0, sizeof(q));
    q.nz = c->nz;
    q.M = c->ndir;
    q.ntiles = ntz;
    q.coff = (int)(r * c->nz);
    q.toff = (int)(r * ntz);
    q.uoff = r * ntz * c->ndir;
    q.kappa_dV = g.kappa_dV;
    q.inv_dV = g.inv_dV;
  }
  S.Ptot = C * c->ndir;
  S.U = R * ntz * c->ndir;
  S.U32 = 0;
  S.NZ = (int)C;
  S.MT = c->ndir;
  S.NT = (int)(R * ntz);
  S.Mmax = c->ndir;
  return nullptr;
}

Layout layout3(const Shape& S, size_t nrows) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t NZ = (size_t)S.NZ, MT = (size_t)S.MT;
  L.geo = take(sizeof(BoxGeo));
  L.dts = take(sizeof(double));
  L.nmax = take(sizeof(double));
  L.A = take(sizeof(double) * kNA * NZ);
  L.At = take(sizeof(double) * kNT * NZ);
  L.mom = take(sizeof(double) * kNM * NZ);
  L.partial = take(sizeof(double) * (size_t)(kMaxWarps + S.NT) * kSlot);
  L.W = take(0);
  L.err = take(sizeof(int));
  L.dirtab = take(sizeof(double) * 6 * MT);
  L.shift = take(sizeof(int) * 12 * MT);
  L.wtab = take(0);
  L.bar = take(sizeof(unsigned) * 2);
  L.species = take(sizeof(double) * 8 * NZ);
  L.dirs = take(sizeof(double) * 3 * MT);
  L.diag = take(sizeof(double) * 63);
  L.scalar = take(sizeof(double) * 4);
  L.rowgeo = take(sizeof(BoxGeo) * nrows);
  L.bw3 = take(sizeof(double) * (size_t)kNC * (size_t)S.Ptot);
  L.gf3 = take(sizeof(double) * (size_t)kNC * (size_t)S.Ptot);
  L.wdir3 = take(sizeof(double) * 4 * 3 * 5 * MT);
  L.total = off;
  return L;
}

Box3 box3_view(const emu_box* b) {
  const emu3_config& c = b->c3;
  Box3 v;
  v.n[0] = c.nx; v.n[1] = c.ny; v.n[2] = c.nz;
  v.M = c.ndir;
  v.R = c.nx * c.ny;
  v.C = v.R * c.nz;
  v.ntz = b->ntz;
  v.T = b->S.T;
  v.nw = batch_view(b).nw;
  v.ntz32 = (c.nz + kLanes - 1) / kLanes;
  v.U32 = (int64_t)v.ntz32 * c.nx * c.ny * c.ndir;
  {
    const int64_t warps = (int64_t)b->blocks * kWarps;
    v.nw32 = (int)(v.U32 < warps ? v.U32 : warps);
  }
  v.use_dirs = b->S.geo[0].use_dirs;
  v.U = b->S.U;
  v.P = b->S.Ptot;
  const double L[3] = {c.Lx, c.Ly, c.Lz};
  for (int a = 0; a < 3; ++a) {
    v.L[a] = L[a];
    v.h[a] = L[a] / v.n[a];
    v.inv_h[a] = 1.0 / v.h[a];
    v.n_d[a] = (double)v.n[a];
  }
  v.kappa_dV = b->S.geo[0].kappa_dV;
  v.inv_dV = b->S.geo[0].inv_dV;
  v.c_light = c.c_light;
  v.alpha = b->S.geo[0].alpha;
  v.seed = b->S.geo[0].seed;
  v.dt = b->dts;
  v.g = b->geo_d;
  return v;
}

// The deposit combination's batch: the box's cell rows.
Batch row_view(const emu_box* b) {
  Batch B = batch_view(b);
  B.box = b->rows_d;
  B.nbox = (int)b->rows.size();
  return B;
}

// The lattice shifts of nrows position offsets and the directions' weights there.
int launch3_shifts(emu_box* b, const double* fracs, int nrows) {
  Fracs f{};
  for (int s = 0; s < nrows; ++s) f.v[s] = fracs[s];
  double* wtab = (double*)(b->ws + b->L.wdir3);
  before_launch(b, CLS_SHIFT);
  by_order(b->S.order, [&](auto O) {
    pdl(b->stream, k3_shifts<decltype(O)::value>, dim3((unsigned)((b->c3.ndir + kThreads - 1) / kThreads)),
        box3_view(b), b->x3, b->y3, b->pt.z, b->dirtab, f, nrows, b->shift, wtab);
    return 0;
  });
  return after_launch(b, "3D shift kernel");
}

// The stage's rows of the direction weight table (k3_shifts).
const double* wrow3(const emu_box* b, int s) {
  return (const double*)(b->ws + b->L.wdir3) + (size_t)(s - 1) * 3 * 5 * b->S.MT;
}

// One separable pass (k3_pass) over every (direction, cell).
template <int AXIS, bool SPREAD>
int launch3_pass(emu_box* b, const double* in, const double* wrow, double* out) {
  before_launch(b, CLS_OTHER);
  by_order(b->S.order, [&](auto O) {
    pdl(b->stream, k3_pass<decltype(O)::value, AXIS, SPREAD>, dim3((unsigned)((b->S.Ptot + kThreads - 1) / kThreads)),
        box3_view(b), in, wrow, out);
    return 0;
  });
  return after_launch(b, "3D separable pass kernel");
}

// Deposit of the state (rnu, rnb) at positions x + frac dt c Omega with the
// shift rows srow ([3][M]) into out; modes as k3_deposit (0, 1, 2, 4).
int launch3_deposit(emu_box* b, int mode, const double* rnu, const double* rnb, const int* srow, double frac,
                    double* out) {
  const Box3 v = box3_view(b);
  const dim3 grid = persist_grid(b);
  cudaStream_t st = b->stream;
  const double *x = b->x3, *y = b->y3, *z = b->pt.z, *N = b->pt.N, *Nb = b->pt.Nbar;
  before_launch(b, CLS_DEPOSIT);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    if (mode == 0)
      pdl(st, k3_deposit<0, R>, grid, v, x, y, z, N, Nb, rnu, rnb, b->dirtab, srow, frac, b->partial, b->err);
    else if (mode == 1)
      pdl(st, k3_deposit<1, R>, grid, v, x, y, z, N, Nb, rnu, rnb, b->dirtab, srow, frac, b->partial, b->err);
    else if (mode == 2)
      pdl(st, k3_deposit<2, R>, grid, v, x, y, z, N, Nb, rnu, rnb, b->dirtab, srow, frac, b->partial, b->err);
    else
      pdl(st, k3_deposit<4, R>, grid, v, x, y, z, N, Nb, rnu, rnb, b->dirtab, srow, frac, b->partial, b->err);
    return 0;
  });
  if (int rc = after_launch(b, "3D deposit kernel")) return rc;
  const Batch B = row_view(b);
  const int split = combine_split(b->S, B.nw);
  const int rows = kNA;
  const int potential = mode == 0 ? 1 : 0;
  before_launch(b, CLS_COMBINE);
  pdl(st, k_combine, dim3(combine_blocks(rows, B.NZ, split)), B, b->partial, out, rows, potential, split, b->err);
  return after_launch(b, "deposit combine kernel");
}

// The RK stage of stage s: G = A0 - Omega . A of every (direction, cell)
// (k3_gfield), interpolated along x and y (k3_pass), then k3_rk_stage
// (along z, commutators, RK update).
int launch3_rk(emu_box* b, int s, const int* srow, int dry) {
  const Box3 v = box3_view(b);
  double* F0 = (double*)(b->ws + b->L.bw3);
  double* F1 = (double*)(b->ws + b->L.gf3);
  const double* wrow = wrow3(b, s);
  before_launch(b, CLS_OTHER);
  pdl(b->stream, k3_gfield, dim3((unsigned)((b->S.Ptot + kThreads - 1) / kThreads)), v, (const double*)b->At,
      (const double*)b->dirtab, F1);
  if (int rc = after_launch(b, "3D G field kernel")) return rc;
  if (int rc = launch3_pass<0, false>(b, F1, wrow, F0)) return rc;
  if (int rc = launch3_pass<1, false>(b, F0, wrow, F1)) return rc;
  before_launch(b, CLS_RK);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    if (b->pot)
      pdl(b->stream, k3_rk_stage<true, R>, persist_grid(b), v, b->pt, b->x3, b->y3, b->dirtab, srow,
          (const double*)F1, wrow, s, dry);
    else
      pdl(b->stream, k3_rk_stage<false, R>, persist_grid(b), v, b->pt, b->x3, b->y3, b->dirtab, srow,
          (const double*)F1, wrow, s, dry);
    return 0;
  });
  return after_launch(b, "3D RK stage kernel");
}

// The step's deposit of stage s, separable: every particle's B at its cell
// (k3_prep, with the lattice check), spread along z and y (k3_pass), then
// along x and summed over directions into the traceless potential At
// (k3_spread_x_sum).
int launch3_step_deposit(emu_box* b, int s, const int* srow) {
  const size_t P = (size_t)b->S.Ptot;
  const double* rnu = (s == 1) ? b->pt.rho : b->pt.stage;
  const double* rnb = (s == 1) ? b->pt.rhobar : b->pt.stage + 9 * P;
  double* F0 = (double*)(b->ws + b->L.bw3);
  double* F1 = (double*)(b->ws + b->L.gf3);
  const double* wrow = wrow3(b, s);
  const Box3 v = box3_view(b);
  before_launch(b, CLS_OTHER);
  pdl(b->stream, k3_prep, dim3((unsigned)((P + kThreads - 1) / kThreads)), v, (const double*)b->x3,
      (const double*)b->y3, (const double*)b->pt.z, (const double*)b->pt.N, (const double*)b->pt.Nbar, rnu, rnb,
      (const double*)b->dirtab, srow, kStageFrac[s - 1], F0, b->err);
  if (int rc = after_launch(b, "3D prep kernel")) return rc;
  if (int rc = launch3_pass<2, true>(b, F0, wrow, F1)) return rc;
  if (int rc = launch3_pass<1, true>(b, F1, wrow, F0)) return rc;
  before_launch(b, CLS_DEPOSIT);
  by_order(b->S.order, [&](auto O) {
    pdl(b->stream, k3_spread_x_sum<decltype(O)::value>, dim3((unsigned)((v.C + kThreads - 1) / kThreads)), v,
        (const double*)F0, wrow, (const double*)b->dirtab, b->At, b->err);
    return 0;
  });
  return after_launch(b, "3D deposit sum kernel");
}

int launch3_stage(emu_box* b, int s, int dry) {
  const int* srow = b->shift + (size_t)(s - 1) * 3 * b->S.MT;
  if (int rc = launch3_step_deposit(b, s, srow)) return rc;
  return launch3_rk(b, s, srow, dry);
}

int launch3_step(emu_box* b, int dry) {
  if (int rc = launch3_shifts(b, kStageFrac, 4)) return rc;
  for (int s = 1; s <= 4; ++s)
    if (int rc = launch3_stage(b, s, dry)) return rc;
  return EMU_OK;
}

int run3_moments(emu_box* b) {
  const double zero = 0.0;
  if (int rc = launch3_shifts(b, &zero, 1)) return rc;
  if (int rc = launch3_deposit(b, 1, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom)) return rc;
  return launch3_deposit(b, 2, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom + (size_t)kNA * b->S.NZ);
}

int rebuild_dirtable3(emu_box* b) {
  before_launch(b, CLS_OTHER);
  k3_dirtable<<<(unsigned)((b->S.Ptot + kThreads - 1) / kThreads), kThreads, 0, b->stream>>>(box3_view(b), b->pt,
                                                                                               b->dirtab, b->err);
  return after_launch(b, "3D direction table kernel");
}

int no_3d(emu_box* b, const char* what) {
  return fail(b, EMU_EINVAL, "%s is not available for a 3D box", what);
}


// ------------------------------------------------- particles anywhere (1D)
//
// The path of kernels_general.cuh: per stage, sort the particles by the cell
// containing their stage position (stable radix sort), deposit with one warp
// per cell in sorted order, then one thread per particle for the RK stage.

// Stable sort of the particles by containing cell at z + frac dt c Omega_z;
// leaves the cell starts in b->gstart and returns the sorted particle ids.
int gsort(emu_box* b, double frac, const int** ids_out) {
  const Batch B = batch_view(b);
  const int64_t P = b->S.Ptot;
  unsigned* k0 = (unsigned*)(b->ws + b->L.gkeys);
  unsigned* k1 = (unsigned*)(b->ws + b->L.gkeys2);
  int* v0 = (int*)(b->ws + b->L.gids);
  int* v1 = (int*)(b->ws + b->L.gids2);
  int* hist = (int*)(b->ws + b->L.ghist);
  int* start = (int*)(b->ws + b->L.gstart);
  const unsigned pblocks = (unsigned)((P + kThreads - 1) / kThreads);
  before_launch(b, CLS_OTHER);
  pdl(b->stream, k_gkeys, dim3(pblocks), B, b->pt.z, b->pt.oz, frac, k0, v0, b->err);
  if (int rc = after_launch(b, "sort key kernel")) return rc;
  int bits = 0;
  while (bits < 31 && (int64_t(1) << bits) < (int64_t)b->S.NZ) ++bits;
  const int nblk = (int)((P + kRadixTile - 1) / kRadixTile);
  for (int shift = 0; shift < bits; shift += kRadixBits) {
    before_launch(b, CLS_OTHER);
    k_radix_hist<<<nblk, kThreads, 0, b->stream>>>(k0, P, shift, hist, nblk);
    if (int rc = after_launch(b, "radix histogram kernel")) return rc;
    before_launch(b, CLS_OTHER);
    k_scan_exclusive<<<1, kThreads, 0, b->stream>>>(hist, (int64_t)kRadixBuckets * nblk);
    if (int rc = after_launch(b, "radix scan kernel")) return rc;
    before_launch(b, CLS_OTHER);
    k_radix_scatter<<<nblk, kThreads, 0, b->stream>>>(k0, v0, P, shift, hist, nblk, k1, v1);
    if (int rc = after_launch(b, "radix scatter kernel")) return rc;
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  before_launch(b, CLS_OTHER);
  k_cell_start<<<(unsigned)((P + 1 + kThreads - 1) / kThreads), kThreads, 0, b->stream>>>(k0, P, b->S.NZ, start);
  if (int rc = after_launch(b, "cell start kernel")) return rc;
  *ids_out = v0;
  return EMU_OK;
}

// Deposit of particles anywhere (modes as k_deposit) into out.
int launch_gdeposit(emu_box* b, int mode, const double* rnu, const double* rnb, double frac, double* out) {
  const int* ids = nullptr;
  if (int rc = gsort(b, frac, &ids)) return rc;
  const Batch B = batch_view(b);
  const int* start = (const int*)(b->ws + b->L.gstart);
  const int64_t wb = ((int64_t)B.NZ + kWarps - 1) / kWarps;
  const dim3 grid((unsigned)(wb < 8 * kPersistBlocks ? wb : 8 * kPersistBlocks));
  before_launch(b, CLS_DEPOSIT);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    cudaStream_t st = b->stream;
    if (mode == 0) pdl(st, k_gdeposit<0, R>, grid, B, b->pt, rnu, rnb, frac, ids, start, out, b->err);
    else if (mode == 1) pdl(st, k_gdeposit<1, R>, grid, B, b->pt, rnu, rnb, frac, ids, start, out, b->err);
    else if (mode == 2) pdl(st, k_gdeposit<2, R>, grid, B, b->pt, rnu, rnb, frac, ids, start, out, b->err);
    else if (mode == 4) pdl(st, k_gdeposit<4, R>, grid, B, b->pt, rnu, rnb, frac, ids, start, out, b->err);
    else pdl(st, k_gdeposit<5, R>, grid, B, b->pt, rnu, rnb, frac, ids, start, out, b->err);
    return 0;
  });
  return after_launch(b, "deposit kernel (particles anywhere)");
}

// The step's deposit of particles anywhere: sort, every particle's weights,
// B and direction in sorted order (k_gprep; the weights in the lattice path's
// weight buffer, unused here), then the deposit from them (k_gdeposit_sorted).
int launch_gstep_deposit(emu_box* b, const double* rnu, const double* rnb, double frac) {
  const int* ids = nullptr;
  if (int rc = gsort(b, frac, &ids)) return rc;
  const Batch B = batch_view(b);
  const int64_t P = b->S.Ptot;
  const int* start = (const int*)(b->ws + b->L.gstart);
  double* Bs = (double*)(b->ws + b->L.gprep);
  double* Os = Bs + (size_t)kNC * P;
  before_launch(b, CLS_OTHER);
  by_order(b->S.order, [&](auto O) {
    pdl(b->stream, k_gprep<decltype(O)::value>, dim3((unsigned)((P + kThreads - 1) / kThreads)), B, b->pt, rnu, rnb,
        frac, ids, b->W, Bs, Os, b->err);
    return 0;
  });
  if (int rc = after_launch(b, "deposit prep kernel (particles anywhere)")) return rc;
  const int64_t groups = kWarps / kGSplit, nb = ((int64_t)B.NZ + groups - 1) / groups;
  before_launch(b, CLS_DEPOSIT);
  by_order(b->S.order, [&](auto O) {
    pdl(b->stream, k_gdeposit_sorted<decltype(O)::value>,
        dim3((unsigned)(nb < 8 * kPersistBlocks ? nb : 8 * kPersistBlocks)), B, (const double*)b->W,
        (const double*)Bs, (const double*)Os, start, b->At, b->err);
    return 0;
  });
  return after_launch(b, "deposit kernel (particles anywhere)");
}

int launch_gstage(emu_box* b, int s, int dry) {
  const size_t P = (size_t)b->S.Ptot;
  const double* rnu = (s == 1) ? b->pt.rho : b->pt.stage;
  const double* rnb = (s == 1) ? b->pt.rhobar : b->pt.stage + 9 * P;
  if (int rc = launch_gstep_deposit(b, rnu, rnb, kStageFrac[s - 1])) return rc;
  before_launch(b, CLS_RK);
  by_order(b->S.order, [&](auto O) {
    constexpr int R = decltype(O)::value;
    const dim3 grid((unsigned)((P + kThreads - 1) / kThreads));
    if (b->pot) pdl(b->stream, k_grk_stage<true, R>, grid, batch_view(b), b->pt, (const double*)b->At, s, dry);
    else pdl(b->stream, k_grk_stage<false, R>, grid, batch_view(b), b->pt, (const double*)b->At, s, dry);
    return 0;
  });
  return after_launch(b, "RK stage kernel (particles anywhere)");
}

int launch_gstep(emu_box* b, int dry) {
  for (int s = 1; s <= 4; ++s)
    if (int rc = launch_gstage(b, s, dry)) return rc;
  return EMU_OK;
}

// Does every particle keep the lattice contract?  (Synchronises.)  Returns
// EMU_OK and sets *on_lattice.
int check_lattice(emu_box* b, bool* on_lattice) {
  int* flag = (int*)(b->ws + b->L.gflag);
  if (int rc = cuda_check(b, cudaMemsetAsync(flag, 0, sizeof(int), b->stream), "clear lattice flag")) return rc;
  before_launch(b, CLS_OTHER);
  k_lattice_check<<<(unsigned)((b->S.Ptot + kThreads - 1) / kThreads), kThreads, 0, b->stream>>>(batch_view(b),
                                                                                                 b->pt, flag);
  if (int rc = after_launch(b, "lattice check kernel")) return rc;
  int h = 0;
  if (int rc = cuda_check(b, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
                          "read lattice flag"))
    return rc;
  if (int rc = cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise after lattice check")) return rc;
  *on_lattice = h == 0;
  return EMU_OK;
}

// Chooses the path after particles were installed (layout -1: by the check).
int choose_layout(emu_box* b) {
  bool general = b->layout == 1;
  if (b->layout == -1) {
    bool on = true;
    if (int rc = check_lattice(b, &on)) return rc;
    general = !on;
  }
  if (general != b->general) invalidate_graph(b);
  b->general = general;
  return EMU_OK;
}

int needs_lattice(emu_box* b, const char* what) {
  return fail(b, EMU_EINVAL, "%s needs the particles on their lattice sites (emu_set_layout)", what);
}

int bind_common(emu_box* b, const emu_particles* parts, void* workspace, int64_t workspace_bytes, void* stream);

int create_common(const emu_config* cfgs, int nbox, emu_box** out) {
  if (!out) return fail(nullptr, EMU_EINVAL, "out is NULL");
  *out = nullptr;
  Shape S;
  if (const char* why = make_shape(cfgs, nbox, S)) return fail(nullptr, EMU_EINVAL, "%s", why);
  emu_box* b = new (std::nothrow) emu_box();
  if (!b) return fail(nullptr, EMU_EINVAL, "host allocation failed");
  b->S = std::move(S);
  b->L = layout(b->S);
  b->cfg.assign(cfgs, cfgs + nbox);
  *out = b;
  return EMU_OK;
}

int init_common(emu_box* b, const double* n_nu, const double* n_nubar, const double* f_nu, const double* f_nubar,
                const double* dirs, const double* alpha, const uint64_t* seed) {
  if (!n_nu || !n_nubar || !f_nu || !f_nubar || !alpha || !seed)
    return fail(b, EMU_EINVAL, "species arrays must not be NULL");
  const Shape& S = b->S;
  // per box: n_nu[nz], n_nubar[nz], f_nu[3 nz], f_nubar[3 nz] at 8 * coff
  std::vector<double> sp((size_t)8 * S.NZ);
  for (int i = 0; i < S.nbox; ++i) {
    BoxGeo& g = b->S.geo[i];
    const size_t nz = (size_t)g.nz, c = (size_t)g.coff;
    double* dst = sp.data() + 8 * c;
    std::memcpy(dst, n_nu + c, sizeof(double) * nz);
    std::memcpy(dst + nz, n_nubar + c, sizeof(double) * nz);
    std::memcpy(dst + 2 * nz, f_nu + 3 * c, sizeof(double) * 3 * nz);
    std::memcpy(dst + 5 * nz, f_nubar + 3 * c, sizeof(double) * 3 * nz);
    g.use_dirs = dirs ? 1 : 0;
    g.alpha = alpha[i];
    g.seed = seed[i];
  }
  cudaStream_t st = b->stream;
  if (int rc = upload_geo(b)) return rc;
  if (int rc = cuda_check(b, cudaMemcpyAsync(b->species, sp.data(), sizeof(double) * sp.size(),
                                             cudaMemcpyHostToDevice, st), "copy species"))
    return rc;
  if (dirs)
    if (int rc = cuda_check(b, cudaMemcpyAsync(b->dirs, dirs, sizeof(double) * 3 * (size_t)S.MT,
                                               cudaMemcpyHostToDevice, st), "copy directions"))
      return rc;
  const int blocks = (int)((S.Ptot + kThreads - 1) / kThreads);
  before_launch(b, CLS_OTHER);
  k_init<<<blocks, kThreads, 0, st>>>(batch_view(b), b->pt, b->species, b->dirs, b->err);
  if (int rc = after_launch(b, "init kernel")) return rc;
  if (int rc = rebuild_dirtable(b)) return rc;
  b->next_stage = 1;
  if ((b->layout == 1) != b->general) invalidate_graph(b);
  b->general = b->layout == 1;   // initial particles sit on their lattice sites
  return read_errors(b);  // synchronises: the host staging vector may go
}

}  // namespace

// --------------------------------------------------------------------- C ABI

extern "C" {

int64_t emu_workspace_bytes(const emu_config* cfg) { return emu_batch_workspace_bytes(cfg, 1); }

int64_t emu_batch_workspace_bytes(const emu_config* cfgs, int32_t nbox) {
  Shape S;
  if (make_shape(cfgs, nbox, S)) return EMU_EINVAL;
  return (int64_t)layout(S).total;
}

int64_t emu_batch_particles(const emu_config* cfgs, int32_t nbox) {
  Shape S;
  if (make_shape(cfgs, nbox, S)) return EMU_EINVAL;
  return S.Ptot;
}

int64_t emu_batch_cells(const emu_config* cfgs, int32_t nbox) {
  Shape S;
  if (make_shape(cfgs, nbox, S)) return EMU_EINVAL;
  return S.NZ;
}

int emu_create(const emu_config* cfg, emu_box** out) { return create_common(cfg, 1, out); }

int emu_batch_create(const emu_config* cfgs, int32_t nbox, emu_box** out) { return create_common(cfgs, nbox, out); }

int emu_bind(emu_box* b, const emu_particles* parts, void* workspace, int64_t workspace_bytes, void* stream) {
  if (!b) return EMU_EINVAL;
  if (b->is3d) return fail(b, EMU_EINVAL, "a 3D box is bound with emu3_bind");
  return bind_common(b, parts, workspace, workspace_bytes, stream);
}

}  // extern "C"

namespace {
int bind_common(emu_box* b, const emu_particles* parts, void* workspace, int64_t workspace_bytes, void* stream) {
  if (!parts || !workspace) return fail(b, EMU_EINVAL, "particles or workspace is NULL");
  if (parts->P != b->S.Ptot)
    return fail(b, EMU_EINVAL, "parts->P = %lld, expected %lld particles", (long long)parts->P,
                (long long)b->S.Ptot);
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
  b->geo_d = (BoxGeo*)(b->ws + L.geo);
  b->dts = (double*)(b->ws + L.dts);
  b->nmax = (double*)(b->ws + L.nmax);
  b->A = (double*)(b->ws + L.A);
  b->At = (double*)(b->ws + L.At);
  b->mom = (double*)(b->ws + L.mom);
  b->partial = (double*)(b->ws + L.partial);
  b->W = (double*)(b->ws + L.W);
  b->frame = (double*)(b->ws + L.frame);
  b->err = (int*)(b->ws + L.err);
  b->dirtab = (double*)(b->ws + L.dirtab);
  b->shift = (int*)(b->ws + L.shift);
  b->wtab = (double*)(b->ws + L.wtab);
  b->bar = (unsigned*)(b->ws + L.bar);
  b->rows_d = b->is3d ? (BoxGeo*)(b->ws + L.rowgeo) : nullptr;
  b->species = (double*)(b->ws + L.species);
  b->dirs = (double*)(b->ws + L.dirs);
  b->diag = (double*)(b->ws + L.diag);
  b->scalar = (double*)(b->ws + L.scalar);
  invalidate_graph(b);
  if (int rc = cuda_check(b, cudaMemsetAsync(workspace, 0, L.total, b->stream), "clear workspace")) return rc;
  if (int rc = upload_geo(b)) return rc;
  if (b->is3d)
    if (int rc = cuda_check(b, cudaMemcpyAsync(b->rows_d, b->rows.data(), sizeof(BoxGeo) * b->rows.size(),
                                               cudaMemcpyHostToDevice, b->stream), "upload row descriptors"))
      return rc;
  b->dt_set = false;
  b->step_valid = false;
  b->bound = true;
  b->next_stage = 1;
  return EMU_OK;
}
}  // namespace

extern "C" {

int emu_init_particles(emu_box* b, const double* n_nu, const double* n_nubar, const double* f_nu,
                       const double* f_nubar, const double* dirs, double alpha, uint64_t seed) {
  if (int rc = check_single(b)) return rc;
  if (b->is3d) return fail(b, EMU_EINVAL, "a 3D box is initialised with emu3_init_particles");
  return init_common(b, n_nu, n_nubar, f_nu, f_nubar, dirs, &alpha, &seed);
}

int emu_batch_init_particles(emu_box* b, const double* n_nu, const double* n_nubar, const double* f_nu,
                             const double* f_nubar, const double* dirs, const double* alpha, const uint64_t* seed) {
  if (int rc = check_bound(b)) return rc;
  if (b->is3d) return fail(b, EMU_EINVAL, "a 3D box is initialised with emu3_init_particles");
  return init_common(b, n_nu, n_nubar, f_nu, f_nubar, dirs, alpha, seed);
}

int emu_set_particles(emu_box* b, const double* z, const double* ox, const double* oy, const double* oz,
                      const double* N, const double* Nbar, const double* rho, const double* rhobar, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (on_host < 0 || on_host > 2) return fail(b, EMU_EINVAL, "on_host must be 0, 1 or 2");
  const size_t P = (size_t)b->S.Ptot;
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
  // the layout is checked when positions come from host memory or directions
  // change; a device-to-device copy of positions alone (a checkpoint of this
  // box restored) keeps the layout in use
  if (!b->is3d && ((z && on_host) || ox || oy || oz))
    if (int rc = choose_layout(b)) return rc;
  if ((ox || oy || oz) && !b->general)
    if (int rc = rebuild_dirtable(b)) return rc;
  if (on_host == 1) return cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise after copy in");
  return EMU_OK;   // (on_host = 2: the copies stay in flight on the stream)
}

int emu_get_particles(emu_box* b, double* z, double* ox, double* oy, double* oz, double* N, double* Nbar,
                      double* rho, double* rhobar, int on_host) {
  if (int rc = check_bound(b)) return rc;
  const size_t P = (size_t)b->S.Ptot;
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
  if (int rc = check_single(b)) return rc;
  if (src != 0 && src != 1) return fail(b, EMU_EINVAL, "src must be 0 (rho) or 1 (stage buffer)");
  if (!std::isfinite(pos_dt)) return fail(b, EMU_EINVAL, "pos_dt must be finite");
  if (int rc = set_dts(b, &pos_dt)) return rc;
  const double one = 1.0;
  const size_t P = (size_t)b->S.Ptot;
  const double* rnu = src ? b->pt.stage : b->pt.rho;
  const double* rnb = src ? b->pt.stage + 9 * P : b->pt.rhobar;
  if (b->is3d) {
    if (int rc = launch3_shifts(b, &one, 1)) return rc;
    if (int rc = launch3_deposit(b, 0, rnu, rnb, b->shift, 1.0, b->A)) return rc;
  } else if (b->general) {
    if (int rc = launch_gdeposit(b, 0, rnu, rnb, 1.0, b->A)) return rc;
  } else {
    if (int rc = launch_shifts(b, &one, 1)) return rc;
    if (int rc = launch_deposit(b, 0, rnu, rnb, b->shift, 1.0, b->A)) return rc;
  }
  b->next_stage = 1;
  if (A_out) return copy_out(b, A_out, b->A, sizeof(double) * kNA * b->S.NZ, on_host);
  return EMU_OK;
}

int emu_interpolate_H(emu_box* b, double pos_dt, double* H_out, int on_host) {
  if (int rc = check_single(b)) return rc;
  if (!H_out) return fail(b, EMU_EINVAL, "H_out is NULL");
  if (!std::isfinite(pos_dt)) return fail(b, EMU_EINVAL, "pos_dt must be finite");
  if (int rc = set_dts(b, &pos_dt)) return rc;
  const double one = 1.0;
  if (!b->general)
    if (int rc = b->is3d ? launch3_shifts(b, &one, 1) : launch_shifts(b, &one, 1)) return rc;
  double* dst = H_out;
  if (on_host) dst = b->pt.acc;  // staging: the RK scratch holds 18 P doubles
  before_launch(b, CLS_OTHER);
  by_order(b->S.order, [&](auto O) {
    if (b->general)
      k_ginterpolate<decltype(O)::value><<<(unsigned)((b->S.Ptot + kThreads - 1) / kThreads), kThreads, 0,
                                           b->stream>>>(batch_view(b), b->pt, b->A, 1.0, dst);
    else if (b->is3d)
      k3_interpolate<decltype(O)::value><<<persist_grid(b), kThreads, 0, b->stream>>>(
          box3_view(b), b->x3, b->y3, b->pt.z, b->dirtab, b->shift, b->A, 1.0, dst, b->err);
    else
      k_interpolate<decltype(O)::value><<<persist_grid(b), kThreads, 0, b->stream>>>(
          batch_view(b), b->pt.z, b->dirtab, b->shift, b->A, 1.0, dst, b->err);
    return 0;
  });
  if (int rc = after_launch(b, "interpolation kernel")) return rc;
  b->next_stage = 1;  // the staging above may overwrite the RK scratch
  if (on_host) return copy_out(b, H_out, dst, sizeof(double) * 9 * (size_t)b->S.Ptot, 1);
  return EMU_OK;
}

int emu_rk_stage(emu_box* b, int s, double dt) {
  if (int rc = check_single(b)) return rc;
  if (s < 1 || s > 4) return fail(b, EMU_EINVAL, "stage must be 1..4");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(b, EMU_EINVAL, "dt must be positive and finite");
  if (s != b->next_stage) return fail(b, EMU_EINVAL, "stage %d called, expected stage %d", s, b->next_stage);
  if (s > 1 && dt != b->dt_h[0]) return fail(b, EMU_EINVAL, "dt changed within a step");
  if (s == 1) {
    if (int rc = set_dts(b, &dt)) return rc;
    if (!b->general)
      if (int rc = b->is3d ? launch3_shifts(b, kStageFrac, 4) : launch_shifts(b, kStageFrac, 4)) return rc;
  }
  if (int rc = b->general ? launch_gstage(b, s, 0) : b->is3d ? launch3_stage(b, s, 0) : launch_stage(b, s, 0))
    return rc;
  b->next_stage = s == 4 ? 1 : s + 1;
  return EMU_OK;
}

int emu_timestep(emu_box* b, double* dt_out) {
  if (int rc = check_single(b)) return rc;
  if (!dt_out) return fail(b, EMU_EINVAL, "dt_out is NULL");
  return run_timestep(b, dt_out);
}

int emu_step(emu_box* b, int64_t nsteps, double dt) {
  if (int rc = check_single(b)) return rc;
  if (nsteps < 0) return fail(b, EMU_EINVAL, "nsteps must be >= 0");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  if (!(dt > 0)) {
    if (!b->step_valid)
      if (int rc = run_timestep(b, nullptr)) return rc;
    dt = b->step_dt[0];
  }
  if (!std::isfinite(dt)) return fail(b, EMU_EINVAL, "dt must be positive and finite");
  if (int rc = set_dts(b, &dt)) return rc;
  return run_steps(b, nsteps);
}

int emu_batch_timestep(emu_box* b, double* dt_out) {
  if (int rc = check_bound(b)) return rc;
  return run_timestep(b, dt_out);
}

int emu_batch_set_dt(emu_box* b, const double* dt) {
  if (int rc = check_bound(b)) return rc;
  if (!dt) return fail(b, EMU_EINVAL, "dt is NULL");
  for (int i = 0; i < b->S.nbox; ++i)
    if (!(dt[i] > 0) || !std::isfinite(dt[i])) return fail(b, EMU_EINVAL, "dt[%d] must be positive and finite", i);
  b->step_dt.assign(dt, dt + b->S.nbox);
  b->step_valid = true;
  return set_dts(b, dt);
}

int emu_batch_step(emu_box* b, int64_t nsteps) {
  if (int rc = check_bound(b)) return rc;
  if (nsteps < 0) return fail(b, EMU_EINVAL, "nsteps must be >= 0");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  if (!b->step_valid)
    if (int rc = run_timestep(b, nullptr)) return rc;
  if (int rc = set_dts(b, b->step_dt.data())) return rc;
  return run_steps(b, nsteps);
}

int emu_moments(emu_box* b, double* out, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (!out) return fail(b, EMU_EINVAL, "out is NULL");
  if (int rc = run_moments(b)) return rc;
  return copy_out(b, out, b->mom, sizeof(double) * kNM * b->S.NZ, on_host);
}

int emu_batch_diagnostics(emu_box* b, double* out, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (!out) return fail(b, EMU_EINVAL, "out is NULL");
  // the diagnostics read n, f_x, nbar, fbar_x: one deposit pass of both species
  const double zero = 0.0;
  if (b->is3d) {
    if (int rc = launch3_shifts(b, &zero, 1)) return rc;
    if (int rc = launch3_deposit(b, 4, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom)) return rc;
  } else if (b->general) {
    if (int rc = launch_gdeposit(b, 4, b->pt.rho, b->pt.rhobar, 0.0, b->mom)) return rc;
  } else {
    if (int rc = launch_shifts(b, &zero, 1)) return rc;
    if (int rc = launch_deposit(b, 4, b->pt.rho, b->pt.rhobar, b->shift, 0.0, b->mom)) return rc;
  }
  before_launch(b, CLS_OTHER);
  k_diagnostics<<<dim3((unsigned)b->S.nbox, 63), kThreads, 0, b->stream>>>(batch_view(b), b->mom, b->diag);
  if (int rc = after_launch(b, "diagnostics kernel")) return rc;
  return copy_out(b, out, b->diag, sizeof(double) * 63 * b->S.nbox, on_host);
}

int emu_diagnostics(emu_box* b, double* out, int on_host) {
  if (int rc = check_single(b)) return rc;
  return emu_batch_diagnostics(b, out, on_host);
}

int emu_set_grid(emu_box* b, int32_t blocks) {
  if (int rc = check_bound(b)) return rc;
  if (blocks < 1 || blocks > kMaxBlocks) return fail(b, EMU_EINVAL, "blocks must be in 1..%d", kMaxBlocks);
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  b->blocks = blocks;
  b->rk_form = -1;
  if (b->step_form == 1 && blocks > fused_max_blocks(b)) b->step_form = 0;   // cannot be all resident
  invalidate_graph(b);
  return EMU_OK;
}

int emu_set_rk_form(emu_box* b, int32_t form) {
  if (int rc = check_bound(b)) return rc;
  if (form < -1 || form > 1) return fail(b, EMU_EINVAL, "form must be -1, 0 or 1");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  b->rk_form = form;
  invalidate_graph(b);
  return EMU_OK;
}

int emu_set_deposit_form(emu_box* b, int32_t form) {
  if (int rc = check_bound(b)) return rc;
  if (form < 0 || form > 2) return fail(b, EMU_EINVAL, "form must be 0, 1 or 2");
  if (form != 0 && b->is3d) return no_3d(b, "the cluster deposit");
  if (form != 0 && b->general) return needs_lattice(b, "the cluster deposit");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  if (form != 0 && dep_cluster_capacity(b, form) <= 0)
    return fail(b, EMU_EINVAL, "the device cannot run clusters of %d blocks for the deposit", dep_cluster_size(form));
  b->dep_form = form;
  invalidate_graph(b);
  return EMU_OK;
}

int emu_autotune(emu_box* b, int trial_steps, int32_t* choice_out, double* ms_out) {
  if (int rc = check_bound(b)) return rc;
  if (trial_steps < 1) return fail(b, EMU_EINVAL, "trial_steps must be >= 1");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  if (!b->step_valid)
    if (int rc = run_timestep(b, nullptr)) return rc;
  if (int rc = set_dts(b, b->step_dt.data())) return rc;
  // candidate c: step form, grid and RK form (see emu.h)
  const int grids[EMU_AUTOTUNE_CANDIDATES] = {kPersistBlocks, kPersistBlocks, kPersistBlocks / 2, kPersistBlocks / 2,
                                              kMaxBlocks, kMaxBlocks, kPersistBlocks, kPersistBlocks,
                                              kPersistBlocks / 2, kPersistBlocks / 2, kPersistBlocks,
                                              kPersistBlocks / 2, kMaxBlocks, kPersistBlocks, kPersistBlocks,
                                              kPersistBlocks, kPersistBlocks};
  auto apply = [&](int c) {
    b->blocks = grids[c];
    b->rk_form = c < 10 || c >= 13 ? c % 2 : -1;
    b->step_form = c >= 13 ? 0 : c >= 10 ? 2 : c >= 6 ? 1 : 0;
    b->dep_form = c >= 15 ? 2 : c >= 13 ? 1 : 0;
  };
  const bool dep_ok[2] = {!b->is3d && !b->general && dep_cluster_capacity(b, 1) > 0,
                          !b->is3d && !b->general && dep_cluster_capacity(b, 2) > 0};
  const int maxb = fused_max_blocks(b);
  const bool rd_ok = rd_possible(b) && rd_step_sizes_ok(b);
  if (rd_ok)
    if (int rc = rd_prepare(b)) return rc;
  const bool prof = b->prof;
  b->prof = false;
  cudaEvent_t e0 = take_event(b), e1 = take_event(b);
  int best = 0;
  float best_ms = 0.f;
  int rc = EMU_OK;
  for (int c = 0; c < EMU_AUTOTUNE_CANDIDATES && rc == EMU_OK; ++c) {
    apply(c);
    if ((b->step_form == 1 && (b->is3d || b->general || b->blocks > maxb)) ||
        (b->step_form == 2 && !rd_ok) || (b->dep_form != 0 && !dep_ok[b->dep_form - 1])) {   // not a candidate
      if (ms_out) ms_out[c] = -1.0;
      continue;
    }
    rc = launch_step(b, 1, true);  // warm-up (dry: the particle state is left as it was)
    if (rc) break;
    cudaEventRecord(e0, b->stream);
    for (int n = 0; n < trial_steps && rc == EMU_OK; ++n) rc = launch_step(b, 1, false);
    cudaEventRecord(e1, b->stream);
    if (rc) break;
    rc = cuda_check(b, cudaEventSynchronize(e1), "autotune timing");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= trial_steps;
    if (ms_out) ms_out[c] = ms;
    if (c == 0 || ms < best_ms) { best = c; best_ms = ms; }
  }
  b->pool.push_back(e0);
  b->pool.push_back(e1);
  b->prof = prof;
  apply(best);
  invalidate_graph(b);
  if (rc) return rc;
  if (choice_out) *choice_out = best;
  return read_errors(b);
}

int emu_set_step_form(emu_box* b, int32_t form) {
  if (int rc = check_bound(b)) return rc;
  if (form < 0 || form > 2) return fail(b, EMU_EINVAL, "form must be 0, 1 or 2");
  if (form >= 1 && b->is3d) return no_3d(b, form == 1 ? "the fused step form" : "step form 2");
  if (form >= 1 && b->general) return needs_lattice(b, form == 1 ? "the fused step form" : "step form 2");
  if (form == 2 && b->S.order > 2) return fail(b, EMU_EINVAL, "step form 2 covers the shape orders 0-2");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  if (form == 1) {
    const int maxb = fused_max_blocks(b);
    if (maxb <= 0) return fail(b, EMU_EINVAL, "the device cannot launch the fused (cooperative) step");
    if (b->blocks > maxb)
      return fail(b, EMU_EINVAL, "the fused step needs all %d blocks resident at once; at most %d fit (emu_set_grid)",
                  b->blocks, maxb);
  }
  b->step_form = form;
  invalidate_graph(b);
  return EMU_OK;
}

int emu_set_layout(emu_box* b, int32_t layout) {
  if (int rc = check_bound(b)) return rc;
  if (b->is3d) return no_3d(b, "a particle layout other than the lattice");
  if (layout < -1 || layout > 1) return fail(b, EMU_EINVAL, "layout must be -1, 0 or 1");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  b->layout = layout;
  if (int rc = choose_layout(b)) return rc;
  if (!b->general) return rebuild_dirtable(b);
  return EMU_OK;
}

int emu_get_layout(emu_box* b, int32_t* general) {
  if (int rc = check_bound(b)) return rc;
  if (!general) return fail(b, EMU_EINVAL, "general is NULL");
  *general = b->general ? 1 : 0;
  return EMU_OK;
}

int emu_set_barrier_timeout(emu_box* b, int64_t ns) {
  if (int rc = check_bound(b)) return rc;
  if (ns < 0) return fail(b, EMU_EINVAL, "the timeout must be >= 0 ns");
  b->limit_ns = (unsigned long long)ns;
  invalidate_graph(b);
  return EMU_OK;
}

int64_t emu3_workspace_bytes(const emu3_config* cfg) {
  Shape S;
  std::vector<BoxGeo> rows;
  int ntz = 0;
  if (make_shape3(cfg, S, rows, ntz)) return EMU_EINVAL;
  return (int64_t)layout3(S, rows.size()).total;
}

int emu3_create(const emu3_config* cfg, emu_box** out) {
  if (!out) return fail(nullptr, EMU_EINVAL, "out is NULL");
  *out = nullptr;
  Shape S;
  std::vector<BoxGeo> rows;
  int ntz = 0;
  if (const char* why = make_shape3(cfg, S, rows, ntz)) return fail(nullptr, EMU_EINVAL, "%s", why);
  emu_box* b = new (std::nothrow) emu_box();
  if (!b) return fail(nullptr, EMU_EINVAL, "host allocation failed");
  b->is3d = true;
  b->c3 = *cfg;
  b->S = std::move(S);
  b->rows = std::move(rows);
  b->ntz = ntz;
  b->L = layout3(b->S, b->rows.size());
  emu_config c{};   // the physics values the shared calls read (kappa for the matter term)
  c.nz = cfg->nz;
  c.ndir = cfg->ndir;
  c.Lz = cfg->Lz;
  c.area = cfg->Lx * cfg->Ly;
  c.kappa = cfg->kappa;
  c.c_light = cfg->c_light;
  c.cfl_adv = cfg->cfl_adv;
  c.cfl_flavor = cfg->cfl_flavor;
  c.shape_order = cfg->shape_order;
  b->cfg.assign(1, c);
  *out = b;
  return EMU_OK;
}

int emu3_bind(emu_box* b, const emu_particles* parts, double* x, double* y, void* workspace, int64_t workspace_bytes,
              void* stream) {
  if (!b) return EMU_EINVAL;
  if (!b->is3d) return fail(b, EMU_EINVAL, "emu3_bind takes a box made by emu3_create");
  if (!x || !y) return fail(b, EMU_EINVAL, "x or y is NULL");
  b->x3 = x;
  b->y3 = y;
  return bind_common(b, parts, workspace, workspace_bytes, stream);
}

int emu3_init_particles(emu_box* b, const double* n_nu, const double* n_nubar, const double* f_nu,
                        const double* f_nubar, const double* dirs, double alpha, uint64_t seed) {
  if (int rc = check_bound(b)) return rc;
  if (!b->is3d) return fail(b, EMU_EINVAL, "emu3_init_particles takes a 3D box");
  if (!n_nu || !n_nubar || !f_nu || !f_nubar) return fail(b, EMU_EINVAL, "species arrays must not be NULL");
  const size_t C = (size_t)b->S.NZ, M = (size_t)b->S.MT;
  std::vector<double> sp(8 * C);
  std::memcpy(sp.data(), n_nu, sizeof(double) * C);
  std::memcpy(sp.data() + C, n_nubar, sizeof(double) * C);
  std::memcpy(sp.data() + 2 * C, f_nu, sizeof(double) * 3 * C);
  std::memcpy(sp.data() + 5 * C, f_nubar, sizeof(double) * 3 * C);
  BoxGeo& g = b->S.geo[0];
  g.use_dirs = dirs ? 1 : 0;
  g.alpha = alpha;
  g.seed = seed;
  if (int rc = upload_geo(b)) return rc;
  if (int rc = cuda_check(b, cudaMemcpyAsync(b->species, sp.data(), sizeof(double) * sp.size(),
                                             cudaMemcpyHostToDevice, b->stream), "copy species"))
    return rc;
  if (dirs)
    if (int rc = cuda_check(b, cudaMemcpyAsync(b->dirs, dirs, sizeof(double) * 3 * M, cudaMemcpyHostToDevice,
                                               b->stream), "copy directions"))
      return rc;
  before_launch(b, CLS_OTHER);
  k3_init<<<(unsigned)((b->S.Ptot + kThreads - 1) / kThreads), kThreads, 0, b->stream>>>(
      box3_view(b), b->pt, b->x3, b->y3, b->species, b->dirs, b->err);
  if (int rc = after_launch(b, "3D init kernel")) return rc;
  if (int rc = rebuild_dirtable3(b)) return rc;
  b->next_stage = 1;
  b->step_valid = false;
  return read_errors(b);   // synchronises: the host staging vector may go
}

static int positions3(emu_box* b, double* xd, double* yd, const double* xs, const double* ys, cudaMemcpyKind kind,
                      int sync) {
  const size_t bytes = sizeof(double) * (size_t)b->S.Ptot;
  if (xs && xd)
    if (int rc = cuda_check(b, cudaMemcpyAsync(xd, xs, bytes, kind, b->stream), "copy x")) return rc;
  if (ys && yd)
    if (int rc = cuda_check(b, cudaMemcpyAsync(yd, ys, bytes, kind, b->stream), "copy y")) return rc;
  if (sync) return cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise after copy");
  return EMU_OK;
}

int emu3_get_positions(emu_box* b, double* x, double* y, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (!b->is3d) return fail(b, EMU_EINVAL, "emu3_get_positions takes a 3D box");
  return positions3(b, x, y, x ? b->x3 : nullptr, y ? b->y3 : nullptr,
                    on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, on_host);
}

int emu3_set_positions(emu_box* b, const double* x, const double* y, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (!b->is3d) return fail(b, EMU_EINVAL, "emu3_set_positions takes a 3D box");
  b->next_stage = 1;
  return positions3(b, x ? b->x3 : nullptr, y ? b->y3 : nullptr, x, y,
                    on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, on_host);
}

int emu_set_oscillation(emu_box* b, int32_t box, const emu_oscillation* osc) {
  if (!b) return EMU_EINVAL;
  if (box < -1 || box >= b->S.nbox) return fail(b, EMU_EINVAL, "box index %d out of range", box);
  double vn[9] = {0}, vb[9] = {0}, ne = 0.0;
  if (osc) {
    const double* m = osc->mass_eV;
    if (!(osc->energy_erg > 0) || !(osc->hbar > 0) || !(osc->erg_per_eV > 0) || !std::isfinite(osc->n_e))
      return fail(b, EMU_EINVAL, "oscillation parameters: energy, hbar and erg_per_eV must be positive");
    typedef std::complex<double> cd;
    const double c12 = std::cos(osc->theta12), s12 = std::sin(osc->theta12);
    const double c13 = std::cos(osc->theta13), s13 = std::sin(osc->theta13);
    const double c23 = std::cos(osc->theta23), s23 = std::sin(osc->theta23);
    const cd e = std::polar(1.0, osc->delta_cp);
    // standard three-angle mixing matrix (flavour <- mass)
    const cd U[3][3] = {{c12 * c13, s12 * c13, s13 * std::conj(e)},
                        {-s12 * c23 - c12 * s23 * s13 * e, c12 * c23 - s12 * s23 * s13 * e, s23 * c13},
                        {s12 * s23 - c12 * c23 * s13 * e, -c12 * s23 - s12 * c23 * s13 * e, c23 * c13}};
    double w[3];
    for (int i = 0; i < 3; ++i) {
      const double mc2 = m[i] * osc->erg_per_eV;
      w[i] = mc2 * mc2 / (2.0 * osc->energy_erg) / osc->hbar;
    }
    cd Hv[3][3];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        cd v = 0.0;
        for (int i = 0; i < 3; ++i) v += U[a][i] * w[i] * std::conj(U[c][i]);
        Hv[a][c] = v;
      }
    ne = osc->n_e;
    const int pk[6][2] = {{0, 1}, {0, 1}, {0, 2}, {0, 2}, {1, 2}, {1, 2}};
    for (int k = 0; k < 3; ++k) { vn[k] = Hv[k][k].real(); vb[k] = Hv[k][k].real(); }
    for (int q = 0; q < 6; ++q) {
      const cd v = Hv[pk[q][0]][pk[q][1]];
      vn[3 + q] = (q & 1) ? v.imag() : v.real();
      vb[3 + q] = (q & 1) ? -v.imag() : v.real();   // H_vacuum^*
    }
  }
  bool any = false;
  for (int i = 0; i < b->S.nbox; ++i) {
    BoxGeo& g = b->S.geo[i];
    if (box == -1 || box == i) {
      const double mat = b->cfg[i].kappa * ne;   // kappa n_e on the electron flavour; Hbar gets -H_matter
      // traceless components (the trace commutes with every rho): H_11 - H_22, H_22 - H_33, off-diagonals
      g.vnu[0] = (vn[0] + mat) - vn[1];
      g.vnu[1] = vn[1] - vn[2];
      g.vnubar[0] = (vb[0] - mat) - vb[1];
      g.vnubar[1] = vb[1] - vb[2];
      for (int q = 0; q < 6; ++q) { g.vnu[2 + q] = vn[3 + q]; g.vnubar[2 + q] = vb[3 + q]; }
      g.n_e = ne;
    }
    for (int c = 0; c < kNC; ++c) any = any || g.vnu[c] != 0.0 || g.vnubar[c] != 0.0;
  }
  b->pot = any;
  b->step_valid = false;
  invalidate_graph(b);
  if (b->bound) return upload_geo(b);
  return EMU_OK;
}

// ------------------------------------------------------------------ adjoint

}  // extern "C"

namespace {
// Adjoint scratch: stage states y2, y3 and three stage adjoints [18][P] each,
// then the shape weights and grid potential of stages 1-3 kept from the
// recomputed forward stages ([3][NWS][P] and [3][32][NZ], traceless potentials).
size_t adjoint_doubles(const Shape& S) {
  return (size_t)90 * S.Ptot + 3 * ((size_t)kept_weights(S.order) * S.Ptot + (size_t)kNT * S.NZ);
}

// Record of one step for the adjoint: the stage states y2, y3, y4 ([3][18][P]),
// the shape weights of stages 1-4 ([4][NWS][P]) and their grid potentials
// ([4][32][NZ], traceless).
size_t record_doubles(const Shape& S) {
  return (size_t)54 * S.Ptot + 4 * ((size_t)kept_weights(S.order) * S.Ptot + (size_t)kNT * S.NZ);
}

// One forward step (as launch_step) that also writes its record: the stage
// kernels write their weights, potentials and next stage states straight into it.
int record_step(emu_box* b, double* rec) {
  const size_t P = (size_t)b->S.Ptot;
  const size_t nws = (size_t)kept_weights(b->S.order) * P, na = (size_t)kNT * b->S.NZ;
  double* Y = rec;                 // y2, y3, y4
  double* Wr = Y + 54 * P;         // weights of stages 1..4
  double* Ar = Wr + 4 * nws;       // potentials of stages 1..4
  if (int rc = launch_shifts(b, kStageFrac, 4)) return rc;
  for (int s = 1; s <= 4; ++s) {
    const double* src = s == 1 ? b->pt.stage : Y + (s - 2) * 18 * P;   // y_s (stages 2-4)
    const double* rnu = (s == 1) ? b->pt.rho : src;
    const double* rnb = (s == 1) ? b->pt.rhobar : src + 9 * P;
    const int* srow = b->shift + (size_t)(s - 1) * b->S.MT;
    double* Ws = nws ? Wr + (s - 1) * nws : b->W;   // (order 0 keeps no weights)
    double* As = Ar + (s - 1) * na;
    if (int rc = launch_deposit(b, 5, rnu, rnb, srow, kStageFrac[s - 1], As, Ws)) return rc;
    Parts ps = b->pt;
    if (s < 4) ps.stage = Y + (s - 1) * 18 * P;   // y_{s+1}
    if (int rc = launch_rk_on(b, s, srow, 0, ps, Ws, As, src)) return rc;
  }
  return EMU_OK;
}

// The backward stages of one adjoint step from a record (no recomputation).
int adjoint_recorded_body(emu_box* b, const double* rec, double* lambda, double* gN, double* gNbar, void* adj_ws) {
  const size_t P = (size_t)b->S.Ptot;
  const size_t nws = (size_t)kept_weights(b->S.order) * P, na = (size_t)kNT * b->S.NZ;
  const double* Y = rec;
  const double* Wr = Y + 54 * P;
  const double* Ar = Wr + 4 * nws;
  double* La = (double*)adj_ws;
  double* Lb = La + 18 * P;
  double* Lt = Lb + 18 * P;
  const size_t bytes18 = sizeof(double) * 18 * P;
  if (int rc = launch_shifts(b, kStageFrac, 4)) return rc;
  if (int rc = cuda_check(b, cudaMemcpyAsync(Lt, lambda, bytes18, cudaMemcpyDeviceToDevice, b->stream),
                          "copy adjoint"))
    return rc;
  const Batch B = batch_view(b);
  double* Lnext = nullptr;
  for (int s = 4; s >= 1; --s) {
    double* ys = s == 1 ? b->pt.rho : const_cast<double*>(Y + (s - 2) * 18 * P);
    double* ysb = s == 1 ? b->pt.rhobar : ys + 9 * P;
    const int* srow = b->shift + (size_t)(s - 1) * b->S.MT;
    const double* Hs = Ar + (s - 1) * na;
    const double* Ws = Wr + (s - 1) * nws;
    Parts ps = b->pt;
    ps.rho = ys;
    ps.rhobar = ysb;
    double* Lcur = (s % 2 == 0) ? La : Lb;
    before_launch(b, CLS_OTHER);
    by_order(b->S.order, [&](auto O) {
      constexpr int R = decltype(O)::value;
      if (b->pot)
        pdl(b->stream, k_adj_a<true, R>, persist_grid(b), B, ps, Ws, b->dirtab, srow, Hs, lambda,
            Lnext, s, Lcur, b->pt.acc);
      else
        pdl(b->stream, k_adj_a<false, R>, persist_grid(b), B, ps, Ws, b->dirtab, srow, Hs, lambda,
            Lnext, s, Lcur, b->pt.acc);
      return 0;
    });
    if (int rc = after_launch(b, "adjoint stage kernel")) return rc;
    if (int rc = launch_deposit(b, 3, b->pt.acc, nullptr, srow, kStageFrac[s - 1], b->mom)) return rc;
    before_launch(b, CLS_OTHER);
    by_order(b->S.order, [&](auto O) {
      pdl(b->stream, k_adj_b<decltype(O)::value>, persist_grid(b), B, ps, Ws, b->dirtab, srow, b->mom,
          Lcur, Lt, gN, gNbar);
      return 0;
    });
    if (int rc = after_launch(b, "adjoint interpolation kernel")) return rc;
    Lnext = Lcur;
  }
  return cuda_check(b, cudaMemcpyAsync(lambda, Lt, bytes18, cudaMemcpyDeviceToDevice, b->stream), "copy adjoint");
}

// The launches of one adjoint step (emu_adjoint_step; the step sizes are on the device).
int adjoint_body(emu_box* b, double* lambda, double* gN, double* gNbar, void* adj_ws) {
  const size_t P = (size_t)b->S.Ptot;
  double* Y2 = (double*)adj_ws;  // stage states y2, y3 (y4 stays in the stage buffer)
  double* Y3 = Y2 + 18 * P;
  double* La = Y3 + 18 * P;      // adjoints of two consecutive stage states
  double* Lb = La + 18 * P;
  double* Lt = Lb + 18 * P;      // running sum: lambda + sum over stages
  const size_t nws = (size_t)kept_weights(b->S.order) * P, na = (size_t)kNT * b->S.NZ;
  double* Wk = Lt + 18 * P;      // weights of stages 1..3
  double* Ak = Wk + 3 * nws;     // grid potential of stages 1..3
  const size_t bytes18 = sizeof(double) * 18 * P;
  if (int rc = launch_shifts(b, kStageFrac, 4)) return rc;
  // forward stages 1..3: y2, y3 copied out, y4 left in the stage buffer; each
  // stage's weights and potential kept for the backward pass
  for (int s = 1; s <= 3; ++s) {
    if (int rc = launch_stage(b, s, 0)) return rc;
    if (nws)
      if (int rc = cuda_check(b, cudaMemcpyAsync(Wk + (s - 1) * nws, b->W, sizeof(double) * nws,
                                                 cudaMemcpyDeviceToDevice, b->stream), "keep stage weights"))
        return rc;
    if (int rc = cuda_check(b, cudaMemcpyAsync(Ak + (s - 1) * na, b->At, sizeof(double) * na,
                                               cudaMemcpyDeviceToDevice, b->stream), "keep stage potential"))
      return rc;
    if (s < 3)
      if (int rc = cuda_check(b, cudaMemcpyAsync(s == 1 ? Y2 : Y3, b->pt.stage, bytes18, cudaMemcpyDeviceToDevice,
                                                 b->stream), "copy stage state"))
        return rc;
  }
  if (int rc = cuda_check(b, cudaMemcpyAsync(Lt, lambda, bytes18, cudaMemcpyDeviceToDevice, b->stream),
                          "copy adjoint"))
    return rc;
  // backward: stage adjoint lam_s = J(y_s)^T mu_s with mu_4 = dt/6 lam,
  // mu_3 = dt/3 lam + dt lam_4, mu_2 = dt/3 lam + dt/2 lam_3, mu_1 = dt/6 lam + dt/2 lam_2
  const Batch B = batch_view(b);
  double* Lnext = nullptr;
  for (int s = 4; s >= 1; --s) {
    double* ys = s == 1 ? b->pt.rho : s == 2 ? Y2 : s == 3 ? Y3 : b->pt.stage;
    double* ysb = s == 1 ? b->pt.rhobar : ys + 9 * P;
    const int* srow = b->shift + (size_t)(s - 1) * b->S.MT;
    const double frac = kStageFrac[s - 1];
    // H and weights of the stage state: stage 4 deposits them now, stages 1-3 kept theirs
    const double* Hs = s == 4 ? b->At : Ak + (s - 1) * na;
    const double* Ws = s == 4 ? b->W : Wk + (s - 1) * nws;
    if (s == 4)
      if (int rc = launch_deposit(b, 5, ys, ysb, srow, frac, b->At)) return rc;
    Parts ps = b->pt;
    ps.rho = ys;
    ps.rhobar = ysb;
    double* Lcur = (s % 2 == 0) ? La : Lb;
    before_launch(b, CLS_OTHER);
    by_order(b->S.order, [&](auto O) {
      constexpr int R = decltype(O)::value;
      if (b->pot)
        pdl(b->stream, k_adj_a<true, R>, persist_grid(b), B, ps, Ws, b->dirtab, srow, Hs, lambda,
            Lnext, s, Lcur, b->pt.acc);
      else
        pdl(b->stream, k_adj_a<false, R>, persist_grid(b), B, ps, Ws, b->dirtab, srow, Hs, lambda,
            Lnext, s, Lcur, b->pt.acc);
      return 0;
    });
    if (int rc = after_launch(b, "adjoint stage kernel")) return rc;
    if (int rc = launch_deposit(b, 3, b->pt.acc, nullptr, srow, frac, b->mom)) return rc;
    before_launch(b, CLS_OTHER);
    by_order(b->S.order, [&](auto O) {
      pdl(b->stream, k_adj_b<decltype(O)::value>, persist_grid(b), B, ps, Ws, b->dirtab, srow, b->mom,
          Lcur, Lt, gN, gNbar);
      return 0;
    });
    if (int rc = after_launch(b, "adjoint interpolation kernel")) return rc;
    Lnext = Lcur;
  }
  return cuda_check(b, cudaMemcpyAsync(lambda, Lt, bytes18, cudaMemcpyDeviceToDevice, b->stream), "copy adjoint");
}

}  // namespace

extern "C" {

int64_t emu_adjoint_workspace_bytes(const emu_config* cfg) { return emu_batch_adjoint_workspace_bytes(cfg, 1); }

int64_t emu_batch_adjoint_workspace_bytes(const emu_config* cfgs, int32_t nbox) {
  Shape S;
  if (make_shape(cfgs, nbox, S)) return EMU_EINVAL;
  return (int64_t)(sizeof(double) * adjoint_doubles(S));
}

int emu_adjoint_seed(emu_box* b, const double* dmom, double* lambda, double* gN, double* gNbar) {
  if (int rc = check_bound(b)) return rc;
  if (b->is3d) return no_3d(b, "the adjoint");
  if (b->general) return needs_lattice(b, "the adjoint");
  if (!dmom || !lambda || !gN || !gNbar) return fail(b, EMU_EINVAL, "adjoint seed: NULL pointer");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  const double zero = 0.0;
  if (int rc = launch_shifts(b, &zero, 1)) return rc;
  before_launch(b, CLS_OTHER);
  by_order(b->S.order, [&](auto O) {
    k_adj_seed<decltype(O)::value><<<persist_grid(b), kThreads, 0, b->stream>>>(
        batch_view(b), b->pt, b->dirtab, b->shift, dmom, lambda, gN, gNbar, b->err);
    return 0;
  });
  return after_launch(b, "adjoint seed kernel");
}

int emu_adjoint_step(emu_box* b, double dt, double* lambda, double* gN, double* gNbar, void* adj_ws,
                     int64_t adj_ws_bytes) {
  if (int rc = check_bound(b)) return rc;
  if (b->is3d) return no_3d(b, "the adjoint");
  if (b->general) return needs_lattice(b, "the adjoint");
  if (dt != 0.0) {
    if (b->S.nbox != 1) return fail(b, EMU_EINVAL, "a batch takes dt = 0 (each box's own step size)");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(b, EMU_EINVAL, "dt must be positive and finite, or 0");
  } else if (!b->step_valid) {
    return fail(b, EMU_EINVAL, "dt = 0 needs the boxes' step sizes (emu_batch_set_dt or a time-step call)");
  }
  if (!lambda || !gN || !gNbar || !adj_ws) return fail(b, EMU_EINVAL, "adjoint step: NULL pointer");
  const size_t need = sizeof(double) * adjoint_doubles(b->S);
  if (adj_ws_bytes < (int64_t)need)
    return fail(b, EMU_EINVAL, "adjoint workspace too small: %lld < %lld bytes", (long long)adj_ws_bytes,
                (long long)need);
  if (((uintptr_t)adj_ws) & 255) return fail(b, EMU_EINVAL, "adjoint workspace must be 256-byte aligned");
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  if (int rc = set_dts(b, dt != 0.0 ? &dt : b->step_dt.data())) return rc;
  b->next_stage = 1;
  if (b->prof) return adjoint_body(b, lambda, gN, gNbar, adj_ws);
  // the graph reads the step sizes from the device: it depends on the buffers only
  const void* key[4] = {lambda, gN, gNbar, adj_ws};
  const bool same = b->adj_graph && std::memcmp(key, b->adj_key, sizeof(key)) == 0;
  if (!same) {
    if (b->adj_graph) { cudaGraphExecDestroy(b->adj_graph); b->adj_graph = nullptr; }
    if (int rc = capture(b, &b->adj_graph, &b->adj_launches,
                         [&] { return adjoint_body(b, lambda, gN, gNbar, adj_ws); }))
      return rc;
    std::memcpy(b->adj_key, key, sizeof(key));
  }
  return launch_graph(b, b->adj_graph, b->adj_launches);
}

int64_t emu_batch_adjoint_record_bytes(const emu_config* cfgs, int32_t nbox) {
  Shape S;
  if (make_shape(cfgs, nbox, S)) return EMU_EINVAL;
  return (int64_t)(sizeof(double) * record_doubles(S));
}

// Shared checks of the recording calls: step size (dt > 0 single box, 0 =
// each box's own), a buffer of at least `need` bytes, 256-byte aligned.
static int record_checks(emu_box* b, double dt, const void* buf, int64_t bytes, size_t need, const char* what) {
  if (int rc = check_bound(b)) return rc;
  if (b->is3d) return no_3d(b, "the adjoint");
  if (b->general) return needs_lattice(b, "the adjoint");
  if (dt != 0.0) {
    if (b->S.nbox != 1) return fail(b, EMU_EINVAL, "a batch takes dt = 0 (each box's own step size)");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(b, EMU_EINVAL, "dt must be positive and finite, or 0");
  } else if (!b->step_valid) {
    return fail(b, EMU_EINVAL, "dt = 0 needs the boxes' step sizes (emu_batch_set_dt or a time-step call)");
  }
  if (!buf) return fail(b, EMU_EINVAL, "%s: NULL pointer", what);
  if (bytes < (int64_t)need)
    return fail(b, EMU_EINVAL, "%s too small: %lld < %lld bytes", what, (long long)bytes, (long long)need);
  if (((uintptr_t)buf) & 255) return fail(b, EMU_EINVAL, "%s must be 256-byte aligned", what);
  if (b->next_stage != 1) return fail(b, EMU_EINVAL, "a step is in progress (stage %d next)", b->next_stage);
  return EMU_OK;
}

int emu_adjoint_record_step(emu_box* b, double dt, void* rec, int64_t rec_bytes) {
  if (int rc = record_checks(b, dt, rec, rec_bytes, b ? sizeof(double) * record_doubles(b->S) : 0, "record"))
    return rc;
  if (int rc = set_dts(b, dt != 0.0 ? &dt : b->step_dt.data())) return rc;
  b->next_stage = 1;
  if (b->prof) return record_step(b, (double*)rec);
  // the graph reads the step sizes from the device: it depends on the buffer only
  const void* key[6] = {(const void*)1, rec, nullptr, nullptr, nullptr, nullptr};
  return keyed_graph(b, key, [&] { return record_step(b, (double*)rec); });
}

int emu_adjoint_step_recorded(emu_box* b, double dt, const void* rec, double* lambda, double* gN, double* gNbar,
                              void* adj_ws, int64_t adj_ws_bytes) {
  if (int rc = record_checks(b, dt, adj_ws, adj_ws_bytes, b ? sizeof(double) * 54 * (size_t)b->S.Ptot : 0,
                             "adjoint workspace"))
    return rc;
  if (!rec || (((uintptr_t)rec) & 255)) return fail(b, EMU_EINVAL, "record: NULL or not 256-byte aligned");
  if (!lambda || !gN || !gNbar) return fail(b, EMU_EINVAL, "adjoint step: NULL pointer");
  if (int rc = set_dts(b, dt != 0.0 ? &dt : b->step_dt.data())) return rc;
  b->next_stage = 1;
  if (b->prof) return adjoint_recorded_body(b, (const double*)rec, lambda, gN, gNbar, adj_ws);
  const void* key[6] = {(const void*)2, rec, lambda, gN, gNbar, adj_ws};
  return keyed_graph(b, key, [&] { return adjoint_recorded_body(b, (const double*)rec, lambda, gN, gNbar, adj_ws); });
}

int emu_weight_gradient(emu_box* b, const double* gN, const double* gNbar, double* out, int on_host) {
  if (int rc = check_bound(b)) return rc;
  if (b->is3d) return no_3d(b, "the adjoint");
  if (!gN || !gNbar || !out) return fail(b, EMU_EINVAL, "weight gradient: NULL pointer");
  double* dst = on_host ? b->mom : out;  // staging: the moments buffer holds 72 NZ doubles
  const int blocks = (b->S.NZ + kThreads - 1) / kThreads;
  before_launch(b, CLS_OTHER);
  k_weight_grad<<<blocks, kThreads, 0, b->stream>>>(batch_view(b), gN, gNbar, b->dirtab, dst);
  if (int rc = after_launch(b, "weight gradient kernel")) return rc;
  if (on_host) return copy_out(b, out, dst, sizeof(double) * 8 * b->S.NZ, 1);
  return EMU_OK;
}

int emu_sync(emu_box* b) {
  if (int rc = check_bound(b)) return rc;
  if (int rc = cuda_check(b, cudaStreamSynchronize(b->stream), "synchronise")) return rc;
  if (b->cap)
    if (int rc = cuda_check(b, cudaStreamSynchronize(b->cap), "synchronise graph stream")) return rc;
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
// Some callers cannot allocate device memory at all but may still enqueue
// stream work and wait for it: code inside another library's allocation-free
// region, or code that must not call into any allocator (for example while a
// memory pool is being torn down or resized).  They cannot provide the
// workspace that emu_bind expects, so this entry point keeps the deposit's
// scratch (box descriptor, per-direction table, lattice shifts, partial sums
// of the warps, error word) in one static device array that the library
// itself holds on every GPU that loads it.  It launches kernels, copies and
// synchronises, so it must not run inside a host function (CUDA forbids CUDA
// calls there) or on a stream being captured.

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

// Forgets the current device's cached address (after a CUDA error: the next
// call looks it up again).
void forget_static_address() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  g_static_addr[dev] = nullptr;
}

}  // namespace

extern "C" int emu_deposit_static(const emu_config* cfg, const double* z, const double* ox, const double* oy,
                                  const double* oz, const double* N, const double* Nbar, const double* rho,
                                  const double* rhobar, double pos_dt, double* A_out, void* stream) {
  Shape S;
  if (const char* why = make_shape(cfg, 1, S)) return fail(nullptr, EMU_EINVAL, "%s", why);
  if (S.order != 2) return fail(nullptr, EMU_EINVAL, "emu_deposit_static takes the quadratic shape (shape_order 2)");
  if (!z || !ox || !oy || !oz || !N || !Nbar || !rho || !rhobar || !A_out)
    return fail(nullptr, EMU_EINVAL, "a particle array or A_out is NULL");
  if (!std::isfinite(pos_dt)) return fail(nullptr, EMU_EINVAL, "pos_dt must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return fail(nullptr, EMU_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(nullptr, EMU_EINVAL, "emu_deposit_static synchronises its stream: it cannot run on a stream "
                  "that is being captured");
  }
  // carve the static array: box descriptor, step size, partial sums, error word, direction table, shifts
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t o_geo = take(sizeof(BoxGeo));
  const size_t o_dt = take(sizeof(double));
  const size_t o_partial = take(sizeof(double) * (size_t)(kPersistBlocks * kWarps + S.NT) * kSlot);
  const size_t o_err = take(sizeof(int));
  const size_t o_dirtab = take(sizeof(double) * 4 * (size_t)S.MT);
  const size_t o_shift = take(sizeof(int) * (size_t)S.MT);
  if (off > kStaticScratchBytes)
    return fail(nullptr, EMU_EINVAL,
                "emu_deposit_static: this box needs %zu bytes of scratch, more than the %zu-byte static array "
                "(use emu_deposit with a caller workspace)", off, kStaticScratchBytes);
  void* base = nullptr;
  if (int rc = static_scratch_address(&base)) return rc;
  char* s = (char*)base;
  BoxGeo* geo = (BoxGeo*)(s + o_geo);
  double* dtp = (double*)(s + o_dt);
  double* partial = (double*)(s + o_partial);
  int* err = (int*)(s + o_err);
  double* dirtab = (double*)(s + o_dirtab);
  int* shift = (int*)(s + o_shift);
  auto check = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return EMU_OK;
    forget_static_address();
    return fail(nullptr, EMU_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  // the error word must start at zero; the array keeps what the last call left
  if (int rc = check(cudaMemsetAsync(err, 0, sizeof(int), st), "clear static scratch")) return rc;
  k_write_geo<<<1, 1, 0, st>>>(S.geo[0], pos_dt, geo, dtp);
  if (int rc = check(cudaGetLastError(), "descriptor kernel")) return rc;
  Batch B;
  B.box = geo;
  B.dt = dtp;
  B.nbox = 1;
  B.nw = (int)(S.U < kPersistBlocks * kWarps ? S.U : kPersistBlocks * kWarps);
  B.NZ = S.NZ;
  B.MT = S.MT;
  B.NT = S.NT;
  B.T = S.T;
  B.U = S.U;
  B.Ptot = S.Ptot;
  B.U32 = 0;
  B.nw32 = 0;
  Parts pt{const_cast<double*>(z), const_cast<double*>(ox), const_cast<double*>(oy), const_cast<double*>(oz),
           const_cast<double*>(N), const_cast<double*>(Nbar), const_cast<double*>(rho),
           const_cast<double*>(rhobar), nullptr, nullptr};
  const int pblocks = (int)((S.Ptot + kThreads - 1) / kThreads);
  k_dirtable<<<pblocks, kThreads, 0, st>>>(B, pt, dirtab, err);
  if (int rc = check(cudaGetLastError(), "direction table kernel")) return rc;
  Fracs f{};
  f.v[0] = 1.0;
  k_shifts<2><<<(S.MT + kThreads - 1) / kThreads, kThreads, 0, st>>>(B, z, dirtab, f, 1, shift, nullptr);
  if (int rc = check(cudaGetLastError(), "shift kernel")) return rc;
  k_deposit<0, 2><<<dim3(kPersistBlocks), kThreads, 0, st>>>(B, z, N, Nbar, rho, rhobar, dirtab, shift, nullptr, 1.0,
                                                            partial, nullptr, err);
  if (int rc = check(cudaGetLastError(), "deposit kernel")) return rc;
  const int split = combine_split(S, B.nw);
  k_combine<<<combine_blocks(kNA, S.NZ, split), kThreads, 0, st>>>(B, partial, A_out, kNA, 1, split, err);
  if (int rc = check(cudaGetLastError(), "deposit combine kernel")) return rc;
  int h = 0;
  if (int rc = check(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st), "read error word")) return rc;
  if (int rc = check(cudaStreamSynchronize(st), "synchronise")) return rc;
  if (h & ERR_RING) return fail(nullptr, EMU_ELATTICE, "a ring of particles does not share one direction");
  if (h & ERR_LATTICE) return fail(nullptr, EMU_ELATTICE, "a particle is off its lattice site");
  if (h & ERR_NONFINITE) return fail(nullptr, EMU_ENUMERIC, "non-finite value on the grid");
  return EMU_OK;
}
