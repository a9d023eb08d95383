// C ABI of the library (include/molt.h): contexts, descriptor validation,
// per-axis sweep planning and the time-step drivers.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "coeffs.h"
#include "line_constants.h"
#include "nonuniform.cuh"
#include "molt.h"
#include "sweep_launch.h"
#include "sweep_lanes_launch.h"
#include "batch.cuh"

using namespace molt;

namespace {

thread_local std::string g_create_error;

struct Problem {
  molt_desc d;
  int64_t n[3];
  double h[3];
  int64_t total;
  void* acc = nullptr;      // compute-type accumulator (total elements)
  void* stage1 = nullptr;   // heat RK stages (state type)
  void* stage2 = nullptr;
  void* hx = nullptr;       // HJ H^_x, or sigma_x of AFFINE_SQ (state type)
  void* hx2 = nullptr;      // HJ AFFINE_SQ: delta_x (state type)
  void* src = nullptr;      // HJ source coefficients F_0..F_src_deg (state type), or null
  int src_deg = 0;
  void* tu = nullptr;       // HJ, transposed y pass: u^T and (H^_x)^T / u^{n+1}^T
  void* thx = nullptr;
  float* shadow = nullptr;  // FP32 copy of the state the sweeps read (mixed precision)
  void* gp = nullptr;       // advection-diffusion: split fluxes g^+, g^- (compute type)
  void* gm = nullptr;
  void* hv[4] = {nullptr, nullptr, nullptr, nullptr};  // HJ with RK3: S_R, S_L per axis (state type)
  // non-uniform axes: the nodes of one period or of a Dirichlet line (empty =
  // uniform), and device caches (mutable: filled on first use by sweeps that
  // see the problem as const) -- the tables of the last (alpha, rule)
  // applied, transposed copies and the axis sums of molt_step
  std::vector<double> nodes[3];
  struct NuCache {
    double alpha = 0.0;
    int npts = 0;
    int weights = -1;
    void* dev = nullptr;         // cR[K n], cL[K n], q[n] of the compute type (K = 6, WENO-Z 30)
    size_t count = 0;            // values allocated
  };
  mutable NuCache nu[3];
  mutable void* nu_tmp[2] = {nullptr, nullptr};   // transposed copies for strided non-uniform 2-D sweeps
  mutable void* nu_sum = nullptr;                 // S of one axis in the compute type (molt_step)
  void* acc2 = nullptr;     // heat with concurrent axes: the y (and z) sums (compute type)
  int64_t hj_steps = 0;     // HJ steps taken (rotates the speed slots)
  bool hj_lag_ready = false;
  bool hj_flipped = false;  // HJ with a transposed y pass: the state sits in tu (transposed) between steps
  // heat with concurrent axis sweeps: one step captured as a CUDA graph (for
  // the state array it was captured with) and replayed per step
  cudaGraphExec_t heat_graph = nullptr;
  const void* heat_graph_u = nullptr;
  int heat_steps_direct = 0;   // steps launched directly since the state array changed
  bool heat_graph_off = false; // capture refused (e.g. the legacy default stream)
};

}  // namespace

struct BatchState {
  bool checked = false, supported = false, tuned = false;
  std::vector<int> E[2];                 // tuned points per lane per problem, per axis
  BatchSweep* d_sweeps = nullptr;
  BatchUpdate* d_updates = nullptr;
  unsigned int* d_bar = nullptr;         // [count, generation]
  BatchParams params{};
  size_t smem = 0;
  int grid = 0;
  std::vector<void*> last_u;
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
};

struct molt_ctx {
  cudaStream_t stream = nullptr;
  BatchState batch;
  long long wait_limit = 2000000000LL;   // cycles a device-side wait may take
  bool test_skip_arrive = false;         // test hook: one CTA skips the first grid barrier
  std::vector<Problem> probs;
  int* status_dev = nullptr;       // device status word
  unsigned long long* speed_dev = nullptr;  // per problem: 2 speed slots (double bits)
  double* t_dev = nullptr;         // per problem time (HJ)
  double* tnow_dev = nullptr;      // per problem time at the start of the step (HJ source)
  bool no_tma = false;             // force the plain kernels (molt_set_option)
  int lanes = 1;                   // line-per-lane FP32 sweeps: 0 off, 1 auto, 2 whenever the shape allows
  int xlines = 1;                  // x lines of those sweeps one warp per line (0: line-per-lane tiles)
  void* mlp_blob = nullptr;        // learned weights: the BF16 network (MlpBlob)
  unsigned long long* mlp_stats = nullptr;  // [stencils evaluated, fallbacks]
  bool mlp_ready = false;          // molt_set_mlp has been called
  bool profile = false;
  // small heat problems: the axes' sweeps of a stage on two streams at once
  // (MOLT_OPT_AXIS_STREAMS), joined by events before the stage update
  int axis_streams = 1;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  struct Rec { int kind; cudaEvent_t start, stop; };
  std::vector<Rec> recs;
  std::string err;
};

namespace {

molt_status fail(molt_ctx* c, molt_status s, const std::string& m) {
  if (c) c->err = m; else g_create_error = m;
  return s;
}

molt_status cuda_fail(molt_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MOLT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_f64_sweep(const molt_desc& d) { return d.prec == MOLT_PREC_F64; }
bool is_f32_state(const molt_desc& d) { return d.prec == MOLT_PREC_F32; }
bool is_mixed(const molt_desc& d) { return d.prec == MOLT_PREC_F32_F64UPDATE; }
size_t state_bytes(const molt_desc& d) { return is_f32_state(d) ? 4 : 8; }
size_t compute_bytes(const molt_desc& d) { return is_f64_sweep(d) ? 8 : 4; }

// Small heat problems run a stage's axis sweeps on two streams at once: one
// sweep launch covers too few lines to fill the GPU, and the axes read the
// same stage input and write their own accumulators.
constexpr long long kAxisStreamsMaxPoints = 1LL << 18;

std::string validate(const molt_desc& d) {
  if (d.ndim < 1 || d.ndim > 3) return "ndim must be 1, 2 or 3";
  for (int ax = 0; ax < 3; ++ax) {
    if (ax < d.ndim) {
      if (d.n[ax] < 1) return "n must be >= 1 on every used axis";
      if (d.n[ax] > (1 << 20)) return "n above 2^20 points per axis";
      if (d.bc[ax] != MOLT_BC_PERIODIC && d.bc[ax] != MOLT_BC_DIRICHLET) return "unknown boundary type";
      if (d.bc[ax] == MOLT_BC_DIRICHLET && d.n[ax] < 2) return "Dirichlet axes need n >= 2";
      if (!(d.hi[ax] > d.lo[ax])) return "hi must exceed lo";
    } else if (d.n[ax] != 1 && d.n[ax] != 0) {
      return "unused axes must have n = 1";
    }
  }
  if (d.P < 1 || d.P > 64) return "P must be in 1..64";
  if (d.quad_points != 3 && d.quad_points != 5 && d.quad_points != 6) return "quad_points must be 3, 5 or 6";
  if (d.weights != MOLT_W_LINEAR && d.weights != MOLT_W_WENOZ && d.weights != MOLT_W_LEARNED)
    return "unknown weights";
  if (d.weights != MOLT_W_LINEAR && d.quad_points != 5) return "WENO weights need quad_points = 5";
  if (d.prec < 0 || d.prec > 2) return "unknown precision";
  if (d.pde < 0 || d.pde > 3) return "unknown pde";
  if (d.flux != MOLT_FLUX_LINEAR && d.flux != MOLT_FLUX_BURGERS) return "unknown flux";
  if (!(d.beta > 0)) return "beta must be positive";
  if (d.hamiltonian < MOLT_H_HALF_SQ || d.hamiltonian > MOLT_H_AFFINE_SQ) return "unknown hamiltonian";
  for (int ax = 0; ax < 3; ++ax)
    if (!std::isfinite(d.velocity[ax])) return "velocity must be finite";
  if (!std::isfinite(d.h0)) return "h0 must be finite";
  if (d.integrator < MOLT_INT_DEFAULT || d.integrator > MOLT_INT_RK3) return "unknown integrator";
  if (d.integrator != MOLT_INT_DEFAULT && d.pde == MOLT_PDE_WAVE) return "the wave equation runs leapfrog";
  return "";
}

int64_t axis_n(const Problem& p, int ax) { return ax < p.d.ndim ? p.n[ax] : 1; }

// Geometry of the lines along `ax` in a C-ordered [z][y][x] grid.
LineGeom geom(const Problem& p, int ax) {
  const int64_t nx = axis_n(p, 0), ny = axis_n(p, 1), nz = axis_n(p, 2);
  LineGeom g{};
  if (ax == 0) {
    g.n = int(nx);
    g.nlines = ny * nz;
    g.nlo = ny;
    g.s_lo = nx;
    g.s_hi = nx * ny;
    g.stride = 1;
  } else if (ax == 1) {
    g.n = int(ny);
    g.nlines = nx * nz;
    g.nlo = nx;
    g.s_lo = 1;
    g.s_hi = nx * ny;
    g.stride = nx;
  } else {
    g.n = int(nz);
    g.nlines = nx * ny;
    g.nlo = nx;
    g.s_lo = 1;
    g.s_hi = nx;
    g.stride = nx * ny;
  }
  return g;
}

struct Plan {
  SweepArgs a;
  int grid, block;
  size_t smem;
  int ax = 0;
  bool use_tma = false;
  TmaPlan tma;
};

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Builds the kernel arguments for sum_{p<=P} D_mode^p along `ax` with alpha.
int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
  }
  return sms;
}

// Points per lane for a line of n points: the largest of 16, 8, 4 whose
// tile fits the line exactly (n = 32 * E * nwl, nwl <= 16 warps), else 16
// with masked (ragged) tiles.  FP64 sweeps of grids with few lines (fewer
// than 16 warps per SM at that E; nlines counts the lines of every sweep
// running at the same time) are bound by the latency of their recurrences
// on the FP64 pipe, not by bandwidth, and take a shorter chain per lane:
// two warps per line from 512 points on, and the largest E that still puts
// 3 warps per SM in flight, else the smallest that fits.  Measured FP64 heat
// steps (ms; axes one after another / both at once):
//   256^2:  E=4 0.130/0.095  E=8 0.166/0.089
//   512^2:  E=4 0.345/0.285  E=8 0.301/0.255  E=16 0.337/0.588
//   1024^2: E=8 1.064        E=16 0.996      2048^2: E=8 3.91  E=16 3.68
#ifndef MOLT_PREFER_E
#define MOLT_PREFER_E 16
#endif
#ifndef MOLT_F64_SMALL_E
#define MOLT_F64_SMALL_E 1
#endif
#ifndef MOLT_F64_WARPS_PER_SM
#define MOLT_F64_WARPS_PER_SM 3
#endif
#ifndef MOLT_SMALL_TILE_THREADS
#define MOLT_SMALL_TILE_THREADS 256
#endif
constexpr int kSmallTileThreads = MOLT_SMALL_TILE_THREADS;

int choose_E(int n, bool f64, long long nlines) {
  auto fits = [n](int E) { return n % (32 * E) == 0 && n / (32 * E) <= kMaxThreads / 32; };
  static const int kOrder[4] = {MOLT_PREFER_E, 16, 8, 4};
  int first = 0;
  for (int i = 0; i < 4 && !first; ++i)
    if (fits(kOrder[i])) first = kOrder[i];
  if (!first) return kE;
  const long long sms = device_sms();
  if (f64 && MOLT_F64_SMALL_E && nlines * (n / (32 * first)) < 16 * sms) {
    int smallest = 0;
    for (int E : {16, 8, 4}) {
      if (!fits(E) || (n >= 512 && n / (32 * E) < 2)) continue;
      smallest = E;
      if (nlines * (n / (32 * E)) >= (long long)MOLT_F64_WARPS_PER_SM * sms) return E;
    }
    if (smallest) return smallest;
  }
  return first;
}

// E = 0: the planner chooses E and, for grids with few lines, fewer lines per
// CTA so that at least two CTAs per SM are launched.  E != 0: that E and the
// full-CTA tile shape (the batched kernel's tiles).
molt_status plan_axis(molt_ctx* c, const Problem& p, int ax, int mode, int P, double alpha, Plan* out,
                      int E = 0, int concurrent_sweeps = 1) {
  SweepArgs& a = out->a;
  std::memset(&a, 0, sizeof(a));
  out->ax = ax;
  out->use_tma = false;
  a.g = geom(p, ax);
  const int n = a.g.n;
  const bool auto_shape = E == 0;
  if (auto_shape) E = choose_E(n, compute_bytes(p.d) == 8, a.g.nlines * concurrent_sweeps);
  a.E = E;
  a.bc = p.d.bc[ax];
  a.mode = mode;
  a.P = P;
  a.contiguous = a.g.stride == 1;
  a.alpha = alpha;
  const double h = p.h[ax];
  const double nu = alpha * h;
  if (!(nu > 0) || !std::isfinite(nu)) return fail(c, MOLT_EINVAL, "alpha*h must be positive and finite");
  QuadTable qt;
  if (!build_quadrature(p.d.quad_points, nu, &qt)) return fail(c, MOLT_EINVAL, "quadrature table construction failed");
  const int N = a.bc == MOLT_BC_PERIODIC ? n : n - 1;  // intervals
  set_line_constants(a, qt, N, E, compute_bytes(p.d) == 4);
  if (mode == MODE_RL) {
    a.ham = p.d.hamiltonian;
    a.vel = p.d.velocity[ax];
    a.velf = float(a.vel);
    a.h0 = p.d.h0;
    for (int d = 0; d < p.d.ndim; ++d) a.vmax = std::max(a.vmax, std::fabs(p.d.velocity[d]) / p.h[d]);
    a.two_out = a.ham == MOLT_H_AFFINE_SQ ? 1 : 0;
  }
  if (a.g.nlines >= (1LL << 31)) return fail(c, MOLT_EUNSUPPORTED, "more than 2^31 lines along an axis");
  // tile shape: nwl warps per line, W lines per CTA, <= kMaxThreads threads
  const int nwl = (n + 32 * E - 1) / (32 * E);
  if (nwl > kMaxThreads / 32) return fail(c, MOLT_EUNSUPPORTED, "line longer than 8192 points");
  // contiguous lines: tiles of at most kSmallTileThreads threads where a line
  // fits in them, so the register-heavy sweeps (128 per thread) keep two CTAs
  // per SM and one computes while the other waits at a barrier (strided lines
  // keep the wider tiles: their W lines are the width of every row they read)
  const int tmax =
      (auto_shape && a.contiguous && nwl * 32 <= kSmallTileThreads) ? kSmallTileThreads : kMaxThreads;
  int W = (tmax / 32) / nwl;
  int Wp = 1;
  while (Wp * 2 <= W) Wp *= 2;
  W = Wp;
  while (W > 1 && (long long)W / 2 >= a.g.nlines) W /= 2;
  if (auto_shape)
    while (W > 1 && (a.g.nlines + W - 1) / W < 2LL * device_sms()) W /= 2;
  const int cap = nwl * 32 * E;
  int LS = (E == 16 ? phys<16>(cap + 3) : (E == 8 ? phys<8>(cap + 3) : phys<4>(cap + 3))) + 1;
  LS = (LS + 31) / 32 * 32 + (W < 32 ? 32 / W : 1);
  a.W = W;
  a.nwl = nwl;
  a.LS = LS;
  const size_t tb = compute_bytes(p.d);
  size_t off = (size_t(4 * W) * 8 + size_t(W * nwl * 4) * tb + 15) & ~size_t(15);
  out->smem = off + size_t(W) * LS * tb;
  if (a.two_out) out->smem += 16 + size_t(W) * LS * tb;   // second line buffer (carve order)
  if (p.d.weights == MOLT_W_LEARNED) {
    if (!c->mlp_ready) return fail(c, MOLT_EINVAL, "learned weights: call molt_set_mlp first");
    out->smem += learned_extra_bytes(W, LS);
    a.mlp = static_cast<const MlpBlob*>(c->mlp_blob);
    a.mlp_stats = c->mlp_stats;
  }
  if (out->smem > kSmemTileBudget) return fail(c, MOLT_EUNSUPPORTED, "tile does not fit in shared memory");
  out->block = 32 * nwl * W;
  out->grid = int((a.g.nlines + W - 1) / W);
  a.status = c->status_dev;
  return MOLT_OK;
}

// Chooses the persistent TMA kernel when the line is an exact fit and the
// array geometry meets the tensor-copy alignment rules (16-byte global
// strides, a 16-byte multiple of bytes in the innermost box dimension, tiles
// that do not straddle rows); otherwise the plain kernel runs.
void plan_tma(const Problem& p, int ax, const void* in, size_t in_bytes, Plan* pl) {
  pl->use_tma = false;
  SweepArgs& a = pl->a;
  if (!exact_fit(a)) return;
  if (plan_E(a) != kE) return;   // the TMA kernel runs 16 points per lane
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return;
  if (reinterpret_cast<uintptr_t>(in) & 15) return;
  const int64_t nx = axis_n(p, 0), ny = axis_n(p, 1), nz = axis_n(p, 2);
  if ((nx * int64_t(in_bytes)) % 16 != 0) return;
  const int n = a.g.n;
  TmaGeom tg{};
  tg.box_p = n < 256 ? n : 256;
  if (n % tg.box_p != 0 || (tg.box_p & (tg.box_p - 1)) != 0) return;
  tg.nbox = n / tg.box_p;
  tg.nx = int(nx);
  const int W = a.W;
  CUtensorMap map;
  const CUtensorMapDataType dt = in_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r;
  if (ax == 0) {
    tg.kind = 0;
    cuuint64_t dims[2] = {cuuint64_t(nx), cuuint64_t(ny * nz)};
    cuuint64_t strides[1] = {cuuint64_t(nx * in_bytes)};
    cuuint32_t box[2] = {cuuint32_t(tg.box_p), cuuint32_t(W)};
    r = enc(&map, dt, 2, const_cast<void*>(in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    // boxes of bw >= W columns starting on a 16-byte boundary (tiles of
    // fewer than 16 bytes of lines load a wider box and use part of it)
    tg.xalign = int(16 / in_bytes);
    if (nx % W != 0) return;
    if (W < tg.xalign) {
      if (nx % tg.xalign != 0) return;
      tg.bw = tg.xalign;
    } else {
      if (W % tg.xalign != 0) return;
      tg.bw = W;
    }
    tg.kind = ax == 1 ? 1 : 2;
    cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(nz)};
    cuuint64_t strides[2] = {cuuint64_t(nx * in_bytes), cuuint64_t(nx * ny * in_bytes)};
    cuuint32_t box[3] = {cuuint32_t(tg.bw), ax == 1 ? cuuint32_t(tg.box_p) : 1u, ax == 2 ? cuuint32_t(tg.box_p) : 1u};
    r = enc(&map, dt, 3, const_cast<void*>(in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return;
  tg.tx_bytes = unsigned(size_t(tg.nbox) * tg.box_p * (tg.kind == 0 ? W : tg.bw) * in_bytes);
  const size_t bar_off = (pl->smem + 15) & ~size_t(15);
  const size_t stage_off = (bar_off + 16 + 127) & ~size_t(127);
  const size_t total = stage_off + size_t(tg.tx_bytes);
  if (total > kSmemOptIn) return;
  pl->tma.tg = tg;
  pl->tma.map = map;
  pl->tma.smem = total;
  pl->use_tma = true;
}

#define TMA (pl.use_tma ? &pl.tma : nullptr)

template <typename T, typename TIN, typename TST>
cudaError_t dispatch_lin(int epi, const Plan& pl, cudaStream_t s) {
  const SweepArgs& a = pl.a;
  switch (epi) {
    case EPI_STORE: return launch_sweep<T, TIN, TST, JQ_LINEAR, EPI_STORE>(a, TMA, pl.grid, pl.block, pl.smem, s);
    case EPI_ACC_SET: return launch_sweep<T, TIN, TST, JQ_LINEAR, EPI_ACC_SET>(a, TMA, pl.grid, pl.block, pl.smem, s);
    case EPI_ACC_ADD: return launch_sweep<T, TIN, TST, JQ_LINEAR, EPI_ACC_ADD>(a, TMA, pl.grid, pl.block, pl.smem, s);
    case EPI_HEAT_FINAL: return launch_sweep<T, TIN, TST, JQ_LINEAR, EPI_HEAT_FINAL>(a, TMA, pl.grid, pl.block, pl.smem, s);
    case EPI_WAVE_FINAL: return launch_sweep<T, TIN, TST, JQ_LINEAR, EPI_WAVE_FINAL>(a, TMA, pl.grid, pl.block, pl.smem, s);
    case EPI_ACC_AXPY: return launch_sweep<T, TIN, TST, JQ_LINEAR, EPI_ACC_AXPY>(a, TMA, pl.grid, pl.block, pl.smem, s);
    default: return cudaErrorNotSupported;
  }
}

template <typename T>
cudaError_t dispatch_same(int jq, int epi, const Plan& pl, cudaStream_t s) {
  const SweepArgs& a = pl.a;
  if (jq == JQ_WENOZ) {
    if (epi == EPI_STORE) return launch_sweep<T, T, T, JQ_WENOZ, EPI_STORE>(a, TMA, pl.grid, pl.block, pl.smem, s);
    if (epi == EPI_HJ_X) return launch_sweep<T, T, T, JQ_WENOZ, EPI_HJ_X>(a, TMA, pl.grid, pl.block, pl.smem, s);
    if (epi == EPI_HJ_Y) return launch_sweep<T, T, T, JQ_WENOZ, EPI_HJ_Y>(a, TMA, pl.grid, pl.block, pl.smem, s);
    if (epi == EPI_HJ_XG) return launch_sweep<T, T, T, JQ_WENOZ, EPI_HJ_XG>(a, TMA, pl.grid, pl.block, pl.smem, s);
    if (epi == EPI_HJ_YG) return launch_sweep<T, T, T, JQ_WENOZ, EPI_HJ_YG>(a, TMA, pl.grid, pl.block, pl.smem, s);
    if (epi == EPI_ACC_AXPY) return launch_sweep<T, T, T, JQ_WENOZ, EPI_ACC_AXPY>(a, TMA, pl.grid, pl.block, pl.smem, s);
    return cudaErrorNotSupported;
  }
  if (jq == JQ_LEARNED) {
    if constexpr (sizeof(T) == 4) {
      if (epi == EPI_STORE) return launch_sweep<T, T, T, JQ_LEARNED, EPI_STORE>(a, nullptr, pl.grid, pl.block, pl.smem, s);
      if (epi == EPI_HJ_X) return launch_sweep<T, T, T, JQ_LEARNED, EPI_HJ_X>(a, nullptr, pl.grid, pl.block, pl.smem, s);
      if (epi == EPI_HJ_Y) return launch_sweep<T, T, T, JQ_LEARNED, EPI_HJ_Y>(a, nullptr, pl.grid, pl.block, pl.smem, s);
    }
    return cudaErrorNotSupported;
  }
  if (epi == EPI_HJ_X) return launch_sweep<T, T, T, JQ_LINEAR, EPI_HJ_X>(a, TMA, pl.grid, pl.block, pl.smem, s);
  if (epi == EPI_HJ_Y) return launch_sweep<T, T, T, JQ_LINEAR, EPI_HJ_Y>(a, TMA, pl.grid, pl.block, pl.smem, s);
  if (epi == EPI_HJ_XG) return launch_sweep<T, T, T, JQ_LINEAR, EPI_HJ_XG>(a, TMA, pl.grid, pl.block, pl.smem, s);
  if (epi == EPI_HJ_YG) return launch_sweep<T, T, T, JQ_LINEAR, EPI_HJ_YG>(a, TMA, pl.grid, pl.block, pl.smem, s);
  return dispatch_lin<T, T, T>(epi, pl, s);
}

int jquad(const molt_desc& d) {
  return d.weights == MOLT_W_WENOZ ? JQ_WENOZ : (d.weights == MOLT_W_LEARNED ? JQ_LEARNED : JQ_LINEAR);
}

// apply_D in mixed precision reads the FP64 array directly; molt_step's
// sweeps read the FP32 copy of the state.
cudaError_t launch(const Problem& p, int epi, const Plan& pl, cudaStream_t s, bool from_state_copy) {
  const int jq = jquad(p.d);
  if (is_f64_sweep(p.d)) return dispatch_same<double>(jq, epi, pl, s);
  if (is_f32_state(p.d)) return dispatch_same<float>(jq, epi, pl, s);
  if (jq == JQ_LEARNED) return cudaErrorNotSupported;
  if (!from_state_copy) {
    if (epi != EPI_STORE) return cudaErrorNotSupported;
    if (jq == JQ_WENOZ)
      return launch_sweep<float, double, double, JQ_WENOZ, EPI_STORE>(pl.a, TMA, pl.grid, pl.block, pl.smem, s);
    return launch_sweep<float, double, double, JQ_LINEAR, EPI_STORE>(pl.a, TMA, pl.grid, pl.block, pl.smem, s);
  }
  if (jq == JQ_WENOZ) return cudaErrorNotSupported;
  return dispatch_lin<float, float, double>(epi, pl, s);
}

// Line-per-lane FP32 sweeps (csrc/sweep_lanes.cuh): FP32 input, linear rule,
// D_0 / D_R / D_L with P <= 2, lines of 16..512 points (multiples of 16) in
// tiles of 32 lines, epilogues STORE (FP32 state), ACC_SET, ACC_ADD,
// ACC_AXPY.  In auto mode they run when a segment's look-back reaches at most
// kLanesAutoDepth segments (nu >= ~0.22 for 16-point segments): below that
// the look-back grows with 1/nu while the scan kernel's cost does not.
constexpr int kLanesAutoDepth = 8;
constexpr double kLanesTailWeight = 1.4901161193847656e-08;   // 2^-26

bool lane_constants(const Problem& p, const Plan& pl, LanesArgs* Lp);

bool plan_lanes(const molt_ctx* c, const Problem& p, int epi, const Plan& pl, bool f32_input, LanesArgs* la,
                CUtensorMap* map) {
  if (c->lanes == 0) return false;
  const SweepArgs& a = pl.a;
  if (compute_bytes(p.d) != 4 || !f32_input || p.d.weights != MOLT_W_LINEAR) return false;
  if (!p.nodes[pl.ax].empty()) return false;
  if (a.mode != MODE_0 && a.mode != MODE_R && a.mode != MODE_L) return false;
  if (a.P < 1 || a.P > 2) return false;
  const bool wave_final = epi == EPI_WAVE_FINAL && is_mixed(p.d) && pl.ax > 0 && a.shadow && a.dst;
  if (epi != EPI_ACC_SET && epi != EPI_ACC_ADD && epi != EPI_ACC_AXPY && !(epi == EPI_STORE && is_f32_state(p.d)) &&
      !wave_final)
    return false;
  const int n = a.g.n;
  if (n % kLE != 0 || n < kLE || n > kLE * kLMaxSeg) return false;
  const void* outp = epi == EPI_STORE ? a.out : (wave_final ? a.dst : a.acc);
  if (!a.in || !outp || ((reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(outp)) & 15)) return false;
  LanesArgs L;
  std::memset(&L, 0, sizeof(L));
  L.n = n;
  L.S = n / kLE;
  L.bc = a.bc;
  L.mode = a.mode;
  L.P = a.P;
  L.in = static_cast<const float*>(a.in);
  L.out = static_cast<float*>(a.out);
  L.acc = static_cast<float*>(a.acc);
  L.coef = float(a.coefS);
  L.status = a.status;
  if (wave_final) {
    L.un = static_cast<const double*>(a.un);
    L.us = static_cast<const double*>(a.us);
    L.dst = static_cast<double*>(a.dst);
    L.dst2 = static_cast<double*>(a.dst2);
    L.shadow = a.shadow;
    L.coefS = a.coefS;
    L.from_rest = a.from_rest;
  }
  // every wait of this kernel normally lasts microseconds (a tile takes a few)
  L.wait_limit = std::min<long long>(c->wait_limit, 200000000LL);
  const int64_t nx = axis_n(p, 0), ny = axis_n(p, 1), nz = axis_n(p, 2);
  std::memset(map, 0, sizeof(*map));
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  if (pl.ax == 0) {
    // boxes of 32 points x 32 lines, 128-byte swizzle (csrc/sweep_lanes.cuh)
    if (a.g.nlines % kLW != 0 || n % 32 != 0) return false;
    L.contiguous = 1;
    L.ntiles = a.g.nlines / kLW;
    cuuint64_t dims[2] = {cuuint64_t(n), cuuint64_t(a.g.nlines)};
    cuuint64_t strides[1] = {cuuint64_t(n) * 4};
    cuuint32_t box[2] = {32u, cuuint32_t(kLW)};
    cuuint32_t estr[2] = {1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(a.in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  } else {
    if (nx % kLW != 0) return false;
    L.contiguous = 0;
    L.kind = pl.ax;
    L.tiles_per_row = nx / kLW;
    L.ntiles = L.tiles_per_row * (pl.ax == 1 ? nz : ny);
    L.s_hi = pl.ax == 1 ? nx * ny : nx;
    L.stride = pl.ax == 1 ? nx : nx * ny;
    L.nbox = n <= 256 ? 1 : 2;
    L.box_p = n / L.nbox;
    cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(nz)};
    cuuint64_t strides[2] = {cuuint64_t(nx * 4), cuuint64_t(nx * ny * 4)};
    cuuint32_t box[3] = {cuuint32_t(kLW), pl.ax == 1 ? cuuint32_t(L.box_p) : 1u, pl.ax == 2 ? cuuint32_t(L.box_p) : 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(a.in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  if (L.ntiles < 1 || L.ntiles >= (1LL << 31)) return false;
  if (!lane_constants(p, pl, &L)) return false;
  if (c->lanes == 1 && L.lb > kLanesAutoDepth) return false;
  *la = L;
  return true;
}

// The FP32 filter taps, decays, FP64 boundary constants and look-back depth
// of a linear-rule line sweep in difference form (L->n, S, bc, mode set).
bool lane_constants(const Problem& p, const Plan& pl, LanesArgs* Lp) {
  LanesArgs& L = *Lp;
  const SweepArgs& a = pl.a;
  const int n = L.n;
  // quadrature weights (FP64) and the FP32 decay the kernel runs
  const double nu = a.alpha * p.h[pl.ax];
  QuadTable qt;
  if (!build_quadrature(p.d.quad_points, nu, &qt)) return false;
  const float q32 = float(qt.q);
  const double lq = std::log(double(q32));
  L.q = q32;
  L.qE = float(std::exp(lq * kLE));
  // first-difference taps b_m, m = -2..2 (c[0..5] are the J_R weights on offsets -3..2)
  const double* cw = qt.c;
  const double b[5] = {cw[0], cw[0] + cw[1], cw[0] + cw[1] + cw[2] + qt.q, -(cw[4] + cw[5]), -cw[5]};
  const double sR = a.mode == MODE_0 ? 0.5 : (a.mode == MODE_R ? 1.0 : 0.0);
  const double sL = a.mode == MODE_0 ? -0.5 : (a.mode == MODE_L ? -1.0 : 0.0);
  for (int i = 0; i < 5; ++i) {
    L.bR[i] = float(sR * b[i]);
    L.bL[i] = float(sL * b[i]);
  }
  // line constants C = kA T_same + kB T_other
  if (a.bc == MOLT_BC_PERIODIC) {
    L.kA = 1.0 / (-std::expm1(lq * n));
    L.kB = 0.0;
  } else if (a.mode == MODE_0) {
    const double N = double(n - 1), mu = std::exp(lq * N);
    const double k = 1.0 / (-std::expm1(2.0 * lq * N)) * std::exp(-lq);
    L.kA = mu < kLanesTailWeight ? 0.0 : mu * k;
    L.kB = -k;
  } else {
    L.kA = 0.0;
    L.kB = 0.0;
  }
  L.needA = L.kA != 0.0;
  L.needB = L.kB != 0.0;
  // look-back depth: segment weights (q^16)^j >= 2^-26
  double w = 1.0;
  int lb = 0;
  const double qE = std::exp(lq * kLE);
  while (lb < L.S && w >= kLanesTailWeight) {
    w *= qE;
    ++lb;
  }
  L.lb = lb;
  return true;
}

// Warp-per-line FP32 sweeps of x lines (csrc/sweep_xlines.cuh): the same
// operations, inputs and epilogues as the line-per-lane kernel's x lines,
// for any number of lines; a line of n = 16 S points takes S lanes.
bool plan_xlines(const molt_ctx* c, const Problem& p, int epi, const Plan& pl, bool f32_input, XLineArgs* xa) {
  if (c->lanes == 0 || c->xlines == 0 || pl.ax != 0) return false;
  const SweepArgs& a = pl.a;
  if (compute_bytes(p.d) != 4 || !f32_input || p.d.weights != MOLT_W_LINEAR) return false;
  if (!p.nodes[pl.ax].empty() || a.g.stride != 1) return false;
  if (a.mode != MODE_0 && a.mode != MODE_R && a.mode != MODE_L) return false;
  if (a.P < 1 || a.P > 2) return false;
  if (epi != EPI_ACC_SET && epi != EPI_ACC_ADD && epi != EPI_ACC_AXPY && !(epi == EPI_STORE && is_f32_state(p.d)))
    return false;
  const int n = a.g.n;
  if (n % kXlSeg != 0 || n < kXlSeg || n > kXlSeg * 32) return false;
  const void* outp = epi == EPI_STORE ? a.out : a.acc;
  if (!a.in || !outp || ((reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(outp)) & 15)) return false;
  LanesArgs L;
  std::memset(&L, 0, sizeof(L));
  L.n = n;
  L.S = n / kXlSeg;
  L.bc = a.bc;
  L.mode = a.mode;
  L.P = a.P;
  if (!lane_constants(p, pl, &L)) return false;
  if (c->lanes == 1 && L.lb > kLanesAutoDepth) return false;
  XLineArgs X;
  std::memset(&X, 0, sizeof(X));
  X.n = n;
  X.S = L.S;
  X.G = (L.S & (L.S - 1)) == 0 ? 32 / L.S : 1;
  X.width = X.G > 1 ? L.S : 32;
  X.nlines = a.g.nlines;
  X.ngroups = (X.nlines + X.G - 1) / X.G;
  X.bc = L.bc;
  X.mode = L.mode;
  X.P = L.P;
  X.lb = L.lb;
  X.needA = L.needA;
  X.needB = L.needB;
  for (int i = 0; i < 5; ++i) {
    X.bR[i] = L.bR[i];
    X.bL[i] = L.bL[i];
  }
  X.q = L.q;
  // Kogge-Stone multipliers (q^16)^(2^k), from the FP32 q the scans run
  double qk = std::pow(double(L.q), double(kXlSeg));
  for (int k = 0; k < 5; ++k, qk *= qk) X.qd[k] = float(qk);
  X.kA = L.kA;
  X.kB = L.kB;
  X.coef = float(a.coefS);
  X.in = static_cast<const float*>(a.in);
  X.out = static_cast<float*>(a.out);
  X.acc = static_cast<float*>(a.acc);
  *xa = X;
  return true;
}

molt_status run_nonuniform(molt_ctx* c, const Problem& p, int epi, const Plan& pl);

// s: the launch stream (nullptr: the context's)
molt_status run(molt_ctx* c, const Problem& p, int epi, Plan& pl, bool from_state_copy = true,
                cudaStream_t s = nullptr) {
  if (!s) s = c->stream;
  if (!p.nodes[pl.ax].empty()) return run_nonuniform(c, p, epi, pl);
  // element size of the sweep input: FP64 except FP32 state or the FP32 copy
  const size_t in_bytes = is_f32_state(p.d) || (is_mixed(p.d) && from_state_copy) ? 4 : 8;
  {
    XLineArgs xa;
    if (plan_xlines(c, p, epi, pl, in_bytes == 4, &xa)) {
      molt_ctx::Rec rec{epi == EPI_STORE ? int(MOLT_KERNEL_XLINES_STORE)
                        : epi == EPI_ACC_SET ? int(MOLT_KERNEL_XLINES_ACC_SET)
                                             : int(MOLT_KERNEL_XLINES_ACC_ADD),
                        nullptr, nullptr};
      if (c->profile) {
        cudaEventCreate(&rec.start);
        cudaEventCreate(&rec.stop);
        cudaEventRecord(rec.start, s);
      }
      const cudaError_t e = launch_xlines(epi, xa, s);
      if (c->profile) {
        cudaEventRecord(rec.stop, s);
        c->recs.push_back(rec);
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "warp-per-line sweep launch");
      return MOLT_OK;
    }
  }
  {
    LanesArgs la;
    CUtensorMap lmap;
    if (plan_lanes(c, p, epi, pl, in_bytes == 4, &la, &lmap)) {
      molt_ctx::Rec rec{epi == EPI_STORE        ? int(MOLT_KERNEL_LANES_STORE)
                        : epi == EPI_ACC_SET    ? int(MOLT_KERNEL_LANES_ACC_SET)
                        : epi == EPI_WAVE_FINAL ? int(MOLT_KERNEL_LANES_WAVE_FINAL)
                                                : int(MOLT_KERNEL_LANES_ACC_ADD),
                        nullptr, nullptr};
      if (c->profile) {
        cudaEventCreate(&rec.start);
        cudaEventCreate(&rec.stop);
        cudaEventRecord(rec.start, s);
      }
      const cudaError_t e = launch_lanes(epi, la, lmap, s);
      if (c->profile) {
        cudaEventRecord(rec.stop, s);
        c->recs.push_back(rec);
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "line-per-lane sweep launch");
      return MOLT_OK;
    }
  }
  if (!c->no_tma && p.d.weights != MOLT_W_LEARNED) plan_tma(p, pl.ax, pl.a.in, in_bytes, &pl);
  // profiling kind: the general Hamilton-Jacobi passes count as HJ_X / HJ_Y
  // (the advection-diffusion accumulations count as ACC_ADD)
  molt_ctx::Rec rec{epi_hj_x(epi) ? int(EPI_HJ_X)
                                   : (epi_hj_y(epi) ? int(EPI_HJ_Y) : (epi == EPI_ACC_AXPY ? int(EPI_ACC_ADD) : epi)),
                    nullptr, nullptr};
  if (c->profile) {
    cudaEventCreate(&rec.start);
    cudaEventCreate(&rec.stop);
    cudaEventRecord(rec.start, s);
  }
  cudaError_t e = launch(p, epi, pl, s, from_state_copy);
  if (c->profile) {
    cudaEventRecord(rec.stop, s);
    c->recs.push_back(rec);
  }
  if (e == cudaErrorNotSupported)
    return fail(c, MOLT_EUNSUPPORTED, "no kernel for this precision/weights/epilogue combination");
  if (e != cudaSuccess) return cuda_fail(c, e, "sweep launch");
  return MOLT_OK;
}

double step_alpha(const Problem& p) {
  const molt_desc& d = p.d;
  if (d.pde == MOLT_PDE_HEAT) return d.beta / std::sqrt(d.diffusivity * d.dt);
  if (d.pde == MOLT_PDE_WAVE) return d.beta / (d.c * d.dt);
  double hmin = p.h[0];
  for (int ax = 1; ax < d.ndim; ++ax) hmin = std::min(hmin, p.h[ax]);
  return d.beta / (d.cfl * hmin);
}

bool hj_transposed_y(molt_ctx* c, const Problem& p);

}  // namespace

namespace {
molt_status apply_D_nonuniform(molt_ctx* c, const Problem& p, int axis, int mode, int P, double alpha,
                               const void* in, void* out, bool io_compute = false);
molt_status transpose(molt_ctx* c, const Problem& p, const void* in, void* out, long long ny, long long nx,
                      size_t elem = 0);
Problem transposed(const Problem& p);

// Sizes and spacings of a validated descriptor (periodic axes: n intervals,
// Dirichlet axes: n - 1).
Problem make_problem(const molt_desc& d) {
  Problem p;
  p.d = d;
  p.total = 1;
  for (int ax = 0; ax < 3; ++ax) {
    p.n[ax] = ax < p.d.ndim ? p.d.n[ax] : 1;
    p.total *= p.n[ax];
    if (ax < p.d.ndim) {
      const int64_t N = p.d.bc[ax] == MOLT_BC_PERIODIC ? p.n[ax] : p.n[ax] - 1;
      p.h[ax] = (p.d.hi[ax] - p.d.lo[ax]) / double(N);
    } else {
      p.h[ax] = 1.0;
    }
  }
  return p;
}
}  // namespace

extern "C" {

molt_status molt_create(const molt_desc* descs, int count, void* cuda_stream, molt_ctx** out) {
  if (!descs || count < 1 || !out) return fail(nullptr, MOLT_EINVAL, "null descriptor/out or count < 1");
  *out = nullptr;
  molt_ctx* c = new molt_ctx();
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < count; ++i) {
    const std::string v = validate(descs[i]);
    if (!v.empty()) {
      delete c;
      return fail(nullptr, MOLT_EINVAL, "problem " + std::to_string(i) + ": " + v);
    }
    Problem p = make_problem(descs[i]);
    if (p.d.pde == MOLT_PDE_HJ) {
      for (int ax = 0; ax < p.d.ndim; ++ax)
        if (p.d.bc[ax] != MOLT_BC_PERIODIC) {
          delete c;
          return fail(nullptr, MOLT_EUNSUPPORTED, "Hamilton-Jacobi needs periodic axes");
        }
      if (p.d.ndim > 2) {
        delete c;
        return fail(nullptr, MOLT_EUNSUPPORTED, "Hamilton-Jacobi runs in 1-D and 2-D");
      }
      if (p.d.prec == MOLT_PREC_F32_F64UPDATE) {
        delete c;
        return fail(nullptr, MOLT_EUNSUPPORTED, "Hamilton-Jacobi runs in MOLT_PREC_F32 or MOLT_PREC_F64");
      }
      if (!(p.d.cfl > 0)) {
        delete c;
        return fail(nullptr, MOLT_EINVAL, "cfl must be positive");
      }
    }
    if (p.d.weights == MOLT_W_LEARNED && p.d.prec != MOLT_PREC_F32) {
      delete c;
      return fail(nullptr, MOLT_EUNSUPPORTED, "learned weights run with MOLT_PREC_F32");
    }
    if (p.d.weights == MOLT_W_LEARNED && p.d.hamiltonian != MOLT_H_HALF_SQ) {
      delete c;
      return fail(nullptr, MOLT_EUNSUPPORTED, "learned weights run with H = |grad u|^2/2");
    }
    if (p.d.pde == MOLT_PDE_ADVDIFF) {
      std::string why;
      for (int ax = 0; ax < p.d.ndim; ++ax)
        if (p.d.bc[ax] != MOLT_BC_PERIODIC) why = "advection-diffusion needs periodic axes";
      if (!(p.d.c > 0) || !std::isfinite(p.d.c)) why = "advection-diffusion needs the splitting bound c > 0";
      if (!(p.d.diffusivity >= 0) || !std::isfinite(p.d.diffusivity)) why = "diffusivity must be >= 0";
      if (p.d.weights == MOLT_W_LEARNED || (p.d.weights == MOLT_W_WENOZ && is_mixed(p.d)))
        why = "advection-diffusion runs linear weights, or WENO-Z in MOLT_PREC_F64 / MOLT_PREC_F32";
      if (!why.empty()) {
        delete c;
        return fail(nullptr, MOLT_EUNSUPPORTED, why);
      }
    }
    c->probs.push_back(p);
  }
  cudaError_t e;
  if ((e = cudaMalloc(&c->status_dev, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&c->speed_dev, sizeof(unsigned long long) * 2 * count)) != cudaSuccess ||
      (e = cudaMalloc(&c->t_dev, sizeof(double) * count)) != cudaSuccess ||
      (e = cudaMalloc(&c->tnow_dev, sizeof(double) * count)) != cudaSuccess) {
    molt_destroy(c);
    return fail(nullptr, MOLT_ENOMEM, std::string("workspace: ") + cudaGetErrorString(e));
  }
  cudaMemset(c->status_dev, 0, sizeof(int));
  cudaMemset(c->speed_dev, 0, sizeof(unsigned long long) * 2 * count);
  bool learned = false;
  for (const auto& p : c->probs) learned = learned || p.d.weights == MOLT_W_LEARNED;
  if (learned) {
    if ((e = cudaMalloc(&c->mlp_blob, sizeof(MlpBlob))) != cudaSuccess ||
        (e = cudaMalloc(&c->mlp_stats, 2 * sizeof(unsigned long long))) != cudaSuccess) {
      molt_destroy(c);
      return fail(nullptr, MOLT_ENOMEM, std::string("network workspace: ") + cudaGetErrorString(e));
    }
    cudaMemset(c->mlp_stats, 0, 2 * sizeof(unsigned long long));
  }
  for (auto& p : c->probs) {
    const size_t cb = compute_bytes(p.d), sb = state_bytes(p.d);
    const size_t tot = size_t(p.total);
    bool ok = true;
    if ((p.d.ndim > 1 || is_mixed(p.d) || p.d.pde == MOLT_PDE_ADVDIFF) && p.d.pde != MOLT_PDE_HJ)
      ok = ok && cudaMalloc(&p.acc, cb * tot) == cudaSuccess;
    if (p.d.pde == MOLT_PDE_ADVDIFF) {
      ok = ok && cudaMalloc(&p.gp, cb * tot) == cudaSuccess && cudaMalloc(&p.gm, cb * tot) == cudaSuccess;
      if (p.d.integrator != MOLT_INT_EULER)
        ok = ok && cudaMalloc(&p.stage1, sb * tot) == cudaSuccess && cudaMalloc(&p.stage2, sb * tot) == cudaSuccess;
    }
    if (p.d.pde == MOLT_PDE_HEAT && p.d.integrator != MOLT_INT_EULER) {
      ok = ok && cudaMalloc(&p.stage1, sb * tot) == cudaSuccess;
      ok = ok && cudaMalloc(&p.stage2, sb * tot) == cudaSuccess;
    }
    if (p.d.pde == MOLT_PDE_HJ && p.d.ndim > 1) ok = ok && cudaMalloc(&p.hx, sb * tot) == cudaSuccess;
    if (p.d.pde == MOLT_PDE_HJ && p.d.ndim > 1 && p.d.hamiltonian == MOLT_H_AFFINE_SQ)
      ok = ok && cudaMalloc(&p.hx2, sb * tot) == cudaSuccess;
    if (p.d.pde == MOLT_PDE_HJ && p.d.integrator == MOLT_INT_RK3) {
      for (int k = 0; k < 2 * p.d.ndim; ++k) ok = ok && cudaMalloc(&p.hv[k], sb * tot) == cudaSuccess;
      ok = ok && cudaMalloc(&p.stage1, sb * tot) == cudaSuccess && cudaMalloc(&p.stage2, sb * tot) == cudaSuccess;
    }
    if (ok && hj_transposed_y(c, p)) {
      ok = cudaMalloc(&p.tu, sb * tot) == cudaSuccess && cudaMalloc(&p.thx, sb * tot) == cudaSuccess;
    }
    if (is_mixed(p.d) && p.d.pde != MOLT_PDE_HJ) ok = ok && cudaMalloc(&p.shadow, 4 * tot) == cudaSuccess;
    if (p.d.pde == MOLT_PDE_HEAT && p.d.ndim > 1 && p.total <= kAxisStreamsMaxPoints)
      ok = ok && cudaMalloc(&p.acc2, cb * tot) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      molt_destroy(c);
      return fail(nullptr, MOLT_ENOMEM, "workspace allocation failed");
    }
  }
  bool any_acc2 = false;
  for (const auto& p : c->probs) any_acc2 = any_acc2 || p.acc2;
  if (any_acc2 && ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess ||
                   (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
                   (e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess)) {
    molt_destroy(c);
    return fail(nullptr, MOLT_ECUDA, std::string("side stream: ") + cudaGetErrorString(e));
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    molt_destroy(c);
    return fail(nullptr, MOLT_ECUDA, std::string("create: ") + cudaGetErrorString(e));
  }
  *out = c;
  return MOLT_OK;
}

molt_status molt_apply_D(molt_ctx* c, int problem, int axis, int op, int P, double alpha, const void* in,
                         void* out) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (problem < 0 || problem >= int(c->probs.size())) return fail(c, MOLT_EINVAL, "problem index out of range");
  const Problem& p = c->probs[problem];
  if (axis < 0 || axis >= p.d.ndim) return fail(c, MOLT_EINVAL, "axis out of range");
  if (op != MOLT_OP_L && op != MOLT_OP_R && op != MOLT_OP_0) return fail(c, MOLT_EINVAL, "unknown op");
  if (P < 1 || P > 64) return fail(c, MOLT_EINVAL, "P must be in 1..64");
  if (!in || !out) return fail(c, MOLT_EINVAL, "null array");
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15)
    return fail(c, MOLT_EINVAL, "arrays must be 16-byte aligned");
  const int mode = op == MOLT_OP_L ? MODE_L : (op == MOLT_OP_R ? MODE_R : MODE_0);
  if (!p.nodes[axis].empty()) return apply_D_nonuniform(c, c->probs[problem], axis, mode, P, alpha, in, out);
  Plan pl;
  molt_status st = plan_axis(c, p, axis, mode, P, alpha, &pl);
  if (st != MOLT_OK) return st;
  // in == out is safe: every CTA reads its whole lines before writing them
  pl.a.in = in;
  pl.a.out = out;
  return run(c, p, EPI_STORE, pl, false);
}

molt_status molt_plan_sweep(const molt_desc* d, int axis, int op, int P, double alpha, molt_sweep_plan* out) {
  if (!d || !out) return fail(nullptr, MOLT_EINVAL, "null descriptor or plan");
  const std::string v = validate(*d);
  if (!v.empty()) return fail(nullptr, MOLT_EINVAL, v);
  if (axis < 0 || axis >= d->ndim) return fail(nullptr, MOLT_EINVAL, "axis out of range");
  if (op != MOLT_OP_L && op != MOLT_OP_R && op != MOLT_OP_0) return fail(nullptr, MOLT_EINVAL, "unknown op");
  if (P < 1 || P > 64) return fail(nullptr, MOLT_EINVAL, "P must be in 1..64");
  if (d->weights == MOLT_W_LEARNED)
    return fail(nullptr, MOLT_EUNSUPPORTED, "learned sweeps are planned with their network");
  const Problem p = make_problem(*d);
  molt_ctx host;                 // planning reads no device state
  Plan pl;
  const int mode = op == MOLT_OP_L ? MODE_L : (op == MOLT_OP_R ? MODE_R : MODE_0);
  const molt_status st = plan_axis(&host, p, axis, mode, P, alpha, &pl);
  if (st != MOLT_OK) return fail(nullptr, st, host.err);
  out->points_per_lane = pl.a.E;
  out->warps_per_line = pl.a.nwl;
  out->lines_per_cta = pl.a.W;
  out->threads_per_cta = pl.block;
  out->ctas = pl.grid;
  out->smem_bytes = int64_t(pl.smem);
  out->exact_fit = exact_fit(pl.a) ? 1 : 0;
  out->reserved = 0;
  return MOLT_OK;
}

}  // extern "C"

namespace {

// FP32 copy of an FP64 state (integer-pattern conversion, grid-stride, four
// points per thread with their loads issued first).
__global__ void shadow_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    double v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k * stride < n) v[k] = in[i0 + k * stride];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k * stride < n) out[i0 + k * stride] = d2f(v[k]);
  }
}

// FP64 state updates of the FP32-sweep (mixed) forms, as streaming kernels:
// every warp of the GPU can overlap their loads, stores and FP64 FMAs, which
// the sweep kernel's epilogue (one CTA per SM, after its scans) cannot.
//   heat:  u_s = a0 u^n + a1 (u_{s-1} + coefS * acc)       (SSP-RK3 stage)
//   wave:  u^{n+1} = 2u^n - u^{n-1} + coefS * acc          (leapfrog)
//          from rest: u^1 = u^0 + coefS/2 * acc            (Taylor start)
// acc holds sum_d S_{P,d} of the stage input in FP32.  Each also refreshes
// the FP32 copy the next sweeps read and flags non-finite values.
#ifndef MOLT_UPD_PER
#define MOLT_UPD_PER 8
#endif
#ifndef MOLT_UPD_BLOCKS_PER_SM
#define MOLT_UPD_BLOCKS_PER_SM 8
#endif
constexpr int kUpdPer = MOLT_UPD_PER;   // points per thread and iteration; their loads are issued first

__global__ void heat_update_kernel(const float* __restrict__ acc, const double* un, const double* us, double* dst,
                                   float* __restrict__ shadow, double a0, double a1, double coefS, long long n,
                                   int* status) {
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kUpdPer) {
    double x[kUpdPer], y[kUpdPer];
    float w[kUpdPer];
#pragma unroll
    for (int k = 0; k < kUpdPer; ++k) {
      const long long i = i0 + k * stride;
      if (i < n) {
        x[k] = un[i];
        y[k] = us[i];
        w[k] = acc[i];
      }
    }
#pragma unroll
    for (int k = 0; k < kUpdPer; ++k) {
      const long long i = i0 + k * stride;
      if (i < n) {
        const double r = fma(a0, x[k], a1 * fma(coefS, f2d(w[k]), y[k]));
        dst[i] = r;
        shadow[i] = d2f(r);
        bad |= nonfinite(r);
      }
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

__global__ void wave_update_kernel(const float* __restrict__ acc, const double* un, const double* uprev,
                                   double* dst, double* dst2, float* __restrict__ shadow, double coefS,
                                   int from_rest, long long n, int* status) {
  bool bad = false;
  const double half = 0.5 * coefS;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kUpdPer) {
    double x[kUpdPer], y[kUpdPer];
    float w[kUpdPer];
#pragma unroll
    for (int k = 0; k < kUpdPer; ++k) {
      const long long i = i0 + k * stride;
      if (i < n) {
        x[k] = un[i];
        y[k] = from_rest ? 0.0 : uprev[i];
        w[k] = acc[i];
      }
    }
#pragma unroll
    for (int k = 0; k < kUpdPer; ++k) {
      const long long i = i0 + k * stride;
      if (i < n) {
        const double wd = f2d(w[k]);
        const double r = from_rest ? fma(half, wd, x[k]) : fma(coefS, wd, fma(2.0, x[k], -y[k]));
        if (dst2) dst2[i] = x[k];
        dst[i] = r;
        shadow[i] = d2f(r);
        bad |= nonfinite(r);
      }
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

int stream_grid(long long n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + 255) / 256;
  if (blocks > (long long)MOLT_UPD_BLOCKS_PER_SM * sms) blocks = (long long)MOLT_UPD_BLOCKS_PER_SM * sms;
  return int(blocks < 1 ? 1 : blocks);
}

molt_status record_begin(molt_ctx* c, molt_ctx::Rec* rec, int kind) {
  rec->kind = kind;
  rec->start = rec->stop = nullptr;
  if (c->profile) {
    cudaEventCreate(&rec->start);
    cudaEventCreate(&rec->stop);
    cudaEventRecord(rec->start, c->stream);
  }
  return MOLT_OK;
}

void record_end(molt_ctx* c, molt_ctx::Rec* rec) {
  if (c->profile) {
    cudaEventRecord(rec->stop, c->stream);
    c->recs.push_back(*rec);
  }
}

// sum_{p<=P} D^p along a non-uniform axis, periodic or Dirichlet (point-local
// weights).
// io_compute: in and out hold the compute type (molt_step's FP32 copy and
// axis sums), else the state type (molt_apply_D).
molt_status apply_D_nonuniform(molt_ctx* c, const Problem& p, int axis, int mode, int P, double alpha, const void* in,
                               void* out, bool io_compute) {
  if (p.d.weights == MOLT_W_LEARNED) return fail(c, MOLT_EUNSUPPORTED, "non-uniform axes run linear or WENO-Z weights");
  if (!(alpha > 0) || !std::isfinite(alpha)) return fail(c, MOLT_EINVAL, "alpha must be positive and finite");
  const std::vector<double>& x = p.nodes[axis];
  const int n = int(x.size());
  const bool dir = p.d.bc[axis] == MOLT_BC_DIRICHLET;
  const double L = dir ? 0.0 : p.d.hi[axis] - p.d.lo[axis];   // 0: the tables of a Dirichlet line
  const bool f64 = is_f64_sweep(p.d);
  const bool weno = p.d.weights == MOLT_W_WENOZ;
  const size_t slots = weno ? size_t(kNuWeno) : 6;
  const size_t tb = f64 ? 8 : 4;
  Problem::NuCache& cch = p.nu[axis];
  const size_t io_bytes = io_compute ? compute_bytes(p.d) : state_bytes(p.d);
  cudaError_t e;
  if (!cch.dev || cch.alpha != alpha || cch.npts != p.d.quad_points || cch.weights != int(p.d.weights)) {
    std::vector<double> cR, cL, q;
    build_nonuniform_tables(x, L, alpha, p.d.quad_points, &cR, &cL, &q);
    if (weno) build_nonuniform_weno_tables(x, L, alpha, &cR, &cL);
    std::vector<double> all(cR);
    all.insert(all.end(), cL.begin(), cL.end());
    all.insert(all.end(), q.begin(), q.end());
    if (all.size() != (2 * slots + 1) * size_t(n)) return fail(c, MOLT_EINVAL, "non-uniform table size");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "table sync");
    if (cch.dev && cch.count < all.size()) {
      cudaFree(cch.dev);
      cch.dev = nullptr;
    }
    if (!cch.dev) {
      if ((e = cudaMalloc(&cch.dev, all.size() * tb)) != cudaSuccess) {
        cudaGetLastError();
        cch.dev = nullptr;
        cch.count = 0;
        return fail(c, MOLT_ENOMEM, "non-uniform tables");
      }
      cch.count = all.size();
    }
    cch.weights = -1;            // invalid until the upload completes
    if (f64) {
      e = cudaMemcpy(cch.dev, all.data(), all.size() * 8, cudaMemcpyHostToDevice);
    } else {
      std::vector<float> f(all.begin(), all.end());
      e = cudaMemcpy(cch.dev, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "table upload");
    cch.alpha = alpha;
    cch.npts = p.d.quad_points;
    cch.weights = int(p.d.weights);
  }
  // y lines of a 2-D grid run on the transposed array, where they are rows
  // (the sweep reads and writes each strided line with one sector per point)
  const bool trans = p.d.ndim == 2 && axis == 1;
  const long long nx = p.n[0], ny = p.n[1];
  const void* kin = in;
  void* kout = out;
  if (trans) {
    for (void*& t : p.nu_tmp)
      if (!t && cudaMalloc(&t, state_bytes(p.d) * size_t(p.total)) != cudaSuccess) {
        cudaGetLastError();
        t = nullptr;
        return fail(c, MOLT_ENOMEM, "non-uniform transposed copies");
      }
    molt_status st = transpose(c, p, in, p.nu_tmp[0], ny, nx, io_bytes);
    if (st != MOLT_OK) return st;
    kin = p.nu_tmp[0];
    kout = p.nu_tmp[1];
  }
  NuArgs a{};
  a.g = trans ? geom(transposed(p), 0) : geom(p, axis);
  a.mode = mode;
  a.P = P;
  a.bc = dir ? 1 : 0;
  if (dir) {
    const double w = x[size_t(n - 1)] - x[0];
    a.mu = std::exp(-alpha * w);
    a.kdir = 2.0 / (-std::expm1(-2.0 * alpha * w));
  } else {
    a.inv1mmu = 1.0 / (-std::expm1(-alpha * L));
  }
  a.in = kin;
  a.out = kout;
  a.status = c->status_dev;
  // one CTA per line, its scan positions split between up to 16 warps (at
  // most 512 each: the kernel keeps a segment's local integrals in registers)
  const int nw = std::max(1, (n + 511) / 512);
  if (nw > 16) return fail(c, MOLT_EUNSUPPORTED, "non-uniform line longer than 8192 points");
  const size_t smem = (size_t(2 * n + 6) + size_t(2 * nw)) * tb;
  if (smem > kSmemTileBudget) return fail(c, MOLT_EUNSUPPORTED, "non-uniform line too long for shared memory");
  if (a.g.nlines >= (1LL << 31)) return fail(c, MOLT_EUNSUPPORTED, "more than 2^31 lines along an axis");
  const long long blocks = a.g.nlines;
  const int warps = nw;
  molt_ctx::Rec rec;
  record_begin(c, &rec, MOLT_KERNEL_STORE);
  auto launch = [&](auto kernel, auto tables) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemOptIn));
    kernel<<<unsigned(blocks), 32 * warps, smem, c->stream>>>(a, tables);
  };
  if (f64) {
    const double* d = static_cast<const double*>(cch.dev);
    NuTables<double> t{d, d + slots * n, d + 2 * slots * n};
    if (weno) launch(nonuniform_kernel<double, double, true>, t);
    else launch(nonuniform_kernel<double, double, false>, t);
  } else {
    const float* d = static_cast<const float*>(cch.dev);
    NuTables<float> t{d, d + slots * n, d + 2 * slots * n};
    if (io_bytes == 4) {
      if (weno) launch(nonuniform_kernel<float, float, true>, t);
      else launch(nonuniform_kernel<float, float, false>, t);
    } else {
      if (weno) launch(nonuniform_kernel<float, double, true>, t);
      else launch(nonuniform_kernel<float, double, false>, t);
    }
  }
  record_end(c, &rec);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "non-uniform sweep");
  return trans ? transpose(c, p, p.nu_tmp[1], out, nx, ny, io_bytes) : MOLT_OK;
}

// A sweep's epilogue applied point by point to axis sums that another kernel
// wrote (the non-uniform axes of molt_step): the arithmetic of the fused
// epilogues, with S[i] in the compute type and the natural layout.
template <typename T, typename TST, int EPI>
__global__ void point_epilogue_kernel(const SweepArgs a, const T* __restrict__ S, long long n) {
  const Epilogue<T, TST, EPI> ep{a, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const EpiOps<T, TST> o = ep.load(i);
    ep.store(i, S[i], o);
  }
}

template <typename T, typename TST>
cudaError_t launch_point_epilogue(int epi, const SweepArgs& a, const void* S, long long n, cudaStream_t s) {
  const T* sp = static_cast<const T*>(S);
  const int g = stream_grid(n);
  switch (epi) {
    case EPI_ACC_SET: point_epilogue_kernel<T, TST, EPI_ACC_SET><<<g, 256, 0, s>>>(a, sp, n); break;
    case EPI_ACC_ADD: point_epilogue_kernel<T, TST, EPI_ACC_ADD><<<g, 256, 0, s>>>(a, sp, n); break;
    case EPI_ACC_AXPY: point_epilogue_kernel<T, TST, EPI_ACC_AXPY><<<g, 256, 0, s>>>(a, sp, n); break;
    case EPI_HEAT_FINAL: point_epilogue_kernel<T, TST, EPI_HEAT_FINAL><<<g, 256, 0, s>>>(a, sp, n); break;
    case EPI_WAVE_FINAL: point_epilogue_kernel<T, TST, EPI_WAVE_FINAL><<<g, 256, 0, s>>>(a, sp, n); break;
    default: return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}

// One axis of a heat, wave or advection-diffusion step along a non-uniform
// axis: S = sum_{p<=P} D^p of the planned operator into the problem's sum
// buffer by the non-uniform sweep, then the planned epilogue point by point
// (EPI_STORE: S into the output array).
molt_status run_nonuniform(molt_ctx* c, const Problem& p, int epi, const Plan& pl) {
  // S straight into the output array (the one-sided sums of the generic
  // Hamilton-Jacobi step), in the state type
  if (epi == EPI_STORE) return apply_D_nonuniform(c, p, pl.ax, pl.a.mode, pl.a.P, pl.a.alpha, pl.a.in, pl.a.out);
  if (epi != EPI_ACC_SET && epi != EPI_ACC_ADD && epi != EPI_ACC_AXPY && epi != EPI_HEAT_FINAL &&
      epi != EPI_WAVE_FINAL)
    return fail(c, MOLT_EUNSUPPORTED, "non-uniform axes run heat, wave, advection-diffusion and Hamilton-Jacobi steps");
  if (!p.nu_sum) return fail(c, MOLT_EINVAL, "non-uniform axis without its sum buffer");
  molt_status st = apply_D_nonuniform(c, p, pl.ax, pl.a.mode, pl.a.P, pl.a.alpha, pl.a.in, p.nu_sum, true);
  if (st != MOLT_OK) return st;
  molt_ctx::Rec rec;
  record_begin(c, &rec, epi == EPI_ACC_AXPY ? int(MOLT_KERNEL_ACC_ADD) : epi);
  cudaError_t e;
  if (is_f64_sweep(p.d))
    e = launch_point_epilogue<double, double>(epi, pl.a, p.nu_sum, p.total, c->stream);
  else if (is_f32_state(p.d))
    e = launch_point_epilogue<float, float>(epi, pl.a, p.nu_sum, p.total, c->stream);
  else
    e = launch_point_epilogue<float, double>(epi, pl.a, p.nu_sum, p.total, c->stream);
  record_end(c, &rec);
  if (e != cudaSuccess) return cuda_fail(c, e, "non-uniform step epilogue");
  return MOLT_OK;
}


molt_status refresh_shadow(molt_ctx* c, Problem& p, const void* u) {
  if (!p.shadow) return MOLT_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long n = p.total;
  long long blocks = (n + 255) / 256;
  if (blocks > 8LL * sms) blocks = 8LL * sms;
  shadow_kernel<<<int(blocks), 256, 0, c->stream>>>(static_cast<const double*>(u), p.shadow, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MOLT_OK : cuda_fail(c, e, "state copy");
}

// Sweep input of molt_step: the FP32 copy in mixed precision, else the state.
const void* sweep_input(const Problem& p, const void* state) { return p.shadow ? p.shadow : state; }

// Runge-Kutta stage of a heat step whose axis sums sit in two accumulators
// (x in acc, y and z in acc2): dst = a0 u^n + a1 (u_s + coefS (acc + acc2)),
// the arithmetic of the fused last-axis epilogue (acc + S in the compute
// type first); FP32 copy for mixed precision.
template <typename TC, typename TS>
__global__ void heat_update2_kernel(const TC* __restrict__ acc, const TC* __restrict__ acc2, const TS* un,
                                    const TS* us, TS* dst, float* __restrict__ shadow, double a0, double a1,
                                    double coefS, long long n, int* status) {
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const TC tot = acc[i] + acc2[i];
    const TS r = fma(TS(a0), un[i], TS(a1) * fma(TS(coefS), cvt<TS>(tot), us[i]));
    dst[i] = r;
    if (shadow) shadow[i] = cvt<float>(r);
    bad |= nonfinite(r);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

bool heat_axis_streams(const molt_ctx* c, const Problem& p) {
  if (!c->axis_streams || !c->side || !p.acc2) return false;
  for (int ax = 0; ax < p.d.ndim; ++ax)
    if (!p.nodes[ax].empty()) return false;
  return true;
}

molt_status heat_step_axis_streams(molt_ctx* c, Problem& p, void* u) {
  const double alpha = step_alpha(p);
  const double coefS = -p.d.beta * p.d.beta;
  static const double rk[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  const bool euler = p.d.integrator == MOLT_INT_EULER;
  void* ins[3] = {u, p.stage1, p.stage2};
  void* dsts[3] = {euler ? u : p.stage1, p.stage2, u};
  cudaError_t e;
  for (int s = 0; s < (euler ? 1 : 3); ++s) {
    if ((e = cudaEventRecord(c->ev_fork, c->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(c->side, c->ev_fork, 0)) != cudaSuccess)
      return cuda_fail(c, e, "stream fork");
    for (int ax = 0; ax < p.d.ndim; ++ax) {
      Plan pl;
      molt_status st = plan_axis(c, p, ax, MODE_0, p.d.P, alpha, &pl, 0, 2);   // two sweeps at once
      if (st != MOLT_OK) return st;
      pl.a.in = sweep_input(p, ins[s]);
      pl.a.acc = ax == 0 ? p.acc : p.acc2;
      if ((st = run(c, p, ax <= 1 ? EPI_ACC_SET : EPI_ACC_ADD, pl, true, ax == 0 ? c->stream : c->side)) != MOLT_OK)
        return st;
    }
    if ((e = cudaEventRecord(c->ev_join, c->side)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(c->stream, c->ev_join, 0)) != cudaSuccess)
      return cuda_fail(c, e, "stream join");
    molt_ctx::Rec rec;
    record_begin(c, &rec, MOLT_KERNEL_UPDATE);
    const int g = stream_grid(p.total);
    if (is_f64_sweep(p.d))
      heat_update2_kernel<double, double><<<g, 256, 0, c->stream>>>(
          static_cast<const double*>(p.acc), static_cast<const double*>(p.acc2), static_cast<const double*>(u),
          static_cast<const double*>(ins[s]), static_cast<double*>(dsts[s]), nullptr, rk[s][0], rk[s][1], coefS,
          p.total, c->status_dev);
    else if (is_f32_state(p.d))
      heat_update2_kernel<float, float><<<g, 256, 0, c->stream>>>(
          static_cast<const float*>(p.acc), static_cast<const float*>(p.acc2), static_cast<const float*>(u),
          static_cast<const float*>(ins[s]), static_cast<float*>(dsts[s]), nullptr, rk[s][0], rk[s][1], coefS,
          p.total, c->status_dev);
    else
      heat_update2_kernel<float, double><<<g, 256, 0, c->stream>>>(
          static_cast<const float*>(p.acc), static_cast<const float*>(p.acc2), static_cast<const double*>(u),
          static_cast<const double*>(ins[s]), static_cast<double*>(dsts[s]), p.shadow, rk[s][0], rk[s][1], coefS,
          p.total, c->status_dev);
    record_end(c, &rec);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "heat update");
  }
  return MOLT_OK;
}

// One concurrent-axes heat step as a graph launch: the step's launches
// (sweeps on two streams joined by events, three stage updates) are captured
// once per state array and replayed, so a step costs one launch on the host
// and the graph's tighter launch spacing on the device.  The first step on a
// state array runs its launches directly (it also configures the kernels'
// attributes outside any capture); profiling, and streams that cannot be
// captured (the legacy default stream), always run them directly.
molt_status heat_step_graph(molt_ctx* c, Problem& p, void* u) {
  cudaError_t e;
  if (p.heat_graph_u != u) {
    if (p.heat_graph) cudaGraphExecDestroy(p.heat_graph);
    p.heat_graph = nullptr;
    p.heat_graph_u = u;
    p.heat_steps_direct = 0;
  }
  if (p.heat_graph_off || (!p.heat_graph && p.heat_steps_direct == 0)) {
    ++p.heat_steps_direct;
    return heat_step_axis_streams(c, p, u);
  }
  if (!p.heat_graph) {
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      p.heat_graph_off = true;
      return heat_step_axis_streams(c, p, u);
    }
    const molt_status st = heat_step_axis_streams(c, p, u);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->stream, &g);
    if (st != MOLT_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "heat step capture");
    e = cudaGraphInstantiate(&p.heat_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p.heat_graph = nullptr;
      return cuda_fail(c, e, "heat step graph");
    }
  }
  if ((e = cudaGraphLaunch(p.heat_graph, c->stream)) != cudaSuccess) return cuda_fail(c, e, "heat step graph launch");
  return MOLT_OK;
}

molt_status heat_step(molt_ctx* c, Problem& p, void* u) {
  if (heat_axis_streams(c, p))
    return c->profile ? heat_step_axis_streams(c, p, u) : heat_step_graph(c, p, u);
  const double alpha = step_alpha(p);
  const double coefS = -p.d.beta * p.d.beta;
  static const double rk[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  // forward Euler is the first stage written straight into u (pointwise, and
  // every tile reads its lines before writing them)
  const bool euler = p.d.integrator == MOLT_INT_EULER;
  void* ins[3] = {u, p.stage1, p.stage2};
  void* dsts[3] = {euler ? u : p.stage1, p.stage2, u};
  for (int s = 0; s < (euler ? 1 : 3); ++s) {
    for (int ax = 0; ax < p.d.ndim; ++ax) {
      Plan pl;
      molt_status st = plan_axis(c, p, ax, MODE_0, p.d.P, alpha, &pl);
      if (st != MOLT_OK) return st;
      pl.a.in = sweep_input(p, ins[s]);
      pl.a.acc = p.acc;
      int epi;
      const bool last = ax + 1 == p.d.ndim;
      if (!last || p.shadow) {
        epi = ax == 0 ? EPI_ACC_SET : EPI_ACC_ADD;
      } else {
        epi = EPI_HEAT_FINAL;
        if (p.d.ndim == 1) pl.a.acc = nullptr;
        pl.a.un = u;
        pl.a.us = ins[s];
        pl.a.dst = dsts[s];
        pl.a.a0 = rk[s][0];
        pl.a.a1 = rk[s][1];
        pl.a.coefS = coefS;
      }
      if ((st = run(c, p, epi, pl)) != MOLT_OK) return st;
      if (last && p.shadow) {
        molt_ctx::Rec rec;
        record_begin(c, &rec, MOLT_KERNEL_UPDATE);
        heat_update_kernel<<<stream_grid(p.total), 256, 0, c->stream>>>(
            static_cast<const float*>(p.acc), static_cast<const double*>(u), static_cast<const double*>(ins[s]),
            static_cast<double*>(dsts[s]), p.shadow, rk[s][0], rk[s][1], coefS, p.total, c->status_dev);
        record_end(c, &rec);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "heat update");
      }
    }
  }
  return MOLT_OK;
}

// ---------------------------------------------------------------- advection-diffusion
// Split fluxes of one axis from the state (Sec. 2.5): g^{+-} = (g(u) +- c u)/2,
// g = a u or u^2/2, evaluated in the state's precision and stored in the
// sweeps' compute type.
template <typename TS, typename TC>
__global__ void flux_kernel(const TS* __restrict__ u, TC* __restrict__ gp, TC* __restrict__ gm, int burgers, double a,
                            double c, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const TS v = u[i];
    const TS g = burgers ? TS(0.5) * v * v : TS(a) * v;
    const TS cu = TS(c) * v;
    gp[i] = TC(TS(0.5) * (g + cu));
    gm[i] = TC(TS(0.5) * (g - cu));
  }
}

// Runge-Kutta stage (or Euler step) of the advection-diffusion problem:
// dst = a0 u^n + a1 (u_s + dt F), dt F accumulated in acc; FP32 copy for
// mixed precision.
template <typename TC, typename TS>
__global__ void advdiff_update_kernel(const TC* __restrict__ acc, const TS* un, const TS* us, TS* dst,
                                      float* __restrict__ shadow, double a0, double a1, long long n, int* status) {
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const TS r = fma(TS(a0), un[i], TS(a1) * (us[i] + TS(acc[i])));
    dst[i] = r;
    if (shadow) shadow[i] = float(r);
    bad |= nonfinite(r);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

molt_status advdiff_step(molt_ctx* c, Problem& p, void* u) {
  static const double rk[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  const bool euler = p.d.integrator == MOLT_INT_EULER;
  void* ins[3] = {u, p.stage1, p.stage2};
  void* dsts[3] = {euler ? u : p.stage1, p.stage2, u};
  const double dt = p.d.dt, cb = p.d.c, beta = p.d.beta, kappa = p.d.diffusivity;
  const double alpha = beta / (cb * dt);
  const double alpha_nu = kappa > 0 ? beta / std::sqrt(kappa * dt) : 0.0;
  const bool f64 = is_f64_sweep(p.d), f32s = is_f32_state(p.d);
  cudaError_t e;
  for (int s = 0; s < (euler ? 1 : 3); ++s) {
    if ((e = cudaMemsetAsync(p.acc, 0, compute_bytes(p.d) * size_t(p.total), c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "memset");
    for (int ax = 0; ax < p.d.ndim; ++ax) {
      molt_ctx::Rec rec;
      record_begin(c, &rec, MOLT_KERNEL_FLUX);
      const int burgers = p.d.flux == MOLT_FLUX_BURGERS ? 1 : 0;
      const double av = p.d.velocity[ax];
      if (f64)
        flux_kernel<double, double><<<stream_grid(p.total), 256, 0, c->stream>>>(
            static_cast<const double*>(ins[s]), static_cast<double*>(p.gp), static_cast<double*>(p.gm), burgers, av,
            cb, p.total);
      else if (f32s)
        flux_kernel<float, float><<<stream_grid(p.total), 256, 0, c->stream>>>(
            static_cast<const float*>(ins[s]), static_cast<float*>(p.gp), static_cast<float*>(p.gm), burgers, av, cb,
            p.total);
      else
        flux_kernel<double, float><<<stream_grid(p.total), 256, 0, c->stream>>>(
            static_cast<const double*>(ins[s]), static_cast<float*>(p.gp), static_cast<float*>(p.gm), burgers, av,
            cb, p.total);
      record_end(c, &rec);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "flux");
      // -dt alpha S_R[g^+] + dt alpha S_L[g^-]  (dt alpha = beta / c)
      const struct { int mode; const void* in; double coef; double al; } terms[3] = {
          {MODE_R, p.gp, -beta / cb, alpha}, {MODE_L, p.gm, beta / cb, alpha},
          {MODE_0, sweep_input(p, ins[s]), -beta * beta, alpha_nu}};
      for (int t = 0; t < (kappa > 0 ? 3 : 2); ++t) {
        Plan pl;
        molt_status st = plan_axis(c, p, ax, terms[t].mode, p.d.P, terms[t].al, &pl);
        if (st != MOLT_OK) return st;
        pl.a.in = terms[t].in;
        pl.a.acc = p.acc;
        pl.a.coefS = terms[t].coef;
        if ((st = run(c, p, EPI_ACC_AXPY, pl)) != MOLT_OK) return st;
      }
    }
    molt_ctx::Rec rec;
    record_begin(c, &rec, MOLT_KERNEL_UPDATE);
    if (f64)
      advdiff_update_kernel<double, double><<<stream_grid(p.total), 256, 0, c->stream>>>(
          static_cast<const double*>(p.acc), static_cast<const double*>(u), static_cast<const double*>(ins[s]),
          static_cast<double*>(dsts[s]), nullptr, rk[s][0], rk[s][1], p.total, c->status_dev);
    else if (f32s)
      advdiff_update_kernel<float, float><<<stream_grid(p.total), 256, 0, c->stream>>>(
          static_cast<const float*>(p.acc), static_cast<const float*>(u), static_cast<const float*>(ins[s]),
          static_cast<float*>(dsts[s]), nullptr, rk[s][0], rk[s][1], p.total, c->status_dev);
    else
      advdiff_update_kernel<float, double><<<stream_grid(p.total), 256, 0, c->stream>>>(
          static_cast<const float*>(p.acc), static_cast<const double*>(u), static_cast<const double*>(ins[s]),
          static_cast<double*>(dsts[s]), p.shadow, rk[s][0], rk[s][1], p.total, c->status_dev);
    record_end(c, &rec);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "advection-diffusion update");
  }
  return MOLT_OK;
}

// Mixed precision: the FP64 leapfrog update runs as its own streaming kernel
// after the last axis (default), or, with MOLT_WAVE_FUSED_UPDATE=1, in the
// last sweep's epilogue (the line-per-lane kernel's where it takes the last
// axis).  Fused, the FP64 work (two FMAs per point on GB300's narrow FP64
// pipe) arrives in bursts at the end of every tile and stalls the sweep:
// 1.36 ms for z + update at 512^3 against 0.37 + 0.79 ms apart.
#ifndef MOLT_WAVE_FUSED_UPDATE
#define MOLT_WAVE_FUSED_UPDATE 0
#endif
molt_status wave_step(molt_ctx* c, Problem& p, void* cur, void* prev, bool from_rest, bool in_place_variant) {
  const double alpha = step_alpha(p);
  for (int ax = 0; ax < p.d.ndim; ++ax) {
    Plan pl;
    molt_status st = plan_axis(c, p, ax, MODE_0, p.d.P, alpha, &pl);
    if (st != MOLT_OK) return st;
    pl.a.in = sweep_input(p, cur);
    pl.a.acc = p.acc;
    int epi;
    const bool last = ax + 1 == p.d.ndim;
    // mixed precision: a streaming kernel does the FP64 update after the
    // accumulating sweep of the last axis (with MOLT_WAVE_FUSED_UPDATE, the
    // line-per-lane kernel's epilogue does it where that kernel takes the
    // last axis)
    bool split_update = p.shadow && !MOLT_WAVE_FUSED_UPDATE;
    if (MOLT_WAVE_FUSED_UPDATE && last && p.shadow && ax > 0) {
      split_update = true;
      Plan probe = pl;
      probe.a.shadow = p.shadow;
      probe.a.un = cur;
      probe.a.us = prev;
      probe.a.dst = in_place_variant ? cur : prev;
      probe.a.dst2 = in_place_variant ? prev : nullptr;
      LanesArgs la;
      CUtensorMap lmap;
      if (plan_lanes(c, p, EPI_WAVE_FINAL, probe, true, &la, &lmap)) split_update = false;
    }
    if (!last || split_update) {
      epi = ax == 0 ? EPI_ACC_SET : EPI_ACC_ADD;
    } else {
      epi = EPI_WAVE_FINAL;
      if (p.d.ndim == 1) pl.a.acc = nullptr;
      pl.a.shadow = p.shadow;
      pl.a.un = cur;
      pl.a.us = prev;
      pl.a.coefS = -p.d.beta * p.d.beta;
      pl.a.from_rest = from_rest ? 1 : 0;
      if (in_place_variant) {
        pl.a.dst = cur;
        pl.a.dst2 = prev;
      } else {
        pl.a.dst = prev;
      }
    }
    if ((st = run(c, p, epi, pl)) != MOLT_OK) return st;
    if (last && split_update) {
      molt_ctx::Rec rec;
      record_begin(c, &rec, MOLT_KERNEL_UPDATE);
      wave_update_kernel<<<stream_grid(p.total), 256, 0, c->stream>>>(
          static_cast<const float*>(p.acc), static_cast<const double*>(cur), static_cast<const double*>(prev),
          static_cast<double*>(in_place_variant ? cur : prev), in_place_variant ? static_cast<double*>(prev) : nullptr,
          p.shadow, -p.d.beta * p.d.beta, from_rest ? 1 : 0, p.total, c->status_dev);
      record_end(c, &rec);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(c, e, "wave update");
    }
  }
  return MOLT_OK;
}

// out[x][y] = in[y][x] for an ny x nx array, through 64 x 64 shared tiles;
// each of the 32 x 8 threads moves 16 elements, all loads issued first.
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ in, T* __restrict__ out, long long ny, long long nx) {
  __shared__ T tile[64][65];
  const long long x0 = (long long)blockIdx.x * 64, y0 = (long long)blockIdx.y * 64;
  T v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int j = threadIdx.y + 8 * (k >> 1), cx = threadIdx.x + 32 * (k & 1);
    const long long y = y0 + j, x = x0 + cx;
    v[k] = (y < ny && x < nx) ? in[y * nx + x] : T(0);
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) tile[threadIdx.y + 8 * (k >> 1)][threadIdx.x + 32 * (k & 1)] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int j = threadIdx.y + 8 * (k >> 1), cy = threadIdx.x + 32 * (k & 1);
    const long long x = x0 + j, y = y0 + cy;
    if (x < nx && y < ny) out[x * ny + y] = tile[cy][j];
  }
}

molt_status transpose(molt_ctx* c, const Problem& p, const void* in, void* out, long long ny, long long nx,
                      size_t elem) {
  molt_ctx::Rec rec;
  record_begin(c, &rec, MOLT_KERNEL_TRANSPOSE);
  const dim3 grid(unsigned((nx + 63) / 64), unsigned((ny + 63) / 64)), block(32, 8);
  if ((elem ? elem : state_bytes(p.d)) == 4)
    transpose_kernel<float><<<grid, block, 0, c->stream>>>(static_cast<const float*>(in), static_cast<float*>(out),
                                                           ny, nx);
  else
    transpose_kernel<double><<<grid, block, 0, c->stream>>>(static_cast<const double*>(in),
                                                            static_cast<double*>(out), ny, nx);
  record_end(c, &rec);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MOLT_OK : cuda_fail(c, e, "transpose");
}

// 2-D Hamilton-Jacobi: y lines long enough that a tile holds less than 32
// bytes of them (four FP32 lines of 2048 points, two of 4096, one of 8192)
// make the y pass a strided gather and scatter of a few bytes per row.  Such
// problems run the y pass on the transposed state instead, where the lines
// are rows.
bool hj_transposed_y(molt_ctx* c, const Problem& p) {
  if (p.d.pde != MOLT_PDE_HJ || p.d.ndim != 2) return false;
  // sigma/delta of AFFINE_SQ and source terms stay in the natural layout
  if (p.d.hamiltonian == MOLT_H_AFFINE_SQ || p.src) return false;
  Problem q = p;                     // the tile shape does not depend on the weights
  q.d.weights = MOLT_W_WENOZ;
  Plan pl;
  if (plan_axis(c, q, 1, MODE_RL, 1, step_alpha(q), &pl) != MOLT_OK) {
    c->err.clear();
    return false;
  }
  return size_t(pl.a.W) * state_bytes(p.d) < 32;
}

// The problem with x and y exchanged (the transposed state's geometry).
Problem transposed(const Problem& p) {
  Problem t = p;
  std::swap(t.n[0], t.n[1]);
  std::swap(t.h[0], t.h[1]);
  std::swap(t.d.n[0], t.d.n[1]);
  std::swap(t.d.lo[0], t.d.lo[1]);
  std::swap(t.d.hi[0], t.d.hi[1]);
  std::swap(t.d.bc[0], t.d.bc[1]);
  std::swap(t.d.velocity[0], t.d.velocity[1]);
  return t;
}

// dst == nullptr: u is the destination; speed_only: the last pass only
// measures the wave speeds (no store, no time advance).
molt_status hj_pass(molt_ctx* c, Problem& p, int idx, void* u, int ax, int epi, unsigned long long* speed,
                    const unsigned long long* lag, void* hx, void* dst = nullptr, bool speed_only = false) {
  Plan pl;
  molt_status st = plan_axis(c, p, ax, MODE_RL, 1, step_alpha(p), &pl);
  if (st != MOLT_OK) return st;
  double hmin = p.h[0];
  for (int a = 1; a < p.d.ndim; ++a) hmin = std::min(hmin, p.h[a]);
  pl.a.in = u;
  pl.a.un = u;
  pl.a.out = hx;
  pl.a.dst = dst ? dst : u;
  pl.a.speed = speed;
  pl.a.lag = lag;
  pl.a.cfl = p.d.cfl;
  pl.a.inv_h = 1.0 / p.h[ax];
  pl.a.dt_max = 10.0 * hmin;
  pl.a.t_dev = c->t_dev + idx;
  if (hx && p.d.hamiltonian == MOLT_H_AFFINE_SQ) pl.a.out2 = p.hx2;
  // the general kernels: other Hamiltonians, a source, speed-only passes
  const bool general = p.d.hamiltonian != MOLT_H_HALF_SQ || (epi == EPI_HJ_Y && (p.src || speed_only));
  if (epi == EPI_HJ_Y && p.src && !speed_only) {
    pl.a.src = p.src;
    pl.a.src_deg = p.src_deg;
    pl.a.src_stride = p.total;
    pl.a.t_now = c->tnow_dev + idx;
  }
  if (speed_only) {
    pl.a.dst = nullptr;
    pl.a.lag = nullptr;
    pl.a.t_dev = nullptr;
  }
  if (general) epi = epi == EPI_HJ_X ? EPI_HJ_XG : EPI_HJ_YG;
  return run(c, p, epi, pl);
}

// ---------------------------------------------------------------- HJ, SSP-RK3
// One Runge-Kutta stage of the Hamilton-Jacobi step from the P-term sums
// S_R, S_L of every axis (v^- = alpha S_R, v^+ = -alpha S_L): the local
// Lax-Friedrichs Hamiltonian (r_d the largest |dH/dp_d| over the box of
// one-sided derivatives), the source at the stage time, and
// dst = a0 u^n + a1 (u_s - dt (H^ - F)); dt from the lagged speed (as the
// Euler passes); the first stage publishes the speeds max_d r_d / h_d.
struct HjStageArgs {
  const void* sr[2];
  const void* sl[2];
  const void* un;
  const void* us;
  void* dst;            // null: a pass that only measures speeds
  int ndim, ham;
  double alpha, vel[2], inv_h[2], h0, a0, a1, cstage;
  const void* src;
  int src_deg;
  long long src_stride, n;
  const unsigned long long* lag;   // null: dt = 0 (speed-only pass)
  unsigned long long* speed;       // null: no speed published
  double cfl, dt_max;
  const double* t_now;             // time of u^n
  double* t_next;                  // block 0 of the last stage writes t^n + dt (or null)
  int* status;
};

template <typename T>
__global__ void hj_rk3_stage_kernel(const HjStageArgs g) {
  double dt = 0.0;
  if (g.lag) {
    const double cl = __longlong_as_double((long long)g.lag[0]);
    dt = g.dt_max;
    if (cl > 0.0 && g.cfl / cl < dt) dt = g.cfl / cl;
  }
  const double tn = g.t_now ? *g.t_now : 0.0;
  if (g.t_next && blockIdx.x == 0 && threadIdx.x == 0) *g.t_next = tn + dt;
  const T tst = T(tn + g.cstage * dt);
  const T al = T(g.alpha);
  double rmax = 0.0;
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
    T vm[2], vp[2];
    for (int d = 0; d < g.ndim; ++d) {
      vm[d] = al * static_cast<const T*>(g.sr[d])[i];
      vp[d] = -al * static_cast<const T*>(g.sl[d])[i];
    }
    T H = T(0), r[2] = {T(0), T(0)};
    if (g.ham == HAM_AFFINE_SQ) {
      T sbar = T(g.h0), dsum = T(0), dabs = T(0), delta[2];
      for (int d = 0; d < g.ndim; ++d) {
        const T ad = T(g.vel[d]);
        sbar += ad * T(0.5) * (vm[d] + vp[d]);
        delta[d] = fabs(ad) * T(0.5) * (vp[d] - vm[d]);
        dsum += delta[d];
        dabs += fabs(delta[d]);
      }
      const T m = fabs(sbar) + dabs;
      H = T(0.5) * sbar * sbar - m * dsum;
      for (int d = 0; d < g.ndim; ++d) r[d] = fabs(T(g.vel[d])) * m;
    } else {
      for (int d = 0; d < g.ndim; ++d) {
        const T mean = T(0.5) * (vm[d] + vp[d]);
        if (g.ham == HAM_LINEAR) {
          r[d] = fabs(T(g.vel[d]));
          H += T(g.vel[d]) * mean;
        } else {
          r[d] = fmax(fabs(vm[d]), fabs(vp[d]));
          H += T(0.5) * mean * mean;
        }
        H -= r[d] * T(0.5) * (vp[d] - vm[d]);
      }
    }
    for (int d = 0; d < g.ndim; ++d) rmax = fmax(rmax, double(r[d]) * g.inv_h[d]);
    if (g.src) {
      const T* f = static_cast<const T*>(g.src) + i;
      T F = f[g.src_deg * g.src_stride];
      for (int k = g.src_deg - 1; k >= 0; --k) F = fma(F, tst, f[k * g.src_stride]);
      H -= F;
    }
    if (g.dst) {
      const T res = fma(T(g.a0), static_cast<const T*>(g.un)[i],
                        T(g.a1) * fma(-T(dt), H, static_cast<const T*>(g.us)[i]));
      static_cast<T*>(g.dst)[i] = res;
      bad |= nonfinite(res);
    }
  }
  if (g.speed) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if ((threadIdx.x & 31) == 0 && rmax > 0.0) atomicMax(g.speed, (unsigned long long)__double_as_longlong(rmax));
  }
  if (bad) atomicOr(g.status, ST_NONFINITE);
}

// The P-term sums S_R, S_L of every axis of `in` into p.hv.
molt_status hj_rk3_sums(molt_ctx* c, Problem& p, const void* in) {
  for (int ax = 0; ax < p.d.ndim; ++ax) {
    for (int side = 0; side < 2; ++side) {
      Plan pl;
      molt_status st = plan_axis(c, p, ax, side == 0 ? MODE_R : MODE_L, p.d.P, step_alpha(p), &pl);
      if (st != MOLT_OK) return st;
      pl.a.in = in;
      pl.a.out = p.hv[2 * ax + side];
      if ((st = run(c, p, EPI_STORE, pl)) != MOLT_OK) return st;
    }
  }
  return MOLT_OK;
}

molt_status hj_rk3_stage(molt_ctx* c, const Problem& p, HjStageArgs g) {
  molt_ctx::Rec rec;
  record_begin(c, &rec, MOLT_KERNEL_UPDATE);
  if (state_bytes(p.d) == 4) hj_rk3_stage_kernel<float><<<stream_grid(p.total), 256, 0, c->stream>>>(g);
  else hj_rk3_stage_kernel<double><<<stream_grid(p.total), 256, 0, c->stream>>>(g);
  record_end(c, &rec);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MOLT_OK : cuda_fail(c, e, "Hamilton-Jacobi stage");
}

// The Hamilton-Jacobi step from the one-sided sums S_R, S_L of every axis
// (EPI_STORE sweeps into hv) and one pointwise stage kernel per stage: the
// 3-stage SSP Runge-Kutta method, or (stages == 1: a0 = 0, a1 = 1, the stage
// at t^n) forward Euler -- the form non-uniform axes take, whose sums come
// from the non-uniform sweep.
molt_status hj_rk3_step(molt_ctx* c, Problem& p, int idx, void* u, int stages = 3) {
  static const double rk[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  static const double cst[3] = {0.0, 1.0, 0.5};   // stage times t^n + c dt
  unsigned long long* slots = c->speed_dev + 2 * idx;
  double hmin = p.h[0];
  for (int a = 1; a < p.d.ndim; ++a) hmin = std::min(hmin, p.h[a]);
  HjStageArgs g{};
  g.ndim = p.d.ndim;
  g.ham = p.d.hamiltonian;
  g.alpha = step_alpha(p);
  g.h0 = p.d.h0;
  for (int d = 0; d < p.d.ndim; ++d) {
    g.sr[d] = p.hv[2 * d];
    g.sl[d] = p.hv[2 * d + 1];
    g.vel[d] = p.d.velocity[d];
    g.inv_h[d] = 1.0 / p.h[d];
  }
  g.cfl = p.d.cfl;
  g.dt_max = 10.0 * hmin;
  g.n = p.total;
  g.status = c->status_dev;
  cudaError_t e;
  molt_status st;
  if (!p.hj_lag_ready) {
    // speeds of u^0 serve as the lagged speeds of the first step (Algorithm 1)
    if ((e = cudaMemsetAsync(slots + 1, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "memset");
    if ((st = hj_rk3_sums(c, p, u)) != MOLT_OK) return st;
    HjStageArgs s0 = g;
    s0.speed = slots + 1;
    if ((st = hj_rk3_stage(c, p, s0)) != MOLT_OK) return st;
    p.hj_lag_ready = true;
    p.hj_steps = 0;
  }
  const int cur = int(p.hj_steps & 1);
  if ((e = cudaMemsetAsync(slots + cur, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "memset");
  void* ins[3] = {u, p.stage1, p.stage2};
  void* dsts[3] = {stages == 1 ? u : p.stage1, p.stage2, u};
  for (int s = 0; s < stages; ++s) {
    if ((st = hj_rk3_sums(c, p, ins[s])) != MOLT_OK) return st;
    HjStageArgs gs = g;
    gs.un = u;
    gs.us = ins[s];
    gs.dst = dsts[s];
    gs.a0 = rk[s][0];
    gs.a1 = rk[s][1];
    gs.cstage = cst[s];
    gs.lag = slots + (cur ^ 1);
    gs.speed = s == 0 ? slots + cur : nullptr;
    gs.t_now = c->t_dev + idx;
    gs.t_next = s == stages - 1 ? c->tnow_dev + idx : nullptr;
    if (p.src) {
      gs.src = p.src;
      gs.src_deg = p.src_deg;
      gs.src_stride = p.total;
    }
    if ((st = hj_rk3_stage(c, p, gs)) != MOLT_OK) return st;
  }
  // t^{n+1} = t^n + dt (written apart from t^n, which every stage reads)
  if ((e = cudaMemcpyAsync(c->t_dev + idx, c->tnow_dev + idx, sizeof(double), cudaMemcpyDeviceToDevice,
                           c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "time copy");
  p.hj_steps++;
  return MOLT_OK;
}

molt_status hj_step(molt_ctx* c, Problem& p, int idx, void* u) {
  if (p.d.integrator == MOLT_INT_RK3) return hj_rk3_step(c, p, idx, u);
  for (int ax = 0; ax < p.d.ndim; ++ax)
    if (!p.nodes[ax].empty()) return hj_rk3_step(c, p, idx, u, 1);
  unsigned long long* slots = c->speed_dev + 2 * idx;
  cudaError_t e;
  const bool ty = p.tu && p.thx && hj_transposed_y(c, p);
  Problem pt;
  if (ty) pt = transposed(p);
  const long long ny = p.n[1], nx = p.n[0];
  void* hxp = p.d.ndim > 1 ? p.hx : nullptr;
  if (!p.hj_lag_ready) {
    // speeds of u^0 serve as the lagged speeds of the first step (Algorithm 1)
    if ((e = cudaMemsetAsync(slots + 1, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "memset");
    for (int ax = 0; ax < p.d.ndim; ++ax) {
      molt_status st;
      if (p.d.hamiltonian == MOLT_H_AFFINE_SQ) {
        // the speed needs every axis: the x pass, then a last pass that only measures
        const bool last = ax + 1 == p.d.ndim;
        st = hj_pass(c, p, idx, u, ax, last ? EPI_HJ_Y : EPI_HJ_X, slots + 1, nullptr, hxp, nullptr, last);
      } else if (ty && ax == 1) {
        if ((st = transpose(c, p, u, p.tu, ny, nx)) != MOLT_OK) return st;
        st = hj_pass(c, pt, idx, p.tu, 0, EPI_HJ_X, slots + 1, nullptr, nullptr);
      } else {
        st = hj_pass(c, p, idx, u, ax, EPI_HJ_X, slots + 1, nullptr, nullptr);
      }
      if (st != MOLT_OK) return st;
    }
    p.hj_lag_ready = true;
    p.hj_steps = 0;
  }
  const int cur = int(p.hj_steps & 1);
  unsigned long long* slot = slots + cur;
  const unsigned long long* lag = slots + (cur ^ 1);
  if ((e = cudaMemsetAsync(slot, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "memset");
  if (ty) {
    // The y lines run as rows of the transposed state.  The state alternates
    // between the layouts from step to step, so a step transposes twice (the
    // state and the first pass's H^ part) and molt_step transposes the state
    // back once at the end of an odd run:
    //   natural u:     x pass on u -> hx; u, hx -> tu, thx; y pass on tu
    //                  (reads thx) writes u^{n+1} into tu
    //   transposed tu: y pass on tu -> thx; tu, thx -> u, hx; x pass on u
    //                  (reads hx) writes u^{n+1} into u
    // The two one-axis parts of H^ add in either order (the sum is exact in
    // either order), and the speeds are one maximum over both axes.
    molt_status st;
    if (!p.hj_flipped) {
      if ((st = hj_pass(c, p, idx, u, 0, EPI_HJ_X, slot, lag, hxp)) != MOLT_OK) return st;
      if ((st = transpose(c, p, u, p.tu, ny, nx)) != MOLT_OK) return st;
      if ((st = transpose(c, p, p.hx, p.thx, ny, nx)) != MOLT_OK) return st;
      if ((st = hj_pass(c, pt, idx, p.tu, 0, EPI_HJ_Y, slot, lag, p.thx, p.tu)) != MOLT_OK) return st;
    } else {
      if ((st = hj_pass(c, pt, idx, p.tu, 0, EPI_HJ_X, slot, lag, p.thx)) != MOLT_OK) return st;
      if ((st = transpose(c, p, p.tu, u, nx, ny)) != MOLT_OK) return st;
      if ((st = transpose(c, p, p.thx, p.hx, nx, ny)) != MOLT_OK) return st;
      if ((st = hj_pass(c, p, idx, u, 0, EPI_HJ_Y, slot, lag, hxp)) != MOLT_OK) return st;
    }
    p.hj_flipped = !p.hj_flipped;
    p.hj_steps++;
    return MOLT_OK;
  }
  for (int ax = 0; ax < p.d.ndim; ++ax) {
    const bool last = ax + 1 == p.d.ndim;
    const int epi = last ? EPI_HJ_Y : EPI_HJ_X;
    molt_status st;
    if (last && p.src &&
        (e = cudaMemcpyAsync(c->tnow_dev + idx, c->t_dev + idx, sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "time copy");
    st = hj_pass(c, p, idx, u, ax, epi, slot, lag, hxp);
    if (st != MOLT_OK) return st;
  }
  p.hj_steps++;
  return MOLT_OK;
}

// A Hamilton-Jacobi state left in the transposed layout goes back into u.
molt_status hj_unflip(molt_ctx* c, Problem& p, void* u) {
  if (!p.hj_flipped) return MOLT_OK;
  molt_status st = transpose(c, p, p.tu, u, p.n[0], p.n[1]);
  if (st == MOLT_OK) p.hj_flipped = false;
  return st;
}

// ------------------------------------------------------------------ batch
// Shapes a batch problem's line tile may take on one axis: points per lane E
// with n = 32 * nwl * E exactly and nwl | 16 (so 32 * nwl * W = 512).
bool shape_ok(int64_t n, int E) {
  if (n % (32 * E) != 0) return false;
  const int64_t nwl = n / (32 * E);
  return nwl >= 1 && nwl <= 16 && (16 % nwl) == 0;
}

bool batch_supported(const molt_ctx* c) {
  if (c->probs.size() < 2) return false;
  for (const auto& p : c->probs) {
    const molt_desc& d = p.d;
    if (d.pde != MOLT_PDE_HEAT || d.prec != MOLT_PREC_F32_F64UPDATE || d.ndim != 2 || d.weights != MOLT_W_LINEAR ||
        d.integrator == MOLT_INT_EULER)
      return false;
    for (int ax = 0; ax < 2; ++ax)
      if (!shape_ok(p.n[ax], 16) && !shape_ok(p.n[ax], 8) && !shape_ok(p.n[ax], 4)) return false;
  }
  return true;
}

// Fills the device tables for the selected problems and returns the params.
molt_status batch_build(molt_ctx* c, void* const* u, const std::vector<int>& sel, int phase_mask, int stages,
                        BatchParams* out, size_t* smem) {
  BatchState& B = c->batch;
  std::vector<BatchSweep> hs;
  std::vector<BatchUpdate> hu;
  int items[2] = {0, 0};
  long long chunks = 0;
  size_t sm = 0;
  for (int i : sel) {
    Problem& p = c->probs[i];
    const double alpha = step_alpha(p);
    for (int ax = 0; ax < 2; ++ax) {
      Plan pl;
      molt_status st = plan_axis(c, p, ax, MODE_0, p.d.P, alpha, &pl, B.E[ax][i]);
      if (st != MOLT_OK) return st;
      if (pl.block != 512) return fail(c, MOLT_EUNSUPPORTED, "batch tile does not fill 512 threads");
      pl.a.in = p.shadow;
      pl.a.acc = p.acc;
      pl.a.status = c->status_dev;
      BatchSweep bs;
      bs.a = pl.a;
      bs.E = B.E[ax][i];
      bs.first_item = items[ax];
      bs.ntiles = int((pl.a.g.nlines + pl.a.W - 1) / pl.a.W);
      items[ax] += bs.ntiles;
      hs.push_back(bs);
      if (pl.smem > sm) sm = pl.smem;
    }
    BatchUpdate bu;
    bu.acc = static_cast<const float*>(p.acc);
    bu.u = static_cast<double*>(u ? u[i] : nullptr);
    bu.st1 = static_cast<double*>(p.stage1);
    bu.st2 = static_cast<double*>(p.stage2);
    bu.copy = p.shadow;
    bu.total = p.total;
    bu.first_chunk = chunks;
    chunks += (p.total + kChunk - 1) / kChunk;
    hu.push_back(bu);
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(B.d_sweeps, hs.data(), hs.size() * sizeof(BatchSweep), cudaMemcpyHostToDevice,
                           c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(B.d_updates, hu.data(), hu.size() * sizeof(BatchUpdate), cudaMemcpyHostToDevice,
                           c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "batch tables");
  BatchParams prm{};
  prm.nprob = int(sel.size());
  prm.sweeps = B.d_sweeps;
  prm.items[0] = items[0];
  prm.items[1] = items[1];
  prm.updates = B.d_updates;
  prm.chunks = chunks;
  prm.coefS = -c->probs[sel[0]].d.beta * c->probs[sel[0]].d.beta;
  prm.stages = stages;
  prm.phase_mask = phase_mask;
  prm.bar_count = B.d_bar;
  prm.bar_gen = B.d_bar + 1;
  prm.status = c->status_dev;
  prm.wait_limit = c->wait_limit;
  prm.skip_arrive = c->test_skip_arrive ? 1 : 0;
  prm.stage_off = unsigned((sm + 127) & ~size_t(127));
  *out = prm;
  *smem = prm.stage_off + size_t(kStageFloats) * sizeof(float);
  return MOLT_OK;
}

// Cooperative launch: every CTA is resident, so the grid barriers complete.
molt_status batch_launch(molt_ctx* c, const BatchParams& prm, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(batch_heat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return cuda_fail(c, e, "batch attribute");
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_heat_kernel, 512, smem)) != cudaSuccess)
    return cuda_fail(c, e, "batch occupancy");
  if (per_sm < 1) return fail(c, MOLT_EUNSUPPORTED, "batch kernel does not fit on an SM");
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((e = cudaMemsetAsync(c->batch.d_bar, 0, 2 * sizeof(unsigned int), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "batch barrier reset");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(sms * per_sm));
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  molt_ctx::Rec rec;
  record_begin(c, &rec, MOLT_KERNEL_BATCH);
  e = cudaLaunchKernelEx(&cfg, batch_heat_kernel, prm);
  record_end(c, &rec);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch launch");
  return MOLT_OK;
}

// Autotuner: for every size class and axis, time each admissible tile shape
// (points per lane E in {16, 8, 4}) on that class's sweeps and keep the fastest.
molt_status batch_tune(molt_ctx* c) {
  BatchState& B = c->batch;
  const int np = int(c->probs.size());
  for (int ax = 0; ax < 2; ++ax) {
    std::vector<int64_t> sizes;
    for (int i = 0; i < np; ++i) {
      const int64_t n = c->probs[i].n[ax];
      if (std::find(sizes.begin(), sizes.end(), n) == sizes.end()) sizes.push_back(n);
    }
    for (int64_t n : sizes) {
      std::vector<int> sel;
      for (int i = 0; i < np; ++i)
        if (c->probs[i].n[ax] == n) sel.push_back(i);
      std::vector<int> cands;
      for (int E : {16, 8, 4})
        if (shape_ok(n, E)) cands.push_back(E);
      int best = cands[0];
      if (cands.size() > 1) {
        float best_ms = 1e30f;
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        for (int E : cands) {
          for (int i : sel) B.E[ax][i] = E;
          BatchParams prm;
          size_t smem;
          molt_status st = batch_build(c, nullptr, sel, 1 << ax, 1, &prm, &smem);
          if (st != MOLT_OK) return st;
          if ((st = batch_launch(c, prm, smem)) != MOLT_OK) return st;
          cudaEventRecord(t0, c->stream);
          for (int r = 0; r < 3; ++r)
            if ((st = batch_launch(c, prm, smem)) != MOLT_OK) return st;
          cudaEventRecord(t1, c->stream);
          cudaEventSynchronize(t1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, t0, t1);
          if (ms < best_ms) {
            best_ms = ms;
            best = E;
          }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
      }
      for (int i : sel) B.E[ax][i] = best;
    }
  }
  B.tuned = true;
  return MOLT_OK;
}

molt_status batch_prepare(molt_ctx* c) {
  BatchState& B = c->batch;
  if (B.checked) return MOLT_OK;
  B.checked = true;
  B.supported = batch_supported(c);
  if (!B.supported) return MOLT_OK;
  const int np = int(c->probs.size());
  for (int ax = 0; ax < 2; ++ax) {
    B.E[ax].resize(np);
    for (int i = 0; i < np; ++i) {
      const int64_t n = c->probs[i].n[ax];
      B.E[ax][i] = shape_ok(n, 16) ? 16 : (shape_ok(n, 8) ? 8 : 4);
    }
  }
  if (cudaMalloc(&B.d_sweeps, sizeof(BatchSweep) * 2 * np) != cudaSuccess ||
      cudaMalloc(&B.d_updates, sizeof(BatchUpdate) * np) != cudaSuccess ||
      cudaMalloc(&B.d_bar, 2 * sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MOLT_ENOMEM, "batch tables");
  }
  return MOLT_OK;
}

// One graph-captured persistent launch per time step.
molt_status batch_steps(molt_ctx* c, void* const* u, int nsteps) {
  BatchState& B = c->batch;
  const int np = int(c->probs.size());
  molt_status st;
  if (!B.tuned && (st = batch_tune(c)) != MOLT_OK) return st;
  std::vector<void*> cur(u, u + np);
  if (cur != B.last_u || (!B.graph && !B.graph_failed)) {
    if (B.graph) {
      cudaGraphExecDestroy(B.graph);
      B.graph = nullptr;
    }
    std::vector<int> all(np);
    for (int i = 0; i < np; ++i) all[i] = i;
    if ((st = batch_build(c, u, all, 7, 3, &B.params, &B.smem)) != MOLT_OK) return st;
    B.last_u = cur;
    B.graph_failed = true;
    if (c->stream && !c->profile) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const molt_status lst = batch_launch(c, B.params, B.smem);
        const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
        if (lst == MOLT_OK && ce == cudaSuccess && g &&
            cudaGraphInstantiate(&B.graph, g, 0) == cudaSuccess)
          B.graph_failed = false;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
    }
  }
  for (int k = 0; k < nsteps; ++k) {
    if (B.graph) {
      molt_ctx::Rec rec;
      record_begin(c, &rec, MOLT_KERNEL_BATCH);
      cudaError_t e = cudaGraphLaunch(B.graph, c->stream);
      record_end(c, &rec);
      if (e != cudaSuccess) return cuda_fail(c, e, "batch graph launch");
    } else if ((st = batch_launch(c, B.params, B.smem)) != MOLT_OK) {
      return st;
    }
  }
  return MOLT_OK;
}

}  // namespace

extern "C" {

molt_status molt_step(molt_ctx* c, void* const* u, void* const* u_prev, int nsteps, double* t_inout) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (!u || !t_inout || nsteps < 0) return fail(c, MOLT_EINVAL, "null u/t_inout or negative nsteps");
  const int np = int(c->probs.size());
  bool any_nonuniform = false;   // the batched heat step runs uniform grids
  for (int i = 0; i < np; ++i) {
    if (!u[i]) return fail(c, MOLT_EINVAL, "null state pointer");
    if (c->probs[i].d.pde == MOLT_PDE_WAVE && (!u_prev || !u_prev[i]))
      return fail(c, MOLT_EINVAL, "wave problems need u_prev");
    if (c->probs[i].d.pde != MOLT_PDE_HJ && !(c->probs[i].d.dt > 0))
      return fail(c, MOLT_EINVAL, "heat and wave steps need dt > 0");
    for (int ax = 0; ax < 3; ++ax)
      if (!c->probs[i].nodes[ax].empty()) any_nonuniform = true;
  }
  cudaError_t e;
  std::vector<double> t0(np);
  for (int i = 0; i < np; ++i) t0[i] = t_inout[i];
  if ((e = cudaMemcpyAsync(c->t_dev, t0.data(), sizeof(double) * np, cudaMemcpyHostToDevice, c->stream)) !=
      cudaSuccess)
    return cuda_fail(c, e, "t upload");
  for (int i = 0; i < np && nsteps > 0; ++i) {
    molt_status st = refresh_shadow(c, c->probs[i], u[i]);
    if (st != MOLT_OK) return st;
  }
  molt_status bst = batch_prepare(c);
  if (bst != MOLT_OK) return bst;
  const bool batched = c->batch.supported && !any_nonuniform;
  if (batched && nsteps > 0) {
    if ((bst = batch_steps(c, u, nsteps)) != MOLT_OK) return bst;
    for (int i = 0; i < np; ++i) t_inout[i] += nsteps * c->probs[i].d.dt;
  }
  for (int k = 0; k < (batched ? 0 : nsteps); ++k) {
    for (int i = 0; i < np; ++i) {
      Problem& p = c->probs[i];
      molt_status st = MOLT_OK;
      if (p.d.pde == MOLT_PDE_HEAT) {
        st = heat_step(c, p, u[i]);
        t_inout[i] += p.d.dt;
      } else if (p.d.pde == MOLT_PDE_WAVE) {
        const bool from_rest = (k == 0 && t0[i] == 0.0);
        const bool even = (k % 2) == 0;
        void* cur = even ? u[i] : u_prev[i];
        void* prev = even ? u_prev[i] : u[i];
        const bool variant = (k == nsteps - 1) && even;   // keep u = newest on return
        st = wave_step(c, p, cur, prev, from_rest, variant);
        t_inout[i] += p.d.dt;
      } else if (p.d.pde == MOLT_PDE_ADVDIFF) {
        st = advdiff_step(c, p, u[i]);
        t_inout[i] += p.d.dt;
      } else {
        st = hj_step(c, p, i, u[i]);
      }
      if (st != MOLT_OK) return st;
    }
  }
  for (int i = 0; i < np; ++i) {
    molt_status st = hj_unflip(c, c->probs[i], u[i]);
    if (st != MOLT_OK) return st;
  }
  int status = 0;
  std::vector<double> tdev(np);
  if ((e = cudaMemcpyAsync(&status, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "status read");
  if ((e = cudaMemcpyAsync(tdev.data(), c->t_dev, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream)) !=
      cudaSuccess)
    return cuda_fail(c, e, "t read");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "step");
  for (int i = 0; i < np; ++i)
    if (c->probs[i].d.pde == MOLT_PDE_HJ) t_inout[i] = tdev[i];
  if (status & ST_NONFINITE) {
    cudaMemsetAsync(c->status_dev, 0, sizeof(int), c->stream);
    return fail(c, MOLT_ENONFINITE, "a non-finite value reached the state");
  }
  if (status & ST_TIMEOUT) {
    cudaMemsetAsync(c->status_dev, 0, sizeof(int), c->stream);
    return fail(c, MOLT_ETIMEOUT,
                "a device-side wait timed out (a grid barrier or a copy: a copy may still have been in flight, so "
                "treat the CUDA context as suspect: destroy this context and do not reuse its buffers)");
  }
  return MOLT_OK;
}

molt_status molt_set_source(molt_ctx* c, int problem, const void* coef, int degree) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (problem < 0 || problem >= int(c->probs.size())) return fail(c, MOLT_EINVAL, "problem index out of range");
  Problem& p = c->probs[problem];
  if (p.d.pde != MOLT_PDE_HJ) return fail(c, MOLT_EINVAL, "source terms are for Hamilton-Jacobi problems");
  if (coef && p.d.weights == MOLT_W_LEARNED)
    return fail(c, MOLT_EUNSUPPORTED, "source terms run with linear or WENO-Z weights");
  cudaError_t e;
  if (!coef) {
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "source sync");
    cudaFree(p.src);
    p.src = nullptr;
    p.src_deg = 0;
    return MOLT_OK;
  }
  if (degree < 0 || degree > 4) return fail(c, MOLT_EINVAL, "source degree must be in 0..4");
  if (reinterpret_cast<uintptr_t>(coef) & 15) return fail(c, MOLT_EINVAL, "source array must be 16-byte aligned");
  const size_t bytes = size_t(degree + 1) * size_t(p.total) * state_bytes(p.d);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "source sync");
  cudaFree(p.src);
  p.src = nullptr;
  if ((e = cudaMalloc(&p.src, bytes)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MOLT_ENOMEM, "source allocation failed");
  }
  if ((e = cudaMemcpyAsync(p.src, coef, bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "source copy");
  p.src_deg = degree;
  return MOLT_OK;
}

// Nodes of a non-uniform line: strictly increasing and finite; a periodic
// line (period > 0) fits in one period, a Dirichlet line (period == 0) has
// at least 4 nodes.
static bool nonuniform_nodes_ok(const double* x, int64_t n, double period) {
  if (!x || n < 1 || !std::isfinite(period) || period < 0) return false;
  if (period == 0 && n < 4) return false;
  for (int64_t i = 0; i < n; ++i) {
    if (!std::isfinite(x[i])) return false;
    if (i > 0 && !(x[i] > x[i - 1])) return false;
  }
  return period == 0 || x[n - 1] - x[0] < period;
}

molt_status molt_nonuniform_weights(const double* x, int64_t n, double period, double alpha, int quad_points,
                                    double* cR, double* cL, double* q) {
  if (!cR || !cL || !q || !nonuniform_nodes_ok(x, n, period) || !(alpha > 0) || !std::isfinite(alpha))
    return MOLT_EINVAL;
  if (quad_points != 3 && quad_points != 5 && quad_points != 6) return MOLT_EINVAL;
  std::vector<double> nodes(x, x + n), r, l, qq;
  build_nonuniform_tables(nodes, period, alpha, quad_points, &r, &l, &qq);
  std::copy(r.begin(), r.end(), cR);
  std::copy(l.begin(), l.end(), cL);
  std::copy(qq.begin(), qq.end(), q);
  return MOLT_OK;
}

molt_status molt_nonuniform_weno_weights(const double* x, int64_t n, double period, double alpha, double* wR,
                                         double* wL) {
  if (!wR || !wL || !nonuniform_nodes_ok(x, n, period) || !(alpha > 0) || !std::isfinite(alpha)) return MOLT_EINVAL;
  std::vector<double> nodes(x, x + n), r, l;
  build_nonuniform_weno_tables(nodes, period, alpha, &r, &l);
  std::copy(r.begin(), r.end(), wR);
  std::copy(l.begin(), l.end(), wL);
  return MOLT_OK;
}

molt_status molt_set_grid_axis(molt_ctx* c, int problem, int axis, const double* x, int64_t n) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (problem < 0 || problem >= int(c->probs.size())) return fail(c, MOLT_EINVAL, "problem index out of range");
  Problem& p = c->probs[problem];
  if (axis < 0 || axis >= p.d.ndim) return fail(c, MOLT_EINVAL, "axis out of range");
  cudaError_t e;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "grid sync");
  cudaFree(p.nu[axis].dev);
  p.nu[axis] = Problem::NuCache{};
  if (!x) {
    p.nodes[axis].clear();
    p.h[axis] = make_problem(p.d).h[axis];
    return MOLT_OK;
  }
  if (n != p.n[axis]) return fail(c, MOLT_EINVAL, "node count differs from the axis size");
  const bool dir = p.d.bc[axis] == MOLT_BC_DIRICHLET;
  const double L = p.d.hi[axis] - p.d.lo[axis];
  if (dir && n < 4) return fail(c, MOLT_EINVAL, "a Dirichlet axis needs at least 4 nodes");
  for (int64_t i = 0; i < n; ++i) {
    if (!std::isfinite(x[i])) return fail(c, MOLT_EINVAL, "nodes must be finite");
    if (i > 0 && !(x[i] > x[i - 1])) return fail(c, MOLT_EINVAL, "nodes must increase strictly");
  }
  if (!dir && !(x[n - 1] - x[0] < L)) return fail(c, MOLT_EINVAL, "nodes must lie within one period");
  if (!p.nu_sum && (e = cudaMalloc(&p.nu_sum, compute_bytes(p.d) * size_t(p.total))) != cudaSuccess) {
    cudaGetLastError();
    p.nu_sum = nullptr;
    return fail(c, MOLT_ENOMEM, "non-uniform axis sums");
  }
  // Hamilton-Jacobi on non-uniform axes: the one-sided sums of every axis
  if (p.d.pde == MOLT_PDE_HJ)
    for (int k = 0; k < 2 * p.d.ndim; ++k)
      if (!p.hv[k] && (e = cudaMalloc(&p.hv[k], state_bytes(p.d) * size_t(p.total))) != cudaSuccess) {
        cudaGetLastError();
        p.hv[k] = nullptr;
        return fail(c, MOLT_ENOMEM, "Hamilton-Jacobi axis sums");
      }
  p.nodes[axis].assign(x, x + n);
  // the axis's spacing is its smallest cell (the periodic wrap cell
  // included): the Hamilton-Jacobi alpha = beta/(cfl min h) and dt = cfl
  // min_d h_d / c_d take it, as on uniform grids
  double hmin = dir ? x[n - 1] - x[0] : L - (x[n - 1] - x[0]);
  for (int64_t i = 1; i < n; ++i) hmin = std::min(hmin, x[i] - x[i - 1]);
  p.h[axis] = hmin;
  return MOLT_OK;
}

static void clear_records(molt_ctx* c);

molt_status molt_set_option(molt_ctx* c, int option, int64_t value) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (option == MOLT_OPT_WAIT_LIMIT) {
    if (value < 1000) return fail(c, MOLT_EINVAL, "wait limit below 1000 cycles");
    c->wait_limit = value;
  } else if (option == MOLT_OPT_LANES) {
    if (value < 0 || value > 2) return fail(c, MOLT_EINVAL, "MOLT_OPT_LANES takes 0, 1 or 2");
    c->lanes = int(value);
  } else if (option == MOLT_OPT_AXIS_STREAMS) {
    if (value != 0 && value != 1) return fail(c, MOLT_EINVAL, "option value must be 0 or 1");
    c->axis_streams = int(value);
  } else if (option == MOLT_OPT_XLINES) {
    if (value != 0 && value != 1) return fail(c, MOLT_EINVAL, "option value must be 0 or 1");
    c->xlines = int(value);
  } else {
    if (value != 0 && value != 1) return fail(c, MOLT_EINVAL, "option value must be 0 or 1");
    if (option == MOLT_OPT_TMA) c->no_tma = value == 0;
    else if (option == MOLT_OPT_PROFILE) {
      c->profile = value == 1;
      clear_records(c);
    }
    else if (option == MOLT_OPT_TEST_SKIP_ARRIVE) c->test_skip_arrive = value == 1;
    else return fail(c, MOLT_EINVAL, "unknown option");
  }
  // baked into the captured batch and heat steps: rebuild them on the next step
  c->batch.last_u.clear();
  for (auto& p : c->probs) p.heat_graph_u = nullptr;
  return MOLT_OK;
}

molt_status molt_batch_tile_shape(molt_ctx* c, int problem, int axis, int* points_per_lane, int* warps_per_line,
                                  int* lines_per_tile) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (problem < 0 || problem >= int(c->probs.size()) || axis < 0 || axis > 1)
    return fail(c, MOLT_EINVAL, "problem or axis out of range");
  if (!c->batch.supported || !c->batch.tuned) return fail(c, MOLT_EUNSUPPORTED, "no tuned batch step yet");
  const int E = c->batch.E[axis][problem];
  const int nwl = int(c->probs[problem].n[axis] / (32 * E));
  if (points_per_lane) *points_per_lane = E;
  if (warps_per_line) *warps_per_line = nwl;
  if (lines_per_tile) *lines_per_tile = 16 / nwl;
  return MOLT_OK;
}

static void clear_records(molt_ctx* c) {
  for (auto& r : c->recs) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  c->recs.clear();
}

molt_status molt_profile_read(molt_ctx* c, int kind, double* total_ms, int64_t* launches) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  double tot = 0.0;
  int64_t cnt = 0;
  std::vector<molt_ctx::Rec> keep;
  for (auto& r : c->recs) {
    if (r.kind != kind) {
      keep.push_back(r);
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      tot += ms;
      ++cnt;
    }
    if (r.start) cudaEventDestroy(r.start);
    if (r.stop) cudaEventDestroy(r.stop);
  }
  c->recs.swap(keep);
  if (total_ms) *total_ms = tot;
  if (launches) *launches = cnt;
  return MOLT_OK;
}

molt_status molt_destroy(molt_ctx* c) {
  if (!c) return MOLT_OK;
  cudaStreamSynchronize(c->stream);
  clear_records(c);
  for (auto& p : c->probs) {
    cudaFree(p.acc);
    cudaFree(p.stage1);
    cudaFree(p.stage2);
    cudaFree(p.hx);
    cudaFree(p.hx2);
    cudaFree(p.src);
    cudaFree(p.gp);
    cudaFree(p.gm);
    for (auto& cch : p.nu) cudaFree(cch.dev);
    for (void* t : p.nu_tmp) cudaFree(t);
    cudaFree(p.nu_sum);
    cudaFree(p.acc2);
    if (p.heat_graph) cudaGraphExecDestroy(p.heat_graph);
    for (void* v : p.hv) cudaFree(v);
    cudaFree(p.tu);
    cudaFree(p.thx);
    cudaFree(p.shadow);
  }
  if (c->batch.graph) cudaGraphExecDestroy(c->batch.graph);
  cudaFree(c->batch.d_sweeps);
  cudaFree(c->batch.d_updates);
  cudaFree(c->batch.d_bar);
  cudaFree(c->status_dev);
  cudaFree(c->speed_dev);
  cudaFree(c->t_dev);
  cudaFree(c->tnow_dev);
  cudaFree(c->mlp_blob);
  cudaFree(c->mlp_stats);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
  return MOLT_OK;
}

molt_status molt_set_mlp(molt_ctx* c, const void* blob, size_t bytes) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (!blob) return fail(c, MOLT_EINVAL, "null network");
  if (bytes != sizeof(MlpBlob)) return fail(c, MOLT_EINVAL, "network blob must be MOLT_MLP_BLOB_BYTES bytes");
  if (!c->mlp_blob) return fail(c, MOLT_EINVAL, "no problem of this context uses learned weights");
  cudaError_t e = cudaMemcpyAsync(c->mlp_blob, blob, bytes, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "molt_set_mlp");
  c->mlp_ready = true;
  return MOLT_OK;
}

molt_status molt_mlp_stats(molt_ctx* c, int64_t* stencils, int64_t* fallbacks, int reset) {
  if (!c) return fail(nullptr, MOLT_EINVAL, "null context");
  if (!c->mlp_stats) return fail(c, MOLT_EINVAL, "no problem of this context uses learned weights");
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h, c->mlp_stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && reset) {
    e = cudaMemsetAsync(c->mlp_stats, 0, sizeof(h), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "molt_mlp_stats");
  if (stencils) *stencils = int64_t(h[0]);
  if (fallbacks) *fallbacks = int64_t(h[1]);
  return MOLT_OK;
}

const char* molt_last_error(const molt_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

}  // extern "C"
