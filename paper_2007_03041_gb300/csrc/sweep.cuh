// Line-sweep kernel: the O(N) fast summation of L^{-1} and the successive-
// convolution partial sums S_P = sum_{p=1}^P D^p along one axis of a grid
// (arXiv 2007.03041, Sec. 2.1-2.4), with a fused epilogue that consumes S_P
// (store, accumulate, or the time-integrator update).
//
// Mapping.  A CTA owns W lines of one axis.  The lines are staged in shared
// memory (converted to the compute type T) with ghost cells on both ends;
// each line is processed by `nwl` warps and every lane owns kE consecutive
// points of it in registers.  Per application of D:
//   1. local integrals J_R(x_e) = sum_l c_l v_{e+l} and J_L(x_e) =
//      sum_l c_l v_{e-l} (Sec. 2.4 / App. C, optionally WENO-Z weighted) from
//      a register window of the lane's points plus 3 neighbours per side;
//   2. the recurrences I_R(x_i) = q I_R(x_{i-1}) + J_R(x_i) and
//      I_L(x_i) = q I_L(x_{i+1}) + J_L(x_i) (Sec. 2.4) as affine scans:
//      a serial fold per lane, a shuffle scan across the warp, a shared-
//      memory scan across the warps of a line (the exact block split of the
//      convolution sums, Sec. 3, without any truncation);
//   3. the boundary constants from the line totals in FP64 (Sec. 2.3:
//      periodic A = I(b)/(1-mu), B = I(a)/(1-mu); Dirichlet: the 2x2 system
//      with determinant 1-mu^2, Sec. 3.3), folded into the scans as their
//      initial values so that A e^{-alpha(x-a)} needs no pow();
//   4. a fix-up pass giving L^{-1} (in FP32 the recurrence is accumulated
//      with a compensation term: exact product error by FMA, TwoSum for the
//      addition), then D = v - L^{-1}.
// D is written back to shared memory for the next power.  The epilogue runs
// in the coalesced load mapping.
//
// Precision plumbing.  GB300 executes FP64 arithmetic and FP64<->FP32
// conversions at a small fraction of the FP32 rate, so per-point FP64 work is
// kept to the update itself: sweeps read an FP32 copy of the state (written
// by the previous update), conversions are done with integer bit operations,
// and only the state update uses FP64 fused multiply-adds.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp.cuh"

namespace molt {

constexpr int kE = 16;   // points per lane
constexpr int kG = 16;   // ghost slots per side in shared memory (3 used)
#ifndef MOLT_MAX_THREADS
#define MOLT_MAX_THREADS 512
#endif
constexpr int kMaxThreads = MOLT_MAX_THREADS;
#ifndef MOLT_MIN_BLOCKS
#define MOLT_MIN_BLOCKS 1
#endif
constexpr int kMinBlocks = MOLT_MIN_BLOCKS;   // resident CTAs per SM the register budget targets
// Shared memory per CTA (the GPU allows 227 KB): a sweep tile's budget, and the
// dynamic size the sweep kernels opt into (a TMA tile plus its staging buffer
// must fit it).
constexpr size_t kSmemTileBudget = 200 * 1024;
constexpr size_t kSmemOptIn = 210 * 1024;

enum Epi {
  EPI_STORE = 0,       // out = S
  EPI_ACC_SET = 1,     // acc = S
  EPI_ACC_ADD = 2,     // acc += S
  EPI_HEAT_FINAL = 3,  // dst = a0*un + a1*(us + coefS*(acc + S))
  EPI_WAVE_FINAL = 4,  // dst = 2u - uprev + coefS*(acc+S)  (or from rest)
  EPI_HJ_X = 5,        // hx = H^_x(D_R, D_L); speed max
  EPI_HJ_Y = 6,        // u -= dt*H^; speed max
  EPI_HJ_XG = 7,       // EPI_HJ_X for every Hamiltonian (HamKind)
  EPI_HJ_YG = 8,       // EPI_HJ_Y for every Hamiltonian, a source F(x, t), speed-only passes
  EPI_ACC_AXPY = 9     // acc += coefS * S (advection-diffusion terms)
};
// The general Hamilton-Jacobi kernels (XG/YG) carry more operands per point;
// the |grad u|^2/2 kernels without a source keep their own instantiations.
__host__ __device__ constexpr bool epi_hj_x(int e) { return e == EPI_HJ_X || e == EPI_HJ_XG; }
__host__ __device__ constexpr bool epi_hj_y(int e) { return e == EPI_HJ_Y || e == EPI_HJ_YG; }
__host__ __device__ constexpr bool epi_hj_gen(int e) { return e == EPI_HJ_XG || e == EPI_HJ_YG; }
// Hamiltonian of the Hamilton-Jacobi step (values of molt_hamiltonian).
//   HALF_SQ:   H = |grad u|^2/2, separable: each pass adds its axis's part of
//              the local Lax-Friedrichs Hamiltonian
//   LINEAR:    H = sum_d a_d u_d, separable (upwind: H^_d = a_d v^-_d for
//              a_d > 0, a_d v^+_d for a_d < 0)
//   AFFINE_SQ: H = (h0 + sum_d a_d u_d)^2/2, not separable: the x pass leaves
//              sigma_x = a_x mean_x and delta_x = |a_x| (v^+_x - v^-_x)/2, the
//              last pass forms H^ from all axes
enum HamKind { HAM_HALF_SQ = 0, HAM_LINEAR = 1, HAM_AFFINE_SQ = 2 };
enum Mode { MODE_L = 0, MODE_R = 1, MODE_0 = 2, MODE_RL = 3 };
enum StatusBits { ST_NONFINITE = 1, ST_TIMEOUT = 2 };

struct LineGeom {
  int n;              // stored points per line
  long long nlines;   // lines in this pass
  long long nlo;      // line l = hi*nlo + lo
  long long s_lo, s_hi;
  long long stride;   // element stride along the line
};

struct SweepArgs {
  LineGeom g;
  int W, nwl, LS;     // lines per CTA, warps per line, shared line stride (elements)
  int E;              // points per lane of the plain kernel (16, 8 or 4; others mean 16)
  int bc;             // 0 periodic, 1 Dirichlet
  int mode;           // Mode
  int P;
  int contiguous;     // stride == 1
  double c[6];        // J_R weights on offsets -3..2
  double sub[3][4];   // WENO substencil weights (5-point rule)
  double d[3];        // linear weights
  double q;           // e^{-nu}
  double qE;          // e^{-nu E}
  double invq;        // e^{+nu}
  double inv1mmu;     // 1/(1-mu)
  double mu;          // e^{-alpha(b-a)}
  double invdet;      // 1/(1-mu^2)
  double k2det, k2detq;  // 2/(1-mu^2) and 2 e^{nu}/(1-mu^2) (Dirichlet L_0 carries)
  double alpha;
  // the same coefficients rounded to FP32 on the host (FP32 kernels read
  // these; converting on the device would use the FP64 pipe)
  float cf[6], subf[3][3], df[3], qf, qEf, alphaf;
  // epilogue operands
  const void* in;     // sweep input (TIN)
  void* out;          // EPI_STORE destination / HJ: H^_x buffer (state type)
  void* acc;          // accumulator (compute type)
  const void* un;     // heat: u^n; wave: u^n; HJ: u (state type)
  const void* us;     // heat: stage state; wave: u^{n-1}
  void* dst;          // final destination (state type)
  void* dst2;         // wave: receives u^n (old state) when non-null
  float* shadow;      // FP32 copy of dst written by final epilogues (or null)
  double a0, a1, coefS;
  int from_rest;      // wave Taylor start
  // Hamilton-Jacobi
  const unsigned long long* lag;  // lagged speed (double bits)
  unsigned long long* speed;      // this pass's speed slot (double bits)
  // adaptive step (Eq. "adaptive time rule"): dt = cfl min_d h_d / c_d =
  // cfl / max_d (c_d / h_d); the passes publish c_d / h_d
  double cfl, dt_max, inv_h;   // inv_h = 1 / h of this pass's axis
  double* t_dev;            // time accumulator (HJ_Y, block 0)
  int ham;                  // HamKind
  int two_out;              // MODE_RL with AFFINE_SQ: a second line buffer (delta)
  double vel, h0, vmax;     // a_d of this axis, h0, max_d |a_d| / h_d
  float velf;
  void* out2;               // AFFINE_SQ: delta_x (state type; written by the x pass, read by the last)
  const void* src;          // source coefficients F_k, k = 0..src_deg (state type) or null
  int src_deg;
  long long src_stride;     // elements between F_k and F_{k+1}
  const double* t_now;      // time of the state being advanced (read with a source)
  int* status;
  // learned weights (JQ_LEARNED kernels)
  const MlpBlob* mlp;               // BF16 network
  unsigned long long* mlp_stats;    // [stencils evaluated, WENO-Z fallbacks]
};

// Local-quadrature kind of a sweep kernel (template parameter JQ).
enum JQuad { JQ_LINEAR = 0, JQ_WENOZ = 1, JQ_LEARNED = 2 };

// Shared-memory index of point e of a line whose lanes own E points each: one
// pad word after every E words (kG is a multiple of E), so lane chunks start
// (E+1) words apart -- an odd stride, hence bank-conflict free.
template <int E>
__host__ __device__ constexpr int log2i() { return E == 16 ? 4 : (E == 8 ? 3 : (E == 4 ? 2 : -1)); }

template <int E = kE>
__host__ __device__ constexpr int phys(int e) {
  static_assert(log2i<E>() > 0, "points per lane must be 4, 8 or 16");
  return (e + kG) + ((e + kG) >> log2i<E>());
}

// For a lane chunk starting at e0 = E*t: phys(e0 + j) = (E+1)*t +
// chunk_off<E>(j), a compile-time constant for unrolled j.
template <int E = kE>
__host__ __device__ constexpr int chunk_off(int j) { return (j + kG) + ((j + kG) >> log2i<E>()); }

// Base offset of line l (32-bit division: the host keeps nlines < 2^31; a
// 64-bit division would run on the FP64 pipe).
__device__ __forceinline__ long long line_base(const LineGeom& g, long long l) {
  const unsigned int lu = unsigned(l), nlo = unsigned(g.nlo);
  const unsigned int hi = lu / nlo, lo = lu - hi * nlo;
  return (long long)hi * g.s_hi + (long long)lo * g.s_lo;
}

// ------------------------------------------------------------ conversions
// The hardware conversions between FP32 and FP64 run on the FP64 pipe, which
// is narrow on this part; the common operands are converted by integer
// operations on the bit patterns instead.  The rare operands leave through a
// call, so that the hardware conversion runs for them alone (a plain branch
// to it would be if-converted, executing it for every operand).  A
// translation unit whose kernels have no registers to spare for a call
// defines MOLT_CONV_SELECT 1: the hardware conversion is then selected in
// place (measured: the batched heat step, 6.78 ms with it, 8.18 with calls;
// the 512^3 wave step, 1.93 ms with it, 1.76 with calls).
#ifndef MOLT_CONV_SELECT
#define MOLT_CONV_SELECT 0
#endif
static __device__ __noinline__ float d2f_rare(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double f2d_rare(float x) { return double(x); }

// double -> float, round to nearest even: normal results by integer
// operations; results that round to zero (|x| < 2^-150) give the signed
// zero; subnormal results, overflow, inf and NaN take the hardware conversion.
__device__ __forceinline__ float d2f(double x) {
  const unsigned int hi = __double2hiint(x);
  const unsigned int lo = __double2loint(x);
  const unsigned int e11 = (hi >> 20) & 0x7FFu;
  if (e11 < 897u || e11 > 1150u) {
    if (e11 < 873u) return __uint_as_float(hi & 0x80000000u);
    if constexpr (MOLT_CONV_SELECT) return __double2float_rn(x);
    else return d2f_rare(x);
  }
  const unsigned int mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned int rest = lo & 0x1FFFFFFFu;           // 29 dropped bits
  const unsigned int half = 0x10000000u;
  const unsigned int up = (rest > half) | ((rest == half) & (mant & 1u));
  const unsigned int bits = (hi & 0x80000000u) | (((e11 - 896u) << 23) + mant + up);
  return __uint_as_float(bits);
}

// float -> double (exact): normal numbers and zeros by integer operations;
// subnormals, inf and NaN take the hardware conversion.
__device__ __forceinline__ double f2d(float x) {
  const unsigned int u = __float_as_uint(x);
  const unsigned int e8 = (u >> 23) & 0xFFu;
  if (e8 == 0u || e8 == 255u) {
    if ((u << 1) == 0u) return __hiloint2double(int(u & 0x80000000u), 0);
    if constexpr (MOLT_CONV_SELECT) return double(x);
    else return f2d_rare(x);
  }
  const unsigned int hi = (u & 0x80000000u) | ((e8 + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  const unsigned int lo = u << 29;
  return __hiloint2double(int(hi), int(lo));
}

template <typename T>
__device__ __forceinline__ T pick(double d, float f) {
  if constexpr (sizeof(T) == 4) return f; else return d;
}

// Non-finite test on the exponent bits (no floating-point instruction).
__device__ __forceinline__ bool nonfinite(double x) { return (__double2hiint(x) & 0x7FF00000) == 0x7FF00000; }
__device__ __forceinline__ bool nonfinite(float x) { return (__float_as_uint(x) & 0x7F800000u) == 0x7F800000u; }

// Global load; CG = true reads through L2 only (data written earlier in the
// same kernel by other CTAs must not come from a stale L1 line).
template <bool CG, typename V>
__device__ __forceinline__ V gload(const V* p) {
  if constexpr (CG) return __ldcg(p); else return *p;
}

template <typename TO, typename FROM>
__device__ __forceinline__ TO cvt(FROM x) {
  if constexpr (sizeof(TO) == 4 && sizeof(FROM) == 8) return d2f(x);
  else if constexpr (sizeof(TO) == 8 && sizeof(FROM) == 4) return f2d(x);
  else return TO(x);
}

// ---------------------------------------------------------------- arithmetic
// y <- a*y + b on y = hi + lo.  FP32: compensated (exact product error by FMA,
// TwoSum for the addition).  FP64: plain FMA.
#ifndef MOLT_SHARED_BETA
#define MOLT_SHARED_BETA 1   // WENO-Z: smoothness indicators from per-triple products shared by neighbouring points
#endif
#ifndef MOLT_COMPENSATED
#define MOLT_COMPENSATED 1
#endif
template <typename T>
struct Acc {
  T hi, lo;
  __device__ __forceinline__ void step(T a, T b) {
    if constexpr (sizeof(T) == 4 && MOLT_COMPENSATED) {
      const T p = a * hi;
      const T pe = fmaf(a, hi, -p);
      const T s = p + b;
      const T bb = s - p;
      const T se = (p - (s - bb)) + (b - bb);
      lo = fmaf(a, lo, pe + se);
      hi = s;
    } else {
      hi = fma(a, hi, b);
    }
  }
  __device__ __forceinline__ T value() const {
    if constexpr (sizeof(T) == 4 && MOLT_COMPENSATED) return hi + lo; else return hi;
  }
};

template <typename T>
__device__ __forceinline__ T shfl_up(T v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <typename T>
__device__ __forceinline__ T shfl_down(T v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

// WENO-Z weighted local integral from the 5 values w[0..4] = v at offsets
// -3..1 relative to the target node, in the orientation of J_R (J_L passes
// the mirrored values).  Smoothness indicators: beta_r = int_{-1}^0
// (p_r')^2 + (p_r'')^2 dt for the quadratic through substencil r, worked out
// in closed form with s1 = (c-a)/2, s2 = a-2b+c:
//   beta_0 = s1^2 + 3 s1 s2 + 10/3 s2^2,  beta_1 = s1^2 + s1 s2 + 4/3 s2^2,
//   beta_2 = s1^2 - s1 s2 + 4/3 s2^2.
// WENO-Z (Sec. 2.4): w~_r = d_r (1 + tau/(eps+beta_r)), tau = |beta_0-beta_2|.
// Reciprocal for the nonlinear weights: FP32 takes the hardware
// approximation (at most 1 ulp; the arguments eps + beta_r and sum_r w~_r are
// at least 1e-6 and about 1), FP64 the division.
__device__ __forceinline__ float weight_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double weight_rcp(double x) { return 1.0 / x; }

template <typename T>
__device__ __forceinline__ T wenoz_from_beta(const T* w, const T (&beta)[3], const T (&sub)[3][3], const T (&d)[3]) {
  T J[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) J[r] = sub[r][0] * w[r] + sub[r][1] * w[r + 1] + sub[r][2] * w[r + 2];
  const T tau = fabs(beta[0] - beta[2]);
  const T eps = T(1e-6);
  T wt[3], sum = T(0);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    wt[r] = fma(d[r] * tau, weight_rcp(eps + beta[r]), d[r]);   // d_r (1 + tau/(eps+beta_r))
    sum += wt[r];
  }
  return (wt[0] * J[0] + wt[1] * J[1] + wt[2] * J[2]) * weight_rcp(sum);
}

// The smoothness indicator of substencil r from the products of its node
// triple (a, b, c): with s1 = (c - a)/2 and s2 = a - 2b + c, beta_r = s1^2 +
// k_r s1 s2 + m_r s2^2 (k = 3, 1, -1; m = 10/3, 4/3, 4/3).  A triple serves
// three points' J_R and, mirrored (s1 -> -s1), three points' J_L, so the
// products are formed once per triple.
template <typename T>
__device__ __forceinline__ void triple_products(T a, T b, T c, T* p11, T* p12, T* p22) {
  const T s1 = T(0.5) * (c - a);
  const T s2 = a - T(2) * b + c;
  *p11 = s1 * s1;
  *p12 = s1 * s2;
  *p22 = s2 * s2;
}
template <typename T>
__device__ __forceinline__ T beta_from_products(int r, T p11, T p12, T p22, bool mirrored) {
  const T k = r == 0 ? T(3) : (r == 1 ? T(1) : T(-1));
  const T m = r == 0 ? T(10.0 / 3.0) : T(4.0 / 3.0);
  return p11 + (mirrored ? -k : k) * p12 + m * p22;
}

template <typename T>
__device__ __forceinline__ T wenoz_integral(const T* w, const T (&sub)[3][3], const T (&d)[3]) {
  T J[3], beta[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const T a = w[r], b = w[r + 1], c = w[r + 2];
    J[r] = sub[r][0] * a + sub[r][1] * b + sub[r][2] * c;
    const T s1 = T(0.5) * (c - a);
    const T s2 = a - T(2) * b + c;
    const T k = r == 0 ? T(3) : (r == 1 ? T(1) : T(-1));
    const T m = r == 0 ? T(10.0 / 3.0) : T(4.0 / 3.0);
    beta[r] = s1 * s1 + k * s1 * s2 + m * s2 * s2;
  }
  const T tau = fabs(beta[0] - beta[2]);
  const T eps = T(1e-6);
  T wt[3], sum = T(0);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    wt[r] = fma(d[r] * tau, weight_rcp(eps + beta[r]), d[r]);   // d_r (1 + tau/(eps+beta_r))
    sum += wt[r];
  }
  return (wt[0] * J[0] + wt[1] * J[1] + wt[2] * J[2]) * weight_rcp(sum);
}

// -------------------------------------------------------------- tile staging
// Contiguous lines: the nwl warps of line lw read it with consecutive lanes.
// Strided lines: thread (p, w) with w fastest, so a warp reads whole rows of
// W neighbouring lines.
template <typename T, typename TIN, int E = kE, bool CG = false>
__device__ __forceinline__ void load_tile(const SweepArgs& a, const TIN* in, T* lines, long long line0,
                                          int lw, int tl) {
  const int W = a.W, n = a.g.n;
  if (a.contiguous) {
    const long long gl = line0 + lw;
    if (gl >= a.g.nlines) return;
    const TIN* src = in + line_base(a.g, gl);
    T* dstl = lines + lw * a.LS;
    const int step = a.nwl * 32;
#pragma unroll 4
    for (int p = tl; p < n; p += step) dstl[phys<E>(p)] = cvt<T>(gload<CG>(src + p));
  } else {
    // prow = blockDim/W is a multiple of 16, so phys<E>() advances by a constant
    const int w = threadIdx.x % W;
    const int prow = blockDim.x / W;
    const long long gl = line0 + w;
    if (gl >= a.g.nlines) return;
    const long long st = a.g.stride;
    int p = threadIdx.x / W;
    const TIN* src = in + line_base(a.g, gl) + p * st;
    const long long sstep = prow * st;
    T* dst = lines + w * a.LS + phys<E>(p);
    const int dstep = prow + prow / E;
#pragma unroll 8
    for (; p < n; p += prow) {
      *dst = cvt<T>(gload<CG>(src));
      src += sstep;
      dst += dstep;
    }
  }
}

template <typename T, int E = kE>
__device__ __forceinline__ void fill_ghosts(const SweepArgs& a, T* lines) {
  const int n = a.g.n;
  for (int t = threadIdx.x; t < a.W * 6; t += blockDim.x) {
    const int w = t / 6, g = t - w * 6;
    T* b = lines + w * a.LS;
    if (g < 3) {
      const int j = g + 1;  // ghost e = -j
      T val;
      if (a.bc == 0) {
        int s = (-j) % n;
        if (s < 0) s += n;
        val = b[phys<E>(s)];
      } else {
        const int m = j < n - 1 ? j : n - 1;
        val = T(2) * b[phys<E>(0)] - b[phys<E>(m)];
      }
      b[phys<E>(-j)] = val;
    } else {
      const int j = g - 2;  // ghost e = n-1+j
      T val;
      if (a.bc == 0) {
        val = b[phys<E>((n - 1 + j) % n)];
      } else {
        const int m = n - 1 - j > 0 ? n - 1 - j : 0;
        val = T(2) * b[phys<E>(n - 1)] - b[phys<E>(m)];
      }
      b[phys<E>(n - 1 + j)] = val;
    }
  }
}

// ------------------------------------------------------------------- kernels
// T: compute type; TIN: sweep input element type; TST: state type of the
// epilogue operands.

struct TileSmem {
  double* carries;   // [W][4] compute-type (hi, lo) carry pairs (room for FP64)
  void* totals;      // [W][nwl][4] of T
  void* lines;       // [W][LS] of T
  void* lines2;      // two_out: [W][LS] of T (delta of AFFINE_SQ)
  float* jloc;       // JQ_LEARNED: [W][2][LS] local integrals J_R, J_L
  MlpNet* net;       // JQ_LEARNED: the network
};

// Shared bytes of a tile beyond the lines for learned weights (the host
// planner adds the same amount).
__host__ __device__ constexpr size_t learned_extra_bytes(int W, int LS) {
  return 16 + size_t(2) * W * LS * sizeof(float) + sizeof(MlpNet);
}

template <typename T, int JQ = JQ_LINEAR>
__device__ __forceinline__ TileSmem carve(unsigned char* smem, const SweepArgs& a, size_t* used) {
  TileSmem t;
  t.carries = reinterpret_cast<double*>(smem);
  t.totals = reinterpret_cast<T*>(t.carries + 4 * a.W);
  const size_t off = (size_t(4 * a.W) * sizeof(double) + size_t(a.W * a.nwl * 4) * sizeof(T) + 15) & ~size_t(15);
  t.lines = smem + off;
  *used = off + size_t(a.W) * a.LS * sizeof(T);
  t.lines2 = nullptr;
  if (a.two_out) {
    const size_t l2 = (*used + 15) & ~size_t(15);
    t.lines2 = smem + l2;
    *used = l2 + size_t(a.W) * a.LS * sizeof(T);
  }
  t.jloc = nullptr;
  t.net = nullptr;
  if constexpr (JQ == JQ_LEARNED) {
    const size_t j0 = (*used + 15) & ~size_t(15);
    t.jloc = reinterpret_cast<float*>(smem + j0);
    const size_t n0 = j0 + size_t(2) * a.W * a.LS * sizeof(float);
    t.net = reinterpret_cast<MlpNet*>(smem + n0);
    *used = n0 + sizeof(MlpNet);
  }
  return t;
}

// Fills the ghosts of the staged lines, applies D P times (the whole method
// step of the header comment) and leaves S_P (or, for MODE_RL, the per-axis
// Lax-Friedrichs Hamiltonian) in the line buffers.  Returns the thread's
// largest one-sided derivative magnitude (MODE_RL).  Ends synchronised.
// Pairs of compute-type values advanced together: FP32 pairs use the packed
// FP32x2 instructions of sm_100+ (FFMA2/FADD2/FMUL2), FP64 pairs plain FMAs.
template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ typename Pair<T>::type pair2(T x, T y) {
  typename Pair<T>::type r;
  r.x = x;
  r.y = y;
  return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b exactly as an FMA with -1
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Acc on a pair of independent recurrences (y <- a*y + b per component).
template <typename T>
struct Acc2 {
  using V = typename Pair<T>::type;
  V hi, lo;
  __device__ __forceinline__ void step(V a, V b) {
    if constexpr (sizeof(T) == 4 && MOLT_COMPENSATED) {
      const V p = mul2(a, hi);
      const V pe = fma2(a, hi, pair2<T>(-p.x, -p.y));
      const V s = add2(p, b);
      const V bb = sub2(s, p);
      const V se = add2(sub2(p, sub2(s, bb)), sub2(b, bb));
      lo = fma2(a, lo, add2(pe, se));
      hi = s;
    } else {
      hi = fma2(a, hi, b);
    }
  }
  __device__ __forceinline__ V value() const {
    if constexpr (sizeof(T) == 4 && MOLT_COMPENSATED) return add2(hi, lo); else return hi;
  }
};

// Line boundary constants (Sec. 2.3, Sec. 3.3) in FP64 from the line totals
// I_R(b) = tbR and I_L(a) = tbL, returned as the initial values of the R and
// L scans: periodic -> the cyclic values I(b)/(1-mu), I(a)/(1-mu);
// Dirichlet L_0 -> 2A and 2B from the 2x2 system with determinant 1-mu^2;
// Dirichlet L_R / L_L -> v(a) / v(b).  Exact-fit kernels divide Dirichlet
// values by q (their end nodes keep the map (q, 0)).
template <typename T, bool RAGGED, int E = kE>
__device__ __forceinline__ void boundary_carries(const SweepArgs& a, const T* bw, int n, T tbR, T tbL, double* CR,
                                                 double* CL) {
  const double IRb = cvt<double>(tbR);
  const double ILa = cvt<double>(tbL);
  if (a.bc == 0) {
    *CR = IRb * a.inv1mmu;
    *CL = ILa * a.inv1mmu;
    return;
  }
  const double v0 = cvt<double>(bw[phys<E>(0)]), vN = cvt<double>(bw[phys<E>(n - 1)]);
  double cr, cl;
  if (a.mode == MODE_0) {
    // 2A, 2B (the 1/q of exact-fit kernels folded into the constant)
    const double r0 = fma(-0.5, ILa, v0), r1 = fma(-0.5, IRb, vN);
    const double k = RAGGED ? a.k2det : a.k2detq;
    cr = fma(-a.mu, r1, r0) * k;
    cl = fma(-a.mu, r0, r1) * k;
  } else {
    cr = v0;   // L_R^{-1}(a) = v(a)
    cl = vN;   // L_L^{-1}(b) = v(b)
    if (!RAGGED) {
      cr *= a.invq;
      cl *= a.invq;
    }
  }
  *CR = cr;
  *CL = cl;
}

// Compute-type (hi, lo) pair of an FP64 carry.
template <typename T>
__device__ __forceinline__ void split_carry(double c, T* hi, T* lo) {
  const T h = cvt<T>(c);
  *hi = h;
  *lo = cvt<T>(c - cvt<double>(h));
}

// Ghost cells of one line by the lanes of the warp that owns it.
template <typename T, int E = kE>
__device__ __forceinline__ void warp_fill_ghosts(const SweepArgs& a, T* b, int lane) {
  const int n = a.g.n;
  if (lane < 3) {
    const int j = lane + 1;  // ghost e = -j
    T val;
    if (a.bc == 0) {
      int s = (-j) % n;
      if (s < 0) s += n;
      val = b[phys<E>(s)];
    } else {
      const int m = j < n - 1 ? j : n - 1;
      val = T(2) * b[phys<E>(0)] - b[phys<E>(m)];
    }
    b[phys<E>(-j)] = val;
  } else if (lane < 6) {
    const int j = lane - 2;  // ghost e = n-1+j
    T val;
    if (a.bc == 0) {
      val = b[phys<E>((n - 1 + j) % n)];
    } else {
      const int m = n - 1 - j > 0 ? n - 1 - j : 0;
      val = T(2) * b[phys<E>(n - 1)] - b[phys<E>(m)];
    }
    b[phys<E>(n - 1 + j)] = val;
  }
}

// Learned local integrals of the points a warp owns (32*E consecutive points
// of its line from `first`): for 16 points at a time and each side, the lanes
// gather the 5-value stencils (J_R: v_{e-3..e+1}; J_L mirrored: v_{e+3..e-1})
// from the staged line, the warp evaluates the network on the tensor cores,
// and lanes t = 0, 1 of each row group finish rows g, g+8: WENO-Z fallback
// check, then J = sum_r w_r J^{(r)} into jr / jl (shared, line layout).
template <int E>
__device__ __forceinline__ void learned_local_integrals(const SweepArgs& a, const MlpNet& net, const float* buf,
                                                        float* jr, float* jl, int first, int n, int lane) {
  const int g = lane >> 2, t = lane & 3;
  MlpRegs R;
  mlp_load_regs(net, lane, R);
  float sub[3][3], d[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    d[r] = a.df[r];
#pragma unroll
    for (int j = 0; j < 3; ++j) sub[r][j] = a.subf[r][j];
  }
  unsigned evaluated = 0, fallbacks = 0;
  for (int b = 0; b < 32 * E; b += 16) {
    if (first + b >= n) break;   // warp-uniform
    const int e0 = first + b + g, e1 = e0 + 8;
    const int c0 = e0 < n ? e0 : n - 1, c1 = e1 < n ? e1 : n - 1;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      float v0[5], v1[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        const int o = side == 0 ? j - 3 : 3 - j;
        v0[j] = buf[phys<E>(c0 + o)];
        v1[j] = buf[phys<E>(c1 + o)];
      }
      float x0[5], x1[5];
      mlp_normalise(v0, x0);
      mlp_normalise(v1, x1);
      uint32_t xa[4];
      mlp_input_frag(x0, x1, t, xa);
      MlpCache f;
      float p0[3], p1[3];
      mlp_forward16(R, xa, f, p0, p1);
      const int e = t == 0 ? e0 : e1;
      if (t < 2 && e < n) {
        float v[5], p[3], w[3];
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = t == 0 ? v0[j] : v1[j];
#pragma unroll
        for (int r = 0; r < 3; ++r) p[r] = t == 0 ? p0[r] : p1[r];
        fallbacks += mlp_final_weights(v, p, d, w) ? 1u : 0u;
        ++evaluated;
        float J = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) J = fmaf(w[r], fmaf(sub[r][0], v[r], fmaf(sub[r][1], v[r + 1], sub[r][2] * v[r + 2])), J);
        (side == 0 ? jr : jl)[phys<E>(e)] = J;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o);
    fallbacks += __shfl_xor_sync(0xffffffffu, fallbacks, o);
  }
  if (lane == 0 && a.mlp_stats) {
    atomicAdd(a.mlp_stats, (unsigned long long)evaluated);
    if (fallbacks) atomicAdd(a.mlp_stats + 1, (unsigned long long)fallbacks);
  }
}

// WL (warp-local): every line is owned by a single warp (nwl == 1), so a D
// application needs no CTA-wide barrier: ghosts, line totals and the FP64
// boundary solve stay inside the warp (the solve runs on lane 0 and its
// result is broadcast by shuffles).
// GEN: MODE_RL supports every HamKind (else |grad u|^2/2 only).
template <typename T, int JQ, bool RAGGED, bool WL, int E = kE, bool GEN = false>
__device__ __forceinline__ double compute_lines(const SweepArgs& a, const TileSmem& sm, bool line_ok) {
  static_assert(JQ != JQ_LEARNED || sizeof(T) == 4, "learned weights run in FP32");
  const int nwl = a.nwl, n = a.g.n;
  double* carries = sm.carries;
  T* totals = static_cast<T*>(sm.totals);
  T* lines = static_cast<T*>(sm.lines);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lw = warp / nwl, part = warp - lw * nwl;
  const int tl = part * 32 + lane;
  T* buf = lines + lw * a.LS;
  const int e0 = tl * E;
  T* cbase = buf + (E + 1) * tl;   // phys<E>(e0 + j) = (E+1)*tl + chunk_off<E>(j)
  static_assert(phys<E>(E * 3 + 2) == (E + 1) * 3 + chunk_off<E>(2), "lane base / chunk offset mismatch");

  const T q = pick<T>(a.q, a.qf);
  const T qE = pick<T>(a.qE, a.qEf);
  T c[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) c[i] = pick<T>(a.c[i], a.cf[i]);
  T sub[3][3], dw[3];
  if constexpr (JQ == JQ_WENOZ) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dw[r] = pick<T>(a.d[r], a.df[r]);
#pragma unroll
      for (int j = 0; j < 3; ++j) sub[r][j] = pick<T>(a.sub[r][j], a.subf[r][j]);
    }
  }
  // lines owned by one warp (nwl == 1) need CTA barriers only around the
  // vectorised boundary solve: ghosts, write-backs and the final store of a
  // line are warp-local
  const bool own = nwl == 1;
  if (WL || own) {
    warp_fill_ghosts<T, E>(a, buf, lane);
    __syncwarp();
  } else {
    fill_ghosts<T, E>(a, lines);
    __syncthreads();
  }

  // element maps: (q, J) for points with a local integral, identity for
  // points past the end of the line and for the Dirichlet end nodes where the
  // recurrences start (I_R(x_0) = 0, I_L(x_N) = 0).  RAGGED kernels mask per
  // point.  Exact-fit kernels (n = nwl*32*E) have no points past the end;
  // their Dirichlet end nodes keep the map (q, 0) and the line's initial
  // value is divided by q, which yields the same values (x_0: q*(C/q) + 0 = C).
  const int eR0 = (a.bc == 1) ? 1 : 0;          // first R point with a J
  const int eL1 = (a.bc == 1) ? n - 2 : n - 1;  // last L point with a J
  const bool zeroR0 = !RAGGED && a.bc == 1 && e0 == 0;
  const bool zeroLN = !RAGGED && a.bc == 1 && e0 + E == n;

  // J_R(e0+k) and J_L(e0+E-1-k) share the pair Y[k] so that the R chain
  // (ascending) and the L chain (descending) of the recurrences advance
  // together in packed FP32x2 instructions.
  using T2 = typename Pair<T>::type;
  T v[E], S[E];
  T2 Y[E];
#pragma unroll
  for (int k = 0; k < E; ++k) S[k] = T(0);
  T rmax = T(0);

  for (int p = 0; p < a.P; ++p) {
    // ---- 1. local integrals from a window of E + 6 points
    float* jrl = nullptr;
    if constexpr (JQ == JQ_LEARNED) {
      jrl = sm.jloc + lw * 2 * a.LS;
      if (line_ok) learned_local_integrals<E>(a, *sm.net, buf, jrl, jrl + a.LS, part * 32 * E, n, lane);
      __syncwarp();
    }
    {
      T win[E + 6];
#pragma unroll
      for (int k = 0; k < E + 6; ++k) win[k] = cbase[chunk_off<E>(k - 3)];
#if MOLT_SHARED_BETA
      T p11[E + 4], p12[E + 4], p22[E + 4];   // products of the node triples win[t..t+2]
      if constexpr (JQ == JQ_WENOZ) {
#pragma unroll
        for (int t = 0; t < E + 4; ++t) triple_products<T>(win[t], win[t + 1], win[t + 2], &p11[t], &p12[t], &p22[t]);
      }
#endif
#pragma unroll
      for (int k = 0; k < E; ++k) {
        v[k] = win[k + 3];
        if constexpr (JQ == JQ_LEARNED) {
          Y[k].x = jrl[(E + 1) * tl + chunk_off<E>(k)];
          Y[E - 1 - (k)].y = jrl[a.LS + (E + 1) * tl + chunk_off<E>(k)];
        } else if constexpr (JQ == JQ_WENOZ) {
          T wr[5], wl[5];
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            wr[j] = win[k + j];        // offsets -3..1
            wl[j] = win[k + 6 - j];    // mirrored: v_{e+3} .. v_{e-1}
          }
#if MOLT_SHARED_BETA
          // substencil r of J_R is the triple at k + r; of J_L the triple at
          // k + 4 - r, reversed
          T bR[3], bL[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            bR[r] = beta_from_products<T>(r, p11[k + r], p12[k + r], p22[k + r], false);
            bL[r] = beta_from_products<T>(r, p11[k + 4 - r], p12[k + 4 - r], p22[k + 4 - r], true);
          }
          Y[k].x = wenoz_from_beta<T>(wr, bR, sub, dw);
          Y[E - 1 - (k)].y = wenoz_from_beta<T>(wl, bL, sub, dw);
#else
          Y[k].x = wenoz_integral<T>(wr, sub, dw);
          Y[E - 1 - (k)].y = wenoz_integral<T>(wl, sub, dw);
#endif
        } else {
          T r = T(0), l = T(0);
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            r = fma(c[j], win[k + j], r);       // v_{e + (j-3)}
            l = fma(c[j], win[k + 6 - j], l);   // v_{e - (j-3)}
          }
          Y[k].x = r;
          Y[E - 1 - (k)].y = l;
        }
      }
    }
    if (zeroR0) Y[0].x = T(0);
    if (zeroLN) Y[E - 1 - (E - 1)].y = T(0);
    // ---- 2a. lane folds (R ascending, L descending, interleaved)
    T aR, aL, bR, bL;
    if constexpr (!RAGGED) {
      const T2 q2 = pair2<T>(q, q);
      T2 y = pair2<T>(T(0), T(0));
#pragma unroll
      for (int k = 0; k < E; ++k) y = fma2(q2, y, Y[k]);
      aR = qE;
      aL = qE;
      bR = y.x;
      bL = y.y;
    } else {
      T r = T(0), l = T(0);
      aR = T(1);
      aL = T(1);
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int e = e0 + k;
        if (e >= eR0 && e < n) { r = fma(q, r, Y[k].x); aR *= q; }
        const int eL = e0 + E - 1 - k;
        if (eL <= eL1) { l = fma(q, l, Y[E - 1 - (E - 1 - k)].y); aL *= q; }
      }
      bR = r;
      bL = l;
    }
    // ---- 2b. warp scans (R ascending, L descending)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T ap = shfl_up(aR, o), bp = shfl_up(bR, o);
      const T an = shfl_down(aL, o), bn = shfl_down(bL, o);
      if (lane >= o) { bR = fma(aR, bp, bR); aR *= ap; }
      if (lane + o < 32) { bL = fma(aL, bn, bL); aL *= an; }
    }
    T exaR = shfl_up(aR, 1), exbR = shfl_up(bR, 1);
    T exaL = shfl_down(aL, 1), exbL = shfl_down(bL, 1);
    if (lane == 0) { exaR = T(1); exbR = T(0); }
    if (lane == 31) { exaL = T(1); exbL = T(0); }
    T* tot = totals + (lw * nwl) * 4;
    if constexpr (!WL) {
      if (lane == 31) { tot[part * 4 + 0] = aR; tot[part * 4 + 1] = bR; }
      if (lane == 0) { tot[part * 4 + 2] = aL; tot[part * 4 + 3] = bL; }
      __syncthreads();
    }
    // ---- 2c. across the warps of the line
    T paR = T(1), pbR = T(0), paL = T(1), pbL = T(0);
    for (int j = 0; j < part; ++j) {
      const T A = tot[j * 4 + 0], B = tot[j * 4 + 1];
      pbR = fma(A, pbR, B);
      paR *= A;
    }
    for (int j = nwl - 1; j > part; --j) {
      const T A = tot[j * 4 + 2], B = tot[j * 4 + 3];
      pbL = fma(A, pbL, B);
      paL *= A;
    }
    // ---- 3. boundary constants in FP64
    T cRh, cRl, cLh, cLl;
    if constexpr (WL) {
      // lane 31 holds the R line total, lane 0 the L line total
      const T tbR = __shfl_sync(0xffffffffu, bR, 31);
      const T tbL = __shfl_sync(0xffffffffu, bL, 0);
      T c4[4] = {T(0), T(0), T(0), T(0)};
      if (lane == 0) {
        double CR, CL;
        boundary_carries<T, RAGGED, E>(a, buf, n, tbR, tbL, &CR, &CL);
        split_carry<T>(CR, &c4[0], &c4[1]);
        split_carry<T>(CL, &c4[2], &c4[3]);
      }
      cRh = __shfl_sync(0xffffffffu, c4[0], 0);
      cRl = __shfl_sync(0xffffffffu, c4[1], 0);
      cLh = __shfl_sync(0xffffffffu, c4[2], 0);
      cLl = __shfl_sync(0xffffffffu, c4[3], 0);
    } else {
      // vectorised over the CTA's lines: lane w of warp 0 solves line w
      // (GB300's FP64 pipe is narrow: one warp instruction for all lines)
      if (warp == 0 && lane < a.W) {
        const T* tw = totals + (lane * nwl) * 4;
        T tbR = T(0), tbL = T(0);
        for (int j = 0; j < nwl; ++j) tbR = fma(tw[j * 4 + 0], tbR, tw[j * 4 + 1]);
        for (int j = nwl - 1; j >= 0; --j) tbL = fma(tw[j * 4 + 2], tbL, tw[j * 4 + 3]);
        double CR, CL;
        boundary_carries<T, RAGGED, E>(a, lines + lane * a.LS, n, tbR, tbL, &CR, &CL);
        T* cw = reinterpret_cast<T*>(carries) + lane * 4;
        split_carry<T>(CR, &cw[0], &cw[1]);
        split_carry<T>(CL, &cw[2], &cw[3]);
      }
      __syncthreads();
      const T* cw = reinterpret_cast<const T*>(carries) + lw * 4;
      cRh = cw[0];
      cRl = cw[1];
      cLh = cw[2];
      cLl = cw[3];
    }
    // ---- 4. carries into the lane and the fix-up passes.  The first power
    // accumulates I = L^{-1}[v] with |I| ~ |v| and D = v - L^{-1}[v] cancels,
    // so its recurrences are compensated; later powers act on D^p[v], whose
    // rounding errors enter S_P scaled by |D^p v| / |v| (already below the
    // first power's error from the local integrals), so they run plain.
    {
      const T laR = exaR * paR, lbR = fma(exaR, pbR, exbR);
      const T laL = exaL * paL, lbL = fma(exaL, pbL, exbL);
      if constexpr (!RAGGED) {
        const T2 q2 = pair2<T>(q, q);
        if (p == 0 || sizeof(T) == 8) {
          Acc2<T> y{pair2<T>(fma(laR, cRh, lbR), fma(laL, cLh, lbL)), pair2<T>(laR * cRl, laL * cLl)};
#pragma unroll
          for (int k = 0; k < E; ++k) {
            y.step(q2, Y[k]);
            Y[k] = y.value();
          }
        } else {
          T2 y = pair2<T>(fma(laR, cRh, lbR) + laR * cRl, fma(laL, cLh, lbL) + laL * cLl);
#pragma unroll
          for (int k = 0; k < E; ++k) {
            y = fma2(q2, y, Y[k]);
            Y[k] = y;
          }
        }
      } else {
        Acc<T> yR{fma(laR, cRh, lbR), laR * cRl};
        Acc<T> yL{fma(laL, cLh, lbL), laL * cLl};
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const int e = e0 + k;
          if (e >= eR0 && e < n) yR.step(q, Y[k].x);
          Y[k].x = yR.value();
          const int kl = E - 1 - k;
          if (e0 + kl <= eL1) yL.step(q, Y[E - 1 - (kl)].y);
          Y[E - 1 - (kl)].y = yL.value();
        }
      }
    }
    // ---- 5. D = v - L^{-1}, accumulate, write back for the next power
    if (a.mode == MODE_RL) {
      // one-sided derivatives v^- = alpha D_R, v^+ = -alpha D_L and the
      // per-axis part of the Lax-Friedrichs Hamiltonian (Sec. 2.5)
      const T al = pick<T>(a.alpha, a.alphaf);
      if (!GEN || a.ham == HAM_HALF_SQ) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const T vm = al * (v[k] - Y[k].x);
          const T vp = -al * (v[k] - Y[E - 1 - (k)].y);
          const T r = fmax(fabs(vm), fabs(vp));
          const T mean = T(0.5) * (vm + vp);
          S[k] = T(0.5) * mean * mean + r * T(0.5) * (vm - vp);
          if (line_ok && e0 + k < n) rmax = fmax(rmax, r);
        }
      } else if constexpr (GEN) {
        // H_d' = a_d (LINEAR) has |H_d'| = |a_d| everywhere; AFFINE_SQ
        // leaves (sigma, delta) and the last pass takes the box maximum
        const T av = pick<T>(a.vel, a.velf), aa = fabs(av);
        T* cbase2 = static_cast<T*>(sm.lines2) + (cbase - lines);
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const T vm = al * (v[k] - Y[k].x);
          const T vp = -al * (v[k] - Y[E - 1 - (k)].y);
          const T mean = T(0.5) * (vm + vp);
          if (a.ham == HAM_LINEAR) {
            S[k] = av * mean + aa * T(0.5) * (vm - vp);
          } else {
            S[k] = av * mean;
            if (RAGGED ? e0 + k < n : true) cbase2[chunk_off<E>(k)] = aa * T(0.5) * (vp - vm);
          }
        }
        if (a.ham == HAM_LINEAR && line_ok) rmax = aa;
      }
    } else {
#pragma unroll
      for (int k = 0; k < E; ++k) {
        T linv;
        if (a.mode == MODE_0) linv = T(0.5) * (Y[k].x + Y[E - 1 - (k)].y);
        else if (a.mode == MODE_R) linv = Y[k].x;
        else linv = Y[E - 1 - (k)].y;
        v[k] = v[k] - linv;
        S[k] += v[k];
      }
    }
    if (p + 1 < a.P) {
      if (WL || own) {
        __syncwarp();
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (RAGGED ? e0 + k < n : true) cbase[chunk_off<E>(k)] = v[k];
        __syncwarp();
        warp_fill_ghosts<T, E>(a, buf, lane);
        __syncwarp();
      } else {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < E; ++k)
          if (RAGGED ? e0 + k < n : true) cbase[chunk_off<E>(k)] = v[k];
        __syncthreads();
        fill_ghosts<T, E>(a, lines);
        __syncthreads();
      }
    }
  }

  if (WL || own) __syncwarp(); else __syncthreads();
#pragma unroll
  for (int k = 0; k < E; ++k)
    if (RAGGED ? e0 + k < n : true) cbase[chunk_off<E>(k)] = S[k];
  __syncthreads();
  return cvt<double>(rmax);
}

#ifndef MOLT_WL_MODE
#define MOLT_WL_MODE 0
#endif
template <typename T, int JQ, bool RAGGED, int E = kE, bool GEN = false>
__device__ __forceinline__ double compute_lines_any(const SweepArgs& a, const TileSmem& sm, bool line_ok) {
#if MOLT_WL_MODE == 0
  return compute_lines<T, JQ, RAGGED, false, E, GEN>(a, sm, line_ok);
#elif MOLT_WL_MODE == 2
  return compute_lines<T, JQ, RAGGED, true, E, GEN>(a, sm, line_ok);
#else
  if (a.nwl == 1) return compute_lines<T, JQ, RAGGED, true, E, GEN>(a, sm, line_ok);
  return compute_lines<T, JQ, RAGGED, false, E, GEN>(a, sm, line_ok);
#endif
}

// Epilogue operands of one point, loaded ahead of the stores so that the
// loads of a batch of points are in flight together (the compiler cannot
// move a load past a store to a possibly aliasing array).
template <typename T, typename TST>
struct EpiOps {
  T acc;
  TST x, y;
};

template <typename T, typename TST, int EPI, bool CG = false>
struct Epilogue {
  const SweepArgs& a;
  double dt;
  double tn;   // general HJ_Y with a source: time of the state being advanced

  __device__ __forceinline__ EpiOps<T, TST> load(long long gidx) const {
    EpiOps<T, TST> o{T(0), TST(0), TST(0)};
    if constexpr (EPI == EPI_ACC_ADD || EPI == EPI_ACC_AXPY) {
      o.acc = gload<CG>(static_cast<const T*>(a.acc) + gidx);
    } else if constexpr (EPI == EPI_HEAT_FINAL || EPI == EPI_WAVE_FINAL) {
      if (a.acc) o.acc = gload<CG>(static_cast<const T*>(a.acc) + gidx);
      o.x = gload<CG>(static_cast<const TST*>(a.un) + gidx);
      if (EPI == EPI_HEAT_FINAL || !a.from_rest) o.y = gload<CG>(static_cast<const TST*>(a.us) + gidx);
    } else if constexpr (epi_hj_y(EPI)) {
      o.x = gload<CG>(static_cast<const TST*>(a.un) + gidx);
      if (a.out) o.y = gload<CG>(static_cast<const TST*>(a.out) + gidx);
    }
    return o;
  }

  __device__ __forceinline__ void store(long long gidx, T s, const EpiOps<T, TST>& o) const {
    if constexpr (EPI == EPI_STORE) {
      static_cast<TST*>(a.out)[gidx] = cvt<TST>(s);
    } else if constexpr (EPI == EPI_ACC_SET) {
      static_cast<T*>(a.acc)[gidx] = s;
    } else if constexpr (EPI == EPI_ACC_ADD) {
      static_cast<T*>(a.acc)[gidx] = o.acc + s;
    } else if constexpr (EPI == EPI_ACC_AXPY) {
      static_cast<T*>(a.acc)[gidx] = fma(T(a.coefS), s, o.acc);
    } else if constexpr (EPI == EPI_HEAT_FINAL) {
      // u_s = a0 u^n + a1 (u_{s-1} + dt F), dt F = coefS (acc + S)
      const TST r = fma(TST(a.a0), o.x, TST(a.a1) * fma(TST(a.coefS), cvt<TST>(o.acc + s), o.y));
      static_cast<TST*>(a.dst)[gidx] = r;
      if (a.shadow) a.shadow[gidx] = cvt<float>(r);
      if (nonfinite(r)) atomicOr(a.status, ST_NONFINITE);
    } else if constexpr (EPI == EPI_WAVE_FINAL) {
      // u^{n+1} = 2u^n - u^{n-1} + coefS (acc + S)   (from rest: u^n + coefS/2 (acc + S))
      const TST tot = cvt<TST>(o.acc + s);
      const TST r = a.from_rest ? fma(TST(0.5 * a.coefS), tot, o.x) : fma(TST(a.coefS), tot, fma(TST(2), o.x, -o.y));
      if (a.dst2) static_cast<TST*>(a.dst2)[gidx] = o.x;
      static_cast<TST*>(a.dst)[gidx] = r;
      if (a.shadow) a.shadow[gidx] = cvt<float>(r);
      if (nonfinite(r)) atomicOr(a.status, ST_NONFINITE);
    } else if constexpr (epi_hj_x(EPI)) {
      if (a.out) static_cast<TST*>(a.out)[gidx] = TST(s);
    } else if constexpr (epi_hj_y(EPI)) {
      const TST r = o.x - TST(dt) * (o.y + TST(s));
      static_cast<TST*>(a.dst)[gidx] = r;
      if (nonfinite(r)) atomicOr(a.status, ST_NONFINITE);
    }
  }

  // ---- general Hamilton-Jacobi passes (EPI_HJ_XG / EPI_HJ_YG)
  // z: delta_x of AFFINE_SQ from the x pass (last pass), 0 otherwise
  __device__ __forceinline__ TST load_z(long long gidx) const {
    if constexpr (EPI == EPI_HJ_YG)
      if (a.out2) return gload<CG>(static_cast<const TST*>(a.out2) + gidx);
    return TST(0);
  }

  // F(x, t_n) = sum_k t_n^k F_k(x) (Horner)
  __device__ __forceinline__ TST source(long long gidx) const {
    const TST* f = static_cast<const TST*>(a.src) + gidx;
    const TST t = TST(tn);
    TST F = f[a.src_deg * a.src_stride];
    for (int k = a.src_deg - 1; k >= 0; --k) F = fma(F, t, f[k * a.src_stride]);
    return F;
  }

  // s2: the second line buffer's value (two_out).  Returns the point's
  // scaled wave speed where the last pass determines it (AFFINE_SQ), else 0.
  __device__ __forceinline__ T store_general(long long gidx, T s, const EpiOps<T, TST>& o, TST z, T s2) const {
    if constexpr (EPI == EPI_HJ_XG) {
      if (a.out) static_cast<TST*>(a.out)[gidx] = TST(s);
      if (a.out2) static_cast<TST*>(a.out2)[gidx] = TST(s2);
      return T(0);
    } else {
      TST H;
      T speed = T(0);
      if (a.ham == HAM_AFFINE_SQ) {
        // local Lax-Friedrichs over the box of one-sided derivatives:
        // |dH/dp_d| = |a_d| |h0 + a.p| is largest at a corner, where
        // |h0 + a.p| reaches m = |sbar| + sum_d |delta_d|; then
        // H^ = H(means) - sum_d |a_d| m (v^+_d - v^-_d)/2 = sbar^2/2 - m sum_d delta_d;
        // the speeds c_d = |a_d| m enter as max_d c_d / h_d = m vmax
        const TST sbar = TST(a.h0) + o.y + TST(s);
        const TST m = fabs(sbar) + fabs(z) + fabs(TST(s2));
        H = TST(0.5) * sbar * sbar - m * (z + TST(s2));
        speed = T(TST(a.vmax) * m);
      } else {
        H = o.y + TST(s);
      }
      if (a.src) H -= source(gidx);
      if (a.dst) {
        const TST r = o.x - TST(dt) * H;
        static_cast<TST*>(a.dst)[gidx] = r;
        if (nonfinite(r)) atomicOr(a.status, ST_NONFINITE);
      }
      return speed;
    }
  }
};

// Applies the epilogue to the tile's W lines in the coalesced mapping, in
// batches of kEpiBatch points per thread: all operand loads of a batch are
// issued before its stores.
#ifndef MOLT_EPI_BATCH
#define MOLT_EPI_BATCH 8
#endif
constexpr int kEpiBatch = MOLT_EPI_BATCH;

// The epilogue of the general Hamilton-Jacobi passes over one thread's points
// p0, p0 + pstep, ... of a line: shared values sp[k*pdelta] and sp2[k*pdelta]
// (second line buffer, or null), global index g + k*gstep, B points per
// batch with all loads of a batch issued before its stores.  Returns the
// largest scaled wave speed it determined.
template <typename T, typename TST, int EPI, bool CG, int B>
__device__ __forceinline__ double epilogue_general(const Epilogue<T, TST, EPI, CG>& ep, const T* sp, const T* sp2,
                                                   long long g, int p0, int n, int pstep, long long gstep,
                                                   int pdelta) {
  T rmax = T(0);
  for (int pb = p0; pb < n; pb += B * pstep) {
    EpiOps<T, TST> ops[B];
    T sv[B], sv2[B];
    TST oz[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (pb + k * pstep < n) {
        ops[k] = ep.load(g + k * gstep);
        oz[k] = ep.load_z(g + k * gstep);
        sv[k] = sp[k * pdelta];
        sv2[k] = sp2 ? sp2[k * pdelta] : T(0);
      }
    }
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (pb + k * pstep < n) rmax = fmax(rmax, ep.store_general(g + k * gstep, sv[k], ops[k], oz[k], sv2[k]));
    g += B * gstep;
    sp += B * pdelta;
    if (sp2) sp2 += B * pdelta;
  }
  return cvt<double>(rmax);
}

// Returns the largest wave speed the epilogue determined (HJ_Y with
// AFFINE_SQ), else 0.  lines2: the second line buffer (two_out) or null.
template <typename T, typename TST, int EPI, int E = kE, bool CG = false>
__device__ __forceinline__ double epilogue_tile(const SweepArgs& a, const T* lines, long long line0, double dt,
                                                const T* lines2 = nullptr) {
  const Epilogue<T, TST, EPI, CG> ep{a, dt, (epi_hj_y(EPI) && epi_hj_gen(EPI) && a.src) ? *a.t_now : 0.0};
  const int W = a.W, n = a.g.n, nwl = a.nwl;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  long long g0;
  const T* src0;
  int p0, pstep, sstep;
  long long gstep;
  if (a.contiguous) {
    const int lw = warp / nwl, tl = (warp - lw * nwl) * 32 + lane;
    if (line0 + lw >= a.g.nlines) return 0.0;
    p0 = tl;
    pstep = nwl * 32;
    g0 = line_base(a.g, line0 + lw) + p0;
    gstep = pstep;
    src0 = lines + lw * a.LS;
    sstep = 0;
  } else {
    const int w = tid % W;
    const long long gl = line0 + w;
    if (gl >= a.g.nlines) return 0.0;
    p0 = tid / W;
    pstep = blockDim.x / W;
    g0 = line_base(a.g, gl) + p0 * a.g.stride;
    gstep = pstep * a.g.stride;
    src0 = lines + w * a.LS;
    sstep = 1;
  }
  // shared index of point p: contiguous lines step p by a multiple of 32,
  // strided lines by blockDim/W (a multiple of 16), so phys<E>() advances by a
  // constant in both cases
  const int pdelta = pstep + pstep / E;
  const T* sp = src0 + phys<E>(p0);
  (void)sstep;
  if constexpr (epi_hj_gen(EPI)) {
    // more operands per point: a smaller batch
    return epilogue_general<T, TST, EPI, CG, 4>(ep, sp, lines2 ? lines2 + (sp - lines) : nullptr, g0, p0, n, pstep,
                                                 gstep, pdelta);
  } else {
    long long g = g0;
    for (int pb = p0; pb < n; pb += kEpiBatch * pstep) {
      EpiOps<T, TST> ops[kEpiBatch];
      T sv[kEpiBatch];
#pragma unroll
      for (int k = 0; k < kEpiBatch; ++k) {
        if (pb + k * pstep < n) {
          ops[k] = ep.load(g + k * gstep);
          sv[k] = sp[k * pdelta];
        }
      }
#pragma unroll
      for (int k = 0; k < kEpiBatch; ++k)
        if (pb + k * pstep < n) ep.store(g + k * gstep, sv[k], ops[k]);
      g += kEpiBatch * gstep;
      sp += kEpiBatch * pdelta;
    }
    return 0.0;
  }
}

template <int EPI>
__device__ __forceinline__ double hj_dt(const SweepArgs& a) {
  double dt = 0.0;
  if constexpr (epi_hj_y(EPI)) {
    if (!a.lag) return 0.0;   // a pass that only measures speeds
    const double cl = __longlong_as_double((long long)a.lag[0]);
    dt = a.dt_max;
    if (cl > 0.0 && a.cfl / cl < dt) dt = a.cfl / cl;
  }
  return dt;
}

template <int EPI>
__device__ __forceinline__ void publish_speed(const SweepArgs& a, double rmax) {
  if constexpr (epi_hj_x(EPI) || epi_hj_y(EPI)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if ((threadIdx.x & 31) == 0 && rmax > 0.0 && a.speed)
      atomicMax(a.speed, (unsigned long long)__double_as_longlong(rmax));
  }
}

// One tile per CTA, plain coalesced loads (any size / alignment).
template <typename T, typename TIN, typename TST, int JQ, int EPI, bool RAGGED, int E = kE>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) sweep_kernel(const SweepArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  size_t used;
  const TileSmem sm = carve<T, JQ>(smem_raw, a, &used);
  if constexpr (JQ == JQ_LEARNED) mlp_load_net(*sm.net, a.mlp);
  T* lines = static_cast<T*>(sm.lines);
  const long long line0 = (long long)blockIdx.x * a.W;
  const int warp = threadIdx.x >> 5, lw = warp / a.nwl;
  const int tl = (warp - lw * a.nwl) * 32 + (threadIdx.x & 31);
  load_tile<T, TIN, E>(a, static_cast<const TIN*>(a.in), lines, line0, lw, tl);
  __syncthreads();
  if constexpr (epi_hj_x(EPI) || epi_hj_y(EPI)) {
    const double rmax =
        compute_lines_any<T, JQ, RAGGED, E, epi_hj_gen(EPI)>(a, sm, line0 + lw < a.g.nlines) * a.inv_h;
    // the general last pass finds its speeds in the epilogue
    if constexpr (!epi_hj_gen(EPI)) publish_speed<EPI>(a, rmax);
    const double dt = hj_dt<EPI>(a);
    if (epi_hj_y(EPI) && blockIdx.x == 0 && threadIdx.x == 0 && a.t_dev) *a.t_dev += dt;
    const double re = epilogue_tile<T, TST, EPI, E>(a, lines, line0, dt, static_cast<const T*>(sm.lines2));
    if constexpr (epi_hj_gen(EPI)) publish_speed<EPI>(a, fmax(rmax, re));
  } else {
    compute_lines_any<T, JQ, RAGGED, E>(a, sm, line0 + lw < a.g.nlines);
    epilogue_tile<T, TST, EPI, E>(a, lines, line0, 0.0);
  }
}

}  // namespace molt
