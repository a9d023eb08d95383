// Line-per-lane sweep kernel: S_P = sum_{p<=P} D^p along one axis for FP32
// sweeps with the linear quadrature rule (arXiv 2007.03041, Sec. 2.1-2.4),
// on lines of n = 16 S points (S <= 32).
//
// Mapping.  A tile is 32 lines; lane l of every warp owns line l, and warp m
// owns the 16-point segment [16m, 16m + 16) of all 32 lines.  For y and z
// lines the TMA box of a tile, [point][32 lines] (one 128-byte row per
// point), is exactly the layout the compute reads: lane l reads column l, so
// every shared-memory access of a warp is one conflict-free row, no transpose
// runs, and the epilogue reads and writes coalesced 128-byte rows straight
// from registers.  x lines arrive as TMA boxes of 32 points x 32 lines with
// the 128-byte swizzle (16-byte vector reads of a warp hit distinct banks).
//
// Difference form of the recurrences (Sec. 2.4).  With
//   W_R(x_i) = v_i - L_R^{-1}[v](x_i),  W_L(x_i) = v_i - L_L^{-1}[v](x_i)
// the recurrences I_R(x_i) = q I_R(x_{i-1}) + J_R(x_i) and its mirror give
//   W_R(x_i) = q W_R(x_{i-1}) + K_R(x_i),  K_R(x_i) = v_i - q v_{i-1} - J_R(x_i),
//   W_L(x_i) = q W_L(x_{i+1}) + K_L(x_i),  K_L(x_i) = v_i - q v_{i+1} - J_L(x_i).
// Because the weights of J_R sum to 1 - q (App. C), K is a 5-tap filter of
// the first differences d_j = v_j - v_{j-1}:
//   K_R(x_i) =  sum_{m=-2}^{2} b_m d_{i+m},   K_L(x_i) = -sum_{m=-2}^{2} b_m d_{i+1-m},
//   b_{-2} = c_{-3}, b_{-1} = c_{-3} + c_{-2}, b_0 = c_{-3} + c_{-2} + c_{-1} + q,
//   b_1 = -(c_1 + c_2), b_2 = -c_2.
// So D = W is scanned directly: no value of the size of v is ever subtracted
// from another (no cancellation, hence no compensated arithmetic), and D of a
// constant is exactly zero.  D_0 = (W_R + W_L)/2 (I_0 = (I_L + I_R)/2,
// Sec. 3.3); the 1/2 is folded into the filter taps.
//
// Boundary constants (Sec. 2.3; the 2x2 algebra of Sec. 3.3).  T_R, T_L are
// the line totals of the scans started from zero (K_R at the first node and
// K_L at the last node of a Dirichlet line are zero: the recurrences start
// there).  The scans' initial values C_R (entering the line at the left) and
// C_L (at the right) are
//   periodic:        C_R = T_R / (1 - mu), C_L = T_L / (1 - mu), mu = q^n;
//   Dirichlet, D_0:  D_0 vanishes at both end nodes, i.e. with X = W_R(x_0),
//                    Y = W_L(x_{n-1}), mu = q^{n-1}:
//                    X + mu Y = -T_L, mu X + Y = -T_R, and C_R = X/q, C_L = Y/q;
//   Dirichlet, D_R / D_L: W_R(x_0) = 0 / W_L(x_{n-1}) = 0.
// Written as C_R = kA T_R + kB T_L, C_L = kA T_L + kB T_R with FP64
// coefficients from the host; the kernel evaluates this solve in FP64.
//
// Across segments.  Segment m's scan from zero ends at b_m; the value
// entering segment m from the left is
//   sum_{j=1}^{m} (q^16)^{j-1} b_{m-j} + (q^16)^m C_R
// and symmetrically from the right.  Terms whose weight (q^16)^k is below
// 2^-26 -- a quarter of FP32's unit rounding -- are not added (the
// truncation of the convolution tails that Sec. 3 applies at a tolerance),
// so each thread reads at most `lb` segment totals: lb = 3 at nu = 0.4.
//
// Per power: stage 1 (window, first differences, K, scan of the segment from
// zero -> the segment's totals), stage 2 (initial values from the totals,
// the scan again from them -> D).  Epilogues: store S, set / add to / axpy
// into the FP32 accumulator, or (y and z lines) the FP64 leapfrog update of
// the wave step (u^{n+1} from u^n, u^{n-1} and the axes' summed S in FP64,
// with the FP32 copy of u^{n+1} the next sweeps read).  P <= 2: S_2 = D + D^2 re-reads D from the
// line buffer.  No CTA-wide barrier runs in the tile loop: a segment depends
// only on the segments within its look-back (and, for segments near an end,
// on the segments near both ends), so each segment waits on one mbarrier per
// power that exactly those segments arrive on, the second power's ghost
// points come behind a barrier the two neighbours arrive on, and the two
// stage buffers (the copy of tile t+1 runs during tile t) sit behind
// full/empty mbarriers.  Every wait is bounded; a warp whose wait runs out
// records ST_TIMEOUT and leaves, and the warps waiting on it run out in turn.
#pragma once

#include <cuda.h>

#include "sweep.cuh"
#include "sweep_tma.cuh"

namespace molt {

constexpr int kLE = 16;      // points per thread (one segment)
constexpr int kLW = 32;      // lines per tile (one per lane)
constexpr int kLMaxSeg = 32; // segments per line (warps per CTA)

struct LanesArgs {
  int n, S;              // points per line, segments (warps per CTA)
  int contiguous;        // 1: x lines (array rows); 0: y or z lines
  int nbox, box_p;       // strided: TMA boxes per tile, points per box
  int kind;              // strided: 1 = y lines, 2 = z lines
  long long ntiles;
  long long tiles_per_row;  // strided: nx / 32
  long long s_hi;        // strided: element offset per row of tiles
  long long stride;      // strided: element stride along a line
  int bc, mode, P;
  int lb;                // look-back depth in segments (<= S)
  int needA, needB;      // the line constants use T of the same / the other direction
  float bR[5], bL[5];    // K_R = sum_i bR[i] d[t+i], K_L = sum_i bL[i] d[u+5-i] (window indices)
  float q, qE;           // e^{-nu} (FP32), q^16
  double kA, kB;         // line constants C = kA T_same + kB T_other (FP64)
  float coef;            // EPI_ACC_AXPY coefficient
  long long wait_limit;  // cycles any one wait of the kernel may take
  const float* in;       // contiguous: the sweep input (bulk copies read it)
  float* out;            // EPI_STORE destination
  float* acc;            // accumulator (EPI_WAVE_FINAL: sum of the other axes' S, or null)
  int* status;
  // EPI_WAVE_FINAL: u^{n+1} = 2u^n - u^{n-1} + coefS (acc + S) in FP64 (from
  // rest: u^n + coefS/2 (acc + S)); dst2, if set, receives u^n; shadow the
  // FP32 copy of u^{n+1}
  const double* un;
  const double* us;
  double* dst;
  double* dst2;
  float* shadow;
  double coefS;
  int from_rest;
};

constexpr int kLBuf = 3;     // stage buffers: the copy of tile k+2 is issued while tile k computes

// Bytes of one stage buffer.
__host__ __device__ constexpr size_t lanes_buf_bytes(int n, int contiguous) {
  return size_t(kLW) * size_t(n) * sizeof(float) + size_t(0 * contiguous);
}
// Dynamic shared memory of a CTA: the stage buffers, the segment totals of
// both powers and the mbarriers (3 per segment, 2 per buffer).
__host__ __device__ constexpr size_t lanes_smem_bytes(int n, int contiguous) {
  return 1024 + kLBuf * lanes_buf_bytes(n, contiguous) + size_t(2) * (n / kLE) * kLW * sizeof(float2) +
         (size_t(3) * (n / kLE) + 2 * kLBuf) * sizeof(uint64_t);
}

// x lines: the tile arrives as 32-point chunks of the 32 lines, [chunk][line]
// [32 floats], each chunk by one TMA box with the 128-byte swizzle: the
// 16-byte group g of line l sits at group g ^ (l % 8) of its 128-byte row, so
// the 16-byte reads of a quarter-warp (eight lines, one group) hit distinct
// banks.  Index of (line l, point p), p a multiple of 4 for vector access.
__device__ __forceinline__ int xsw(int l, int p) {
  return ((p >> 5) << 10) + (l << 5) + ((((p >> 2) & 7) ^ (l & 7)) << 2) + (p & 3);
}

// Issues the copies of tile `tile` into `buf` (the producer warp; lane 0 arms the barrier first).
__device__ __forceinline__ void lanes_issue(const LanesArgs& a, const CUtensorMap* map, float* buf, int tile,
                                            uint64_t* bar) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_expect_tx(bar, uint32_t(kLW) * uint32_t(a.n) * 4u);
  __syncwarp();
  if (a.contiguous) {
    // chunk c of the tile: lane c issues it
    for (int c = lane; c < (a.n >> 5); c += 32) tma_load_2d(buf + (c << 10), map, c << 5, tile * kLW, bar);
  } else if (lane == 0) {
    const int tpr = int(a.tiles_per_row);
    const int hi = tile / tpr;
    const int x0 = (tile - hi * tpr) * kLW;
    for (int b = 0; b < a.nbox; ++b) {
      float* dst = buf + b * a.box_p * kLW;
      if (a.kind == 1) tma_load_3d(dst, map, x0, b * a.box_p, hi, bar);
      else tma_load_3d(dst, map, x0, hi, b * a.box_p, bar);
    }
  }
}

// Element offset of (line 0 of the tile, point 0) for strided tiles.
__device__ __forceinline__ long long lanes_origin(const LanesArgs& a, int tile) {
  const int tpr = int(a.tiles_per_row);
  const int hi = tile / tpr;
  return (long long)hi * a.s_hi + (tile - hi * tpr) * kLW;
}

// Window w[k] = v_{p0-3+k}, k = 0..21, of this thread's line (ghost cells:
// periodic wrap; Dirichlet odd reflection about the end value,
// v_{-j} = 2 v_0 - v_j, v_{n-1+j} = 2 v_{n-1} - v_{n-1-j}).
template <bool CONTIG>
__device__ __forceinline__ void lanes_window(const LanesArgs& a, const float* buf, int seg, int lane, float (&w)[22]) {
  const int n = a.n, p0 = seg * kLE;
  if constexpr (CONTIG) {
    auto ld4 = [&](int p) { return *reinterpret_cast<const float4*>(buf + xsw(lane, p)); };
    float c[24];   // v_{p0-4 .. p0+19}
#pragma unroll
    for (int k = 1; k < 5; ++k) {
      const float4 x = ld4(p0 - 4 + 4 * k);
      c[4 * k] = x.x; c[4 * k + 1] = x.y; c[4 * k + 2] = x.z; c[4 * k + 3] = x.w;
    }
    if (seg > 0) {
      const float4 x = ld4(p0 - 4);
      c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
    } else if (a.bc == 0) {
      const float4 x = ld4(n - 4);         // v_{n-4..n-1} = v_{-4..-1}
      c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
    } else {
      const float v0 = c[4];
      c[3] = 2.f * v0 - c[5];
      c[2] = 2.f * v0 - c[6];
      c[1] = 2.f * v0 - c[7];
      c[0] = 0.f;
    }
    if (seg + 1 < a.S) {
      const float4 x = ld4(p0 + 16);
      c[20] = x.x; c[21] = x.y; c[22] = x.z; c[23] = x.w;
    } else if (a.bc == 0) {
      const float4 x = ld4(0);             // v_{0..3} = v_{n..n+3}
      c[20] = x.x; c[21] = x.y; c[22] = x.z; c[23] = x.w;
    } else {
      const float vN = c[19];              // v_{n-1} (p0 + 15)
      c[20] = 2.f * vN - c[18];
      c[21] = 2.f * vN - c[17];
      c[22] = 2.f * vN - c[16];
      c[23] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 22; ++k) w[k] = c[k + 1];
  } else {
    const float* col = buf + lane;
    if (seg > 0 && seg + 1 < a.S) {
#pragma unroll
      for (int k = 0; k < 22; ++k) w[k] = col[(p0 - 3 + k) * kLW];
    } else {
#pragma unroll
      for (int k = 3; k < 19; ++k) w[k] = col[(p0 - 3 + k) * kLW];
      if (seg > 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = col[(p0 - 3 + k) * kLW];
      } else if (a.bc == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = col[(n - 3 + k) * kLW];
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = 2.f * w[3] - w[6 - k];
      }
      if (seg + 1 < a.S) {
#pragma unroll
        for (int k = 19; k < 22; ++k) w[k] = col[(p0 - 3 + k) * kLW];
      } else if (a.bc == 0) {
#pragma unroll
        for (int k = 19; k < 22; ++k) w[k] = col[(k - 19) * kLW];
      } else {
#pragma unroll
        for (int k = 19; k < 22; ++k) w[k] = 2.f * w[18] - w[36 - k];
      }
    }
  }
}

// Own points t = 0..15 of this thread's line segment in the stage buffer.
template <bool CONTIG>
__device__ __forceinline__ void lanes_store_own(const LanesArgs& a, float* buf, int seg, int lane,
                                                const float (&x)[kLE]) {
  if constexpr (CONTIG) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      *reinterpret_cast<float4*>(buf + xsw(lane, seg * kLE + 4 * c)) =
          make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
  } else {
    float* o = buf + seg * kLE * kLW + lane;
#pragma unroll
    for (int t = 0; t < kLE; ++t) o[t * kLW] = x[t];
  }
}
template <bool CONTIG>
__device__ __forceinline__ void lanes_load_own(const LanesArgs& a, const float* buf, int seg, int lane,
                                               float (&x)[kLE]) {
  if constexpr (CONTIG) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 v = *reinterpret_cast<const float4*>(buf + xsw(lane, seg * kLE + 4 * c));
      x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
    }
  } else {
    const float* o = buf + seg * kLE * kLW + lane;
#pragma unroll
    for (int t = 0; t < kLE; ++t) x[t] = o[t * kLW];
  }
}

// ---- cross-warp hand-offs inside a CTA (no CTA-wide barrier in the tile loop)
// Segment m's second stage reads the totals of the segments in
//   J(m) = { c : |c - m| <= lb }  plus, when the line constants need totals,
//          every segment within lb of an end if m is one,
// a set with c in J(m) exactly when m is in J(c).  Each (power, segment) has
// an mbarrier expecting |J(m)| arrivals: after writing its totals, segment c
// arrives on the barriers of every m in J(c) (lane m of the warp, one
// instruction), and segment m waits on its own barrier once; a waiting warp
// is suspended by the hardware instead of spinning.  The ghost points of the
// second power come behind a second barrier per segment on which its
// neighbours arrive after storing D.  A producer cannot arrive twice on one
// phase: when c arrives for tile k+1, m (in J(c)) has finished tile k, so m's
// tile-k phases have completed.
__device__ __forceinline__ bool lanes_in_J(const LanesArgs& a, int m, int c) {
  const int d = m > c ? m - c : c - m;
  if (d <= a.lb) return true;
  if (!(a.needA || a.needB)) return false;
  const bool em = m < a.lb || m >= a.S - a.lb, ec = c < a.lb || c >= a.S - a.lb;
  return em && ec;
}
// Neighbours whose D points are ghost values of segment m (periodic lines wrap).
__device__ __forceinline__ int lanes_left(const LanesArgs& a, int m) {
  const int l = m - 1 >= 0 ? m - 1 : (a.bc == 0 ? a.S - 1 : -1);
  return l == m ? -1 : l;
}
__device__ __forceinline__ int lanes_right(const LanesArgs& a, int m) {
  const int r = m + 1 < a.S ? m + 1 : (a.bc == 0 ? 0 : -1);
  return (r == m || r == lanes_left(a, m)) ? -1 : r;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Wait on an mbarrier phase with a suspend-time hint (the thread may sleep
// until the phase completes or the hint elapses).
#ifndef MOLT_LANES_SUSPEND_NS
#define MOLT_LANES_SUSPEND_NS 20000
#endif
constexpr uint32_t kLanesSuspendNs = MOLT_LANES_SUSPEND_NS;
// Segment whose warp issues the tile copies (the end segments also solve the
// line constants, so a middle one keeps the two roles apart).
#ifndef MOLT_LANES_PRODUCER
#define MOLT_LANES_PRODUCER 0
#endif
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kLanesSuspendNs)
      : "memory");
  return ok != 0;
}
// Polling form of the waits: 0 try_wait with the suspend-time hint, 1
// test_wait with a doubling __nanosleep between polls (32 .. 512 ns), 2
// try_wait without a hint (the default).  Measured on the 512^3 wave step:
// the hint (100 ns .. 200 us) changes nothing, the sleeps cost 10% (the waits
// sit on the tile's critical path, so a late wake-up delays it) and 2 is 1%
// faster than 0.
#ifndef MOLT_LANES_WAIT_MODE
#define MOLT_LANES_WAIT_MODE 2
#endif
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool lanes_poll(uint64_t* bar, uint32_t parity) {
  if constexpr (MOLT_LANES_WAIT_MODE == 1) return mbar_test_wait(bar, parity);
  if constexpr (MOLT_LANES_WAIT_MODE == 2) return mbar_try_wait(bar, parity);
  return mbar_try_wait_sleep(bar, parity);
}
// Bounded wait on an mbarrier phase: the clock is read only once every 16
// polls, and the wait gives up after `limit` cycles.
// Polls between two clock reads of a wait (1: the counted loop).  Measured on
// the 512^3 wave step: 4 is 1% faster than 1, 8 and 16 no faster; the sweeps
// are bound by the tiles' dependency chain, not by the polling instructions.
#ifndef MOLT_LANES_POLL_UNROLL
#define MOLT_LANES_POLL_UNROLL 4
#endif
__device__ __forceinline__ bool lanes_mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (lanes_poll(bar, parity)) return true;
  const long long t0 = clock64();
  if constexpr (MOLT_LANES_POLL_UNROLL > 1) {
    // polls back to back between clock reads: a spinning warp issues two
    // instructions per poll (the wait and its branch) instead of the loop's
    // counter, mask, compare and branches
    for (;;) {
#pragma unroll
      for (int k = 0; k < MOLT_LANES_POLL_UNROLL; ++k)
        if (lanes_poll(bar, parity)) return true;
      if (clock64() - t0 > limit) return false;
    }
  }
  unsigned ns = 32;
  for (int i = 1;; ++i) {
    if constexpr (MOLT_LANES_WAIT_MODE == 1) {
      __nanosleep(ns);
      if (ns < 512) ns <<= 1;
    }
    if (lanes_poll(bar, parity)) return true;
    if ((i & 15) == 0 && clock64() - t0 > limit) return false;
  }
}

// Shared-memory layout of a CTA.
struct LanesSmem {
  float* buf0;                 // stage buffers: buf0 + i * bstride, i < kLBuf
  int bstride;                 // floats per stage buffer
  float2* tot;                 // [2][S][32]: (b_R, b_L) of each segment and line, per power
  uint64_t* tbar;              // [2][S]: totals of J(m) written, per power
  uint64_t* dbar;              // [S]: neighbours' D of the first power written
  uint64_t* full;              // [kLBuf] copy of a tile landed
  uint64_t* empty;             // [kLBuf] every warp is done with a buffer
};

__device__ __forceinline__ LanesSmem lanes_carve(unsigned char* smem, const LanesArgs& a, bool contig) {
  LanesSmem m;
  // the swizzled boxes need 1024-byte aligned destinations
  smem += (1024 - (smem_u32(smem) & 1023)) & 1023;
  const size_t bb = lanes_buf_bytes(a.n, contig ? 1 : 0);
  m.buf0 = reinterpret_cast<float*>(smem);
  m.bstride = int(bb / sizeof(float));
  m.tot = reinterpret_cast<float2*>(smem + kLBuf * bb);
  m.tbar = reinterpret_cast<uint64_t*>(m.tot + 2 * a.S * kLW);
  m.dbar = m.tbar + 2 * a.S;
  m.full = m.dbar + a.S;
  m.empty = m.full + kLBuf;
  return m;
}

// Stage 1 of one application of D: local integrals in difference form and the
// scan of the segment from zero; Y[t] = (K_R(p0+t), K_L(p0+15-t)).  Publishes
// the segment's totals (b_R, b_L) of power `pw` and arrives on the barriers
// of the segments that read them.
template <bool CONTIG>
__device__ __forceinline__ void lanes_stage1(const LanesArgs& a, const float* buf, const LanesSmem& sm, int pw,
                                             int seg, int lane, float2 (&Y)[kLE]) {
  {
    float w[22];
    lanes_window<CONTIG>(a, buf, seg, lane, w);
    float d[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) d[k] = w[k + 1] - w[k];
#pragma unroll
    for (int t = 0; t < kLE; ++t) {
      float r = a.bR[0] * d[t];
#pragma unroll
      for (int i = 1; i < 5; ++i) r = fmaf(a.bR[i], d[t + i], r);
      Y[t].x = r;
    }
#pragma unroll
    for (int u = kLE - 1; u >= 0; --u) {
      float l = a.bL[0] * d[u + 5];
#pragma unroll
      for (int i = 1; i < 5; ++i) l = fmaf(a.bL[i], d[u + 5 - i], l);
      Y[kLE - 1 - u].y = l;
    }
  }
  if (a.bc == 1) {
    if (seg == 0) Y[0].x = 0.f;              // K_R(x_0): the R recurrence starts here
    if (seg + 1 == a.S) Y[0].y = 0.f;        // K_L(x_{n-1})
  }
  const float2 q2 = make_float2(a.q, a.q);
  float2 y = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < kLE; ++t) y = fma2(q2, y, Y[t]);
  sm.tot[(pw * a.S + seg) * kLW + lane] = y;
  __syncwarp();
  if (lane < a.S && lanes_in_J(a, seg, lane)) mbar_arrive(&sm.tbar[pw * a.S + lane]);
}

// Stage 1 of the second power, started from D of the first (in registers):
// D goes to the line buffer and the neighbours are signalled at once; the
// filter outputs that need no ghost point (K_R at t = 3..13, K_L at
// u = 2..12) are computed while the neighbours' D arrive; then the ghost
// points, the remaining outputs, the scan from zero and the totals.
template <bool CONTIG>
__device__ __forceinline__ bool lanes_stage1_second(const LanesArgs& a, float* buf, const LanesSmem& sm,
                                                    uint32_t parity, int seg, int lane, const float (&D)[kLE],
                                                    float2 (&Y)[kLE]) {
  lanes_store_own<CONTIG>(a, buf, seg, lane, D);
  __syncwarp();
  const int l = lanes_left(a, seg), r = lanes_right(a, seg);
  if (lane == 0 && l >= 0) mbar_arrive(&sm.dbar[l]);
  if (lane == 1 && r >= 0) mbar_arrive(&sm.dbar[r]);
  // d[k] = w[k+1] - w[k] with w[k] = D at point p0-3+k: d[3..17] are own differences
  float d[21];
#pragma unroll
  for (int k = 3; k < 18; ++k) d[k] = D[k - 2] - D[k - 3];
  const float D0 = D[0], D15 = D[kLE - 1];
#pragma unroll
  for (int t = 3; t <= 13; ++t) {
    float v = a.bR[0] * d[t];
#pragma unroll
    for (int i = 1; i < 5; ++i) v = fmaf(a.bR[i], d[t + i], v);
    Y[t].x = v;
  }
#pragma unroll
  for (int u = 12; u >= 2; --u) {
    float v = a.bL[0] * d[u + 5];
#pragma unroll
    for (int i = 1; i < 5; ++i) v = fmaf(a.bL[i], d[u + 5 - i], v);
    Y[kLE - 1 - u].y = v;
  }
  if (l >= 0 || r >= 0)
    if (!__all_sync(0xffffffffu, lanes_mbar_wait(&sm.dbar[seg], parity, a.wait_limit))) return false;
  {
    // ghost values g[0..2] = points p0-3..p0-1, g[3..5] = p0+16..p0+18
    float g[6];
    const int p0 = seg * kLE;
    if (seg > 0 && seg + 1 < a.S) {
      if constexpr (CONTIG) {
        const float4 lo = *reinterpret_cast<const float4*>(buf + xsw(lane, p0 - 4));
        const float4 hi = *reinterpret_cast<const float4*>(buf + xsw(lane, p0 + kLE));
        g[0] = lo.y; g[1] = lo.z; g[2] = lo.w;
        g[3] = hi.x; g[4] = hi.y; g[5] = hi.z;
      } else {
        const float* col = buf + lane;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          g[k] = col[(p0 - 3 + k) * kLW];
          g[3 + k] = col[(p0 + kLE + k) * kLW];
        }
      }
    } else {
      float w[22];
      lanes_window<CONTIG>(a, buf, seg, lane, w);   // line ends: reflected or wrapped ghosts
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        g[k] = w[k];
        g[3 + k] = w[19 + k];
      }
    }
    d[0] = g[1] - g[0];
    d[1] = g[2] - g[1];
    d[2] = D0 - g[2];
    d[18] = g[3] - D15;
    d[19] = g[4] - g[3];
    d[20] = g[5] - g[4];
  }
#pragma unroll
  for (int t = 0; t < kLE; ++t) {
    if (t >= 3 && t <= 13) continue;
    float v = a.bR[0] * d[t];
#pragma unroll
    for (int i = 1; i < 5; ++i) v = fmaf(a.bR[i], d[t + i], v);
    Y[t].x = v;
  }
#pragma unroll
  for (int u = kLE - 1; u >= 0; --u) {
    if (u >= 2 && u <= 12) continue;
    float v = a.bL[0] * d[u + 5];
#pragma unroll
    for (int i = 1; i < 5; ++i) v = fmaf(a.bL[i], d[u + 5 - i], v);
    Y[kLE - 1 - u].y = v;
  }
  if (a.bc == 1) {
    if (seg == 0) Y[0].x = 0.f;
    if (seg + 1 == a.S) Y[0].y = 0.f;
  }
  const float2 q2 = make_float2(a.q, a.q);
  float2 y = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < kLE; ++t) y = fma2(q2, y, Y[t]);
  sm.tot[(a.S + seg) * kLW + lane] = y;
  __syncwarp();
  if (lane < a.S && lanes_in_J(a, seg, lane)) mbar_arrive(&sm.tbar[a.S + lane]);
  return true;
}

// Stage 2: once the totals of J(seg) are written, the values entering the
// segment from the left and the right (the look-back over at most LB
// segments; the line constants for segments within reach of an end), the scan
// from them, and D = W_R + W_L.  False if the wait ran out.
template <int LB>
__device__ __forceinline__ bool lanes_stage2(const LanesArgs& a, const LanesSmem& sm, int pw, uint32_t parity,
                                             int seg, int lane, float2 (&Y)[kLE], float (&D)[kLE]) {
  const int S = a.S, lb = a.lb;
  const float qE = a.qE;
  if (!__all_sync(0xffffffffu, lanes_mbar_wait(&sm.tbar[pw * S + seg], parity, a.wait_limit))) return false;
  const float2* tt = sm.tot + size_t(pw) * S * kLW + lane;
  const int rseg = S - 1 - seg;
  float cR = 0.f, cL = 0.f;
  if (seg < lb || rseg < lb) {
    // line totals of the scans from zero (terms of weight below the cut dropped)
    float TR = 0.f, TL = 0.f;
    if (a.needA || a.needB) {
      for (int j = S > lb ? S - lb : 0; j < S; ++j) TR = fmaf(qE, TR, tt[j * kLW].x);
      for (int j = (S < lb ? S : lb) - 1; j >= 0; --j) TL = fmaf(qE, TL, tt[j * kLW].y);
    }
    // line constants in FP64 (Sec. 2.3 / 3.3 solve); GB300's FP64 pipe is
    // narrow, so only the products with a nonzero coefficient run
    const double tr = f2d(TR), tl = f2d(TL);
    if (seg < lb) cR = d2f(a.needA && a.needB ? fma(a.kA, tr, a.kB * tl) : (a.needA ? a.kA * tr : a.kB * tl));
    if (rseg < lb) cL = d2f(a.needA && a.needB ? fma(a.kA, tl, a.kB * tr) : (a.needA ? a.kA * tl : a.kB * tr));
  }
  {
    // Horner from the farthest segment in reach: cR = sum_j qE^{j-1} b_R[seg-j] + qE^seg C_R
    const int jm = seg < lb ? seg : lb;
    const int jr = rseg < lb ? rseg : lb;
    if (jm == LB && jr == LB) {   // segments away from both ends (lb == LB): no predicates
#pragma unroll
      for (int j = LB; j >= 1; --j) {
        cR = fmaf(qE, cR, tt[(seg - j) * kLW].x);
        cL = fmaf(qE, cL, tt[(seg + j) * kLW].y);
      }
    } else {
#pragma unroll
      for (int j = LB; j >= 1; --j) {
        if (j <= jm) cR = fmaf(qE, cR, tt[(seg - j) * kLW].x);
        if (j <= jr) cL = fmaf(qE, cL, tt[(seg + j) * kLW].y);
      }
    }
  }
  const float2 q2 = make_float2(a.q, a.q);
  float2 y = make_float2(cR, cL);
#pragma unroll
  for (int t = 0; t < kLE; ++t) {
    y = fma2(q2, y, Y[t]);
    Y[t] = y;
  }
  // D_0 = W_R + W_L (halves in the taps); D_R = W_R; D_L = W_L
#pragma unroll
  for (int t = 0; t < kLE; ++t) D[t] = Y[t].x + Y[kLE - 1 - t].y;
  return true;
}

__device__ __forceinline__ int lanes_producer(const LanesArgs& a) {
  return MOLT_LANES_PRODUCER < a.S ? MOLT_LANES_PRODUCER : a.S - 1;
}

// A warp gives up (a bounded wait ran out): record it and, in the copy-issuing
// warp, wait (bounded) for the copy it may still have in flight.
__device__ __forceinline__ void lanes_give_up(const LanesArgs& a, const LanesSmem& sm, int seg, int lane,
                                              int inflight_buf, uint32_t inflight_parity) {
  if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
  if (seg == lanes_producer(a) && inflight_buf >= 0)
    lanes_mbar_wait(&sm.full[inflight_buf], inflight_parity, a.wait_limit);
}

template <int EPI, bool CONTIG, int LB>
__global__ void __launch_bounds__(kLMaxSeg * 32, 1)
    lanes_sweep_kernel(const LanesArgs a, const __grid_constant__ CUtensorMap map) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const LanesSmem sm = lanes_carve(smem_raw, a, CONTIG);
  const int S = a.S;
  const int seg = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int prod = lanes_producer(a);
  if (threadIdx.x < S) {
    const int m = threadIdx.x;
    int cnt = 0;
    for (int c = 0; c < S; ++c) cnt += lanes_in_J(a, c, m) ? 1 : 0;
    mbar_init(&sm.tbar[m], cnt);
    mbar_init(&sm.tbar[S + m], cnt);
    int nb = 0;
    for (int c = 0; c < S; ++c) nb += (lanes_left(a, c) == m) + (lanes_right(a, c) == m);
    if (nb > 0) mbar_init(&sm.dbar[m], nb);
  }
  if (threadIdx.x < kLBuf) {
    mbar_init(&sm.full[threadIdx.x], 1);
    mbar_init(&sm.empty[threadIdx.x], S);
  }
  fence_mbar_init();
  __syncthreads();   // the only CTA-wide barrier: the mbarriers are initialised

  const int ntiles = int(a.ntiles);
  int tile = blockIdx.x;
  // tiles k = 0 and 1 of this CTA go into buffers 0 and 1; buffer k % 3 holds
  // tile k, and its u-th use completes phase u of its full/empty barriers
  for (int i = 0; i < kLBuf - 1; ++i)
    if (seg == prod && tile + i * int(gridDim.x) < ntiles)
      lanes_issue(a, &map, sm.buf0 + i * sm.bstride, tile + i * int(gridDim.x), &sm.full[i]);

  int b = 0, use = 0;      // buffer of tile k and its use count
  for (int k = 0; tile < ntiles; tile += gridDim.x, ++k) {
    float* buf = sm.buf0 + b * sm.bstride;
    const uint32_t par = uint32_t(k & 1);   // phase of the per-tile barriers
    // ---- this tile's copy
    if (!__all_sync(0xffffffffu, lanes_mbar_wait(&sm.full[b], uint32_t(use & 1), a.wait_limit))) {
      lanes_give_up(a, sm, seg, lane, b, uint32_t(use & 1));   // once more for the copy in flight
      return;
    }
    // ---- the copy of tile k+2 into the buffer tile k-1 used, once every warp
    // has released it
    const int ahead = tile + (kLBuf - 1) * int(gridDim.x);
    const int bn = b == 0 ? kLBuf - 1 : b - 1;    // (k + 2) % 3 == (k - 1) % 3
    const int use_prev = bn < b ? use : use - 1;  // uses of buffer bn before tile k-1's (k >= 1)
    if (seg == prod && ahead < ntiles) {
      if (k >= 1 &&
          !__all_sync(0xffffffffu, lanes_mbar_wait(&sm.empty[bn], uint32_t(use_prev & 1), a.wait_limit))) {
        lanes_give_up(a, sm, seg, lane, -1, 0);
        return;
      }
      lanes_issue(a, &map, sm.buf0 + bn * sm.bstride, ahead, &sm.full[bn]);
    }
    // the copy a give-up waits for: tile k+2's (phase use_prev + 1 of buffer
    // bn; k = 0: its first phase)
    const int inflight = (seg == prod && ahead < ntiles) ? bn : -1;
    const uint32_t inflight_parity = uint32_t(k >= 1 ? (use_prev + 1) & 1 : 0);
    // L2 prefetch of the rows this warp's epilogue reads
    if constexpr (EPI == EPI_ACC_ADD || EPI == EPI_ACC_AXPY) {
      if constexpr (CONTIG) {
        prefetch_l2(a.acc + (long long)(tile * kLW + lane) * a.n + seg * kLE);
      } else if (lane < kLE) {
        prefetch_l2(a.acc + lanes_origin(a, tile) + (long long)(seg * kLE + lane) * a.stride);
      }
    } else if constexpr (EPI == EPI_WAVE_FINAL && !CONTIG) {
      // FP32 acc rows (128 bytes), FP64 u^n and u^{n-1} rows (256 bytes)
      const long long r = lanes_origin(a, tile) + (long long)(seg * kLE + (lane & 15)) * a.stride;
      if (lane < kLE) {
        if (a.acc) prefetch_l2(a.acc + r);
        prefetch_l2(a.un + r);
        prefetch_l2(a.un + r + 16);
      } else if (!a.from_rest) {
        prefetch_l2(a.us + r);
        prefetch_l2(a.us + r + 16);
      }
    }

    float D[kLE];
    {
      float2 Y[kLE];
      lanes_stage1<CONTIG>(a, buf, sm, 0, seg, lane, Y);
      if (!lanes_stage2<LB>(a, sm, 0, par, seg, lane, Y, D)) {
        lanes_give_up(a, sm, seg, lane, inflight, inflight_parity);
        return;
      }
    }
    if (a.P == 2) {
      // D of the first power over this segment's points (its neighbours have
      // read their ghost values from them: their totals were waited on)
      float D2[kLE];
      {
        float2 Y[kLE];
        if (!lanes_stage1_second<CONTIG>(a, buf, sm, par, seg, lane, D, Y)) {
          lanes_give_up(a, sm, seg, lane, inflight, inflight_parity);
          return;
        }
        if (!lanes_stage2<LB>(a, sm, 1, par, seg, lane, Y, D2)) {
          lanes_give_up(a, sm, seg, lane, inflight, inflight_parity);
          return;
        }
      }
      lanes_load_own<CONTIG>(a, buf, seg, lane, D);   // D of the first power, as stored above
#pragma unroll
      for (int t = 0; t < kLE; ++t) D[t] += D2[t];
    }
    // ---- epilogue (this warp's segment of the 32 lines)
    if constexpr (!CONTIG) {
      const long long g0 = lanes_origin(a, tile) + (long long)(seg * kLE) * a.stride + lane;
      const long long st = a.stride;
      if constexpr (EPI == EPI_ACC_ADD || EPI == EPI_ACC_AXPY) {
        float o[kLE];
        const float* src = a.acc + g0;
#pragma unroll
        for (int t = 0; t < kLE; ++t, src += st) o[t] = *src;
        float* dst = a.acc + g0;
#pragma unroll
        for (int t = 0; t < kLE; ++t, dst += st) *dst = EPI == EPI_ACC_ADD ? o[t] + D[t] : fmaf(a.coef, D[t], o[t]);
      } else if constexpr (EPI == EPI_WAVE_FINAL) {
        // the FP64 leapfrog update, four points at a time (loads first)
        bool bad = false;
        const double half = 0.5 * a.coefS;
#pragma unroll
        for (int t0 = 0; t0 < kLE; t0 += 4) {
          float ac[4];
          double x[4], y[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const long long g = g0 + (t0 + j) * st;
            ac[j] = a.acc ? a.acc[g] : 0.f;
            x[j] = a.un[g];
            y[j] = a.from_rest ? 0.0 : a.us[g];
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const long long g = g0 + (t0 + j) * st;
            const double tot = f2d(ac[j] + D[t0 + j]);
            const double r = a.from_rest ? fma(half, tot, x[j]) : fma(a.coefS, tot, fma(2.0, x[j], -y[j]));
            if (a.dst2) a.dst2[g] = x[j];
            a.dst[g] = r;
            a.shadow[g] = d2f(r);
            bad |= nonfinite(r);
          }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, ST_NONFINITE);
      } else {
        float* dst = (EPI == EPI_STORE ? a.out : a.acc) + g0;
#pragma unroll
        for (int t = 0; t < kLE; ++t, dst += st) *dst = D[t];
      }
    } else {
      // through the segment's points of the line buffer: lane l holds line l;
      // after the exchange lane t writes 16 bytes of line (t%8) + 8c, so one
      // instruction stores 8 lines x 64 contiguous bytes
      lanes_store_own<CONTIG>(a, buf, seg, lane, D);
      __syncwarp();
      const int q = lane >> 3;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int line = (lane & 7) + 8 * c;
        const float4 s4 = *reinterpret_cast<const float4*>(buf + xsw(line, seg * kLE + 4 * q));
        float4* g4 = reinterpret_cast<float4*>((EPI == EPI_STORE ? a.out : a.acc) +
                                               (long long)(tile * kLW + line) * a.n + seg * kLE + 4 * q);
        if constexpr (EPI == EPI_ACC_ADD || EPI == EPI_ACC_AXPY) {
          float4 o = *g4;
          if (EPI == EPI_ACC_ADD) {
            o.x += s4.x; o.y += s4.y; o.z += s4.z; o.w += s4.w;
          } else {
            o.x = fmaf(a.coef, s4.x, o.x); o.y = fmaf(a.coef, s4.y, o.y);
            o.z = fmaf(a.coef, s4.z, o.z); o.w = fmaf(a.coef, s4.w, o.w);
          }
          *g4 = o;
        } else {
          *g4 = s4;
        }
      }
    }
    // ---- release the buffer (the next copy into it is an async-proxy write)
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[b]);
    if (++b == kLBuf) {
      b = 0;
      ++use;
    }
  }
}

}  // namespace molt
