// Warp-per-line FP32 sweeps of x lines (rows of the array): S_P = sum_{p<=P}
// D^p along the contiguous axis for the linear quadrature rule, P <= 2, on
// lines of n = 16 S points, S <= 32 (arXiv 2007.03041, Sec. 2.1-2.4).
//
// Mapping.  Lane s of a line's lane group owns the 16-point segment
// [16 s, 16 s + 16); a warp holds G = 32 / S lines when S is a power of two,
// else one line (lanes S..31 idle).  The G n = 512 points of a warp are one
// contiguous 2 KB run of the array, copied into the warp's shared-memory
// buffer by 16-byte asynchronous copies (coalesced: lane L copies chunks L,
// L + 32, ...) one line group ahead of the compute, and read back as each
// lane's four 16-byte chunks under an XOR swizzle that keeps the reads free
// of bank conflicts.  Everything a segment needs from another -- the ghost
// points of the 5-tap filters, the totals the carries are made of, the line
// totals of the boundary constants -- moves by warp shuffles: no warp waits
// on another, so the SM hides latency with its other warps, not with a
// hand-off chain.
//
// Arithmetic (the difference form of the recurrences, Sec. 2.4).  As in the
// line-per-lane kernel: per power, the first differences of the segment's
// window, K_R and K_L as 5-tap filters of them, the scans of the segment from
// zero -> the segment totals (b_R, b_L).  The value entering segment s from
// the left is sum_{i<s} (q^16)^{s-1-i} b_R[i] + (q^16)^s C_R: the inclusive
// scan X_s = b_R[s] + q^16 X_{s-1} over the lanes runs as a Kogge-Stone scan
// in log2 S shuffle steps with multipliers q^(16 d) (no look-back
// truncation), and the carry is X_{s-1}; mirrored for the left-moving
// recurrence.  The line totals are X_{S-1} (R) and the mirrored scan's value
// at lane 0 (L).  The boundary constants (Sec. 2.3 periodic closure, the 2x2
// Dirichlet solve of Sec. 3.3) C = kA T_same + kB T_other run in FP64 on the
// lanes within reach of an end (segments whose weight (q^16)^s is at least
// 2^-26), one FP64 product chain per lane; the scans again from the carries
// give D = W_R + W_L.  The second power starts from D of the first, whose
// ghost points come from the neighbouring lanes' registers.
#pragma once

#include "sweep.cuh"

namespace molt {

constexpr int kXlSeg = 16;        // points per segment (per lane)
constexpr int kXlWarps = 8;       // warps per CTA
constexpr int kXlBuf = 512;       // floats of one warp's line group (G n)
// resident 8-warp CTAs per SM the kernel is compiled for (3: up to 85
// registers a thread, 24 warps per SM)
#ifndef MOLT_XL_MIN_BLOCKS
#define MOLT_XL_MIN_BLOCKS 3
#endif
// line-group buffers of a warp: the copies of the next kXlStages - 1 groups
// are in flight while one is computed (24 warps x 3 x 2 KB per SM: enough
// bytes in flight for the SM's share of HBM bandwidth)
#ifndef MOLT_XL_STAGES
#define MOLT_XL_STAGES 4
#endif
constexpr int kXlStages = MOLT_XL_STAGES;
// 1: the 5-tap filters of both directions as packed FP32x2 operations (same
// sums in the same order; measured on the 512^3 wave x sweep: 0.304 ms
// against 0.287 with scalar taps -- building the operand pairs costs more
// than the halved FMA count saves)
#ifndef MOLT_XL_PAIRED_TAPS
#define MOLT_XL_PAIRED_TAPS 0
#endif
constexpr size_t kXlSmemBytes = size_t(kXlWarps) * kXlStages * kXlBuf * sizeof(float);

struct XLineArgs {
  int n, S;              // points per line, segments per line
  int G;                 // lines per warp
  int width;             // shuffle width of a lane group: S when G > 1, else 32
  long long nlines;      // lines of the array
  long long ngroups;     // ceil(nlines / G)
  int bc, mode, P;
  int lb;                // segments within reach of an end: (q^16)^s >= 2^-26 for s < lb
  int needA, needB;      // the boundary constants use T of the same / the other direction
  float bR[5], bL[5];    // K_R = sum_i bR[i] d[t+i], K_L = sum_i bL[i] d[u+5-i] (window indices)
  float q;               // e^{-nu} (FP32)
  float qd[5];           // (q^16)^(2^k): multipliers of the Kogge-Stone steps
  double kA, kB;         // boundary constants C = kA T_same + kB T_other (FP64)
  float coef;            // EPI_ACC_AXPY coefficient
  const float* in;       // sweep input, [nlines][n]
  float* out;            // EPI_STORE destination
  float* acc;            // accumulator (EPI_ACC_*)
};

// Float offset of 16-byte chunk c (0..127) of a warp buffer: chunk k of the
// segment owned by lane l (c = 4 l + k) sits at 4 l + (k ^ ((l >> 1) & 3)),
// so the eight lanes of each quarter-warp read eight distinct bank groups.
__device__ __forceinline__ int xl_chunk(int c) {
  const int l = c >> 2, k = c & 3;
  return ((l << 2) | (k ^ ((l >> 1) & 3))) << 2;
}

__device__ __forceinline__ void xl_cp16(float* dst, const float* src) {
  const unsigned int d = static_cast<unsigned int>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void xl_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most kXlStages - 1 of this thread's copy groups are pending
__device__ __forceinline__ void xl_wait_ahead() {
  asm volatile("cp.async.wait_group %0;" ::"n"(kXlStages - 1) : "memory");
}

// Copies line group `grp` (G consecutive lines, G n floats) into `buf`;
// lines past the end of the array are not copied (their lanes' results are
// never stored).
template <int SF>
__device__ __forceinline__ void xl_issue(const XLineArgs& a, long long grp, float* buf, int lane) {
  if constexpr (SF == 32) {
    // one 512-point line per group
    const float* src = a.in + grp * kXlBuf;
#pragma unroll
    for (int j = 0; j < 4; ++j) xl_cp16(buf + xl_chunk(lane + 32 * j), src + 4 * (lane + 32 * j));
  } else {
    const long long line0 = grp * a.G;
    const long long rem = a.nlines - line0;
    const int avail = int((rem < a.G ? rem : a.G) * a.n);    // floats
    const float* src = a.in + line0 * a.n;
    for (int c = lane; 4 * c < avail; c += 32) xl_cp16(buf + xl_chunk(c), src + 4 * c);
  }
}

// Own 16 points of a lane.
__device__ __forceinline__ void xl_load_own(const float* buf, int lane, float (&x)[kXlSeg]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = *reinterpret_cast<const float4*>(buf + xl_chunk(4 * lane + k));
    x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
  }
}
__device__ __forceinline__ void xl_store_own(float* buf, int lane, const float (&x)[kXlSeg]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    *reinterpret_cast<float4*>(buf + xl_chunk(4 * lane + k)) =
        make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
}

// (q^16)^s for 0 <= s < 32, from the Kogge-Stone multipliers.
__device__ __forceinline__ float xl_qpow(const XLineArgs& a, int s) {
  float r = 1.f;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if ((s >> k) & 1) r *= a.qd[k];
  return r;
}

// Lane geometry of a line group (derived where used, so that nothing but
// the lane and its segment stays live across the line loop).
struct XlLane {
  int lane, s;           // lane, segment (s >= S: an idle lane of a one-line warp)
};

// One application of D on the segment: v (own points, registers) ->
// D = W_R + W_L (D_0; the 1/2 is in the taps) or W_R / W_L.  BC: 0 periodic,
// 1 Dirichlet; SF: 32 for 512-point lines (one line a warp, every lane
// active), 0 for the shape in the arguments.
template <int BC, int SF>
__device__ __forceinline__ void xl_apply_D(const XLineArgs& a, const XlLane& L, const float (&v)[kXlSeg],
                                           float (&D)[kXlSeg]) {
  const unsigned FULL = 0xffffffffu;
  const int S = SF ? SF : a.S;
  const int width = SF ? 32 : a.width;
  const bool active = SF ? true : L.s < S;
  const int first = SF ? 0 : L.lane - L.s, last = first + S - 1;
  const int rs = active ? S - 1 - L.s : -1;          // segments to the right
  float2 Y[kXlSeg];
  float2 y;
  {
    // window w[k] = v_{p0-3+k}: own points at k = 3..18, ghosts from the neighbours
    float w[22];
#pragma unroll
    for (int t = 0; t < kXlSeg; ++t) w[t + 3] = v[t];
    // neighbouring segments' lanes (periodic wrap within the group)
    const int left = SF ? ((L.lane + 31) & 31) : (!active ? L.lane : (L.s > 0 ? L.lane - 1 : last));
    const int right = SF ? ((L.lane + 1) & 31) : (!active ? L.lane : (rs > 0 ? L.lane + 1 : first));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      w[k] = __shfl_sync(FULL, v[13 + k], left);
      w[19 + k] = __shfl_sync(FULL, v[k], right);
    }
    if constexpr (BC == 1) {
      // Dirichlet: odd reflection about the end value, v_{-j} = 2 v_0 - v_j
      if (L.s == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = 2.f * w[3] - w[6 - k];
      }
      if (rs == 0) {
#pragma unroll
        for (int k = 19; k < 22; ++k) w[k] = 2.f * w[18] - w[36 - k];
      }
    }
    float d[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) d[k] = w[k + 1] - w[k];
#if MOLT_XL_PAIRED_TAPS
    // Y[t] = (K_R(p0+t), K_L(p0+15-t)) as packed FP32x2 filters: with
    // P[k] = (d[k], d[20-k]), Y[t] = sum_i (bR[i], bL[i]) P[t+i]
#pragma unroll
    for (int t = 0; t < kXlSeg; ++t) {
      float2 r = mul2(make_float2(a.bR[0], a.bL[0]), make_float2(d[t], d[20 - t]));
#pragma unroll
      for (int i = 1; i < 5; ++i)
        r = fma2(make_float2(a.bR[i], a.bL[i]), make_float2(d[t + i], d[20 - t - i]), r);
      Y[t] = r;
    }
#else
#pragma unroll
    for (int t = 0; t < kXlSeg; ++t) {
      float r = a.bR[0] * d[t];
#pragma unroll
      for (int i = 1; i < 5; ++i) r = fmaf(a.bR[i], d[t + i], r);
      Y[t].x = r;
    }
#pragma unroll
    for (int u = kXlSeg - 1; u >= 0; --u) {
      float l = a.bL[0] * d[u + 5];
#pragma unroll
      for (int i = 1; i < 5; ++i) l = fmaf(a.bL[i], d[u + 5 - i], l);
      Y[kXlSeg - 1 - u].y = l;
    }
#endif
  }
  if constexpr (BC == 1) {
    if (L.s == 0) Y[0].x = 0.f;      // K_R(x_0): the right-moving recurrence starts here
    if (rs == 0) Y[0].y = 0.f;     // K_L(x_{n-1})
  }
  const float2 q2 = make_float2(a.q, a.q);
  y = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < kXlSeg; ++t) y = fma2(q2, y, Y[t]);
  // inclusive scans over the segments: X_s = b[s] + q^16 X_{s-1} (R), mirrored (L)
  float XR = y.x, XL = y.y;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int dd = 1 << k;
    if (dd >= S) break;
    const float tR = __shfl_up_sync(FULL, XR, dd, width);
    const float tL = __shfl_down_sync(FULL, XL, dd, width);
    const float nR = fmaf(a.qd[k], tR, XR), nL = fmaf(a.qd[k], tL, XL);
    XR = L.s >= dd ? nR : XR;
    XL = rs >= dd ? nL : XL;
  }
  float cR = __shfl_up_sync(FULL, XR, 1, width);
  float cL = __shfl_down_sync(FULL, XL, 1, width);
  if (L.s == 0) cR = 0.f;
  if (rs == 0) cL = 0.f;
  if (a.needA || a.needB) {
    const float TR = __shfl_sync(FULL, XR, last);
    const float TL = __shfl_sync(FULL, XL, first);
    const bool nR = active && L.s < a.lb, nL = active && rs < a.lb;
    if (nR || nL) {
      // boundary constants in FP64 (Sec. 2.3 / 3.3): C_R near the left end,
      // C_L near the right end, one product chain per lane (the rare lanes
      // of short lines that need both take a second one)
      // one FP64 product for the lines whose constant takes one total
      // (periodic; Dirichlet lines longer than the decay's reach), a second
      // for the rest: each FP64 instruction holds the narrow FP64 pipe for
      // a warp's worth of lanes
      const float same = nR ? TR : TL, other = nR ? TL : TR;
      const double k1 = a.needA ? a.kA : a.kB;
      double C = k1 * f2d(a.needA ? same : other);
      if (a.needA && a.needB) C = fma(a.kB, f2d(other), C);
      if (nR) cR = fmaf(xl_qpow(a, L.s), d2f(C), cR);
      else cL = fmaf(xl_qpow(a, rs), d2f(C), cL);
      if (nR && nL) {
        const double tl = f2d(TL), tr = f2d(TR);
        const double C2 = a.needA && a.needB ? fma(a.kA, tl, a.kB * tr) : (a.needA ? a.kA * tl : a.kB * tr);
        cL = fmaf(xl_qpow(a, rs), d2f(C2), cL);
      }
    }
  }
  y = make_float2(cR, cL);
#pragma unroll
  for (int t = 0; t < kXlSeg; ++t) {
    y = fma2(q2, y, Y[t]);
    Y[t] = y;
  }
#pragma unroll
  for (int t = 0; t < kXlSeg; ++t) D[t] = Y[t].x + Y[kXlSeg - 1 - t].y;
}

template <int EPI, int BC, int SF>
__global__ void __launch_bounds__(kXlWarps * 32, MOLT_XL_MIN_BLOCKS) xline_sweep_kernel(const XLineArgs a) {
  extern __shared__ __align__(128) float xl_smem[];
  const int warp = threadIdx.x >> 5;
  float* wbuf = xl_smem + warp * (kXlStages * kXlBuf);   // this warp's kXlStages group buffers
  XlLane L;
  L.lane = threadIdx.x & 31;
  L.s = (SF == 0 && a.G > 1) ? (L.lane & (a.S - 1)) : L.lane;
  const long long nw = (long long)gridDim.x * kXlWarps;
  long long grp = (long long)blockIdx.x * kXlWarps + warp;
  // copies of the first kXlStages - 1 groups, one commit group each
#pragma unroll
  for (int i = 0; i < kXlStages - 1; ++i) {
    if (grp + i * nw < a.ngroups) xl_issue<SF>(a, grp + i * nw, wbuf + i * kXlBuf, L.lane);
    xl_commit();
  }
  for (int b = 0; grp < a.ngroups; grp += nw, b = b + 1 == kXlStages ? 0 : b + 1) {
    float* buf = wbuf + b * kXlBuf;
    // the copy of the group kXlStages - 1 ahead into the buffer the previous
    // group used (its last reads ended at the __syncwarp closing the previous
    // iteration), then wait for this group's data
    const long long ahead = grp + (kXlStages - 1) * nw;
    const int bn = b == 0 ? kXlStages - 1 : b - 1;
    if (ahead < a.ngroups) xl_issue<SF>(a, ahead, wbuf + bn * kXlBuf, L.lane);
    xl_commit();
    xl_wait_ahead();
    __syncwarp();
    float D[kXlSeg];
    {
      float v[kXlSeg];
      xl_load_own(buf, L.lane, v);
      xl_apply_D<BC, SF>(a, L, v, D);
    }
    if (a.P == 2) {
      xl_store_own(buf, L.lane, D);       // D of the first power, reread below
      float D2[kXlSeg];
      xl_apply_D<BC, SF>(a, L, D, D2);
      xl_load_own(buf, L.lane, D);
#pragma unroll
      for (int t = 0; t < kXlSeg; ++t) D[t] += D2[t];
    }
    // epilogue: through the buffer, so that every global access of the warp
    // is one contiguous 512-byte row
    xl_store_own(buf, L.lane, D);
    __syncwarp();
    const long long line0 = grp * a.G;
    const long long rem = a.nlines - line0;
    const int avail = SF ? kXlBuf : int((rem < a.G ? rem : a.G) * a.n);
    float* dst = (EPI == EPI_STORE ? a.out : a.acc) + line0 * a.n;
#pragma unroll 4
    for (int c = L.lane; 4 * c < avail; c += 32) {
      const float4 s4 = *reinterpret_cast<const float4*>(buf + xl_chunk(c));
      float4* g4 = reinterpret_cast<float4*>(dst + 4 * c);
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
    __syncwarp();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace molt
