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
// from registers.  x lines arrive by one bulk copy per line into rows padded
// to n + 4 floats (16-byte vector reads of a warp hit distinct banks).
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
// 2^-40 -- sixteen binary orders below FP32 rounding -- are not added (the
// truncation of the convolution tails that Sec. 3 applies at a tolerance),
// so each thread reads at most `lb` segment totals: lb = 5 at nu = 0.4.
//
// Per power: stage 1 (window, first differences, K, scan of the segment from
// zero -> segment totals in shared memory), barrier, stage 2 (initial value
// from the totals, the scan again from it -> D), barrier before the next
// power reads the line.  P <= 2: S_2 = D + D^2 re-reads D from the line
// buffer.  Tiles stream through two stage buffers (the copy of tile t+1 runs
// during tile t); every wait on a copy is bounded.
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
  int LS;                // contiguous: floats per staged line (n + 4)
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
  const float* in;       // contiguous: the sweep input (bulk copies read it)
  float* out;            // EPI_STORE destination
  float* acc;            // accumulator
  int* status;
};

// Bytes of one stage buffer.
__host__ __device__ constexpr size_t lanes_buf_bytes(int n, int contiguous) {
  return size_t(kLW) * size_t(contiguous ? n + 4 : n) * sizeof(float);
}
// Dynamic shared memory of a CTA: two stage buffers, segment totals, barriers.
__host__ __device__ constexpr size_t lanes_smem_bytes(int n, int contiguous) {
  return 2 * lanes_buf_bytes(n, contiguous) + size_t(n / kLE) * kLW * sizeof(float2) + 64;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Issues the copies of tile `tile` into `buf` (warp 0; lane 0 arms the barrier first).
__device__ __forceinline__ void lanes_issue(const LanesArgs& a, const CUtensorMap* map, float* buf, int tile,
                                            uint64_t* bar) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_expect_tx(bar, uint32_t(kLW) * uint32_t(a.n) * 4u);
  __syncwarp();
  if (a.contiguous) {
    const float* src = a.in + (long long)(tile * kLW + lane) * a.n;
    bulk_load(buf + lane * a.LS, src, uint32_t(a.n) * 4u, bar);
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
    const float* row = buf + lane * a.LS;
    const float4* r4 = reinterpret_cast<const float4*>(row);
    float c[24];   // v_{p0-4 .. p0+19}
#pragma unroll
    for (int k = 1; k < 5; ++k) {
      const float4 x = r4[(p0 >> 2) - 1 + k];
      c[4 * k] = x.x; c[4 * k + 1] = x.y; c[4 * k + 2] = x.z; c[4 * k + 3] = x.w;
    }
    if (seg > 0) {
      const float4 x = r4[(p0 >> 2) - 1];
      c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
    } else if (a.bc == 0) {
      const float4 x = r4[(n >> 2) - 1];   // v_{n-4..n-1} = v_{-4..-1}
      c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
    } else {
      const float v0 = c[4];
      c[3] = 2.f * v0 - c[5];
      c[2] = 2.f * v0 - c[6];
      c[1] = 2.f * v0 - c[7];
      c[0] = 0.f;
    }
    if (seg + 1 < a.S) {
      const float4 x = r4[(p0 >> 2) + 4];
      c[20] = x.x; c[21] = x.y; c[22] = x.z; c[23] = x.w;
    } else if (a.bc == 0) {
      const float4 x = r4[0];              // v_{0..3} = v_{n..n+3}
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
__device__ __forceinline__ float* lanes_own(const LanesArgs& a, float* buf, int seg, int lane) {
  return CONTIG ? buf + lane * a.LS + seg * kLE : buf + seg * kLE * kLW + lane;
}
template <bool CONTIG>
__device__ __forceinline__ void lanes_store_own(const LanesArgs& a, float* buf, int seg, int lane,
                                                const float (&x)[kLE]) {
  float* o = lanes_own<CONTIG>(a, buf, seg, lane);
  if constexpr (CONTIG) {
    float4* o4 = reinterpret_cast<float4*>(o);
#pragma unroll
    for (int c = 0; c < 4; ++c) o4[c] = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
  } else {
#pragma unroll
    for (int t = 0; t < kLE; ++t) o[t * kLW] = x[t];
  }
}
template <bool CONTIG>
__device__ __forceinline__ void lanes_load_own(const LanesArgs& a, const float* buf, int seg, int lane,
                                               float (&x)[kLE]) {
  const float* o = lanes_own<CONTIG>(a, const_cast<float*>(buf), seg, lane);
  if constexpr (CONTIG) {
    const float4* o4 = reinterpret_cast<const float4*>(o);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 v = o4[c];
      x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int t = 0; t < kLE; ++t) x[t] = o[t * kLW];
  }
}

// One application of D to the staged lines: returns D at the thread's 16
// points.  Ends with every thread past the barrier that follows the reads of
// the line buffer (the caller may overwrite its own points).
template <bool CONTIG>
__device__ __forceinline__ void lanes_apply_D(const LanesArgs& a, const float* buf, float2* tot, int seg, int lane,
                                              float (&D)[kLE]) {
  // ---- stage 1: K from the first differences, scan of the segment from zero
  float2 Y[kLE];
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
  {
    float2 y = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < kLE; ++t) y = fma2(q2, y, Y[t]);
    tot[seg * kLW + lane] = y;
  }
  __syncthreads();
  // ---- stage 2: initial values from the segment totals
  const int S = a.S, lb = a.lb;
  const float qE = a.qE;
  const int rseg = S - 1 - seg;
  float cR = 0.f, cL = 0.f;
  if (seg < lb || rseg < lb) {
    // line totals of the scans from zero (terms of weight below 2^-40 dropped)
    float TR = 0.f, TL = 0.f;
    if (a.needA || a.needB) {
      for (int j = S > lb ? S - lb : 0; j < S; ++j) TR = fmaf(qE, TR, tot[j * kLW + lane].x);
      for (int j = (S < lb ? S : lb) - 1; j >= 0; --j) TL = fmaf(qE, TL, tot[j * kLW + lane].y);
    }
    // line constants in FP64 (Sec. 2.3 / 3.3 solve)
    const double tr = f2d(TR), tl = f2d(TL);
    if (seg < lb) cR = d2f(fma(a.kA, tr, a.kB * tl));
    if (rseg < lb) cL = d2f(fma(a.kA, tl, a.kB * tr));
  }
  {
    const int jm = seg < lb ? seg : lb;
    for (int j = jm; j >= 1; --j) cR = fmaf(qE, cR, tot[(seg - j) * kLW + lane].x);
    const int jr = rseg < lb ? rseg : lb;
    for (int j = jr; j >= 1; --j) cL = fmaf(qE, cL, tot[(seg + j) * kLW + lane].y);
  }
  {
    float2 y = make_float2(cR, cL);
#pragma unroll
    for (int t = 0; t < kLE; ++t) {
      y = fma2(q2, y, Y[t]);
      Y[t] = y;
    }
  }
  // D_0 = W_R + W_L (halves in the taps); D_R = W_R; D_L = W_L
#pragma unroll
  for (int t = 0; t < kLE; ++t) D[t] = Y[t].x + Y[kLE - 1 - t].y;
}

template <int EPI, bool CONTIG>
__global__ void __launch_bounds__(kLMaxSeg * 32, 1)
    lanes_sweep_kernel(const LanesArgs a, const __grid_constant__ CUtensorMap map) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const size_t bb = lanes_buf_bytes(a.n, CONTIG ? 1 : 0);
  float* const buf0 = reinterpret_cast<float*>(smem_raw);
  float2* tot = reinterpret_cast<float2*>(smem_raw + 2 * bb);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * bb + size_t(a.S) * kLW * sizeof(float2));
  int* flag = reinterpret_cast<int*>(bar + 2);
  const int seg = threadIdx.x >> 5, lane = threadIdx.x & 31;

  int tile = blockIdx.x;
  const int ntiles = int(a.ntiles);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (seg == 0 && tile < ntiles) lanes_issue(a, &map, buf0, tile, &bar[0]);

  for (int k = 0; tile < ntiles; tile += gridDim.x, ++k) {
    const int b = k & 1;
    float* buf = reinterpret_cast<float*>(smem_raw + (b ? bb : 0));
    if (threadIdx.x == 0) *flag = mbar_wait_bounded(&bar[b], uint32_t((k >> 1) & 1)) ? 1 : 0;
    __syncthreads();
    if (!*flag) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_TIMEOUT);
      return;
    }
    // the other buffer was released by the previous tile's closing barrier
    const int next = tile + gridDim.x;
    if (seg == 0 && next < ntiles) lanes_issue(a, &map, reinterpret_cast<float*>(smem_raw + (b ? 0 : bb)), next, &bar[b ^ 1]);
    // L2 prefetch of the accumulator rows this tile's epilogue reads
    if constexpr (EPI == EPI_ACC_ADD || EPI == EPI_ACC_AXPY) {
      if ((int)threadIdx.x < a.n) {
        const int i = threadIdx.x;
        if constexpr (CONTIG) {
          const int per = a.n >> 5;   // 128-byte segments per line
          const int line = i / per, sg = i - line * per;
          prefetch_l2(a.acc + (long long)(tile * kLW + line) * a.n + sg * 32);
        } else {
          prefetch_l2(a.acc + lanes_origin(a, tile) + i * a.stride);
        }
      }
    }

    float D[kLE];
    lanes_apply_D<CONTIG>(a, buf, tot, seg, lane, D);
    if (a.P == 2) {
      lanes_store_own<CONTIG>(a, buf, seg, lane, D);
      __syncthreads();
      float D2[kLE];
      lanes_apply_D<CONTIG>(a, buf, tot, seg, lane, D2);
      lanes_load_own<CONTIG>(a, buf, seg, lane, D);
#pragma unroll
      for (int t = 0; t < kLE; ++t) D[t] += D2[t];
    }
    // ---- epilogue
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
      } else {
        float* dst = (EPI == EPI_STORE ? a.out : a.acc) + g0;
#pragma unroll
        for (int t = 0; t < kLE; ++t, dst += st) *dst = D[t];
      }
    } else {
      // through the line buffer: rows of 16-byte vectors, one line per warp
      lanes_store_own<CONTIG>(a, buf, seg, lane, D);
      __syncthreads();
      const int nv = a.n >> 2;
      for (int line = seg; line < kLW; line += a.S) {
        const float4* s4 = reinterpret_cast<const float4*>(buf + line * a.LS);
        const long long g = (long long)(tile * kLW + line) * a.n;
        if constexpr (EPI == EPI_ACC_ADD || EPI == EPI_ACC_AXPY) {
          float4* d4 = reinterpret_cast<float4*>(a.acc + g);
          for (int j = lane; j < nv; j += 32) {
            const float4 s = s4[j];
            float4 o = d4[j];
            if (EPI == EPI_ACC_ADD) {
              o.x += s.x; o.y += s.y; o.z += s.z; o.w += s.w;
            } else {
              o.x = fmaf(a.coef, s.x, o.x); o.y = fmaf(a.coef, s.y, o.y);
              o.z = fmaf(a.coef, s.z, o.z); o.w = fmaf(a.coef, s.w, o.w);
            }
            d4[j] = o;
          }
        } else {
          float4* d4 = reinterpret_cast<float4*>((EPI == EPI_STORE ? a.out : a.acc) + g);
          for (int j = lane; j < nv; j += 32) d4[j] = s4[j];
        }
      }
    }
    // the next copy into this buffer (two tiles on) is an async-proxy write
    fence_proxy_async_smem();
    __syncthreads();
  }
}

}  // namespace molt
