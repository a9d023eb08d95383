// Persistent, TMA-fed variant of the line-sweep kernel.
//
// Each CTA walks over tiles of W lines.  The tile's input is brought into a
// staging buffer by the tensor-memory accelerator (cp.async.bulk.tensor,
// completion tracked by an mbarrier); as soon as the staging buffer has been
// transposed into the padded per-line layout of the compute core, the TMA
// copy of the CTA's next tile is issued, so the HBM reads of tile t+1 overlap
// the scans and the epilogue of tile t.  The epilogue operands of the next
// tile are prefetched into L2 at the same time.
//
// Every wait is bounded: after kWaitLimit cycles the CTA records
// ST_TIMEOUT in the status word, waits (bounded) once more for the copy it
// has in flight and returns.
#pragma once

#include <cuda.h>

#include "sweep.cuh"

namespace molt {

constexpr long long kWaitLimit = 4000000000LL;  // cycles (~2 s at 2 GHz)

struct TmaGeom {
  int box_p;      // points per box along the line (<= 256)
  int nbox;       // boxes per line
  int kind;       // 0: contiguous rows (2-D map {n, rows}); 1: y lines (3-D);
                  // 2: z lines (3-D)
  int nx;         // x extent (strided kinds)
  int bw;         // strided kinds: box columns (>= W, a 16-byte multiple)
  int xalign;     // strided kinds: elements per 16 bytes (box x start alignment)
  unsigned int tx_bytes;   // bytes per tile
};

// Strided kinds: the tile's first line sits at column x0 of its row; the box
// starts at x0 rounded down to a 16-byte boundary (a TMA requirement on the
// innermost coordinate), so the tile's lines are columns off..off+W-1 of the
// box.
__device__ __forceinline__ void strided_origin(const TmaGeom& tg, long long line0, int* hi, int* xbox, int* off) {
  const unsigned int l0 = unsigned(line0), nxu = unsigned(tg.nx);
  *hi = int(l0 / nxu);
  const int x0 = int(l0 - unsigned(*hi) * nxu);
  *xbox = x0 & ~(tg.xalign - 1);
  *off = x0 - *xbox;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitLimit) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Issues the TMA boxes of the tile starting at line `line0` into `stage`.
template <typename TIN>
__device__ __forceinline__ void issue_tile(const SweepArgs& a, const TmaGeom& tg, const CUtensorMap* map, TIN* stage,
                                           long long line0, uint64_t* bar) {
  mbar_expect_tx(bar, tg.tx_bytes);
  if (tg.kind == 0) {
    const int boxel = tg.box_p * a.W;
    for (int b = 0; b < tg.nbox; ++b) tma_load_2d(stage + b * boxel, map, b * tg.box_p, int(line0), bar);
  } else {
    const int boxel = tg.box_p * tg.bw;
    int hi, xbox, off;
    strided_origin(tg, line0, &hi, &xbox, &off);
    for (int b = 0; b < tg.nbox; ++b) {
      if (tg.kind == 1) tma_load_3d(stage + b * boxel, map, xbox, b * tg.box_p, hi, bar);
      else tma_load_3d(stage + b * boxel, map, xbox, hi, b * tg.box_p, bar);
    }
  }
}

// L2 prefetch of the epilogue operands of a tile (one request per 128-byte
// row segment).
template <typename T, typename TST, int EPI>
__device__ __forceinline__ void prefetch_operands(const SweepArgs& a, long long line0) {
  const void* ops[3] = {nullptr, nullptr, nullptr};
  int es[3] = {0, 0, 0};
  if constexpr (EPI == EPI_ACC_ADD || EPI == EPI_ACC_AXPY) { ops[0] = a.acc; es[0] = sizeof(T); }
  if constexpr (EPI == EPI_HEAT_FINAL || EPI == EPI_WAVE_FINAL) {
    ops[0] = a.acc; es[0] = sizeof(T);
    ops[1] = a.un; es[1] = sizeof(TST);
    if (EPI == EPI_HEAT_FINAL || !a.from_rest) { ops[2] = a.us; es[2] = sizeof(TST); }
  }
  if constexpr (epi_hj_y(EPI)) {
    ops[0] = a.un; es[0] = sizeof(TST);
    ops[1] = a.out; es[1] = sizeof(TST);
  }
  const int n = a.g.n;
  for (int o = 0; o < 3; ++o) {
    if (!ops[o]) continue;
    const char* base = static_cast<const char*>(ops[o]);
    if (a.contiguous) {
      const int seg = 128 / es[o];
      const int per_line = (n + seg - 1) / seg;
      for (int t = threadIdx.x; t < a.W * per_line; t += blockDim.x) {
        const int w = t / per_line, sgi = t - w * per_line;
        if (line0 + w < a.g.nlines)
          prefetch_l2(base + (line_base(a.g, line0 + w) + (long long)sgi * seg) * es[o]);
      }
    } else {
      if (line0 >= a.g.nlines) continue;
      const long long b0 = line_base(a.g, line0);
      for (int p = threadIdx.x; p < n; p += blockDim.x) prefetch_l2(base + (b0 + p * a.g.stride) * es[o]);
    }
  }
}

// Staging layout -> padded per-line layout of the compute core.
template <typename T, typename TIN>
__device__ __forceinline__ void transpose_tile(const SweepArgs& a, const TmaGeom& tg, const TIN* stage, T* lines,
                                               long long line0) {
  const int W = a.W, n = a.g.n;
  if (tg.kind == 0) {
    // stage: [box][W][box_p]
    const int warp = threadIdx.x >> 5, lw = warp / a.nwl;
    const int tl = (warp - lw * a.nwl) * 32 + (threadIdx.x & 31);
    const int step = a.nwl * 32;
    T* dst = lines + lw * a.LS;
    // box_p and step are multiples of 16 (or box_p == n < step): phys()
    // advances by a constant along r
    for (int b = 0; b < tg.nbox; ++b) {
      const TIN* src = stage + (b * W + lw) * tg.box_p;
      T* d = dst + phys(b * tg.box_p + tl);
      const int dstep = step + step / kE;
#pragma unroll 4
      for (int r = tl; r < tg.box_p; r += step) {
        *d = cvt<T>(src[r]);
        d += dstep;
      }
    }
  } else {
    // stage: [p][bw], the tile's lines in columns off..off+W-1
    int hi, xbox, off;
    strided_origin(tg, line0, &hi, &xbox, &off);
    const int w = threadIdx.x % W;
    const int prow = blockDim.x / W;
    int p = threadIdx.x / W;
    const TIN* src = stage + p * tg.bw + off + w;
    T* dst = lines + w * a.LS + phys(p);
    const int dstep = prow + prow / kE;
#pragma unroll 8
    for (; p < n; p += prow) {
      *dst = cvt<T>(*src);
      src += prow * tg.bw;
      dst += dstep;
    }
  }
}

template <typename T, typename TIN, typename TST, int JQ, int EPI>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks)
    sweep_tma_kernel(const SweepArgs a, const TmaGeom tg, const __grid_constant__ CUtensorMap map) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  size_t used;
  const TileSmem sm = carve<T>(smem_raw, a, &used);
  T* lines = static_cast<T*>(sm.lines);
  const size_t bar_off = (used + 15) & ~size_t(15);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + bar_off);
  int* flag = reinterpret_cast<int*>(smem_raw + bar_off + 8);
  TIN* stage = reinterpret_cast<TIN*>(smem_raw + ((bar_off + 16 + 127) & ~size_t(127)));

  const long long ntiles = (a.g.nlines + a.W - 1) / a.W;
  const int warp = threadIdx.x >> 5, lw = warp / a.nwl;
  const double dt = hj_dt<EPI>(a);
  if (epi_hj_y(EPI) && blockIdx.x == 0 && threadIdx.x == 0 && a.t_dev) *a.t_dev += dt;

  long long tile = blockIdx.x;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
    if (tile < ntiles) issue_tile<TIN>(a, tg, &map, stage, tile * a.W, bar);
  }
  __syncthreads();
  if (tile < ntiles) prefetch_operands<T, TST, EPI>(a, tile * a.W);

  double rmax = 0.0;
  uint32_t parity = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    const long long line0 = tile * a.W;
    if (threadIdx.x == 0) *flag = mbar_wait_bounded(bar, parity) ? 1 : 0;
    __syncthreads();
    if (!*flag) {
      // record the give-up, then wait (bounded) once more for the copy this
      // CTA issued into its own shared memory, the only one in flight
      if (threadIdx.x == 0) {
        atomicOr(a.status, ST_TIMEOUT);
        mbar_wait_bounded(bar, parity);
      }
      return;
    }
    parity ^= 1u;
    transpose_tile<T, TIN>(a, tg, stage, lines, line0);
    __syncthreads();
    const long long next = tile + gridDim.x;
    if (next < ntiles) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        issue_tile<TIN>(a, tg, &map, stage, next * a.W, bar);
      }
      prefetch_operands<T, TST, EPI>(a, next * a.W);
    }
    rmax = fmax(rmax, compute_lines_any<T, JQ, false, kE, epi_hj_gen(EPI)>(a, sm, line0 + lw < a.g.nlines) *
                          a.inv_h);
    rmax = fmax(rmax, epilogue_tile<T, TST, EPI>(a, lines, line0, dt, static_cast<const T*>(sm.lines2)));
    __syncthreads();
  }
  publish_speed<EPI>(a, rmax);
}

}  // namespace molt
