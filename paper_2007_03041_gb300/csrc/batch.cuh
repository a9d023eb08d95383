// Batched heat step: many independent 2-D problems of uneven sizes advanced
// by ONE persistent, cooperative kernel per time step.
//
// The kernel walks the phases of a 3-stage SSP Runge-Kutta step:
//   for each stage: [x sweeps of every problem] -> [y sweeps] -> [FP64 update]
// and separates the phases with a grid barrier.  Within a sweep phase the CTAs
// take (problem, line tile) work items round-robin; every problem brings its
// own tile shape (points per lane E, warps per line, lines per tile), chosen
// per size class by the host-side autotuner.  Every wait is bounded: a grid
// barrier that does not complete within the wait limit records ST_TIMEOUT and
// the kernel returns.  Data written earlier in the same launch is read through
// L2 only.
#pragma once

#include "sweep.cuh"
#include "sweep_tma.cuh"

namespace molt {

struct BatchSweep {
  SweepArgs a;       // geometry, coefficients and tile shape of one (problem, axis)
  int E;             // points per lane (4, 8 or 16)
  int first_item;    // first work item of this problem in the phase
  int ntiles;
};

struct BatchUpdate {
  const float* acc;
  double* u;         // u^n
  double* st1;       // stage states
  double* st2;
  float* copy;       // FP32 copy the sweeps read
  long long total;
  long long first_chunk;
};

struct BatchParams {
  int nprob;
  const BatchSweep* sweeps;   // [nprob][2]
  int items[2];               // work items of the x and y sweep phases
  const BatchUpdate* updates; // [nprob]
  long long chunks;           // work items of the update phase
  double coefS;               // -beta^2
  int stages;                 // 3 (a full step) or 1 (tuning)
  int phase_mask;             // bit 0: x sweeps, bit 1: y sweeps, bit 2: updates
  unsigned int* bar_count;
  unsigned int* bar_gen;
  int* status;
  long long wait_limit;       // cycles
  int skip_arrive;            // test hook: CTA 0 never arrives at the first barrier
  unsigned int stage_off;     // shared-memory offset of the tile staging buffer
};

// Staging buffer of one tile's raw input (W lines x n points, FP32): the
// asynchronous copy of a CTA's next tile lands here while the current tile
// is computed.
constexpr int kStageFloats = 512 * 16;   // W * n = 512 * E <= 8192

// 16-byte asynchronous copy through L2 only (.cg): the sweep inputs were
// written earlier in the same launch by other CTAs, so no L1 line may serve
// them.
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned int d = static_cast<unsigned int>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Issues the copy of the tile starting at line0 into the staging buffer:
// contiguous lines as [w][n], strided lines as [p][W].  Batch tiles are exact
// fits (n a multiple of 128, the line count a multiple of W), so contiguous
// rows and strided rows of W >= 4 floats move as asynchronous 16-byte
// pieces; rows of one or two floats are loaded synchronously (through L2).
// log2 of a power of two
__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

__device__ __forceinline__ void stage_tile(const SweepArgs& a, float* stage, long long line0) {
  const float* in = static_cast<const float*>(a.in);
  const int n = a.g.n, W = a.W;          // powers of two in batch tiles
  const int ln = ilog2(n), lW = ilog2(W);
  if (a.contiguous) {
    const int lc = ln - 2;               // 16-byte chunks per line
    for (int t = threadIdx.x; t < W << lc; t += blockDim.x) {
      const int w = t >> lc, c = t & ((1 << lc) - 1);
      if (line0 + w < a.g.nlines) cp_async16(stage + (w << ln) + 4 * c, in + line_base(a.g, line0 + w) + 4 * c);
    }
  } else if (line0 < a.g.nlines) {
    const long long b0 = line_base(a.g, line0);
    if (W >= 4) {
      const int lp = lW - 2;             // 16-byte pieces per row
      for (int t = threadIdx.x; t < n << lp; t += blockDim.x) {
        const int q = t >> lp, c = t & ((1 << lp) - 1);
        cp_async16(stage + (q << lW) + 4 * c, in + b0 + q * a.g.stride + 4 * c);
      }
    } else {
      for (int t = threadIdx.x; t < n << lW; t += blockDim.x) {
        const int q = t >> lW, w = t & (W - 1);
        stage[t] = __ldcg(in + b0 + q * a.g.stride + w);
      }
    }
  }
  cp_async_commit();
}

// Staging layout -> padded per-line layout of the compute core.
template <int E>
__device__ __forceinline__ void unstage_tile(const SweepArgs& a, const float* stage, float* lines) {
  const int n = a.g.n, W = a.W;
  const int ln = ilog2(n), lW = ilog2(W);
  if (a.contiguous) {
    for (int t = threadIdx.x; t < W << ln; t += blockDim.x) {
      const int w = t >> ln, q = t & (n - 1);
      lines[w * a.LS + phys<E>(q)] = stage[t];
    }
  } else {
    for (int t = threadIdx.x; t < n << lW; t += blockDim.x) {
      const int q = t >> lW, w = t & (W - 1);
      lines[w * a.LS + phys<E>(q)] = stage[t];
    }
  }
}

#ifndef MOLT_BATCH_CHUNK
#define MOLT_BATCH_CHUNK 4096
#endif
constexpr int kChunk = MOLT_BATCH_CHUNK;  // points per update work item

// Grid barrier with a bounded wait (cooperative launch: all CTAs resident).
__device__ __forceinline__ bool grid_sync(const BatchParams& p, bool skip) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* gen = p.bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    bool done = false;
    if (!skip) {
      const unsigned int arrived = atomicAdd(p.bar_count, 1u) + 1u;
      if (arrived == gridDim.x) {
        *p.bar_count = 0u;
        __threadfence();
        atomicAdd(p.bar_gen, 1u);
        done = true;
      }
    }
    if (!done) {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > p.wait_limit) {
          atomicOr(p.status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// One (problem, line tile) work item: the tile shape fills the CTA exactly
// (32 * nwl * W == blockDim.x) and the lines are an exact fit (n = 32*nwl*E).
// The tile's input is in the staging buffer (copy complete and visible); the
// copy of the next tile (if any) is issued once the buffer has been read.
template <int E>
__device__ __forceinline__ void batch_tile(const SweepArgs& a, const TileSmem& sm, long long line0, int ax,
                                           float* stage, const SweepArgs* next, long long next_line0) {
  float* lines = static_cast<float*>(sm.lines);
  const int warp = threadIdx.x >> 5, lw = warp / a.nwl;
  unstage_tile<E>(a, stage, lines);
  __syncthreads();
  if (next) stage_tile(*next, stage, next_line0);
  compute_lines_any<float, false, false, E>(a, sm, line0 + lw < a.g.nlines);
  if (ax == 0) epilogue_tile<float, double, EPI_ACC_SET, E, true>(a, lines, line0, 0.0);
  else epilogue_tile<float, double, EPI_ACC_ADD, E, true>(a, lines, line0, 0.0);
  __syncthreads();
}

// L2 prefetch of the accumulator a y-phase tile's epilogue reads, issued for
// the CTA's next work item before the current one is computed.  One request
// per 128-byte segment (contiguous lines) or per row (strided lines).
__device__ __forceinline__ void prefetch_acc(const SweepArgs& a, long long line0) {
  const LineGeom& g = a.g;
  const int n = g.n, W = a.W;
  const char* acc = static_cast<const char*>(a.acc);
  if (a.contiguous) {
    const int nseg = (n + 31) / 32;
    for (int t = threadIdx.x; t < W * nseg; t += blockDim.x) {
      const int w = t / nseg, sg = t - w * nseg;
      if (line0 + w < g.nlines) prefetch_l2(acc + (line_base(g, line0 + w) + 32LL * sg) * 4);
    }
  } else if (line0 < g.nlines) {
    const long long b0 = line_base(g, line0);
    for (int q = threadIdx.x; q < n; q += blockDim.x) prefetch_l2(acc + (b0 + q * g.stride) * 4);
  }
}

__device__ __forceinline__ int find_problem(const BatchParams& p, long long item, int ax) {
  int lo = 0, hi = p.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.sweeps[mid * 2 + ax].first_item <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_update(const BatchParams& p, long long chunk) {
  int lo = 0, hi = p.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.updates[mid].first_chunk <= chunk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Compiled for two CTAs per SM (64 registers; more spills than at 128, but
// the second resident CTA covers the phases' memory latency: 64 problems,
// 7.09 -> 6.81 ms per RK3 step).
#ifndef MOLT_BATCH_MIN_BLOCKS
#define MOLT_BATCH_MIN_BLOCKS 2
#endif
#ifndef MOLT_BATCH_KERNEL_TU
// defined in csrc/batch.cu (its own translation unit: FP32 <-> FP64
// conversions selected in place, MOLT_CONV_SELECT)
__global__ void batch_heat_kernel(const BatchParams p);
#else
__global__ void __launch_bounds__(512, MOLT_BATCH_MIN_BLOCKS) batch_heat_kernel(const BatchParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SweepArgs sa;
  __shared__ int s_prob, s_tile, s_nprob, s_ntile;
  static const double rk[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  bool first = true;
  for (int s = 0; s < p.stages; ++s) {
    for (int ax = 0; ax < 2; ++ax) {
      if (p.phase_mask & (1 << ax)) {
        float* stage = reinterpret_cast<float*>(smem_raw + p.stage_off);
        if (blockIdx.x < p.items[ax]) {
          const int p0 = find_problem(p, blockIdx.x, ax);
          const SweepArgs& a0 = p.sweeps[p0 * 2 + ax].a;
          stage_tile(a0, stage, (long long)(blockIdx.x - p.sweeps[p0 * 2 + ax].first_item) * a0.W);
        }
        for (long long item = blockIdx.x; item < p.items[ax]; item += gridDim.x) {
          if (threadIdx.x == 0) {
            s_prob = find_problem(p, item, ax);
            s_tile = int(item - p.sweeps[s_prob * 2 + ax].first_item);
            const long long nx = item + gridDim.x;
            s_nprob = nx < p.items[ax] ? find_problem(p, nx, ax) : -1;
            if (s_nprob >= 0) s_ntile = int(nx - p.sweeps[s_nprob * 2 + ax].first_item);
          }
          cp_async_wait_all();
          __syncthreads();
          const SweepArgs* na = s_nprob >= 0 ? &p.sweeps[s_nprob * 2 + ax].a : nullptr;
          const long long nline0 = na ? (long long)s_ntile * na->W : 0;
          if (na && ax == 1) prefetch_acc(*na, nline0);
          const BatchSweep* bs = p.sweeps + s_prob * 2 + ax;
          const int* src = reinterpret_cast<const int*>(&bs->a);
          int* dst = reinterpret_cast<int*>(&sa);
          for (int w = threadIdx.x; w < int(sizeof(SweepArgs) / 4); w += blockDim.x) dst[w] = src[w];
          const int E = bs->E;
          __syncthreads();
          size_t used;
          const TileSmem sm = carve<float>(smem_raw, sa, &used);
          const long long line0 = (long long)s_tile * sa.W;
          if (E == 16) batch_tile<16>(sa, sm, line0, ax, stage, na, nline0);
          else if (E == 8) batch_tile<8>(sa, sm, line0, ax, stage, na, nline0);
          else batch_tile<4>(sa, sm, line0, ax, stage, na, nline0);
        }
      }
      const bool skip = first && p.skip_arrive && blockIdx.x == 0;
      first = false;
      if (!grid_sync(p, skip)) return;
    }
    if (p.phase_mask & 4) {
      const double a0 = rk[s][0], a1 = rk[s][1];
      bool bad = false;
      for (long long c = blockIdx.x; c < p.chunks; c += gridDim.x) {
        const BatchUpdate& U = p.updates[find_update(p, c)];
        const long long i0 = (c - U.first_chunk) * kChunk;
        const long long i1 = i0 + kChunk < U.total ? i0 + kChunk : U.total;
        const double* us = s == 0 ? U.u : (s == 1 ? U.st1 : U.st2);
        double* dstp = s == 0 ? U.st1 : (s == 1 ? U.st2 : U.u);
        // L2 prefetch of the CTA's next chunk (u, the stage input, acc)
        {
          const long long cn = c + gridDim.x;
          if (cn < p.chunks) {
            const BatchUpdate& V = p.updates[find_update(p, cn)];
            const long long j0 = (cn - V.first_chunk) * kChunk;
            const long long j1 = j0 + kChunk < V.total ? j0 + kChunk : V.total;
            const double* vs = s == 0 ? V.u : (s == 1 ? V.st1 : V.st2);
            for (long long j = j0 + 16LL * threadIdx.x; j < j1; j += 16LL * blockDim.x) {
              prefetch_l2(V.u + j);
              prefetch_l2(j + 8 < j1 ? V.u + j + 8 : V.u + j);
              if (vs != V.u) {
                prefetch_l2(vs + j);
                prefetch_l2(j + 8 < j1 ? vs + j + 8 : vs + j);
              }
              prefetch_l2(V.acc + j);
            }
          }
        }
        // all loads of a thread's points are issued before its stores (the
        // CTA is the SM's only one, so memory parallelism comes from here)
        constexpr int kPer = kChunk / 512;
        double uu[kPer], ss[kPer];
        float aa[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const long long i = i0 + threadIdx.x + (long long)k * blockDim.x;
          if (i < i1) {
            uu[k] = __ldcg(U.u + i);
            ss[k] = __ldcg(us + i);
            aa[k] = __ldcg(U.acc + i);
          }
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const long long i = i0 + threadIdx.x + (long long)k * blockDim.x;
          if (i < i1) {
            const double r = fma(a0, uu[k], a1 * fma(p.coefS, f2d(aa[k]), ss[k]));
            dstp[i] = r;
            U.copy[i] = d2f(r);
            bad |= nonfinite(r);
          }
        }
      }
      if (bad) atomicOr(p.status, ST_NONFINITE);
      if (s + 1 < p.stages && !grid_sync(p, false)) return;
    }
  }
}

#endif  // MOLT_BATCH_KERNEL_TU

}  // namespace molt
