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
};

constexpr int kChunk = 4096;  // points per update work item

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
template <int E>
__device__ __forceinline__ void batch_tile(const SweepArgs& a, const TileSmem& sm, long long line0, int ax) {
  float* lines = static_cast<float*>(sm.lines);
  const int warp = threadIdx.x >> 5, lw = warp / a.nwl;
  const int tl = (warp - lw * a.nwl) * 32 + (threadIdx.x & 31);
  load_tile<float, float, E, true>(a, static_cast<const float*>(a.in), lines, line0, lw, tl);
  __syncthreads();
  compute_lines_any<float, false, false, E>(a, sm, line0 + lw < a.g.nlines);
  if (ax == 0) epilogue_tile<float, double, EPI_ACC_SET, E, true>(a, lines, line0, 0.0);
  else epilogue_tile<float, double, EPI_ACC_ADD, E, true>(a, lines, line0, 0.0);
  __syncthreads();
}

// L2 prefetch of a tile's sweep input (and, for the y phase, of the
// accumulator its epilogue reads): issued for the CTA's next work item
// before the current one is computed, so that the plain loads of the next
// tile hit L2.  One request per 128-byte segment (contiguous lines) or per
// row of the tile (strided lines).
__device__ __forceinline__ void prefetch_tile(const SweepArgs& a, long long line0, int ax) {
  const LineGeom& g = a.g;
  const int n = g.n, W = a.W;
  const char* ops[2] = {static_cast<const char*>(a.in), ax == 1 ? static_cast<const char*>(a.acc) : nullptr};
  for (int o = 0; o < 2; ++o) {
    if (!ops[o]) continue;
    if (a.contiguous) {
      const int nseg = (n + 31) / 32;
      for (int t = threadIdx.x; t < W * nseg; t += blockDim.x) {
        const int w = t / nseg, sg = t - w * nseg;
        if (line0 + w < g.nlines) prefetch_l2(ops[o] + (line_base(g, line0 + w) + 32LL * sg) * 4);
      }
    } else if (line0 < g.nlines) {
      const long long b0 = line_base(g, line0);
      for (int q = threadIdx.x; q < n; q += blockDim.x) prefetch_l2(ops[o] + (b0 + q * g.stride) * 4);
    }
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

__global__ void __launch_bounds__(512, 1) batch_heat_kernel(const BatchParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SweepArgs sa;
  __shared__ int s_prob, s_tile, s_nprob, s_ntile;
  static const double rk[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  bool first = true;
  for (int s = 0; s < p.stages; ++s) {
    for (int ax = 0; ax < 2; ++ax) {
      if (p.phase_mask & (1 << ax)) {
        for (long long item = blockIdx.x; item < p.items[ax]; item += gridDim.x) {
          if (threadIdx.x == 0) {
            s_prob = find_problem(p, item, ax);
            s_tile = int(item - p.sweeps[s_prob * 2 + ax].first_item);
            const long long nx = item + gridDim.x;
            s_nprob = nx < p.items[ax] ? find_problem(p, nx, ax) : -1;
            if (s_nprob >= 0) s_ntile = int(nx - p.sweeps[s_nprob * 2 + ax].first_item);
          }
          __syncthreads();
          if (s_nprob >= 0) {
            const SweepArgs& na = p.sweeps[s_nprob * 2 + ax].a;
            prefetch_tile(na, (long long)s_ntile * na.W, ax);
          }
          const BatchSweep* bs = p.sweeps + s_prob * 2 + ax;
          const int* src = reinterpret_cast<const int*>(&bs->a);
          int* dst = reinterpret_cast<int*>(&sa);
          for (int w = threadIdx.x; w < int(sizeof(SweepArgs) / 4); w += blockDim.x) dst[w] = src[w];
          const int E = bs->E;
          __syncthreads();
          size_t used;
          const TileSmem sm = carve<float>(smem_raw, sa, &used);
          const long long line0 = (long long)s_tile * sa.W;
          if (E == 16) batch_tile<16>(sa, sm, line0, ax);
          else if (E == 8) batch_tile<8>(sa, sm, line0, ax);
          else batch_tile<4>(sa, sm, line0, ax);
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
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
          const double r = fma(a0, __ldcg(U.u + i), a1 * fma(p.coefS, f2d(__ldcg(U.acc + i)), __ldcg(us + i)));
          dstp[i] = r;
          U.copy[i] = d2f(r);
          bad |= nonfinite(r);
        }
      }
      if (bad) atomicOr(p.status, ST_NONFINITE);
      if (s + 1 < p.stages && !grid_sync(p, false)) return;
    }
  }
}

}  // namespace molt
