// Launch entry points of the sweep kernel instantiations (one translation
// unit per precision family, compiled in parallel).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "sweep.cuh"
#include "sweep_tma.cuh"

namespace molt {

// TMA-fed persistent launch: staging geometry, tensor map, shared bytes.
struct TmaPlan {
  TmaGeom tg;
  CUtensorMap map;
  size_t smem;
};

// tma == nullptr: one tile per CTA with plain loads (grid/block/smem given);
// otherwise the persistent TMA kernel on at most `grid` CTAs.
template <typename T, typename TIN, typename TST, int JQ, int EPI>
cudaError_t launch_sweep(const SweepArgs& a, const TmaPlan* tma, int grid, int block, size_t smem,
                         cudaStream_t s);

// Points per lane of a plan (16 unless the planner chose 8 or 4).
inline int plan_E(const SweepArgs& a) { return a.E == 8 || a.E == 4 ? a.E : kE; }

// Exact-fit lines (n = 32*E*nwl) run the unmasked kernels.
inline bool exact_fit(const SweepArgs& a) { return a.g.n == a.nwl * 32 * plan_E(a); }

#define MOLT_DEFINE_LAUNCH                                                                       \
  template <typename T, typename TIN, typename TST, int JQ, int EPI>                             \
  cudaError_t launch_sweep(const SweepArgs& a, const TmaPlan* tma, int grid, int block,          \
                           size_t smem, cudaStream_t s) {                                        \
    if constexpr (JQ == JQ_LEARNED) {                                                            \
      if (tma) return cudaErrorNotSupported;                                                     \
    } else if (tma) {                                                                            \
      auto k = &sweep_tma_kernel<T, TIN, TST, JQ, EPI>;                                          \
      static bool configured = false;                                                            \
      if (!configured) {                                                                         \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                             int(kSmemOptIn));                                   \
        if (e != cudaSuccess) return e;                                                          \
        configured = true;                                                                       \
      }                                                                                          \
      int per_sm = 0, dev = 0, sms = 0;                                                          \
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, tma->smem); \
      if (e != cudaSuccess) return e;                                                            \
      cudaGetDevice(&dev);                                                                       \
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);                         \
      long long ntiles = (a.g.nlines + a.W - 1) / a.W;                                           \
      long long g = (long long)sms * (per_sm > 0 ? per_sm : 1);                                  \
      if (g > ntiles) g = ntiles;                                                                \
      k<<<int(g), block, tma->smem, s>>>(a, tma->tg, tma->map);                                  \
      return cudaGetLastError();                                                                 \
    }                                                                                            \
    const bool fit = exact_fit(a);                                                               \
    const int ei = plan_E(a) == 16 ? 0 : (plan_E(a) == 8 ? 1 : 2);                               \
    using KFn = void (*)(SweepArgs);                                                             \
    static const KFn kfn[3][2] = {                                                               \
        {&sweep_kernel<T, TIN, TST, JQ, EPI, true, 16>, &sweep_kernel<T, TIN, TST, JQ, EPI, false, 16>}, \
        {&sweep_kernel<T, TIN, TST, JQ, EPI, true, 8>, &sweep_kernel<T, TIN, TST, JQ, EPI, false, 8>},   \
        {&sweep_kernel<T, TIN, TST, JQ, EPI, true, 4>, &sweep_kernel<T, TIN, TST, JQ, EPI, false, 4>}};  \
    const KFn k = kfn[ei][fit ? 1 : 0];                                                          \
    static bool configured[3][2] = {};                                                           \
    if (!configured[ei][fit]) {                                                                  \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                           int(kSmemTileBudget));                                \
      if (e != cudaSuccess) return e;                                                            \
      configured[ei][fit] = true;                                                                \
    }                                                                                            \
    k<<<grid, block, smem, s>>>(a);                                                              \
    return cudaGetLastError();                                                                   \
  }

#define MOLT_INST(T, TIN, TST, JQ, EPI)                                                          \
  template cudaError_t launch_sweep<T, TIN, TST, JQ, EPI>(const SweepArgs&, const TmaPlan*, int,   \
                                                            int, size_t, cudaStream_t);

}  // namespace molt
