// Launches of the line-per-lane FP32 sweeps (csrc/sweep_lanes.cuh).
#include "sweep_lanes_launch.h"

namespace molt {

namespace {

template <int EPI, bool CONTIG, int LB>
cudaError_t launch_one(const LanesArgs& a, const CUtensorMap& map, cudaStream_t s) {
  auto k = &lanes_sweep_kernel<EPI, CONTIG, LB>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(lanes_smem_bytes(kLMaxSeg * kLE, 1)));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int block = 32 * a.S;
  const size_t smem = lanes_smem_bytes(a.n, CONTIG ? 1 : 0);
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  long long grid = (long long)sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  k<<<int(grid), block, smem, s>>>(a, map);
  return cudaGetLastError();
}

template <bool CONTIG, int LB>
cudaError_t launch_epi(int epi, const LanesArgs& a, const CUtensorMap& map, cudaStream_t s) {
  switch (epi) {
    case EPI_STORE: return launch_one<EPI_STORE, CONTIG, LB>(a, map, s);
    case EPI_ACC_SET: return launch_one<EPI_ACC_SET, CONTIG, LB>(a, map, s);
    case EPI_ACC_ADD: return launch_one<EPI_ACC_ADD, CONTIG, LB>(a, map, s);
    case EPI_ACC_AXPY: return launch_one<EPI_ACC_AXPY, CONTIG, LB>(a, map, s);
    case EPI_WAVE_FINAL:
      if constexpr (!CONTIG) return launch_one<EPI_WAVE_FINAL, false, LB>(a, map, s);
      return cudaErrorNotSupported;
    default: return cudaErrorNotSupported;
  }
}

// The look-back is unrolled to a compile-time depth: 4 (nu >= 0.33 with
// 16-point segments and the 2^-26 cut), 8, or every segment of a 512-point
// line.
template <bool CONTIG>
cudaError_t launch_lb(int epi, const LanesArgs& a, const CUtensorMap& map, cudaStream_t s) {
  if (a.lb <= 4) return launch_epi<CONTIG, 4>(epi, a, map, s);
  if (a.lb <= 8) return launch_epi<CONTIG, 8>(epi, a, map, s);
  return launch_epi<CONTIG, kLMaxSeg>(epi, a, map, s);
}

}  // namespace

cudaError_t launch_lanes(int epi, const LanesArgs& a, const CUtensorMap& map, cudaStream_t s) {
  if (a.S < 1 || a.S > kLMaxSeg || a.n != a.S * kLE || a.P < 1 || a.P > 2 || a.ntiles < 1 || a.lb < 1 ||
      a.lb > a.S)
    return cudaErrorInvalidValue;
  return a.contiguous ? launch_lb<true>(epi, a, map, s) : launch_lb<false>(epi, a, map, s);
}

}  // namespace molt
