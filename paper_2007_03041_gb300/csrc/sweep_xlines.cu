// Launches of the warp-per-line FP32 sweeps of x lines (csrc/sweep_xlines.cuh).
#include "sweep_lanes_launch.h"

namespace molt {

namespace {

template <int EPI, int BC, int SF>
cudaError_t launch_one(const XLineArgs& a, cudaStream_t s) {
  auto k = &xline_sweep_kernel<EPI, BC, SF>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kXlSmemBytes));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kXlWarps * 32, kXlSmemBytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  // persistent: every resident warp walks the line groups, one ahead in its copies
  long long grid = (long long)sms * per_sm;
  const long long need = (a.ngroups + kXlWarps - 1) / kXlWarps;
  if (grid > need) grid = need;
  k<<<int(grid), kXlWarps * 32, kXlSmemBytes, s>>>(a);
  return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_shape(const XLineArgs& a, cudaStream_t s) {
  const bool full = a.S == 32;
  if (a.bc == 1) return full ? launch_one<EPI, 1, 32>(a, s) : launch_one<EPI, 1, 0>(a, s);
  return full ? launch_one<EPI, 0, 32>(a, s) : launch_one<EPI, 0, 0>(a, s);
}

}  // namespace

cudaError_t launch_xlines(int epi, const XLineArgs& a, cudaStream_t s) {
  if (a.S < 1 || a.S > 32 || a.n != a.S * kXlSeg || a.P < 1 || a.P > 2 || a.nlines < 1 || a.lb < 0 ||
      a.lb > a.S || a.G < 1 || a.G * a.S > 32 || a.ngroups != (a.nlines + a.G - 1) / a.G ||
      (a.G > 1 && (a.S & (a.S - 1)) != 0) || a.width != (a.G > 1 ? a.S : 32) || (a.bc != 0 && a.bc != 1))
    return cudaErrorInvalidValue;
  switch (epi) {
    case EPI_STORE: return launch_shape<EPI_STORE>(a, s);
    case EPI_ACC_SET: return launch_shape<EPI_ACC_SET>(a, s);
    case EPI_ACC_ADD: return launch_shape<EPI_ACC_ADD>(a, s);
    case EPI_ACC_AXPY: return launch_shape<EPI_ACC_AXPY>(a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace molt
