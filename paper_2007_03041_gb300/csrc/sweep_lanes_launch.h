// Launch entry points of the FP32 linear-rule sweeps: line-per-lane tiles
// (csrc/sweep_lanes.cuh) and warp-per-line x lines (csrc/sweep_xlines.cuh).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "sweep_lanes.cuh"
#include "sweep_xlines.cuh"

namespace molt {

// epi: EPI_STORE (float output), EPI_ACC_SET, EPI_ACC_ADD or EPI_ACC_AXPY.
// `map` is the tensor map of the input for strided lines (unused for x lines).
// Persistent launch: at most (SMs x resident CTAs) CTAs walk the tiles.
cudaError_t launch_lanes(int epi, const LanesArgs& a, const CUtensorMap& map, cudaStream_t s);

// epi: EPI_STORE, EPI_ACC_SET, EPI_ACC_ADD or EPI_ACC_AXPY.  Persistent
// launch of 8-warp CTAs, at most (SMs x resident CTAs).
cudaError_t launch_xlines(int epi, const XLineArgs& a, cudaStream_t s);

}  // namespace molt
