// Launch entry point of the line-per-lane FP32 sweeps (csrc/sweep_lanes.cuh).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "sweep_lanes.cuh"

namespace molt {

// epi: EPI_STORE (float output), EPI_ACC_SET, EPI_ACC_ADD or EPI_ACC_AXPY.
// `map` is the tensor map of the input for strided lines (unused for x lines).
// Persistent launch: at most (SMs x resident CTAs) CTAs walk the tiles.
cudaError_t launch_lanes(int epi, const LanesArgs& a, const CUtensorMap& map, cudaStream_t s);

}  // namespace molt
