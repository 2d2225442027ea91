// point.h -- host-side entry points of the L0 (one thread per point) kernels.
#pragma once

#include <cuda_runtime.h>

#include "sweep.cuh"

namespace chessfad {

// fn: FN_ROSENBROCK / FN_ACKLEY / FN_FP; C in {1, 2, 4, 8, 16}.
cudaError_t launch_point_f32c(int fn, int C, bool hvp, const SweepArgs &a, cudaStream_t stream);
cudaError_t launch_point_f64(int fn, int C, bool hvp, const SweepArgs &a, cudaStream_t stream);
size_t smem_point_f32c(int fn, int C, bool hvp, const SweepArgs &a);
size_t smem_point_f64(int fn, int C, bool hvp, const SweepArgs &a);

}  // namespace chessfad
