// dispatch.h -- host-side entry points of the kernel instantiation slices
// (instances.cu compiled once per function and precision).
#pragma once

#include <cuda_runtime.h>

#include "sweep.cuh"

namespace chessfad {

// Residual hDuals held in registers at once by the Fletcher-Powell sweep for
// chunk size C (keeps MB * (2C+1) accumulator registers near 70).
constexpr int fp_mb(int C) { return C <= 4 ? 8 : 32 / C; }

// The launch functions of one (function, precision) slice.  C is the chunk
// size (a compile-time constant inside; an unsupported C returns
// cudaErrorInvalidValue or 0 bytes).
struct SliceOps {
    // plain method (Alg. 7 / Alg. 5), C in {1,2,4,8,16,32}
    cudaError_t (*sweep)(int C, bool hvp, const SweepArgs &a, int block_threads, cudaStream_t stream);
    // registers / local memory of the plain kernel
    cudaError_t (*attr)(int C, bool hvp, cudaFuncAttributes *fa);
    // symmetric method (Alg. 8 / Alg. 6): a.maxpts = points per block,
    // a.tpp = threads per point; and its dynamic shared memory
    cudaError_t (*sym)(int C, bool hvp, const SweepArgs &a, cudaStream_t stream);
    size_t (*sym_smem)(int C, bool hvp, const SweepArgs &a);
    // symmetric method with seed-sparse propagation, C in {4, 8, 16}
    cudaError_t (*sym_sparse)(int C, bool hvp, const SweepArgs &a, cudaStream_t stream);
    // one thread per point (L0, Alg. 9), C in {1..16}; a.maxpts = points per block
    cudaError_t (*point)(int C, bool hvp, const SweepArgs &a, cudaStream_t stream);
    size_t (*point_smem)(int C, bool hvp, const SweepArgs &a);
    // compensated-FP32 slices: n == 1 swept in FP64 with float I/O (null in
    // the FP64 slices)
    cudaError_t (*sweep_f64io32)(bool hvp, const SweepArgs &a, int block_threads, cudaStream_t stream);
};

extern const SliceOps slice_0_0, slice_0_1, slice_1_0, slice_1_1, slice_2_0, slice_2_1;

// The slice of function fn (FN_ROSENBROCK, FN_ACKLEY, FN_FP) in FP64 (f64)
// or compensated FP32.
inline const SliceOps &slice(int fn, bool f64)
{
    switch (fn) {
    case FN_ROSENBROCK: return f64 ? slice_0_1 : slice_0_0;
    case FN_ACKLEY: return f64 ? slice_1_1 : slice_1_0;
    default: return f64 ? slice_2_1 : slice_2_0;
    }
}

}  // namespace chessfad
