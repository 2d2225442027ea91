// dispatch.h -- host-side entry points of the per-(function, precision)
// kernel instantiation units.
#pragma once

#include <cuda_runtime.h>

#include "sweep.cuh"

namespace chessfad {

// Residual hDuals held in registers at once by the Fletcher-Powell sweep for
// chunk size C (keeps MB * (2C+1) accumulator registers near 70).
constexpr int fp_mb(int C) { return C <= 4 ? 8 : 32 / C; }

#define CHESSFAD_DECL(name) \
    cudaError_t name(int C, bool hvp, const SweepArgs &a, int block_threads, cudaStream_t stream)
CHESSFAD_DECL(launch_rosenbrock_f64);
CHESSFAD_DECL(launch_rosenbrock_f32c);
CHESSFAD_DECL(launch_ackley_f64);
CHESSFAD_DECL(launch_ackley_f32c);
CHESSFAD_DECL(launch_fp_f64);
CHESSFAD_DECL(launch_fp_f32c);
#undef CHESSFAD_DECL

// n == 1 under CHESSFAD_FP32_COMP: the Hessian is one entry, a sum of terms
// that can cancel to far below their size; the single sweep runs in FP64 with
// float inputs and output.
cudaError_t launch_rosenbrock_f64io32(bool hvp, const SweepArgs &a, int block_threads, cudaStream_t stream);
cudaError_t launch_ackley_f64io32(bool hvp, const SweepArgs &a, int block_threads, cudaStream_t stream);
cudaError_t launch_fp_f64io32(bool hvp, const SweepArgs &a, int block_threads, cudaStream_t stream);

// Symmetric variants (SCHUNK-HESS, SC-HESS-VEC): a.maxpts = points per block,
// a.tpp = threads per point.
#define CHESSFAD_SYM(name) cudaError_t launch_##name##_sym(int C, bool hvp, const SweepArgs &a, cudaStream_t stream); \
    size_t smem_##name##_sym(int C, bool hvp, const SweepArgs &a)
CHESSFAD_SYM(rosenbrock_f64);
CHESSFAD_SYM(rosenbrock_f32c);
CHESSFAD_SYM(ackley_f64);
CHESSFAD_SYM(ackley_f32c);
CHESSFAD_SYM(fp_f64);
CHESSFAD_SYM(fp_f32c);
#undef CHESSFAD_SYM

// Symmetric method with seed-sparse propagation; C in {4, 8, 16}.
#define CHESSFAD_SPARSE(name) cudaError_t launch_##name##_sym_sparse(int C, bool hvp, const SweepArgs &a, cudaStream_t stream)
CHESSFAD_SPARSE(rosenbrock_f64);
CHESSFAD_SPARSE(rosenbrock_f32c);
CHESSFAD_SPARSE(ackley_f64);
CHESSFAD_SPARSE(ackley_f32c);
CHESSFAD_SPARSE(fp_f64);
CHESSFAD_SPARSE(fp_f32c);
#undef CHESSFAD_SPARSE

// cudaFuncGetAttributes of the instantiation (registers, local memory).
#define CHESSFAD_ATTR(name) cudaError_t name(int C, bool hvp, cudaFuncAttributes *fa)
CHESSFAD_ATTR(attr_rosenbrock_f64);
CHESSFAD_ATTR(attr_rosenbrock_f32c);
CHESSFAD_ATTR(attr_ackley_f64);
CHESSFAD_ATTR(attr_ackley_f32c);
CHESSFAD_ATTR(attr_fp_f64);
CHESSFAD_ATTR(attr_fp_f32c);
#undef CHESSFAD_ATTR

}  // namespace chessfad
