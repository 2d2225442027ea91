// Kernel instantiations: the L0 (one thread per point) kernels, double hDual
// arithmetic, every function, chunk sizes 1..16.
#include "dispatch.h"
#include "point.cuh"
#include "point.h"

namespace chessfad {

template <int FN, int C>
static cudaError_t go(bool hvp, const SweepArgs &a, cudaStream_t s)
{
    constexpr int MB = fp_mb(C);
    return hvp ? launch_point<double, double, C, FN, true, MB>(a, s) : launch_point<double, double, C, FN, false, MB>(a, s);
}

template <int FN, int C>
static size_t bytes(bool hvp, const SweepArgs &a)
{
    constexpr int MB = fp_mb(C);
    return hvp ? point_smem_bytes<double, double, C, FN, true, MB>(a) : point_smem_bytes<double, double, C, FN, false, MB>(a);
}

template <int FN>
static cudaError_t go_fn(int C, bool hvp, const SweepArgs &a, cudaStream_t s)
{
    switch (C) {
    case 1: return go<FN, 1>(hvp, a, s);
    case 2: return go<FN, 2>(hvp, a, s);
    case 4: return go<FN, 4>(hvp, a, s);
    case 8: return go<FN, 8>(hvp, a, s);
    case 16: return go<FN, 16>(hvp, a, s);
    }
    return cudaErrorInvalidValue;
}

template <int FN>
static size_t bytes_fn(int C, bool hvp, const SweepArgs &a)
{
    switch (C) {
    case 1: return bytes<FN, 1>(hvp, a);
    case 2: return bytes<FN, 2>(hvp, a);
    case 4: return bytes<FN, 4>(hvp, a);
    case 8: return bytes<FN, 8>(hvp, a);
    case 16: return bytes<FN, 16>(hvp, a);
    }
    return 0;
}

cudaError_t launch_point_f64(int fn, int C, bool hvp, const SweepArgs &a, cudaStream_t s)
{
    switch (fn) {
    case FN_ROSENBROCK: return go_fn<FN_ROSENBROCK>(C, hvp, a, s);
    case FN_ACKLEY: return go_fn<FN_ACKLEY>(C, hvp, a, s);
    case FN_FP: return go_fn<FN_FP>(C, hvp, a, s);
    }
    return cudaErrorInvalidValue;
}

size_t smem_point_f64(int fn, int C, bool hvp, const SweepArgs &a)
{
    switch (fn) {
    case FN_ROSENBROCK: return bytes_fn<FN_ROSENBROCK>(C, hvp, a);
    case FN_ACKLEY: return bytes_fn<FN_ACKLEY>(C, hvp, a);
    case FN_FP: return bytes_fn<FN_FP>(C, hvp, a);
    }
    return 0;
}

}  // namespace chessfad
