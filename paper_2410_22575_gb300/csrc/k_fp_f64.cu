// Kernel instantiations: fp, double hDual arithmetic (f64), every chunk size.
#include "dispatch.h"

namespace chessfad {

template <int C>
static cudaError_t go(bool hvp, const SweepArgs &a, int bt, cudaStream_t s)
{
    constexpr int MB = fp_mb(C);
    return hvp ? launch_sweep<double, double, C, FN_FP, true, MB>(a, bt, s) : launch_sweep<double, double, C, FN_FP, false, MB>(a, bt, s);
}

cudaError_t launch_fp_f64(int C, bool hvp, const SweepArgs &a, int bt, cudaStream_t s)
{
    switch (C) {
    case 1: return go<1>(hvp, a, bt, s);
    case 2: return go<2>(hvp, a, bt, s);
    case 4: return go<4>(hvp, a, bt, s);
    case 8: return go<8>(hvp, a, bt, s);
    case 16: return go<16>(hvp, a, bt, s);
    case 32: return go<32>(hvp, a, bt, s);
    }
    return cudaErrorInvalidValue;
}

template <int C>
static cudaError_t at(bool hvp, cudaFuncAttributes *fa)
{
    constexpr int MB = fp_mb(C);
    return hvp ? cudaFuncGetAttributes(fa, sweep_kernel<double, double, C, FN_FP, true, MB>)
               : cudaFuncGetAttributes(fa, sweep_kernel<double, double, C, FN_FP, false, MB>);
}

cudaError_t attr_fp_f64(int C, bool hvp, cudaFuncAttributes *fa)
{
    switch (C) {
    case 1: return at<1>(hvp, fa);
    case 2: return at<2>(hvp, fa);
    case 4: return at<4>(hvp, fa);
    case 8: return at<8>(hvp, fa);
    case 16: return at<16>(hvp, fa);
    case 32: return at<32>(hvp, fa);
    }
    return cudaErrorInvalidValue;
}

// One-variable compensated-FP32 calls: FP64 sweep, float x, v and output.
cudaError_t launch_fp_f64io32(bool hvp, const SweepArgs &a, int bt, cudaStream_t s)
{
    return hvp ? launch_sweep<double, float, 1, FN_FP, true, fp_mb(1)>(a, bt, s)
               : launch_sweep<double, float, 1, FN_FP, false, fp_mb(1)>(a, bt, s);
}

// Symmetric variants (SCHUNK-HESS / SC-HESS-VEC): launch and shared-memory size.
template <int C>
static cudaError_t go_sym(bool hvp, const SweepArgs &a, cudaStream_t s)
{
    constexpr int MB = fp_mb(C);
    return hvp ? launch_sym<double, double, C, FN_FP, true, MB>(a, s) : launch_sym<double, double, C, FN_FP, false, MB>(a, s);
}

template <int C>
static size_t bytes_sym(bool hvp, const SweepArgs &a)
{
    constexpr int MB = fp_mb(C);
    return hvp ? sym_smem_bytes<double, double, C, FN_FP, true, MB>(a) : sym_smem_bytes<double, double, C, FN_FP, false, MB>(a);
}

cudaError_t launch_fp_f64_sym(int C, bool hvp, const SweepArgs &a, cudaStream_t s)
{
    switch (C) {
    case 1: return go_sym<1>(hvp, a, s);
    case 2: return go_sym<2>(hvp, a, s);
    case 4: return go_sym<4>(hvp, a, s);
    case 8: return go_sym<8>(hvp, a, s);
    case 16: return go_sym<16>(hvp, a, s);
    case 32: return go_sym<32>(hvp, a, s);
    }
    return cudaErrorInvalidValue;
}

size_t smem_fp_f64_sym(int C, bool hvp, const SweepArgs &a)
{
    switch (C) {
    case 1: return bytes_sym<1>(hvp, a);
    case 2: return bytes_sym<2>(hvp, a);
    case 4: return bytes_sym<4>(hvp, a);
    case 8: return bytes_sym<8>(hvp, a);
    case 16: return bytes_sym<16>(hvp, a);
    case 32: return bytes_sym<32>(hvp, a);
    }
    return 0;
}

// Symmetric method with seed-sparse propagation (chunk sizes 4, 8, 16).
cudaError_t launch_fp_f64_sym_sparse(int C, bool hvp, const SweepArgs &a, cudaStream_t s)
{
    switch (C) {
    case 4: return hvp ? launch_sym<double, double, 4, FN_FP, true, fp_mb(4), true>(a, s)
                       : launch_sym<double, double, 4, FN_FP, false, fp_mb(4), true>(a, s);
    case 8: return hvp ? launch_sym<double, double, 8, FN_FP, true, fp_mb(8), true>(a, s)
                       : launch_sym<double, double, 8, FN_FP, false, fp_mb(8), true>(a, s);
    case 16: return hvp ? launch_sym<double, double, 16, FN_FP, true, fp_mb(16), true>(a, s)
                        : launch_sym<double, double, 16, FN_FP, false, fp_mb(16), true>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace chessfad
