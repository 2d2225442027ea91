// instances.cu -- the kernel instantiations of the batched sweeps for one
// (function, precision) slice.  The build compiles this file once per slice,
// with CHESSFAD_SLICE_FN (0 Rosenbrock, 1 Ackley, 2 Fletcher-Powell) and
// CHESSFAD_SLICE_F64 (1: FP64 arithmetic, 0: compensated FP32) defined, so the
// six slices compile in parallel; each exports its table of launch functions
// (SliceOps, dispatch.h) as chessfad::slice_<fn>_<f64>.
//
// Per slice: the plain method (CHESS-VEC / CHUNK-HESS, Alg. 7 / Alg. 5) for
// chunk sizes 1..32, the symmetric method (SC-HESS-VEC / SCHUNK-HESS, Alg. 8
// / Alg. 6) for 1..32 and its seed-sparse variant for 4, 8, 16, the
// one-thread-per-point kernels (L0, Alg. 9) for 1..16, and, in the
// compensated-FP32 slices, the one-variable FP64 sweep with float I/O.
#include <type_traits>

#include "dispatch.h"
#include "point.cuh"

#if !defined(CHESSFAD_SLICE_FN) || !defined(CHESSFAD_SLICE_F64)
#error "compile with -DCHESSFAD_SLICE_FN=<0|1|2> -DCHESSFAD_SLICE_F64=<0|1>"
#endif

namespace chessfad {
namespace {

constexpr int FN = CHESSFAD_SLICE_FN;
using T = typename std::conditional<CHESSFAD_SLICE_F64 != 0, double, float>::type;

// f(std::integral_constant<int, C>{}) for the run-time chunk size c, when c
// is one of Cs; cudaErrorInvalidValue otherwise.
template <int... Cs, typename F>
cudaError_t with_chunk(int c, F &&f)
{
    cudaError_t e = cudaErrorInvalidValue;
    (void)((c == Cs ? (e = f(std::integral_constant<int, Cs>{}), true) : false) || ...);
    return e;
}

template <int... Cs, typename F>
size_t bytes_for_chunk(int c, F &&f)
{
    size_t b = 0;
    (void)((c == Cs ? (b = f(std::integral_constant<int, Cs>{}), true) : false) || ...);
    return b;
}

cudaError_t sweep(int c, bool hvp, const SweepArgs &a, int bt, cudaStream_t s)
{
    return with_chunk<1, 2, 4, 8, 16, 32>(c, [&](auto C) {
        constexpr int MB = fp_mb(C.value);
        return hvp ? launch_sweep<T, T, C.value, FN, true, MB>(a, bt, s)
                   : launch_sweep<T, T, C.value, FN, false, MB>(a, bt, s);
    });
}

cudaError_t attr(int c, bool hvp, cudaFuncAttributes *fa)
{
    return with_chunk<1, 2, 4, 8, 16, 32>(c, [&](auto C) {
        constexpr int MB = fp_mb(C.value);
        return hvp ? cudaFuncGetAttributes(fa, sweep_kernel<T, T, C.value, FN, true, MB>)
                   : cudaFuncGetAttributes(fa, sweep_kernel<T, T, C.value, FN, false, MB>);
    });
}

cudaError_t sym(int c, bool hvp, const SweepArgs &a, cudaStream_t s)
{
    return with_chunk<1, 2, 4, 8, 16, 32>(c, [&](auto C) {
        constexpr int MB = fp_mb(C.value);
        return hvp ? launch_sym<T, T, C.value, FN, true, MB>(a, s) : launch_sym<T, T, C.value, FN, false, MB>(a, s);
    });
}

size_t sym_smem(int c, bool hvp, const SweepArgs &a)
{
    return bytes_for_chunk<1, 2, 4, 8, 16, 32>(c, [&](auto C) {
        constexpr int MB = fp_mb(C.value);
        return hvp ? sym_smem_bytes<T, T, C.value, FN, true, MB>(a) : sym_smem_bytes<T, T, C.value, FN, false, MB>(a);
    });
}

cudaError_t sym_sparse(int c, bool hvp, const SweepArgs &a, cudaStream_t s)
{
    return with_chunk<4, 8, 16>(c, [&](auto C) {
        constexpr int MB = fp_mb(C.value);
        return hvp ? launch_sym<T, T, C.value, FN, true, MB, true>(a, s)
                   : launch_sym<T, T, C.value, FN, false, MB, true>(a, s);
    });
}

cudaError_t point(int c, bool hvp, const SweepArgs &a, cudaStream_t s)
{
    return with_chunk<1, 2, 4, 8, 16>(c, [&](auto C) {
        constexpr int MB = fp_mb(C.value);
        return hvp ? launch_point<T, T, C.value, FN, true, MB>(a, s) : launch_point<T, T, C.value, FN, false, MB>(a, s);
    });
}

size_t point_smem(int c, bool hvp, const SweepArgs &a)
{
    return bytes_for_chunk<1, 2, 4, 8, 16>(c, [&](auto C) {
        constexpr int MB = fp_mb(C.value);
        return hvp ? point_smem_bytes<T, T, C.value, FN, true, MB>(a) : point_smem_bytes<T, T, C.value, FN, false, MB>(a);
    });
}

#if !CHESSFAD_SLICE_F64
// n == 1 under compensated FP32: the Hessian is one entry, a sum of terms
// that can cancel far below their size; the single sweep runs in FP64 with
// float inputs and output.
cudaError_t sweep_f64io32(bool hvp, const SweepArgs &a, int bt, cudaStream_t s)
{
    return hvp ? launch_sweep<double, float, 1, FN, true, fp_mb(1)>(a, bt, s)
               : launch_sweep<double, float, 1, FN, false, fp_mb(1)>(a, bt, s);
}
#endif

}  // namespace

#define CHESSFAD_SLICE_NAME_(f, d) slice_##f##_##d
#define CHESSFAD_SLICE_NAME(f, d) CHESSFAD_SLICE_NAME_(f, d)

extern const SliceOps CHESSFAD_SLICE_NAME(CHESSFAD_SLICE_FN, CHESSFAD_SLICE_F64) = {
    sweep, attr, sym, sym_smem, sym_sparse, point, point_smem,
#if CHESSFAD_SLICE_F64
    nullptr,
#else
    sweep_f64io32,
#endif
};

}  // namespace chessfad
