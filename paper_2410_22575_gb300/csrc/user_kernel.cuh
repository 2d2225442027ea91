// user_kernel.cuh -- CHESS-VEC (Alg. 7) and CHUNK-HESS (Alg. 5) over a batch
// of points for a user-supplied function.  Compiled at run time (NVRTC) after
// the user's source, with
//   CHESSFAD_USER_T    float or double (the arithmetic precision)
//   CHESSFAD_USER_C    the chunk size (compile-time: the hDual lives in registers)
//   CHESSFAD_USER_FN   the name of the user's function template
//                        template <class R, class X>
//                        R name(const X &x, int n, const double *params);
// Decomposition (the paper's L2 over rows, Sec. VI): one thread per
// (point, row i), sweeping the row's ceil(n/C) chunks; a CTA of 256 threads
// stages the x (and v) of the points its rows belong to in shared memory.
// FP32: the row-times-v products are summed as a Dot2 (TwoProd by FMA plus
// TwoSum); the function's own arithmetic is plain FP32, as written by the
// user.  FP64: fused multiply-add accumulation.
#pragma once

#include "user_num.cuh"

namespace chessfad {
namespace user {

struct UserArgs {
    const void *x;
    const void *v;
    void *out;
    long long batch;
    const double *params;
    int n;
    int maxpts;  // points staged per CTA: min(batch, 255 / n + 2)
};

template <typename T>
struct RowDot;
template <>
struct RowDot<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = __fma_rn(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct RowDot<float> {
    CSum s{0.f, 0.f};
    __device__ __forceinline__ void add(float a, float b) { cdot_add(s, a, b); }
    __device__ __forceinline__ float value() const { return csum_value(s); }
};

template <typename T, int C, bool HVP>
__device__ __forceinline__ void user_sweep(const UserArgs &a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *vs = xs + (size_t)a.maxpts * a.n;
    const int n = a.n;
    const long long items = a.batch * n;
    const long long first = (long long)blockIdx.x * blockDim.x;
    const long long last = (first + blockDim.x <= items ? first + blockDim.x : items) - 1;
    const long long p0 = first / n;
    const int staged = (int)(last / n - p0 + 1) * n;
    const T *xg = static_cast<const T *>(a.x) + p0 * n;
    const T *vg = static_cast<const T *>(a.v) + p0 * n;
    for (int t = threadIdx.x; t < staged; t += blockDim.x) {
        xs[t] = xg[t];
        if (HVP) vs[t] = vg[t];
    }
    __syncthreads();
    const long long item = first + threadIdx.x;
    if (item >= items) return;
    const long long p = item / n;
    const int i = (int)(item - p * n);
    const T *xp = xs + (p - p0) * n;
    const T *vp = vs + (p - p0) * n;
    const T z = opaque_zero<T>();
    const int nch = (n + C - 1) / C;
    RowDot<T> dot;
    for (int cn = 0; cn < nch; ++cn) {
        const int cstart = cn * C;
        const Vars<T, C> x{xp, i, cstart, z};
        const Num<T, C> r = ::CHESSFAD_USER_FN<Num<T, C>, Vars<T, C>>(x, n, a.params);
        if (HVP) {
#pragma unroll
            for (int l = 0; l < C; ++l)
                if (cstart + l < n) dot.add(r.a.h[l], vp[cstart + l]);
        } else {
            T *H = static_cast<T *>(a.out) + (p * n + i) * (long long)n + cstart;
#pragma unroll
            for (int l = 0; l < C; ++l)
                if (cstart + l < n) H[l] = r.a.h[l];
        }
    }
    if (HVP) static_cast<T *>(a.out)[p * n + i] = dot.value();
}

}  // namespace user
}  // namespace chessfad

extern "C" __global__ void __launch_bounds__(256) chessfad_user_hvp(chessfad::user::UserArgs a)
{
    chessfad::user::user_sweep<CHESSFAD_USER_T, CHESSFAD_USER_C, true>(a);
}

extern "C" __global__ void __launch_bounds__(256) chessfad_user_hessian(chessfad::user::UserArgs a)
{
    chessfad::user::user_sweep<CHESSFAD_USER_T, CHESSFAD_USER_C, false>(a);
}
