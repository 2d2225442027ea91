// user_kernel.cuh -- CHESS-VEC (Alg. 7) and CHUNK-HESS (Alg. 5) over a batch
// of points for a user-supplied function.  Compiled at run time (NVRTC) after
// the user's source, with
//   CHESSFAD_USER_T    float or double (the arithmetic precision)
//   CHESSFAD_USER_C    the chunk size (compile-time: the hDual lives in registers)
//   CHESSFAD_USER_FN   the name of the user's function template
//                        template <class R, class X>
//                        R name(const X &x, int n, const double *params);
// Two decompositions:
//  plain (CHESS-VEC / CHUNK-HESS, the paper's L2 over rows, Sec. VI): one
//    thread per (point, row i), sweeping the row's ceil(n/C) chunks; a CTA
//    stages the x (and v) of the points its rows belong to in shared memory;
//  symmetric (SC-HESS-VEC, Alg. 8 / SCHUNK-HESS, Alg. 6): a CTA holds maxpts
//    points with tpp threads each; a point's items (row i, chunk cn >=
//    floor(i/C)) are dealt round-robin to its threads.  The Hessian writes
//    each chunk and its mirror image; the HVP stages the chunks in shared
//    memory (compact upper-block layout) and, after one barrier, every thread
//    sums whole rows, each off-diagonal-chunk entry serving both r_i and r_j.
// FP32: the row-times-v products are summed as a Dot2 (TwoProd by FMA plus
// TwoSum); the function's own arithmetic is plain FP32, as written by the
// user, except at n = 1 (FP64 arithmetic, float I/O).  FP64: fused
// multiply-add accumulation.
#pragma once

#include "sym_layout.cuh"
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
    int maxpts;  // plain: points staged per CTA, min(batch, (blockDim - 1) / n + 2);
                 // symmetric: points per CTA
    int tpp;     // symmetric: threads per point
    int acc;     // symmetric HVP: 0 = stage the chunk matrix, 1 = FP64 row accumulators
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

// T: the arithmetic type; IO: the element type of x, v and the output (IO =
// T except for the one-variable kernels of an FP32 handle, which compute in
// FP64 with float inputs and outputs).
template <typename T, typename IO, int C, bool HVP>
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
    const IO *xg = static_cast<const IO *>(a.x) + p0 * n;
    const IO *vg = static_cast<const IO *>(a.v) + p0 * n;
    for (int t = threadIdx.x; t < staged; t += blockDim.x) {
        xs[t] = (T)xg[t];
        if (HVP) vs[t] = (T)vg[t];
    }
    __syncthreads();
    const long long item = first + threadIdx.x;
    if (item >= items) return;
    const long long p = item / n;
    const int i = (int)(item - p * n);
    const T *xp = xs + (p - p0) * n;
    const T *vp = vs + (p - p0) * n;
    const SeedK<T> z = seed_constants<T>();
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
            IO *H = static_cast<IO *>(a.out) + (p * n + i) * (long long)n + cstart;
#pragma unroll
            for (int l = 0; l < C; ++l)
                if (cstart + l < n) H[l] = (IO)r.a.h[l];
        }
    }
    if (HVP) static_cast<IO *>(a.out)[p * n + i] = (IO)dot.value();
}

template <typename T, int C, bool HVP>
__device__ __forceinline__ void user_sym(const UserArgs &a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, ppb = a.maxpts, tpp = a.tpp;
    // accumulators first (8-byte aligned), then x, v and the staged chunks
    // (accumulator form: the per-iteration stage, SymStage, in their place)
    double *accs = reinterpret_cast<double *>(smem_raw);
    const bool acc_form = HVP && a.acc;
    T *xs = reinterpret_cast<T *>(smem_raw + (acc_form ? (size_t)ppb * n * sizeof(double) : 0));
    T *vs = xs + (size_t)ppb * n;
    T *hs = vs + (HVP ? (size_t)ppb * n : 0);
    const long long p0 = (long long)blockIdx.x * ppb;
    const int npts = (int)(a.batch - p0 < ppb ? a.batch - p0 : ppb);
    const T *xg = static_cast<const T *>(a.x) + p0 * n;
    const T *vg = static_cast<const T *>(a.v) + p0 * n;
    for (int e = threadIdx.x; e < npts * n; e += blockDim.x) {
        xs[e] = xg[e];
        if (HVP) vs[e] = vg[e];
        if (acc_form) accs[e] = 0.0;
    }
    __syncthreads();
    const int q = threadIdx.x / tpp, t = threadIdx.x - q * tpp;
    double *acc = accs + (size_t)q * n;
    const bool active = q < npts;
    const long long p = p0 + q;
    const T *xp = xs + (size_t)q * n;
    T *Hs = hs + (size_t)q * sym_hs_elems(n, C);
    const SeedK<T> z = seed_constants<T>();
    const int nch = (n + C - 1) / C;
    const int items = C * nch * (nch + 1) / 2;
    if (HVP && acc_form) {
        // Alg. 8's two updates (r_i += sum_l H_il v_l; off the diagonal chunk
        // also r_l += H_il v_i) in FP64, reproducibly: each iteration stages
        // every thread's chunk and row dot (SymStage), and each thread adds
        // the contributions to its own rows in thread order.  Every thread
        // runs the same number of iterations (the barriers).
        const size_t soff = ((size_t)(reinterpret_cast<unsigned char *>(hs) - smem_raw) + 15) / 16 * 16;
        const SymStage<T, C> stage(smem_raw + soff, (int)blockDim.x);
        const T *vp = vs + (size_t)q * n;
        const int iters = (items + tpp - 1) / tpp;
        for (int it = 0; it < iters; ++it) {
            const int k = t + it * tpp;
            int i = -1, cn = 0;
            T h[C];
            double own = 0.0;
            if (active && k < items) {
                sym_item(k, C, nch, i, cn);
                if (i >= n) i = -1;
            }
            if (i >= 0) {
                const int cstart = cn * C;
                const Vars<T, C> x{xp, i, cstart, z};
                const Num<T, C> r = ::CHESSFAD_USER_FN<Num<T, C>, Vars<T, C>>(x, n, a.params);
#pragma unroll
                for (int l = 0; l < C; ++l) {
                    h[l] = r.a.h[l];
                    if (cstart + l < n) own = fma((double)h[l], (double)vp[cstart + l], own);
                }
            } else {
#pragma unroll
                for (int l = 0; l < C; ++l) h[l] = T(0);
            }
            stage.put(threadIdx.x, h, own, i, cn);
            __syncthreads();
            if (active) {
                const int t0 = q * tpp;
                for (int srow = t; srow < n; srow += tpp) {
                    const int scn = srow / C, sl = srow - scn * C;
                    double sum = acc[srow];
                    for (int u = 0; u < tpp; ++u) {
                        const int ui = stage.row(t0 + u);
                        if (ui < 0) continue;
                        if (ui == srow) sum += stage.own(t0 + u);
                        const int ucn = stage.chunk(t0 + u);
                        if (ucn == scn && ucn > ui / C) sum += (double)stage.h(t0 + u, sl) * (double)vp[ui];
                    }
                    acc[srow] = sum;
                }
            }
            __syncthreads();
        }
    }
    for (int k = (active && !(HVP && acc_form)) ? t : items; k < items; k += tpp) {
        int i = 0, cn = 0;
        sym_item(k, C, nch, i, cn);
        if (i >= n) continue;
        const int cstart = cn * C;
        const Vars<T, C> x{xp, i, cstart, z};
        const Num<T, C> r = ::CHESSFAD_USER_FN<Num<T, C>, Vars<T, C>>(x, n, a.params);
        if (HVP) {
            T *hrow = Hs + sym_hs_row(i, n, C) - (i / C) * C;
#pragma unroll
            for (int l = 0; l < C; ++l)
                if (cstart + l < n) hrow[cstart + l] = r.a.h[l];
        } else {
            T *H = static_cast<T *>(a.out) + (size_t)p * n * n;
            const bool mirror = cn > i / C;
#pragma unroll
            for (int l = 0; l < C; ++l) {
                const int j = cstart + l;
                if (j < n) {
                    H[(size_t)i * n + j] = r.a.h[l];
                    if (mirror) H[(size_t)j * n + i] = r.a.h[l];
                }
            }
        }
    }
    if (HVP) {
        // r_s = sum_j H_sj v_j: entries right of row s's diagonal chunk from
        // row s, entries left of it from column s (H_sj = H_js).
        __syncthreads();
        if (active && acc_form) {
            T *O = static_cast<T *>(a.out) + p * n;
            for (int srow = t; srow < n; srow += tpp) O[srow] = (T)acc[srow];
        } else if (active) {
            const T *vp = vs + (size_t)q * n;
            T *O = static_cast<T *>(a.out) + p * n;
            for (int srow = t; srow < n; srow += tpp) {
                const int dstart = (srow / C) * C;
                const T *own = Hs + sym_hs_row(srow, n, C) - dstart;
                RowDot<T> dot;
                for (int j = 0; j < dstart; ++j) dot.add(Hs[sym_hs_row(j, n, C) + srow - (j / C) * C], vp[j]);
                for (int j = dstart; j < n; ++j) dot.add(own[j], vp[j]);
                O[srow] = dot.value();
            }
        }
    }
}

}  // namespace user
}  // namespace chessfad

extern "C" __global__ void __launch_bounds__(256) chessfad_user_sym_hvp(chessfad::user::UserArgs a)
{
    chessfad::user::user_sym<CHESSFAD_USER_T, CHESSFAD_USER_C, true>(a);
}

extern "C" __global__ void __launch_bounds__(256) chessfad_user_sym_hessian(chessfad::user::UserArgs a)
{
    chessfad::user::user_sym<CHESSFAD_USER_T, CHESSFAD_USER_C, false>(a);
}

extern "C" __global__ void __launch_bounds__(256) chessfad_user_hvp(chessfad::user::UserArgs a)
{
    chessfad::user::user_sweep<CHESSFAD_USER_T, CHESSFAD_USER_T, CHESSFAD_USER_C, true>(a);
}

extern "C" __global__ void __launch_bounds__(256) chessfad_user_hessian(chessfad::user::UserArgs a)
{
    chessfad::user::user_sweep<CHESSFAD_USER_T, CHESSFAD_USER_T, CHESSFAD_USER_C, false>(a);
}

#if CHESSFAD_USER_F32
// One variable in an FP32 handle: the Hessian is a single entry, a sum of
// terms that can cancel far below their size, so no FP32 evaluation bounds
// its relative error; it is computed in FP64 with float x, v and output.
extern "C" __global__ void __launch_bounds__(256) chessfad_user_hvp_n1(chessfad::user::UserArgs a)
{
    chessfad::user::user_sweep<double, float, 1, true>(a);
}

extern "C" __global__ void __launch_bounds__(256) chessfad_user_hessian_n1(chessfad::user::UserArgs a)
{
    chessfad::user::user_sweep<double, float, 1, false>(a);
}
#endif
