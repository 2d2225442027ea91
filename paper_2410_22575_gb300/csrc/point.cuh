// point.cuh -- the L0 decomposition (Alg. 9, L0-HESS-VEC): one thread per
// point, sweeping every chunk of every row of its point in order, CHESS-VEC
// (Alg. 7) / CHUNK-HESS (Alg. 5) as written, the row's dot accumulated in the
// thread.  A CTA holds maxpts points (one per thread) and stages their x, v
// and per-point tables in shared memory like the other kernels.  All threads
// of a warp are on the same (row, chunk), so the three-segment seeding loop
// applies; for one point per thread the parallelism is the batch size, so this
// form suits very large batches of small problems.
#pragma once

#include "sweep.cuh"

namespace chessfad {

template <typename T, typename IO, int C, int FN, bool HVP, int MB>
__global__ void __launch_bounds__(256, 1) point_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n;
    const int ppb = a.maxpts;
    const Smem<T> L = smem_layout<T>(FN, HVP, n, ppb, a.mt);
    Job job;
    job.x = a.x;
    job.v = a.v;
    job.out = a.out;
    job.A = a.A;
    job.B = a.B;
    job.npoints = a.batch;
    job.row0 = 0;
    job.n = n;
    job.nch = a.nch;
    job.tpr = 1;
    job.maxpts = ppb;
    job.mt = a.mt;
    job.ld = a.ld;
    ContigPoints pm{a.E, n};

    const long long p0 = (long long)blockIdx.x * ppb;
    const int npts = (int)min((long long)ppb, a.batch - p0);
    point_prologue<T, IO, FN, HVP>(job, pm, smem_raw, L, p0, npts);

    const int q = threadIdx.x;
    const bool active = q < npts;
    const long long p = p0 + (active ? q : 0);
    const PointTables<T> pt(smem_raw, L, active ? q : 0, n);
    using Dot = typename std::conditional<IsComp<T>::value, CSum, T>::type;
    for (int i = 0; i < n; ++i) {
        Dot dot;
        if constexpr (IsComp<T>::value) {
            dot.s = 0.f;
            dot.e = 0.f;
        } else {
            dot = T(0);
        }
        for (int cn = 0; cn < a.nch; ++cn) {
            const int cstart = cn * C;
            const HD<T, C> f = row_chunk<T, C, FN, MB, false>(job, smem_raw, L, pt, i, cstart, active, i == 0 && cn == 0);
            if (!active) continue;
            if constexpr (HVP) {
#pragma unroll
                for (int l = 0; l < C; ++l) {
                    if (cstart + l < n) {
                        if constexpr (IsComp<T>::value) cdot_add(dot, f.h[l], pt.v[cstart + l]);
                        else dot = fma_(f.h[l], pt.v[cstart + l], dot);
                    }
                }
            } else {
                IO *H = reinterpret_cast<IO *>(a.out) + ((size_t)p * n + i) * n + cstart;
#pragma unroll
                for (int l = 0; l < C; ++l)
                    if (cstart + l < n) H[l] = (IO)f.h[l];
            }
        }
        if constexpr (HVP) {
            if (active) {
                IO *O = reinterpret_cast<IO *>(a.out) + (size_t)p * n;
                if constexpr (IsComp<T>::value) O[i] = (IO)csum_value(dot);
                else O[i] = (IO)dot;
            }
        }
    }
}

template <typename T, typename IO, int C, int FN, bool HVP, int MB>
size_t point_smem_bytes(const SweepArgs &a)
{
    return smem_layout<T>(FN, HVP, a.n, a.maxpts, a.mt).total;
}

template <typename T, typename IO, int C, int FN, bool HVP, int MB>
cudaError_t launch_point(SweepArgs a, cudaStream_t stream)
{
    const size_t bytes = point_smem_bytes<T, IO, C, FN, HVP, MB>(a);
    auto kern = point_kernel<T, IO, C, FN, HVP, MB>;
    static std::atomic<int> configured[64];
    cudaError_t e = opt_in_smem(kern, bytes, configured);
    if (e != cudaSuccess) return e;
    const long long blocks = (a.batch + a.maxpts - 1) / a.maxpts;
    kern<<<(unsigned)blocks, a.maxpts, bytes, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace chessfad
