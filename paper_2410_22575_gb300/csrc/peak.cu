// peak.cu -- CUDA-core FMA peak microbenchmark (the roofline denominator of
// the ALU-bound sweep kernels).  Every thread runs NCH independent dependent
// chains a = fma(a, m, b) over all SMs at full occupancy; one FMA counts as
// two flops.  The result is folded into a never-taken store so the chains
// cannot be removed.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/chessfad.h"

namespace chessfad {

template <typename T>
__device__ T g_peak_sink;

template <typename T, int NCH>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T seed)
{
    T a[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) a[c] = seed + T(c) * T(1e-3) + T(threadIdx.x) * T(1e-7);
    const T m = T(0.9999999), b = T(1e-7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) a[c] = fma(a[c], m, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += a[c];
    if (s == T(-12345.0)) g_peak_sink<T> = s;
}

template <typename T, int NCH>
static int measure(int iters, double *flops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CHESSFAD_ERR_CUDA;
    }
    fma_peak_kernel<T, NCH><<<blocks, threads>>>(std::max(1, iters / 16), T(1));
    double best = 0.0;
    int rc = CHESSFAD_SUCCESS;
    for (int rep = 0; rep < 3 && rc == CHESSFAD_SUCCESS; ++rep) {
        cudaEventRecord(e0);
        fma_peak_kernel<T, NCH><<<blocks, threads>>>(iters, T(1));
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = CHESSFAD_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double fl = 2.0 * NCH * 16.0 * (double)iters * (double)blocks * threads;
        best = std::max(best, fl / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CHESSFAD_SUCCESS) *flops = best;
    return rc;
}

}  // namespace chessfad

extern "C" CHESSFAD_API int chessfad_peak_flops(int prec, double *flops_per_s)
{
    if (!flops_per_s) return CHESSFAD_ERR_NULL;
    if (prec == CHESSFAD_FP32_COMP) return chessfad::measure<float, 8>(40000, flops_per_s);
    if (prec == CHESSFAD_FP64) return chessfad::measure<double, 8>(800, flops_per_s);
    return CHESSFAD_ERR_PRECISION;
}
