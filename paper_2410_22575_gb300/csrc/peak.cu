// peak.cu -- CUDA-core FMA peak microbenchmark (the measured counterpart of
// the unit-count roofline of the ALU-bound sweep kernels).  Every thread runs
// independent dependent FMA chains over all SMs, either through the
// multiplicand (a = fma(a, m, b)) or through the addend (acc = fma(s, v,
// acc)); one FMA counts as two flops.  The
// result is folded into a never-taken store so the chains cannot be removed.
// Several (chains per thread, CTAs per SM) shapes, with shared or per-chain
// operands, are timed and the best is reported, so the number is the pipe's
// throughput rather than one shape's latency, occupancy or operand limit.
// Thread 0 of CTA 0 reads the SM cycle counter and the global nanosecond
// timer around its loop, which gives the SM clock the run actually saw.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/chessfad.h"

namespace chessfad {

template <typename T>
__device__ T g_peak_sink;

__device__ unsigned long long g_peak_clk[2];

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T, int NCH>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T seed)
{
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        t0 = global_ns();
        c0 = clock64();
    }
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
    if (timer) {
        const unsigned long long c1 = clock64();
        const unsigned long long t1 = global_ns();
        g_peak_clk[0] = c1 - c0;
        g_peak_clk[1] = t1 - t0;
    }
}

// The same with a multiplier and an addend per chain (held in registers,
// not literals), so no two chains read the same operand registers.
template <typename T, int NCH>
__global__ void __launch_bounds__(256) fma_peak_kernel_ops(int iters, T seed)
{
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        t0 = global_ns();
        c0 = clock64();
    }
    T a[NCH], m[NCH], b[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        a[c] = seed + T(c) * T(1e-3) + T(threadIdx.x) * T(1e-7);
        m[c] = T(0.9999999) - T(c) * T(1e-9) - T(threadIdx.x & 7) * T(1e-10);
        b[c] = T(1e-7) + T(c) * T(1e-9);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) a[c] = fma(a[c], m[c], b[c]);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += a[c];
    if (s == T(-12345.0)) g_peak_sink<T> = s;
    if (timer) {
        const unsigned long long c1 = clock64();
        const unsigned long long t1 = global_ns();
        g_peak_clk[0] = c1 - c0;
        g_peak_clk[1] = t1 - t0;
    }
}

// Accumulation chains: acc[l] = fma(s, v[l], acc[l]) for l < L with one
// scalar s per step (the shape of a scalar-times-hDual accumulation), the
// dependency through the addend.  kLiteral: the v[l] are literals, so the
// compiler takes them as constant operands (FP64: constant bank; FP32:
// immediates) instead of general registers.  On GB300 the FP64 pipe sustains
// the register form at 99 % of its nominal rate and the literal form, like
// the chains above with their literal operands, at about 84 %; FFMA runs at
// the same rate either way.
template <typename T, int L, bool kLiteral = false>
__global__ void __launch_bounds__(256) fma_peak_kernel_axpy(int iters, T seed)
{
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        t0 = global_ns();
        c0 = clock64();
    }
    T acc[L], v[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        acc[l] = T(0);
        v[l] = kLiteral ? T(1) + T(l) * T(1e-3) : seed + T(l) * T(1e-3) + T(threadIdx.x) * T(1e-7);
    }
    T s = T(1e-3) * T(threadIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            s = fma(s, T(0.999999), T(1e-9));
#pragma unroll
            for (int l = 0; l < L; ++l) acc[l] = fma(s, v[l], acc[l]);
        }
    }
    T r = T(0);
#pragma unroll
    for (int l = 0; l < L; ++l) r += acc[l];
    if (r == T(-12345.0)) g_peak_sink<T> = r;
    if (timer) {
        const unsigned long long c1 = clock64();
        const unsigned long long t1 = global_ns();
        g_peak_clk[0] = c1 - c0;
        g_peak_clk[1] = t1 - t0;
    }
}

struct PeakResult {
    double flops = 0.0;
    double sm_mhz = 0.0;
};

enum { kChains = 0, kChainsOps = 1, kAxpy = 2, kAxpyLiteral = 3 };

// NCH: chains per thread (kAxpy: L + 1 FMAs per step, L accumulators)
template <typename T, int NCH, int KIND = kChains>
static int measure(int iters, int blocks_per_sm, PeakResult *best)
{
    auto kern = KIND == kAxpy          ? fma_peak_kernel_axpy<T, NCH>
                : KIND == kAxpyLiteral ? fma_peak_kernel_axpy<T, NCH, true>
                : KIND == kChainsOps   ? fma_peak_kernel_ops<T, NCH>
                                       : fma_peak_kernel<T, NCH>;
    const int fmas_per_step = (KIND == kAxpy || KIND == kAxpyLiteral) ? NCH + 1 : NCH;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    const int threads = 256, blocks = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CHESSFAD_ERR_CUDA;
    }
    kern<<<blocks, threads>>>(std::max(1, iters / 16), T(1));
    int rc = CHESSFAD_SUCCESS;
    for (int rep = 0; rep < 3 && rc == CHESSFAD_SUCCESS; ++rep) {
        cudaEventRecord(e0);
        kern<<<blocks, threads>>>(iters, T(1));
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = CHESSFAD_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        unsigned long long clk[2] = {0, 0};
        if (cudaMemcpyFromSymbol(clk, g_peak_clk, sizeof(clk)) != cudaSuccess) {
            rc = CHESSFAD_ERR_CUDA;
            break;
        }
        const double fl = 2.0 * fmas_per_step * 16.0 * (double)iters * (double)blocks * threads;
        const double f = fl / (ms * 1e-3);
        if (f > best->flops) {
            best->flops = f;
            best->sm_mhz = clk[1] ? (double)clk[0] / (double)clk[1] * 1e3 : 0.0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

static int peak(int prec, PeakResult *r)
{
    int rc;
    if (prec == CHESSFAD_FP32_COMP) {
        // FP32: 128 lanes per SM; 8 chains at 8 CTAs of 256 per SM saturate.
        if ((rc = measure<float, 8>(40000, 8, r))) return rc;
        if ((rc = measure<float, 16>(20000, 4, r))) return rc;
        if ((rc = measure<float, 8, kChainsOps>(40000, 8, r))) return rc;
        return measure<float, 17, kAxpy>(20000, 8, r);
    }
    if (prec == CHESSFAD_FP64) {
        // FP64: few lanes per SM and a long pipe: more chains per thread, and
        // both full and half occupancy, to reach the pipe's throughput.
        if ((rc = measure<double, 8>(800, 8, r))) return rc;
        if ((rc = measure<double, 16>(400, 8, r))) return rc;
        if ((rc = measure<double, 16>(800, 4, r))) return rc;
        if ((rc = measure<double, 32>(400, 4, r))) return rc;
        if ((rc = measure<double, 8, kChainsOps>(800, 8, r))) return rc;
        if ((rc = measure<double, 16, kChainsOps>(400, 4, r))) return rc;
        if ((rc = measure<double, 17, kAxpy>(400, 8, r))) return rc;
        return measure<double, 9, kAxpy>(800, 8, r);
    }
    return CHESSFAD_ERR_PRECISION;
}

// The accumulation-chain shape with its multipliers in general registers
// and as literals, at the same shape (17 accumulators, 8 CTAs of 256 per SM
// requested).
static int operand_rates(int prec, PeakResult *reg, PeakResult *lit)
{
    if (prec == CHESSFAD_FP32_COMP) {
        const int rc = measure<float, 17, kAxpy>(20000, 8, reg);
        return rc ? rc : measure<float, 17, kAxpyLiteral>(20000, 8, lit);
    }
    if (prec == CHESSFAD_FP64) {
        const int rc = measure<double, 17, kAxpy>(400, 8, reg);
        return rc ? rc : measure<double, 17, kAxpyLiteral>(400, 8, lit);
    }
    return CHESSFAD_ERR_PRECISION;
}

}  // namespace chessfad

extern "C" CHESSFAD_API int chessfad_peak_operand_rates(int prec, double *register_flops, double *literal_flops)
{
    if (!register_flops || !literal_flops) return CHESSFAD_ERR_NULL;
    chessfad::PeakResult reg, lit;
    const int rc = chessfad::operand_rates(prec, &reg, &lit);
    if (rc == CHESSFAD_SUCCESS) {
        *register_flops = reg.flops;
        *literal_flops = lit.flops;
    }
    return rc;
}

extern "C" CHESSFAD_API int chessfad_peak_flops(int prec, double *flops_per_s)
{
    if (!flops_per_s) return CHESSFAD_ERR_NULL;
    chessfad::PeakResult r;
    const int rc = chessfad::peak(prec, &r);
    if (rc == CHESSFAD_SUCCESS) *flops_per_s = r.flops;
    return rc;
}

extern "C" CHESSFAD_API int chessfad_peak_info(int prec, double *flops_per_s, double *sm_mhz)
{
    if (!flops_per_s) return CHESSFAD_ERR_NULL;
    chessfad::PeakResult r;
    const int rc = chessfad::peak(prec, &r);
    if (rc == CHESSFAD_SUCCESS) {
        *flops_per_s = r.flops;
        if (sm_mhz) *sm_mhz = r.sm_mhz;
    }
    return rc;
}
