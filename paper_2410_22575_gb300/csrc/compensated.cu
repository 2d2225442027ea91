// compensated.cu -- the error-free transformations and compensated sums that
// the compensated-FP32 kernels are built from (hdual.cuh: two_sum, two_prod,
// csum_add, cdot_add, csum_merge, csum_value), run over caller arrays so that
// their defining properties can be checked from outside the sweep kernels:
//   TwoSum (Knuth)        s + e == a + b exactly
//   TwoProd (by FMA)      p + q == a * b exactly (barring underflow)
//   Sum2 / Dot2 (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26(6), 2005)
//                         as accurate as the recursive sum / dot product in
//                         twice the working precision, then rounded.
// The row reductions use the order of the compensated-FP32 row . v
// reduction of the sweep kernels: lane r of a row takes the blocks r,
// r + lanes, r + 2 lanes, ... of `chunk` consecutive elements, in ascending
// order, and the lanes of the row are merged by xor shuffles at distances
// lanes/2, ..., 1 (aligned groups of `lanes` lanes inside one warp).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "../../include/chessfad.h"
#include "hdual.cuh"

namespace chessfad {

__global__ void __launch_bounds__(256) eft_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                  long long count, float *s, float *e, float *p, float *q)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        const float x = a[k], y = b[k];
        float hi, lo;
        two_sum(x, y, hi, lo);
        if (s) s[k] = hi;
        if (e) e[k] = lo;
        two_prod(x, y, hi, lo);
        if (p) p[k] = hi;
        if (q) q[k] = lo;
    }
}

// One row per aligned group of `lanes` lanes; a warp serves 32 / lanes rows
// per step of its loop, and every lane of the warp runs the same number of
// steps (rows past the end accumulate nothing), so the shuffles always see
// the whole warp.  b == nullptr: Sum2 of a's rows; else Dot2 of a's and b's.
__global__ void __launch_bounds__(256) rows_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                   long long rows, int len, int lanes, int chunk,
                                                   float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int per_warp = 32 / lanes;
    const long long groups = (rows + per_warp - 1) / per_warp;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int r = lane % lanes;  // the lane's index inside its row's group
    for (long long g = warp; g < groups; g += nwarps) {
        const long long row = g * per_warp + lane / lanes;
        CSum acc{0.0f, 0.0f};
        if (row < rows) {
            const float *ar = a + row * len;
            const float *br = b ? b + row * len : nullptr;
            for (long long blk = r; blk * chunk < len; blk += lanes) {
                const long long end = (blk + 1) * chunk;
                const int j1 = end < len ? (int)end : len;
                for (int j = (int)(blk * chunk); j < j1; ++j) {
                    if (br) cdot_add(acc, ar[j], br[j]);
                    else csum_add(acc, ar[j]);
                }
            }
        }
        for (int off = lanes >> 1; off > 0; off >>= 1) {
            CSum o;
            o.s = __shfl_xor_sync(0xffffffffu, acc.s, off);
            o.e = __shfl_xor_sync(0xffffffffu, acc.e, off);
            acc = csum_merge(acc, o);
        }
        if (row < rows && r == 0) out[row] = csum_value(acc);
    }
}

static int grid_for(long long threads)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 1;
    const long long blocks = (threads + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(blocks, (long long)sms * 8));
}

}  // namespace chessfad

extern "C" CHESSFAD_API int chessfad_eft(const float *a, const float *b, long long count, float *s, float *e,
                                         float *p, float *q, chessfad_stream_t stream)
{
    if (count < 0) return CHESSFAD_ERR_BATCH;
    if (count == 0) return CHESSFAD_SUCCESS;
    if (!a || !b) return CHESSFAD_ERR_NULL;
    chessfad::eft_kernel<<<chessfad::grid_for(count), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        a, b, count, s, e, p, q);
    return cudaGetLastError() == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}

extern "C" CHESSFAD_API int chessfad_compensated_rows(const float *a, const float *b, long long rows, int len,
                                                      int lanes, int chunk, float *out, chessfad_stream_t stream)
{
    if (rows < 0 || len < 0) return CHESSFAD_ERR_BATCH;
    if (lanes < 1 || lanes > 32 || (lanes & (lanes - 1)) || chunk < 1) return CHESSFAD_ERR_CONFIG;
    if (len > 0 && rows > LLONG_MAX / len) return CHESSFAD_ERR_BATCH;
    if (rows == 0) return CHESSFAD_SUCCESS;
    if (!out || (len > 0 && !a)) return CHESSFAD_ERR_NULL;
    const long long groups = (rows + 32 / lanes - 1) / (32 / lanes);
    chessfad::rows_kernel<<<chessfad::grid_for(groups * 32), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        a, b, rows, len, lanes, chunk, out);
    return cudaGetLastError() == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}
