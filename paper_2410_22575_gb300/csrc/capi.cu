// capi.cu -- the extern "C" boundary of include/chessfad.h: argument checks,
// launch-configuration choice (defaults, autotuned table), dispatch to the
// kernel instantiation units, the autotuner and status strings.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/chessfad.h"
#include "dispatch.h"

namespace chessfad {

static int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Local memory per thread that is not a register spill: the FP64 sin/cos
// argument reduction keeps a 40-byte buffer on the stack for huge arguments.
// Frames above this size are treated as spilling kernels by the autotuner.
static constexpr size_t kMaxFrameNoSpill = 48;

static bool valid_chunk(int c) { return c == 1 || c == 2 || c == 4 || c == 8 || c == 16 || c == 32; }

// Tuned configurations keyed by (fn, n, prec): HVPs and Hessians.
static std::mutex g_mu;
static std::map<std::tuple<int, int, int>, chessfad_config> g_table;
static std::map<std::tuple<int, int, int>, chessfad_config> g_htable;

// Multiprocessors of the current device (queried once per device; 152 on
// GB300 when the query fails, e.g. with no device).
static int device_sms()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int s = cache[dev].load(std::memory_order_relaxed);
    if (s > 0) return s;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) return 152;
    cache[dev].store(s, std::memory_order_relaxed);
    return s;
}

// Threads that fill the GPU several times over: four 256-thread CTAs per
// multiprocessor.
static long long rows_one_lane() { return 4LL * device_sms() * 256; }

static int default_threads_per_point(int n, int csize, long long batch);

// Largest chunk that keeps the plain method's hDual state comfortably in
// registers (its multiplication count (6 + 3/c) n^2 M falls with c, Sec. V).
static int plain_chunk(int fn, int n, int prec)
{
    int cmax = (prec == CHESSFAD_FP64) ? 8 : 16;
    if (fn == CHESSFAD_FLETCHER_POWELL) cmax = (prec == CHESSFAD_FP64) ? 4 : 16;
    return std::min(cmax, next_pow2(n));
}

// The symmetric method's chunk: the Sec. V optimum c = sqrt(n/2), rounded up
// to a power of two, within the plain method's register budget.
static int sym_chunk(int fn, int n, int prec)
{
    return std::min(plain_chunk(fn, n, prec), next_pow2((int)std::ceil(std::sqrt(n / 2.0))));
}

static chessfad_config default_config(int fn, int n, long long batch, int prec)
{
    chessfad_config c{};
    c.csize = plain_chunk(fn, n, prec);
    const int nch = (n + c.csize - 1) / c.csize;
    // Enough rows: one thread per row sweeps all of the row's chunks (the
    // per-point prologue is amortised over the most work).  Few rows: spread
    // a row's chunks over lanes (the paper's L2) to fill the GPU.
    int tpr = 1;
    const long long rows = batch * (long long)n;
    while (tpr < 32 && tpr < nch && rows * tpr < rows_one_lane()) tpr <<= 1;
    c.threads_per_row = tpr;
    c.block_threads = 256;
    c.method = CHESSFAD_METHOD_PLAIN;
    c.threads_per_point = default_threads_per_point(n, sym_chunk(fn, n, prec), batch);
    if (n >= 4) {
        // The symmetric method (about half the evaluations) at the Sec. V
        // optimum c = sqrt(n/2), rounded up to a power of two.
        c.method = CHESSFAD_METHOD_SYMMETRIC;
        c.csize = sym_chunk(fn, n, prec);
        c.block_threads = std::max(128, c.threads_per_point);
    }
    return c;
}

static chessfad_config resolve(int fn, int n, long long batch, int prec, const chessfad_config *cfg, int csize_hint,
                               bool hvp)
{
    chessfad_config c{};
    if (cfg) c = *cfg;
    if (c.csize == 0 && csize_hint != 0) c.csize = csize_hint;
    if (c.csize == 0) {
        chessfad_config base;
        bool tuned = false;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            const auto &table = hvp ? g_table : g_htable;
            auto it = table.find(std::make_tuple(fn, n, prec));
            tuned = it != table.end();
            base = tuned ? it->second : default_config(fn, n, batch, prec);
        }
        // Method 0 with csize 0 is "the default method" (the tuned one, else
        // the default configuration's), not necessarily the plain method.
        if (!cfg || cfg->method == 0) c.method = base.method;
        if (c.method == base.method) {
            c.csize = base.csize;
            if (c.threads_per_row == 0) c.threads_per_row = base.threads_per_row;
            if (c.block_threads == 0) c.block_threads = base.block_threads;
            if (c.threads_per_point == 0) c.threads_per_point = base.threads_per_point;
        } else if (c.method == CHESSFAD_METHOD_SYMMETRIC || c.method == CHESSFAD_METHOD_SYMMETRIC_SPARSE) {
            c.csize = sym_chunk(fn, n, prec);
        } else {
            c.csize = plain_chunk(fn, n, prec);
        }
        // the seed-sparse kernels exist for chunk sizes 4, 8 and 16 only, the
        // one-thread-per-point kernels for 1 .. 16
        if (c.method == CHESSFAD_METHOD_SYMMETRIC_SPARSE) c.csize = std::min(16, std::max(4, c.csize));
        if (c.method == CHESSFAD_METHOD_POINT) c.csize = std::min(16, c.csize);
    }
    if (c.threads_per_point == 0) c.threads_per_point = default_threads_per_point(n, c.csize, batch);
    if (c.threads_per_row == 0 || c.block_threads == 0) {
        chessfad_config d = default_config(fn, n, batch, prec);
        const int nch = (n + c.csize - 1) / c.csize;
        if (c.threads_per_row == 0) c.threads_per_row = std::min(d.threads_per_row, std::max(1, next_pow2(nch)));
        if (c.block_threads == 0) {
            const bool sym = c.method == CHESSFAD_METHOD_SYMMETRIC || c.method == CHESSFAD_METHOD_SYMMETRIC_SPARSE;
            c.block_threads = sym ? std::max(128, c.threads_per_point) : d.block_threads;
        }
    }
    return c;
}

static int check_common(int fn, int n, long long batch, int prec, const chessfad_fp_params *params)
{
    if (fn < 0 || fn > 2) return CHESSFAD_ERR_FUNCTION;
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    if (n < 1 || n > CHESSFAD_MAX_N) return CHESSFAD_ERR_SIZE;
    if (batch < 0) return CHESSFAD_ERR_BATCH;
    if (fn == CHESSFAD_FLETCHER_POWELL) {
        if (!params || !params->A || !params->B || !params->E || params->ld < n) return CHESSFAD_ERR_PARAMS;
    }
    return CHESSFAD_SUCCESS;
}

static int check_config(const chessfad_config &c)
{
    if (!valid_chunk(c.csize)) return CHESSFAD_ERR_CHUNK;
    const int t = c.threads_per_row;
    if (t < 1 || t > 32 || (t & (t - 1))) return CHESSFAD_ERR_CONFIG;
    if (c.block_threads < 32 || c.block_threads > 256 || c.block_threads % 32) return CHESSFAD_ERR_CONFIG;
    if (c.method != CHESSFAD_METHOD_PLAIN && c.method != CHESSFAD_METHOD_SYMMETRIC &&
        c.method != CHESSFAD_METHOD_SYMMETRIC_SPARSE && c.method != CHESSFAD_METHOD_POINT)
        return CHESSFAD_ERR_CONFIG;
    if (c.method == CHESSFAD_METHOD_SYMMETRIC_SPARSE && c.csize != 4 && c.csize != 8 && c.csize != 16)
        return CHESSFAD_ERR_CHUNK;
    if (c.method == CHESSFAD_METHOD_POINT && c.csize > 16) return CHESSFAD_ERR_CHUNK;
    const int p = c.threads_per_point;
    if (p < 8 || p > 256 || (p & (p - 1))) return CHESSFAD_ERR_CONFIG;
    return CHESSFAD_SUCCESS;
}

// Symmetric method: threads per point that fill the GPU several times over,
// but no more than the point has (row, chunk) items (C nch (nch+1) / 2),
// rounded up to a power of two, at least 8: a small point leaves no lanes
// idle for want of items.
static int default_threads_per_point(int n, int csize, long long batch)
{
    const long long nch = (n + csize - 1) / csize;
    const long long items = (long long)csize * nch * (nch + 1) / 2;
    int cap = 8;
    while (cap < 256 && cap < items) cap <<= 1;
    int p = std::min(32, cap);
    while (p < cap && batch * (long long)p < rows_one_lane()) p <<= 1;
    return p;
}

// Rows of A and B staged per shared-memory tile by the Fletcher-Powell sweep:
// all n rows when they fit in ~64 KiB, else the largest multiple of 8.
static int fp_tile_rows(int n, int prec)
{
    const size_t esz = (prec == CHESSFAD_FP64) ? 8 : 4;
    const size_t budget = 64 * 1024;
    int mt = (int)(budget / (2 * (size_t)n * esz));
    mt = std::max(8, mt / 8 * 8);
    return std::min(mt, (n + 7) / 8 * 8);
}

// A launch grid holds at most 2^31 - 1 blocks.  A batch that needs more is
// rejected before anything is launched (the block count would otherwise be
// truncated to 32 bits and part of the batch silently skipped).
constexpr long long kMaxGridBlocks = 0x7fffffffLL;

// batch points at pts_per_block points per block fit in one grid.
static bool grid_fits_points(long long batch, int pts_per_block)
{
    return batch <= kMaxGridBlocks * (long long)pts_per_block;
}

// batch points at threads_per_point threads each, block_threads per block.
static bool grid_fits_threads(long long batch, int threads_per_point, int block_threads)
{
    return batch <= kMaxGridBlocks * (long long)block_threads / threads_per_point;
}

static int launch(int fn, int n, long long batch, const chessfad_config &c, const void *x, const void *v,
                  void *out, const chessfad_fp_params *params, int prec, bool hvp, cudaStream_t stream)
{
    SweepArgs a{};
    a.x = x;
    a.v = v;
    a.out = out;
    if (fn == CHESSFAD_FLETCHER_POWELL) {
        a.A = params->A;
        a.B = params->B;
        a.E = params->E;
        a.ld = params->ld;
    }
    a.batch = batch;
    a.n = n;
    a.nch = (n + c.csize - 1) / c.csize;
    a.tpr = c.threads_per_row;
    a.tpp = n * c.threads_per_row;
    a.maxpts = (int)std::min<long long>(batch, (c.block_threads - 1) / a.tpp + 2);
    a.mt = (fn == CHESSFAD_FLETCHER_POWELL) ? fp_tile_rows(n, prec) : 8;
    if (fn == CHESSFAD_FLETCHER_POWELL && a.mt % fp_mb(c.csize) != 0) return CHESSFAD_ERR_CONFIG;
    cudaError_t e = cudaErrorInvalidValue;
    const bool f64 = (prec == CHESSFAD_FP64);
    const SliceOps &ops = slice(fn, f64);
    const bool sym = c.method == CHESSFAD_METHOD_SYMMETRIC || c.method == CHESSFAD_METHOD_SYMMETRIC_SPARSE;
    if (sym && !(!f64 && n == 1)) {
        const bool sparse = c.method == CHESSFAD_METHOD_SYMMETRIC_SPARSE;
        // Symmetric method: a.maxpts = points per block, a.tpp = threads per
        // point; as many points per CTA as shared memory allows (<= 200 KiB).
        a.tpp = c.threads_per_point;
        auto bytes = [&](int ppb) {
            a.maxpts = ppb;
            return ops.sym_smem(c.csize, hvp, a);
        };
        int ppb = (int)std::min<long long>(batch, std::max(1, c.block_threads / c.threads_per_point));
        const size_t kBudget = 200 * 1024;
        a.sym_acc = 0;
        const int ppb0 = ppb;
        while (ppb > 1 && bytes(ppb) > kBudget) --ppb;
        if (hvp && bytes(ppb) > kBudget) {
            // the chunk matrix of one point does not fit: FP64 row accumulators
            a.sym_acc = 1;
            ppb = ppb0;
            while (ppb > 1 && bytes(ppb) > kBudget) --ppb;
        }
        if (bytes(ppb) > kBudget) return CHESSFAD_ERR_SIZE;
        if (!grid_fits_points(batch, ppb)) return CHESSFAD_ERR_BATCH;
        a.maxpts = ppb;
        e = sparse ? ops.sym_sparse(c.csize, hvp, a, stream) : ops.sym(c.csize, hvp, a, stream);
        return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
    }
    if (c.method == CHESSFAD_METHOD_POINT && !(!f64 && n == 1)) {
        // L0 (Alg. 9): one thread per point; as many points per CTA as the CTA
        // size allows within 200 KiB of shared memory, at least 32.
        a.tpr = 1;
        a.tpp = 1;
        auto bytes = [&](int ppb) {
            a.maxpts = ppb;
            return ops.point_smem(c.csize, hvp, a);
        };
        int ppb = c.block_threads;
        while (ppb > 32 && bytes(ppb) > 200 * 1024) ppb -= 32;
        if (bytes(ppb) > 200 * 1024) return CHESSFAD_ERR_SIZE;
        if (!grid_fits_points(batch, ppb)) return CHESSFAD_ERR_BATCH;
        a.maxpts = ppb;
        e = ops.point(c.csize, hvp, a, stream);
        return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
    }
    if (!grid_fits_threads(batch, a.tpp, c.block_threads)) return CHESSFAD_ERR_BATCH;
    if (!f64 && n == 1) {
        // One variable: compute in FP64 (float I/O), see dispatch.h.
        a.nch = 1;
        e = ops.sweep_f64io32(hvp, a, c.block_threads, stream);
        return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
    }
    e = ops.sweep(c.csize, hvp, a, c.block_threads, stream);
    return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}

static cudaError_t kernel_attr(int fn, int prec, int csize, bool hvp, cudaFuncAttributes *fa)
{
    if (fn < 0 || fn > 2) return cudaErrorInvalidValue;
    return slice(fn, prec == CHESSFAD_FP64).attr(csize, hvp, fa);
}

static int run(int fn, int n, long long batch, const chessfad_config *cfg, int csize_hint, const void *x,
               const void *v, void *out, const chessfad_fp_params *params, int prec, bool hvp,
               cudaStream_t stream)
{
    int st = check_common(fn, n, batch, prec, params);
    if (st) return st;
    if (csize_hint != 0 && !valid_chunk(csize_hint)) return CHESSFAD_ERR_CHUNK;
    if (cfg && cfg->csize != 0 && !valid_chunk(cfg->csize)) return CHESSFAD_ERR_CHUNK;
    const chessfad_config c = resolve(fn, n, batch, prec, cfg, csize_hint, hvp);
    st = check_config(c);
    if (st) return st;
    if (batch == 0) return CHESSFAD_SUCCESS;
    if (!x || !out || (hvp && !v)) return CHESSFAD_ERR_NULL;
    return launch(fn, n, batch, c, x, v, out, params, prec, hvp, stream);
}

// The autotuner of chessfad_autotune_hvp / chessfad_autotune_hessian: times
// every candidate on a prefix of the caller's batch and stores the fastest in
// the HVP or the Hessian table.
static int autotune(int fn, int n, long long batch, const void *x, const void *v, void *out,
                    const chessfad_fp_params *params, int prec, cudaStream_t stream, bool hvp, chessfad_config *best)
{
    int st = check_common(fn, n, batch, prec, params);
    if (st) return st;
    if (batch == 0) return CHESSFAD_ERR_BATCH;
    if (!x || !out || (hvp && !v)) return CHESSFAD_ERR_NULL;

    // Candidate chunk sizes: powers of two up to next_pow2(n), ordered by the
    // Sec. V model of the plain method, whose multiplication count
    // (6 + 3/c) n^2 M falls with c, so large chunks are tried first.
    std::vector<int> chunks;
    for (int c = std::min(32, next_pow2(n)); c >= 1; c >>= 1) chunks.push_back(c);

    // Time on a prefix of the batch big enough to fill the GPU several times.
    const long long want_threads = 2 * rows_one_lane();
    long long sub = std::min<long long>(batch, std::max<long long>(1, want_threads / n));

    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CHESSFAD_ERR_CUDA;
    }
    chessfad_config win{};
    float win_ms = INFINITY;
    int rc = CHESSFAD_SUCCESS;
    // Candidates: plain method over (threads/row, CTA size), symmetric method
    // (Alg. 6 / Alg. 8) over threads/point; kernels that spill are skipped.
    std::vector<chessfad_config> cands;
    for (int c : chunks) {
        cudaFuncAttributes fa{};
        if (kernel_attr(fn, prec, c, hvp, &fa) != cudaSuccess || fa.localSizeBytes > kMaxFrameNoSpill) continue;
        const int nch = (n + c - 1) / c;
        const int tmax = std::min(32, next_pow2(nch));
        for (int t = tmax; t >= std::max(1, tmax / 8); t >>= 1)
            for (int bt : {256, 128}) cands.push_back(chessfad_config{c, t, bt, CHESSFAD_METHOD_PLAIN, 32});
        if (std::max(1, tmax / 8) > 1) cands.push_back(chessfad_config{c, 1, 256, CHESSFAD_METHOD_PLAIN, 32});
        // threads per point: 8 for small n (few items per point), 256 for
        // large n; never more than twice the point's items
        const long long items = (long long)c * nch * (nch + 1) / 2;
        for (int p : {8, 16, 32, 64, 128, 256})
            for (int bt : {128, 256})
                if (bt >= p && (p < 256 || n >= 128) && (p > 8 || n <= 32) && (p <= 8 || p < 2 * items))
                    cands.push_back(chessfad_config{c, 1, bt, CHESSFAD_METHOD_SYMMETRIC, p});
    }
    for (const chessfad_config &cfg : cands) {
        if (launch(fn, n, sub, cfg, x, v, out, params, prec, hvp, stream) != CHESSFAD_SUCCESS) {
            cudaGetLastError();
            continue;  // e.g. a symmetric HVP whose staged chunks exceed shared memory
        }
        cudaEventRecord(e0, stream);
        const int reps = 3;
        for (int k = 0; k < reps; ++k) launch(fn, n, sub, cfg, x, v, out, params, prec, hvp, stream);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = CHESSFAD_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < win_ms) {
            win_ms = ms;
            win = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (!std::isfinite(win_ms)) return CHESSFAD_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        (hvp ? g_table : g_htable)[std::make_tuple(fn, n, prec)] = win;
    }
    if (best) *best = win;
    return CHESSFAD_SUCCESS;
}

}  // namespace chessfad

using namespace chessfad;

extern "C" {

int chessfad_hvp(int fn, int n, long long batch, int csize, const void *x, const void *v, void *out,
                 const chessfad_fp_params *params, int prec, chessfad_stream_t stream)
{
    return run(fn, n, batch, nullptr, csize, x, v, out, params, prec, true, (cudaStream_t)stream);
}

int chessfad_hessian(int fn, int n, long long batch, int csize, const void *x, void *H,
                     const chessfad_fp_params *params, int prec, chessfad_stream_t stream)
{
    return run(fn, n, batch, nullptr, csize, x, nullptr, H, params, prec, false, (cudaStream_t)stream);
}

int chessfad_hvp_config(int fn, int n, long long batch, const chessfad_config *cfg, const void *x, const void *v,
                        void *out, const chessfad_fp_params *params, int prec, chessfad_stream_t stream)
{
    return run(fn, n, batch, cfg, 0, x, v, out, params, prec, true, (cudaStream_t)stream);
}

int chessfad_hessian_config(int fn, int n, long long batch, const chessfad_config *cfg, const void *x, void *H,
                            const chessfad_fp_params *params, int prec, chessfad_stream_t stream)
{
    return run(fn, n, batch, cfg, 0, x, nullptr, H, params, prec, false, (cudaStream_t)stream);
}

int chessfad_default_config(int fn, int n, long long batch, int prec, chessfad_config *cfg)
{
    if (!cfg) return CHESSFAD_ERR_NULL;
    if (fn < 0 || fn > 2) return CHESSFAD_ERR_FUNCTION;
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    if (n < 1 || n > CHESSFAD_MAX_N) return CHESSFAD_ERR_SIZE;
    if (batch < 0) return CHESSFAD_ERR_BATCH;
    *cfg = resolve(fn, n, batch, prec, nullptr, 0, true);
    return CHESSFAD_SUCCESS;
}

int chessfad_resolve_config(int fn, int n, long long batch, int prec, int hvp, const chessfad_config *cfg,
                            chessfad_config *out)
{
    if (!out) return CHESSFAD_ERR_NULL;
    if (fn < 0 || fn > 2) return CHESSFAD_ERR_FUNCTION;
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    if (n < 1 || n > CHESSFAD_MAX_N) return CHESSFAD_ERR_SIZE;
    if (batch < 0) return CHESSFAD_ERR_BATCH;
    if (cfg && cfg->csize != 0 && !valid_chunk(cfg->csize)) return CHESSFAD_ERR_CHUNK;
    const chessfad_config c = resolve(fn, n, batch, prec, cfg, 0, hvp != 0);
    const int st = check_config(c);
    if (st) return st;
    *out = c;
    return CHESSFAD_SUCCESS;
}

int chessfad_autotune_hvp(int fn, int n, long long batch, const void *x, const void *v, void *out,
                          const chessfad_fp_params *params, int prec, chessfad_stream_t stream,
                          chessfad_config *best)
{
    return autotune(fn, n, batch, x, v, out, params, prec, (cudaStream_t)stream, true, best);
}

int chessfad_autotune_hessian(int fn, int n, long long batch, const void *x, void *H, const chessfad_fp_params *params,
                              int prec, chessfad_stream_t stream, chessfad_config *best)
{
    return autotune(fn, n, batch, x, nullptr, H, params, prec, (cudaStream_t)stream, false, best);
}

int chessfad_kernel_info(int fn, int prec, int csize, int hvp, int *registers, long long *local_bytes)
{
    if (!registers || !local_bytes) return CHESSFAD_ERR_NULL;
    if (fn < 0 || fn > 2) return CHESSFAD_ERR_FUNCTION;
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    if (!valid_chunk(csize)) return CHESSFAD_ERR_CHUNK;
    cudaFuncAttributes fa{};
    if (kernel_attr(fn, prec, csize, hvp != 0, &fa) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    *registers = fa.numRegs;
    *local_bytes = (long long)fa.localSizeBytes;
    return CHESSFAD_SUCCESS;
}

const char *chessfad_strerror(int status)
{
    switch (status) {
    case CHESSFAD_SUCCESS: return "success";
    case CHESSFAD_ERR_FUNCTION: return "unknown function id";
    case CHESSFAD_ERR_SIZE: return "n out of range [1, CHESSFAD_MAX_N]";
    case CHESSFAD_ERR_BATCH: return "invalid batch size";
    case CHESSFAD_ERR_CHUNK: return "chunk size not in {1,2,4,8,16,32} (or 0)";
    case CHESSFAD_ERR_NULL: return "required pointer is NULL";
    case CHESSFAD_ERR_PARAMS: return "Fletcher-Powell parameters missing or ld < n";
    case CHESSFAD_ERR_PRECISION: return "unknown precision";
    case CHESSFAD_ERR_WORKSPACE: return "workspace missing or too small";
    case CHESSFAD_ERR_CONFIG: return "launch configuration out of range";
    case CHESSFAD_ERR_CUDA: return "CUDA runtime or launch error";
    case CHESSFAD_ERR_PLAN: return "ragged plan invalid or built for another precision";
    case CHESSFAD_ERR_JIT: return "user function: NVRTC unavailable or compilation failed";
    }
    return "unknown status";
}

int chessfad_version(void) { return 100; }

}  // extern "C"
