// ragged.cu -- Hessian-vector products over an uneven batch: requests of
// different test functions and different n in one persistent launch.
//
// Host side (a plan, built once per request table): requests are grouped by
// (function, n); the point-major row space of each group is cut into tiles of
// one CTA each (blockDim/tpr rows, the same (point, row, lane) decomposition as
// the batched kernel, Sec. VI); tiles are sorted by estimated cost, largest
// first, so the long Fletcher-Powell tiles at large n start early and the short
// ones fill the tail.  The chunk size and the lanes per row are chosen per
// (function, n range): from the table chessfad_ragged_autotune fills, else by
// default.  The tables (tiles, request list, offsets) live in a
// caller-provided device workspace together with a queue counter.
//
// Device side: a persistent kernel, a few CTAs per SM, whose CTAs take tile
// after tile from the counter with atomicAdd and run the tile's sweeps.  No
// CTA ever waits for another one.  A run is {memset of the counters, kernel},
// both stream-ordered, so it can be captured into a CUDA graph and replayed.
//
// Fletcher-Powell requests with n >= kSymMinN (where nearly all of the cost
// is) use the symmetric method, SC-HESS-VEC (Alg. 8): row i evaluates only
// the chunks from its diagonal chunk on, about half the evaluations.  A tile
// holds rows of one request and deals their (row, chunk) items to its
// threads round-robin.  Each off-diagonal-chunk entry H_ij serves r_i in the
// row's own sum and r_j, a row usually in another tile.  A tile sums what its
// items contribute to every column in shared memory, in a fixed order
// (iterations, then threads), writes
// that partial row vector to its own slot in the workspace, and the tile that
// completes a request (a per-request tile counter) adds the request's slots
// in tile order: the result does not depend on the order in which tiles run,
// so FP64 results are bitwise reproducible.  Products of two FP32 values are
// exact in FP64, so the compensated-FP32 path accumulates them in FP64 too.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/chessfad.h"
#include "dispatch.h"

namespace chessfad {

struct RTile {
    long long row0;     // first row of the tile in its group's row space
    long long npoints;  // points (requests) in the group
    int list0;          // group's first entry in the request list
    int fn, n, C, nch, tpr, maxpts, mt;  // tpr: lanes per row (symmetric tiles: kRaggedBlock / rows)
    int sym;            // symmetric tile: rows row0 .. row0+nrows-1 of one point
    int nrows;
    int srows;          // symmetric: rows per tile of the request (the last tile may have fewer)
    int ntiles_req;     // symmetric: tiles of the request
};

constexpr int kRaggedBlock = 256;
constexpr int kSymMinN = 128;  // Fletcher-Powell requests this large use the symmetric method

struct RaggedArgs {
    const void *x;
    const void *v;
    void *out;
    const double *A;
    const double *B;
    const double *Epack;
    const RTile *tiles;
    const int *list;
    const long long *offs;
    const long long *eoffs;
    const long long *soffs;  // per request: first slot element (symmetric requests)
    int *counter;
    int *done;               // per request: tiles completed (symmetric requests)
    double *slots;           // per symmetric tile: its partial row vector (FP64)
    unsigned long long *busy;  // autotuning: SM cycles spent in tiles, summed (null otherwise)
    int ntiles;
    int ld;
};

// Fletcher-Powell residual rows held in registers per pass over the variables
// (each seeded sin/cos hDual serves this many rows): as many as fit the
// register file without spilling at one 256-thread CTA per SM.
__host__ __device__ constexpr int ragged_mb(int C, bool f64) { return f64 ? (C <= 8 ? 4 : 2) : (C <= 8 ? 8 : 4); }

// First column of a symmetric tile's slot: the diagonal chunk of its first
// row (no row of the tile contributes left of it), and the slot's length.
__host__ __device__ inline int sym_slot_base(int i0, int C) { return (i0 / C) * C; }

// Shared memory a symmetric tile needs beyond the sweep's layout L: the
// partial row vector (n doubles) and the per-iteration stage of every
// thread's item (SymStage: its chunk, its row dot, its row and chunk).
template <typename T>
__host__ __device__ inline size_t sym_tile_extra(int n, int C)
{
    const size_t stage = align_up((size_t)kRaggedBlock * C * sizeof(T), 16) +
                         (size_t)kRaggedBlock * (sizeof(double) + 2 * sizeof(int));
    return align_up((size_t)n * sizeof(double), 16) + stage;
}

// The (row, chunk) items of a symmetric tile: the rows i0 .. i0+nrows-1, row
// i with the chunks from its diagonal chunk floor(i/C) on (SC-HESS-VEC,
// Alg. 8), enumerated by chunk row R, then row, then chunk.
__host__ __device__ inline int sym_tile_items(int i0, int nrows, int C, int nch)
{
    int items = 0;
    for (int R = i0 / C; R * C < i0 + nrows; ++R) {
        const int lo = R * C > i0 ? R * C : i0;
        const int hi = (R + 1) * C < i0 + nrows ? (R + 1) * C : i0 + nrows;
        items += (hi - lo) * (nch - R);
    }
    return items;
}

__device__ __forceinline__ void sym_tile_item(int k, int i0, int nrows, int C, int nch, int &i, int &cn)
{
    int R = i0 / C;
    for (;; ++R) {
        const int lo = R * C > i0 ? R * C : i0;
        const int hi = (R + 1) * C < i0 + nrows ? (R + 1) * C : i0 + nrows;
        const int cnt = (hi - lo) * (nch - R);
        if (k < cnt || (R + 1) * C >= i0 + nrows) {
            i = lo + k / (nch - R);
            cn = R + k % (nch - R);
            return;
        }
        k -= cnt;
    }
}

// One symmetric tile: rows i0 .. i0+nrows-1 of one large Fletcher-Powell
// request.  Its (row, chunk) items are dealt round-robin to the CTA's
// threads, so every thread has an item in every iteration but the last
// (rows with few chunks leave no lane idle).  Each iteration stages every
// thread's chunk and row dot; after a barrier each column's owner adds, in
// thread order, the row dots of its own row and the mirrored entries H_is v_i
// of the chunks that hold its column (right of their row's diagonal chunk),
// into the tile's FP64 partial row vector.  The trip count is the same for
// every thread (the sweep's A/B tile loads are block-wide).
template <typename T, int C, int MB>
__device__ __forceinline__ void ragged_sym_tile(const RaggedArgs &a, const RTile &t, const Job &job,
                                                const ListPoints &pm, unsigned char *smem)
{
    __shared__ int s_last;
    const int n = t.n;
    const Smem<T> L = smem_layout<T>(FN_FP, true, n, t.maxpts, t.mt);
    double *part = reinterpret_cast<double *>(smem + align_up(L.total, 16));
    const SymStage<T, C> stage(smem + align_up(L.total, 16) + align_up((size_t)n * sizeof(double), 16),
                               (int)blockDim.x);
    const long long p = t.row0 / n;
    const int i0 = (int)(t.row0 - p * n);
    const int base = sym_slot_base(i0, C);
    const int tid = threadIdx.x;
    for (int e = tid; e < n - base; e += blockDim.x) part[e] = 0.0;
    point_prologue<T, T, FN_FP, true>(job, pm, smem, L, p, 1);  // ends with a barrier
    const PointTables<T> pt(smem, L, 0, n);
    const int q = a.list[t.list0 + p];
    const int items = sym_tile_items(i0, t.nrows, C, t.nch);
    const int iters = (items + (int)blockDim.x - 1) / (int)blockDim.x;
    for (int it = 0; it < iters; ++it) {
        const int k = tid + it * (int)blockDim.x;
        const bool has = k < items;
        int i = i0, cn = i0 / C;
        if (has) sym_tile_item(k, i0, t.nrows, C, t.nch, i, cn);
        const int cstart = cn * C;
        const HD<T, C> f = row_chunk<T, C, FN_FP, MB, true>(job, smem, L, pt, i, cstart, has, it == 0);
        double own = 0.0;  // products of two FP32 values are exact in FP64
        if (has) {
#pragma unroll
            for (int l = 0; l < C; ++l)
                if (cstart + l < n) own = fma((double)f.h[l], (double)pt.v[cstart + l], own);
        }
        stage.put(tid, f.h, own, has ? i : -1, cn);
        __syncthreads();
        for (int col = base + tid; col < n; col += blockDim.x) {
            const int ccn = col / C, cl = col - ccn * C;
            double sum = part[col - base];
            for (int u = 0; u < (int)blockDim.x; ++u) {
                const int ui = stage.row(u);
                if (ui < 0) continue;
                if (ui == col) sum += stage.own(u);
                const int ucn = stage.chunk(u);
                if (ucn == ccn && ucn > ui / C) sum += (double)stage.h(u, cl) * (double)pt.v[ui];
            }
            part[col - base] = sum;
        }
        __syncthreads();  // the stage is rewritten by the next iteration
    }
    // This tile's slot: after the slots of the request's earlier tiles.
    const int ti = i0 / t.srows;
    long long slot = a.soffs[q];
    for (int tt = 0; tt < ti; ++tt) slot += n - sym_slot_base(tt * t.srows, C);
    for (int e = tid; e < n - base; e += blockDim.x) a.slots[slot + e] = part[e];
    // Publish the slot, count the tile; the tile that completes the request
    // adds all of its slots in tile order and writes the output.
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&a.done[q], 1) + 1 == t.ntiles_req);
    __syncthreads();
    if (s_last) {
        __threadfence();
        T *O = reinterpret_cast<T *>(a.out) + pm.off(p);
        for (int col = tid; col < n; col += blockDim.x) {
            double sum = 0.0;
            long long off = a.soffs[q];
            for (int tt = 0; tt < t.ntiles_req; ++tt) {
                const int b = sym_slot_base(tt * t.srows, C);
                if (col >= b) sum += __ldcg(&a.slots[off + col - b]);
                off += n - b;
            }
            O[col] = (T)sum;
        }
    }
}

template <typename T, int C, int FN>
__device__ __forceinline__ void ragged_tile(const RaggedArgs &a, const RTile &t, unsigned char *smem)
{
    Job job;
    job.x = a.x;
    job.v = a.v;
    job.out = a.out;
    job.A = a.A;
    job.B = a.B;
    job.npoints = t.npoints;
    job.row0 = t.row0;
    job.n = t.n;
    job.nch = t.nch;
    job.tpr = t.tpr;
    job.maxpts = t.maxpts;
    job.mt = t.mt;
    job.ld = a.ld;
    ListPoints pm{a.list + t.list0, a.offs, a.eoffs, a.Epack};
    if (FN == FN_FP && t.sym) {
        ragged_sym_tile<T, C, ragged_mb(C, sizeof(T) == 8)>(a, t, job, pm, smem);
    } else {
        block_sweeps<T, T, C, FN, true, ragged_mb(C, sizeof(T) == 8)>(job, pm, smem);
    }
}

template <typename T, int FN>
__device__ __forceinline__ void ragged_tile_c(const RaggedArgs &a, const RTile &t, unsigned char *smem)
{
    if (IsComp<T>::value && t.n == 1) {
        // One variable: FP64 sweep with float I/O (the Hessian is a single
        // entry whose terms can cancel far below their size).
        Job job;
        job.x = a.x;
        job.v = a.v;
        job.out = a.out;
        job.A = a.A;
        job.B = a.B;
        job.npoints = t.npoints;
        job.row0 = t.row0;
        job.n = t.n;
        job.nch = t.nch;
        job.tpr = t.tpr;
        job.maxpts = t.maxpts;
        job.mt = t.mt;
        job.ld = a.ld;
        ListPoints pm{a.list + t.list0, a.offs, a.eoffs, a.Epack};
        block_sweeps<double, float, 1, FN, true, 8>(job, pm, smem);
    } else if (t.C == 8) {
        ragged_tile<T, 8, FN>(a, t, smem);
    } else {
        ragged_tile<T, 16, FN>(a, t, smem);
    }
}

template <typename T>
__global__ void __launch_bounds__(kRaggedBlock, 1) ragged_kernel(const RaggedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_tile;
    long long t_start = -1;  // thread 0, autotuning only: start of the current tile
    for (;;) {
        __syncthreads();  // the previous tile is done with shared memory and s_tile
        if (threadIdx.x == 0) {
            if (a.busy) {
                const long long now = clock64();
                if (t_start >= 0) atomicAdd(a.busy, (unsigned long long)(now - t_start));
                t_start = now;
            }
            s_tile = atomicAdd(a.counter, 1);
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= a.ntiles) break;
        const RTile tile = a.tiles[t];
        switch (tile.fn) {
        case FN_ROSENBROCK: ragged_tile_c<T, FN_ROSENBROCK>(a, tile, smem_raw); break;
        case FN_ACKLEY: ragged_tile_c<T, FN_ACKLEY>(a, tile, smem_raw); break;
        default: ragged_tile_c<T, FN_FP>(a, tile, smem_raw); break;
        }
    }
}

}  // namespace chessfad

using namespace chessfad;

struct chessfad_ragged_plan_s {
    int prec = 0;
    int csize = 0;  // 0: per-group chunk sizes (tuned or default); else every group's
    long long nreq = 0;
    int max_fp_n = 0;
    size_t smem = 0;
    std::vector<RTile> tiles;
    std::vector<int> list;
    std::vector<long long> offs, eoffs, soffs;
    long long slot_elems = 0;  // FP64 partial rows of the symmetric tiles
    // device workspace layout (bytes): tables (uploaded), then the queue
    // counter and the per-request tile counters (zeroed every run), then the
    // symmetric tiles' slots (written before they are read)
    size_t off_tiles = 0, off_list = 0, off_offs = 0, off_eoffs = 0, off_soffs = 0, off_counter = 0, off_done = 0,
           off_slots = 0, table_bytes = 0, total = 0;
    std::vector<unsigned char> image;  // host image of the tables (table_bytes)
    // persistent grid size, computed for the device of the first run (and
    // again when a run is on another device); guarded by mu
    std::mutex mu;
    int grid_dev = -1, grid = 0;
    double est_cost = 0.0;
};

namespace {

size_t align256(size_t a) { return (a + 255) / 256 * 256; }

int pow2_floor(int v)
{
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// Relative cost of one sweep (FP32 instruction estimate of the dense rules).
double sweep_cost(int fn, int n, int C)
{
    switch (fn) {
    case CHESSFAD_ROSENBROCK: return (double)std::max(1, n - 1) * (22.0 * C + 11.0);
    case CHESSFAD_ACKLEY: return (double)n * (9.0 * C + 5.0) + 15.0 * C;
    default: return (double)n * n * (6.0 * C + 8.0) + (double)n * (11.0 * C);
    }
}

// Rows of A and B per shared-memory tile of the Fletcher-Powell sweep: as
// many as fit `budget` bytes (both matrices), a multiple of 8 and of mb, at
// most n rounded up to 8.
int fp_tile_rows_ragged(int n, int prec, int mb, size_t budget)
{
    const size_t esz = (prec == CHESSFAD_FP64) ? 8 : 4;
    int mt = (int)(budget / (2 * (size_t)n * esz));
    mt = std::max(8, mt / 8 * 8);
    mt = std::min(mt, (n + 7) / 8 * 8);
    if (mt % mb) mt = (mt / mb + 1) * mb;
    return mt;
}

// Configuration of one (function, n range) group: chunk size and lanes per
// row (0 = default).  n ranges are the powers of two: bucket b holds
// 2^b <= n < 2^(b+1) (n = 512 joins bucket 8).
struct GroupCfg {
    int C = 0;
    int tpr = 0;
    int ab_kib = 0;  // Fletcher-Powell: A/B tile budget in KiB (0: kAbDefaultKiB)
};

// The default budget of a Fletcher-Powell group's A/B tiles, and the large
// one the tuner also tries: the uneven-batch kernel runs one CTA per SM (its
// registers), so a larger tile costs no occupancy and halves or quarters the
// tile loads and barriers of an evaluation at large n.
constexpr int kAbDefaultKiB = 48;
constexpr int kAbLargeKiB = 144;

int n_bucket(int n)
{
    int b = 0;
    while ((2 << b) <= n && b < 8) ++b;
    return b;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, GroupCfg> g_tuned;  // (prec, fn, bucket)

// Default lanes per row: enough rows per tile to keep the per-point prologue
// small, more lanes only when a row's chunks are many.
int default_tpr(int nch) { return std::min(32, pow2_floor(std::max(1, nch / 8))); }

// Symmetric tiles: rows of one point each, kRaggedBlock / lanes of them (the
// tile's items are dealt to all its threads); at least enough lanes per row that
// a tile's rows do not outnumber the point's.
int sym_tpr(int tpr, int n)
{
    while (tpr < 32 && kRaggedBlock / tpr > n) tpr *= 2;
    return tpr;
}

struct PlanOptions {
    int csize = 0;                               // fixed chunk size for every group (0: per group)
    const std::map<std::pair<int, int>, GroupCfg> *force = nullptr;  // (fn, bucket) -> forced config
};

int build_plan(const chessfad_request *reqs, long long nreq, int prec, const PlanOptions &opt,
               chessfad_ragged_plan_s *pl)
{
    pl->prec = prec;
    pl->csize = opt.csize;
    pl->nreq = nreq;
    const int cdef = (prec == CHESSFAD_FP64) ? 8 : 16;

    // Group by (fn, n); the request list holds each group's requests in order.
    std::map<std::pair<int, int>, std::vector<int>> groups;
    for (long long q = 0; q < nreq; ++q) groups[{reqs[q].fn, reqs[q].n}].push_back((int)q);
    pl->offs.resize(nreq);
    pl->eoffs.resize(nreq);
    pl->soffs.assign(nreq, -1);
    for (long long q = 0; q < nreq; ++q) {
        pl->offs[q] = reqs[q].off;
        pl->eoffs[q] = reqs[q].fn == CHESSFAD_FLETCHER_POWELL ? reqs[q].eoff : 0;
    }
    std::vector<std::pair<double, RTile>> work;
    size_t smem = 0;
    for (auto &g : groups) {
        const int fn = g.first.first, n = g.first.second;
        GroupCfg gc;
        if (opt.force) {
            auto it = opt.force->find({fn, n_bucket(n)});
            if (it != opt.force->end()) gc = it->second;
        } else if (opt.csize == 0) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(std::make_tuple(prec, fn, n_bucket(n)));
            if (it != g_tuned.end()) gc = it->second;
        }
        int C = gc.C ? gc.C : (opt.csize ? opt.csize : cdef);
        if (prec == CHESSFAD_FP32_COMP && n == 1) C = 1;
        const int nch = (n + C - 1) / C;
        const int mb = ragged_mb(C, prec == CHESSFAD_FP64);
        const int tpr = gc.tpr ? std::min(gc.tpr, 32) : default_tpr(nch);
        const int rows = kRaggedBlock / tpr;
        const long long np = (long long)g.second.size();
        const long long total_rows = np * n;
        const int maxpts = (int)std::min<long long>(np, (rows - 1) / n + 2);
        const size_t ab = (size_t)(gc.ab_kib ? gc.ab_kib : kAbDefaultKiB) * 1024;
        const int mt = (fn == CHESSFAD_FLETCHER_POWELL) ? fp_tile_rows_ragged(n, prec, (C == 1) ? 8 : mb, ab) : 8;
        if (fn == CHESSFAD_FLETCHER_POWELL) pl->max_fp_n = std::max(pl->max_fp_n, n);
        const bool f64sweep = (prec == CHESSFAD_FP64) || n == 1;
        const size_t bytes = f64sweep ? smem_layout<double>(fn, true, n, maxpts, mt).total
                                      : smem_layout<float>(fn, true, n, maxpts, mt).total;
        smem = std::max(smem, bytes);
        const int list0 = (int)pl->list.size();
        for (int q : g.second) pl->list.push_back(q);
        if (fn == CHESSFAD_FLETCHER_POWELL && n >= kSymMinN) {
            const int stpr = sym_tpr(tpr, n);
            const int srows = kRaggedBlock / stpr;
            const int ntq = (n + srows - 1) / srows;
            const int smt = fp_tile_rows_ragged(n, prec, mb, ab);
            const size_t sbytes =
                (prec == CHESSFAD_FP64)
                    ? align_up(smem_layout<double>(fn, true, n, 1, smt).total, 16) + sym_tile_extra<double>(n, C)
                    : align_up(smem_layout<float>(fn, true, n, 1, smt).total, 16) + sym_tile_extra<float>(n, C);
            smem = std::max(smem, sbytes);
            long long slot_len = 0;
            for (int tt = 0; tt < ntq; ++tt) slot_len += n - sym_slot_base(tt * srows, C);
            const double sweep = sweep_cost(fn, n, C);
            for (long long pt = 0; pt < np; ++pt) {
                const int q = g.second[pt];
                pl->soffs[q] = pl->slot_elems;
                pl->slot_elems += slot_len;
                for (int i0 = 0; i0 < n; i0 += srows) {
                    RTile t{};
                    t.row0 = pt * n + i0;
                    t.npoints = np;
                    t.list0 = list0;
                    t.fn = fn;
                    t.n = n;
                    t.C = C;
                    t.nch = nch;
                    t.tpr = stpr;
                    t.maxpts = 1;
                    t.mt = smt;
                    t.sym = 1;
                    t.nrows = std::min(srows, n - i0);
                    t.srows = srows;
                    t.ntiles_req = ntq;
                    // the tile's (row, chunk) items, dealt to its threads
                    const int iters = (sym_tile_items(i0, t.nrows, C, nch) + kRaggedBlock - 1) / kRaggedBlock;
                    const double cost = (double)iters * kRaggedBlock * sweep + 2000.0;
                    work.push_back({cost, t});
                    pl->est_cost += cost;
                }
            }
            continue;
        }
        const double per_row = nch * sweep_cost(fn, n, C);
        for (long long r0 = 0; r0 < total_rows; r0 += rows) {
            RTile t{};
            t.row0 = r0;
            t.npoints = np;
            t.list0 = list0;
            t.fn = fn;
            t.n = n;
            t.C = C;
            t.nch = nch;
            t.tpr = tpr;
            t.maxpts = maxpts;
            t.mt = mt;
            t.sym = 0;
            t.nrows = rows;
            const double cost = per_row * (double)std::min<long long>(rows, total_rows - r0) + 2000.0;
            work.push_back({cost, t});
            pl->est_cost += cost;
        }
    }
    if (work.size() > (size_t)0x7fffffff) return CHESSFAD_ERR_BATCH;
    std::stable_sort(work.begin(), work.end(),
                     [](const std::pair<double, RTile> &a, const std::pair<double, RTile> &b) { return a.first > b.first; });
    pl->tiles.reserve(work.size());
    for (auto &w : work) pl->tiles.push_back(w.second);
    pl->smem = smem;

    // Workspace: tiles | list | offs | eoffs | soffs (the tables), then
    // counter | done (zeroed by every run), then the slots.
    pl->off_tiles = 0;
    pl->off_list = align256(pl->off_tiles + pl->tiles.size() * sizeof(RTile));
    pl->off_offs = align256(pl->off_list + pl->list.size() * sizeof(int));
    pl->off_eoffs = align256(pl->off_offs + pl->offs.size() * sizeof(long long));
    pl->off_soffs = align256(pl->off_eoffs + pl->eoffs.size() * sizeof(long long));
    pl->table_bytes = align256(pl->off_soffs + pl->soffs.size() * sizeof(long long));
    pl->off_counter = pl->table_bytes;
    pl->off_done = align256(pl->off_counter + sizeof(int));
    pl->off_slots = align256(pl->off_done + (size_t)nreq * sizeof(int));
    pl->total = align256(pl->off_slots + (size_t)pl->slot_elems * sizeof(double));
    pl->image.assign(pl->table_bytes, 0);
    if (!pl->tiles.empty()) std::memcpy(&pl->image[pl->off_tiles], pl->tiles.data(), pl->tiles.size() * sizeof(RTile));
    if (!pl->list.empty()) std::memcpy(&pl->image[pl->off_list], pl->list.data(), pl->list.size() * sizeof(int));
    if (!pl->offs.empty()) std::memcpy(&pl->image[pl->off_offs], pl->offs.data(), pl->offs.size() * sizeof(long long));
    if (!pl->eoffs.empty())
        std::memcpy(&pl->image[pl->off_eoffs], pl->eoffs.data(), pl->eoffs.size() * sizeof(long long));
    if (!pl->soffs.empty())
        std::memcpy(&pl->image[pl->off_soffs], pl->soffs.data(), pl->soffs.size() * sizeof(long long));
    return CHESSFAD_SUCCESS;
}

int check_requests(const chessfad_request *reqs, long long nreq)
{
    if (nreq < 0) return CHESSFAD_ERR_BATCH;
    if (nreq > 0 && !reqs) return CHESSFAD_ERR_NULL;
    if (nreq > (1LL << 30)) return CHESSFAD_ERR_BATCH;
    for (long long q = 0; q < nreq; ++q) {
        const chessfad_request &r = reqs[q];
        if (r.fn < 0 || r.fn > 2) return CHESSFAD_ERR_FUNCTION;
        if (r.n < 1 || r.n > CHESSFAD_MAX_N) return CHESSFAD_ERR_SIZE;
        if (r.off < 0 || (r.fn == CHESSFAD_FLETCHER_POWELL && r.eoff < 0)) return CHESSFAD_ERR_PLAN;
    }
    return CHESSFAD_SUCCESS;
}

template <typename T>
cudaError_t launch_ragged(chessfad_ragged_plan_s *pl, const RaggedArgs &a, cudaStream_t stream)
{
    auto kern = ragged_kernel<T>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // the kernel's dynamic shared-memory limit only ever grows (several plans
    // share the kernel)
    static std::atomic<int> configured[64];
    e = opt_in_smem(kern, pl->smem, configured);
    if (e != cudaSuccess) return e;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(pl->mu);
        if (pl->grid_dev != dev) {
            int per_sm = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRaggedBlock, pl->smem);
            if (e != cudaSuccess) return e;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            pl->grid = std::max(1, per_sm) * sms;
            pl->grid_dev = dev;
        }
        grid = pl->grid;
    }
    if (a.ntiles == 0) return cudaSuccess;
    // queue counter and per-request tile counters: contiguous
    e = cudaMemsetAsync(a.counter, 0, pl->off_slots - pl->off_counter, stream);
    if (e != cudaSuccess) return e;
    kern<<<std::min(grid, a.ntiles), kRaggedBlock, pl->smem, stream>>>(a);
    return cudaGetLastError();
}

RaggedArgs ragged_args(const chessfad_ragged_plan_s *plan, unsigned char *ws, const void *xpack, const void *vpack,
                       void *outpack, const chessfad_fp_params *params)
{
    RaggedArgs a{};
    a.x = xpack;
    a.v = vpack;
    a.out = outpack;
    if (params) {
        a.A = params->A;
        a.B = params->B;
        a.Epack = params->E;
        a.ld = params->ld;
    }
    a.tiles = reinterpret_cast<const RTile *>(ws + plan->off_tiles);
    a.list = reinterpret_cast<const int *>(ws + plan->off_list);
    a.offs = reinterpret_cast<const long long *>(ws + plan->off_offs);
    a.eoffs = reinterpret_cast<const long long *>(ws + plan->off_eoffs);
    a.soffs = reinterpret_cast<const long long *>(ws + plan->off_soffs);
    a.counter = reinterpret_cast<int *>(ws + plan->off_counter);
    a.done = reinterpret_cast<int *>(ws + plan->off_done);
    a.slots = reinterpret_cast<double *>(ws + plan->off_slots);
    a.ntiles = (int)plan->tiles.size();
    return a;
}

int run_plan(chessfad_ragged_plan_s *plan, unsigned char *ws, const void *xpack, const void *vpack, void *outpack,
             const chessfad_fp_params *params, cudaStream_t s, unsigned long long *busy = nullptr)
{
    RaggedArgs a = ragged_args(plan, ws, xpack, vpack, outpack, params);
    a.busy = busy;
    const cudaError_t e =
        plan->prec == CHESSFAD_FP64 ? launch_ragged<double>(plan, a, s) : launch_ragged<float>(plan, a, s);
    return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}

int check_run(const chessfad_ragged_plan_s *plan, const void *xpack, const void *vpack, const void *outpack,
              const chessfad_fp_params *params)
{
    if (!xpack || !vpack || !outpack) return CHESSFAD_ERR_NULL;
    if (plan->max_fp_n > 0 && (!params || !params->A || !params->B || !params->E || params->ld < plan->max_fp_n))
        return CHESSFAD_ERR_PARAMS;
    return CHESSFAD_SUCCESS;
}

}  // namespace

extern "C" {

int chessfad_ragged_plan_create(const chessfad_request *reqs, long long nreq, int prec, int csize,
                                chessfad_ragged_plan *plan_out)
{
    if (!plan_out) return CHESSFAD_ERR_NULL;
    *plan_out = nullptr;
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    if (csize != 0 && csize != 8 && csize != 16) return CHESSFAD_ERR_CHUNK;
    int st = check_requests(reqs, nreq);
    if (st) return st;
    auto *pl = new (std::nothrow) chessfad_ragged_plan_s();
    if (!pl) return CHESSFAD_ERR_PLAN;
    PlanOptions opt;
    opt.csize = csize;
    st = build_plan(reqs, nreq, prec, opt, pl);
    if (st) {
        delete pl;
        return st;
    }
    *plan_out = pl;
    return CHESSFAD_SUCCESS;
}

int chessfad_ragged_plan_destroy(chessfad_ragged_plan plan)
{
    delete plan;
    return CHESSFAD_SUCCESS;
}

int chessfad_ragged_plan_info(chessfad_ragged_plan plan, size_t *workspace_bytes, long long *ntiles,
                              size_t *smem_bytes)
{
    if (!plan) return CHESSFAD_ERR_PLAN;
    if (workspace_bytes) *workspace_bytes = plan->total;
    if (ntiles) *ntiles = (long long)plan->tiles.size();
    if (smem_bytes) *smem_bytes = plan->smem;
    return CHESSFAD_SUCCESS;
}

int chessfad_ragged_plan_group_config(chessfad_ragged_plan plan, int fn, int n, int *csize, int *threads_per_row,
                                      int *tile_rows)
{
    if (!plan) return CHESSFAD_ERR_PLAN;
    for (const RTile &t : plan->tiles) {
        if (t.fn == fn && t.n == n) {
            if (csize) *csize = t.C;
            if (threads_per_row) *threads_per_row = t.tpr;
            if (tile_rows) *tile_rows = t.mt;
            return CHESSFAD_SUCCESS;
        }
    }
    return CHESSFAD_ERR_SIZE;
}

int chessfad_ragged_plan_upload(chessfad_ragged_plan plan, void *workspace, size_t workspace_bytes,
                                chessfad_stream_t stream)
{
    if (!plan) return CHESSFAD_ERR_PLAN;
    if (!workspace || workspace_bytes < plan->total) return CHESSFAD_ERR_WORKSPACE;
    if (plan->table_bytes == 0) return CHESSFAD_SUCCESS;
    cudaError_t e = cudaMemcpyAsync(workspace, plan->image.data(), plan->table_bytes, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? CHESSFAD_SUCCESS : CHESSFAD_ERR_CUDA;
}

int chessfad_hvp_ragged(chessfad_ragged_plan plan, const void *xpack, const void *vpack, void *outpack,
                        const chessfad_fp_params *params, void *workspace, size_t workspace_bytes,
                        chessfad_stream_t stream)
{
    if (!plan) return CHESSFAD_ERR_PLAN;
    if (!workspace || workspace_bytes < plan->total) return CHESSFAD_ERR_WORKSPACE;
    if (plan->tiles.empty()) return CHESSFAD_SUCCESS;
    const int st = check_run(plan, xpack, vpack, outpack, params);
    if (st) return st;
    return run_plan(plan, static_cast<unsigned char *>(workspace), xpack, vpack, outpack, params,
                    (cudaStream_t)stream);
}

int chessfad_ragged_autotune(const chessfad_request *reqs, long long nreq, int prec, const void *xpack,
                             const void *vpack, void *outpack, const chessfad_fp_params *params, void *workspace,
                             size_t workspace_bytes, chessfad_stream_t stream_, long long *groups_tuned)
{
    const cudaStream_t stream = (cudaStream_t)stream_;
    if (groups_tuned) *groups_tuned = 0;
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    int st = check_requests(reqs, nreq);
    if (st) return st;
    if (nreq == 0) return CHESSFAD_SUCCESS;
    if (!workspace) return CHESSFAD_ERR_WORKSPACE;
    if (!xpack || !vpack || !outpack) return CHESSFAD_ERR_NULL;
    int max_fp_n = 0;
    for (long long q = 0; q < nreq; ++q)
        if (reqs[q].fn == CHESSFAD_FLETCHER_POWELL) max_fp_n = std::max(max_fp_n, reqs[q].n);
    if (max_fp_n > 0 && (!params || !params->A || !params->B || !params->E || params->ld < max_fp_n))
        return CHESSFAD_ERR_PARAMS;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;

    // (fn, n range) groups, each request in its group in table order
    std::map<std::pair<int, int>, std::vector<long long>> groups;
    for (long long q = 0; q < nreq; ++q) groups[{reqs[q].fn, n_bucket(reqs[q].n)}].push_back(q);

    int rc = CHESSFAD_SUCCESS;
    long long tuned = 0;
    for (auto &g : groups) {
        const int fn = g.first.first, bucket = g.first.second;
        // A sample of the group: requests in table order until their rows
        // fill the GPU about four times with the default tiles (symmetric
        // requests: four tiles per SM).
        std::vector<chessfad_request> sample;
        long long rows = 0;
        const long long want_rows = 4LL * sms * kRaggedBlock;
        for (long long q : g.second) {
            sample.push_back(reqs[q]);
            const int n = reqs[q].n;
            rows += (fn == CHESSFAD_FLETCHER_POWELL && n >= kSymMinN) ? (long long)kRaggedBlock * 8 : n;
            if (rows >= want_rows) break;
        }
        int nmax = 0;
        for (const chessfad_request &r : sample) nmax = std::max(nmax, r.n);
        std::vector<GroupCfg> cands;
        // A/B tile budgets that give different tile heights at this group's n
        std::vector<int> abs{kAbDefaultKiB};
        if (fn == CHESSFAD_FLETCHER_POWELL &&
            fp_tile_rows_ragged(nmax, prec, 8, (size_t)kAbLargeKiB * 1024) !=
                fp_tile_rows_ragged(nmax, prec, 8, (size_t)kAbDefaultKiB * 1024))
            abs.push_back(kAbLargeKiB);
        for (int C : {16, 8}) {
            if (prec == CHESSFAD_FP32_COMP && nmax == 1 && C == 8) continue;  // n = 1 runs C = 1 either way
            const int nch = (nmax + C - 1) / C;
            std::vector<int> seen;
            for (int tpr = 1; tpr <= 32; tpr <<= 1) {
                if (tpr > 1 && tpr > 2 * nch) break;
                const int eff = (fn == CHESSFAD_FLETCHER_POWELL && nmax >= kSymMinN) ? sym_tpr(tpr, nmax) : tpr;
                if (std::find(seen.begin(), seen.end(), eff) != seen.end()) continue;
                seen.push_back(eff);
                for (int ab : abs) cands.push_back(GroupCfg{C, eff, ab});
            }
        }
        GroupCfg best;
        float best_ms = INFINITY;  // the objective: summed SM cycles of the sample's tiles
        for (const GroupCfg &c : cands) {
            std::map<std::pair<int, int>, GroupCfg> force;
            force[{fn, bucket}] = c;
            PlanOptions opt;
            opt.force = &force;
            chessfad_ragged_plan_s trial;
            if (build_plan(sample.data(), (long long)sample.size(), prec, opt, &trial) != CHESSFAD_SUCCESS) continue;
            // the busy-cycle counter after the trial plan's workspace
            if (trial.total + 256 > workspace_bytes) continue;
            unsigned char *ws = static_cast<unsigned char *>(workspace);
            unsigned long long *busy = reinterpret_cast<unsigned long long *>(ws + trial.total);
            if (cudaMemcpyAsync(ws, trial.image.data(), trial.table_bytes, cudaMemcpyHostToDevice, stream) !=
                cudaSuccess) {
                rc = CHESSFAD_ERR_CUDA;
                break;
            }
            if (run_plan(&trial, ws, xpack, vpack, outpack, params, stream) != CHESSFAD_SUCCESS) {
                cudaGetLastError();
                continue;
            }
            // The objective is the SM time the group's tiles take, summed over
            // the CTAs (one CTA per SM): the throughput the group gets inside
            // a large mixed run, free of the sample's own tail.
            if (cudaMemsetAsync(busy, 0, sizeof(unsigned long long), stream) != cudaSuccess ||
                run_plan(&trial, ws, xpack, vpack, outpack, params, stream, busy) != CHESSFAD_SUCCESS) {
                rc = CHESSFAD_ERR_CUDA;
                break;
            }
            unsigned long long cycles = 0;
            if (cudaMemcpyAsync(&cycles, busy, sizeof(cycles), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                rc = CHESSFAD_ERR_CUDA;
                break;
            }
            const float ms = (float)cycles;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        if (rc) break;
        if (std::isfinite(best_ms)) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[std::make_tuple(prec, fn, bucket)] = best;
            ++tuned;
        }
    }
    if (groups_tuned) *groups_tuned = tuned;
    return rc;
}

int chessfad_ragged_tuned_config(int prec, int fn, int n, int *csize, int *threads_per_row, int *ab_kib)
{
    if (prec != CHESSFAD_FP64 && prec != CHESSFAD_FP32_COMP) return CHESSFAD_ERR_PRECISION;
    if (fn < 0 || fn > 2) return CHESSFAD_ERR_FUNCTION;
    if (n < 1 || n > CHESSFAD_MAX_N) return CHESSFAD_ERR_SIZE;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(prec, fn, n_bucket(n)));
    if (it == g_tuned.end()) return CHESSFAD_ERR_CONFIG;
    if (csize) *csize = it->second.C;
    if (threads_per_row) *threads_per_row = it->second.tpr;
    if (ab_kib) *ab_kib = it->second.ab_kib ? it->second.ab_kib : kAbDefaultKiB;
    return CHESSFAD_SUCCESS;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation entry point.
//
// Some callers cannot call cudaMalloc: a host framework that owns device
// memory through its own pool (raw allocations would bypass its accounting or
// fail because the pool holds the memory), a plugin or callback that must not
// allocate or implicitly synchronise the device (cudaMalloc may do both), or
// real-time code for which allocation latency is unbounded.  For them the
// uneven-batch run keeps its scratch -- the plan's tables, the queue and tile
// counters and the symmetric tiles' partial rows -- in a file-scope __device__ array of CHESSFAD_RAGGED_STATIC_BYTES
// that every GPU which loads this library holds until the process exits.
//
// In host code the array's name is only a host-side stand-in; its device
// address is taken once per device with cudaGetSymbolAddress, with that device
// current, the first time the entry point runs on it.  Every call shares the
// array: each call copies the plan's tables into it and zeroes the counters
// (stream-ordered) before its kernel, so calls whose work overlaps on the GPU
// race on the shared scratch.
static __device__ __align__(256) unsigned char g_ragged_scratch[CHESSFAD_RAGGED_STATIC_BYTES];

namespace {

constexpr int kMaxScratchDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxScratchDevices] = {};

int ragged_scratch_address(void **addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHESSFAD_ERR_CUDA;
    if (dev < 0 || dev >= kMaxScratchDevices) return CHESSFAD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ragged_scratch) != cudaSuccess || !p) return CHESSFAD_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return CHESSFAD_SUCCESS;
}

}  // namespace

extern "C" int chessfad_hvp_ragged_noalloc(chessfad_ragged_plan plan, const void *xpack, const void *vpack,
                                           void *outpack, const chessfad_fp_params *params,
                                           chessfad_stream_t stream)
{
    if (!plan) return CHESSFAD_ERR_PLAN;
    if (plan->total > (size_t)CHESSFAD_RAGGED_STATIC_BYTES) return CHESSFAD_ERR_WORKSPACE;
    if (plan->tiles.empty()) return CHESSFAD_SUCCESS;
    int st = check_run(plan, xpack, vpack, outpack, params);
    if (st) return st;
    void *scratch = nullptr;
    st = ragged_scratch_address(&scratch);
    if (st != CHESSFAD_SUCCESS) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    // The plan's tables; the run zeroes the counters, and every symmetric
    // tile writes its whole slot before any tile reads it.
    if (cudaMemcpyAsync(scratch, plan->image.data(), plan->table_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return CHESSFAD_ERR_CUDA;
    return run_plan(plan, static_cast<unsigned char *>(scratch), xpack, vpack, outpack, params, s);
}
