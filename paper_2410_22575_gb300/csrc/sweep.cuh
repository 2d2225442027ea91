// sweep.cuh -- the chunked-hDual sweep kernels (Hessian-vector products and
// full Hessians at many independent points).
//
// Work decomposition (the paper's L0/L1/L2 parallelism, Sec. VI, Alg. 9,
// Alg. 10, Fig. 2): one thread per (point p, Hessian row i, lane r), with tpr
// lanes per row; lane r evaluates chunks r, r+tpr, r+2tpr, ... of row i.  An
// evaluation ("sweep") seeds the n variables with CHUNK-INIT (Alg. 4) on the
// fly, runs the test function on register-resident hDual<C> numbers and
// leaves d2f/dx_i dx_{cstart+l}, l < C, in the result's h[] (Alg. 5).  For
// Hessian-vector products the chunk is dotted with v[cstart..cstart+C)
// (Alg. 7) and the tpr lanes of a row are summed with warp shuffles, where
// Fig. 2 goes through shared memory and __syncthreads.
//
// Per-block staging: the points a block touches are contiguous in x and v, so
// the block copies them into shared memory with coalesced loads once, together
// with per-point tables of value-only quantities that every sweep of the point
// would otherwise recompute: cos/sin(2 pi x_k) (Ackley), sin/cos x_j and the
// Fletcher-Powell residuals r_m (FP64), the Ackley sums S = sum x_k^2 and
// C = sum cos(2 pi x_k) (FP64) with the sqrt/exp values taken at them.  The
// value component of an hDual is the same in every sweep of a point; only
// the derivative components depend on (row, chunk).  These FP64 sums are the
// "FP64 islands" of the compensated-FP32 precision.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include <atomic>
#include <mutex>
#include <type_traits>

#include "hdual.cuh"
#include "sym_layout.cuh"

namespace chessfad {

enum { FN_ROSENBROCK = 0, FN_ACKLEY = 1, FN_FP = 2 };

struct SweepArgs {
    const void *x;
    const void *v;
    void *out;
    const double *A;
    const double *B;
    const double *E;
    long long batch;
    int n;
    int ld;
    int nch;     // ceil(n / C)
    int tpr;     // threads per row (power of two <= 32)
    int tpp;     // threads per point = n * tpr
    int maxpts;  // points staged per block (upper bound)
    int mt;      // Fletcher-Powell: rows of A, B per shared-memory tile
    int sym_acc; // symmetric HVP: 0 = stage the chunk matrix, 1 = FP64 row accumulators
};

// Number of Ackley per-point scalars kept in the table.
constexpr int kAckScal = 8;

// Shared-memory layout, computed identically on host and device.
template <typename T>
struct Smem {
    size_t xs, vs, t1, t2, sc, res, dsin, dcos, at, bt, total;
};

__host__ __device__ inline size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

template <typename T>
__host__ __device__ inline Smem<T> smem_layout(int fn, bool hvp, int n, int maxpts, int mt)
{
    Smem<T> s{};
    size_t off = 0;
    const size_t pn = (size_t)maxpts * n;
    s.xs = off; off = align_up(off + pn * sizeof(T), 16);
    s.vs = off; if (hvp) off = align_up(off + pn * sizeof(T), 16);
    s.t1 = s.t2 = s.sc = s.res = s.dsin = s.dcos = s.at = s.bt = off;
    if (fn == FN_ACKLEY) {
        // {x_k, phi'_k, phi''_k, pad} per variable, each point's n entries
        // stored twice so a walk that wraps past n stays contiguous.
        s.t1 = off; off = align_up(off + 2 * pn * 4 * sizeof(T), 16);
        s.t2 = s.t1;
        s.sc = off; off = align_up(off + (size_t)maxpts * kAckScal * sizeof(T), 16);
    } else if (fn == FN_FP) {
        s.t1 = off; off = align_up(off + pn * sizeof(T), 16);    // sin x_j
        s.t2 = off; off = align_up(off + pn * sizeof(T), 16);    // cos x_j
        s.res = off; off = align_up(off + pn * sizeof(T), 16);   // residual r_m (FP64-computed)
        // The FP64 sin/cos scratch of the prologue and the A/B tiles of the
        // sweep are never live together: they share one region.
        const size_t u = off;
        s.dsin = u;
        s.dcos = align_up(u + pn * sizeof(double), 16);
        const size_t end1 = align_up(s.dcos + pn * sizeof(double), 16);
        s.at = u;                                                   // A tile, [j][m]
        s.bt = align_up(u + (size_t)n * mt * sizeof(T), 16);       // B tile, [j][m]
        const size_t end2 = align_up(s.bt + (size_t)n * mt * sizeof(T), 16);
        off = end1 > end2 ? end1 : end2;
    }
    s.total = off;
    return s;
}

// ------------------------------------------------------------------ sums
// Sum over a function's terms.  FP64 (and plain) accumulation adds each term
// with FMAs; the compensated FP32 form runs Sum2 on every component.
template <typename T, int C, bool COMP>
struct TermSum;

// Terms enter as unary-rule applications phi(a) (phi with its derivatives
// at the value): a square u^2 is phi = u^2, phi' = 2u, phi'' = 2, the same
// components as the product rule on u * u with 3C+1 instead of 6C+3 FMAs.
template <typename T, int C>
struct TermSum<T, C, false> {
    HD<T, C> s;
    __device__ __forceinline__ void init() { s = hzero<T, C>(); }
    // += phi(a) + psi(b)
    __device__ __forceinline__ void add_unary2(const HD<T, C> &a, T pa, T da, T d2a, const HD<T, C> &b, T pb, T db,
                                               T d2b)
    {
        ::chessfad::add_unary<true>(s, a, pa, da, d2a);
        ::chessfad::add_unary<true>(s, b, pb, db, d2b);
    }
    // += a^2
    __device__ __forceinline__ void add_sq(const HD<T, C> &a) { ::chessfad::add_unary<true>(s, a, a.v * a.v, T(2) * a.v, T(2)); }
    __device__ __forceinline__ HD<T, C> value() const { return s; }
};

// Compensated FP32: blocked Sum2.  Terms are fused (FMA) into a plain FP32
// block partial; every kSumBlock terms the partial is added into the
// compensated pair (sum, error) with TwoSum, and value() adds the last
// partial and the error.  Each block partial carries at most
// (kSumBlock - 1) u of its own terms' magnitude in rounding error; the
// compensated pair then adds the partials with twice-working-precision
// accuracy (Ogita, Rump & Oishi, Sum2 over the partials).
constexpr int kSumBlock = 8;

template <int C>
struct TermSum<float, C, true> {
    CHD<C> s;
    HD<float, C> blk;
    int cnt;
    __device__ __forceinline__ void init()
    {
        chd_zero(s);
        blk = hzero<float, C>();
        cnt = 0;
    }
    __device__ __forceinline__ void step()
    {
        if (++cnt == kSumBlock) {
            chd_add(s, blk);
            blk = hzero<float, C>();
            cnt = 0;
        }
    }
    __device__ __forceinline__ void add_unary2(const HD<float, C> &a, float pa, float da, float d2a,
                                               const HD<float, C> &b, float pb, float db, float d2b)
    {
        ::chessfad::add_unary<true>(blk, a, pa, da, d2a);
        ::chessfad::add_unary<true>(blk, b, pb, db, d2b);
        step();
    }
    __device__ __forceinline__ void add_sq(const HD<float, C> &a)
    {
        ::chessfad::add_unary<true>(blk, a, a.v * a.v, 2.f * a.v, 2.f);
        step();
    }
    __device__ __forceinline__ HD<float, C> value() const
    {
        CHD<C> t = s;
        chd_add(t, blk);
        return chd_value(t);
    }
};

template <typename T>
struct IsComp {
    static constexpr bool value = false;
};
template <>
struct IsComp<float> {
    static constexpr bool value = true;
};

// ------------------------------------------------------------------ seeding
// The seeded variables y_0 .. y_{n-1} of one sweep (CHUNK-INIT, Alg. 4) are
// visited as: every variable outside the chunk (ascending), then the chunk's.
// Outside the chunk the g part is the constant zero vector; inside, when the
// chunk is unrolled, the constant unit vector e_{k-cstart}; only the d/dx_i
// seed [k == i] is data dependent.  The loop over the variables outside the
// chunk has the same trip count (n - C) for every chunk except a ragged last
// one, so lanes of a warp that work on different chunks do not diverge.
// Chunks wider than the unroll limit walk their variables with the generic
// (select-based) seed.
template <int C, int LIMIT>
struct Unroll {
    static constexpr bool value = C <= LIMIT;
};

template <int P, int END>
struct StaticFor {
    template <typename F>
    __device__ __forceinline__ static void run(F &&f)
    {
        if constexpr (P < END) {
            f(std::integral_constant<int, P>{});
            StaticFor<P + 1, END>::run(f);
        }
    }
};

// f(k, y_k) for every k in 0 .. n-1.  kRemap: the variables outside the chunk
// in one loop of uniform trip count, then the chunk (lanes of a warp on
// different chunks stay converged); otherwise three segments in ascending
// order (cheapest when a warp's lanes share the chunk).
template <typename T, int C, int LIMIT, bool kRemap, bool kSparse = false, typename F>
__device__ __forceinline__ void for_each_seed(const T *__restrict__ xs, int n, int i, int cstart, F &&f)
{
    const SeedK<T> z = seed_constants<T>();
    const int lo = min(cstart, n), hi = min(cstart + C, n);
    auto chunk = [&]() {
        if constexpr (Unroll<C, LIMIT>::value) {
            StaticFor<0, C>::run([&](auto P) {
                const int k = cstart + P.value;
                if (k < n) f(k, seed_at<T, C, P.value>(xs[k], k == i, z));
            });
        } else {
            for (int k = lo; k < hi; ++k) f(k, seed<T, C>(xs[k], k, i, cstart, z));
        }
    };
    if constexpr (kSparse) {
        // Seed-sparse: only y_i and the chunk's variables carry nonzero
        // derivatives; the others add to value components only.
        chunk();
        if (i < lo || i >= hi) f(i, seed_at<T, C, -1>(xs[i], true, z));
    } else if constexpr (kRemap) {
        const int nout = n - (hi - lo);
        for (int kk = 0; kk < nout; ++kk) {
            const int k = kk < lo ? kk : kk + (hi - lo);
            f(k, seed_at<T, C, -1>(xs[k], k == i, z));
        }
        chunk();
    } else {
        for (int k = 0; k < lo; ++k) f(k, seed_at<T, C, -1>(xs[k], k == i, z));
        chunk();
        for (int k = hi; k < n; ++k) f(k, seed_at<T, C, -1>(xs[k], k == i, z));
    }
}

// f(y_k, y_{k+1}) for every k in 0 .. n-2 (functions whose terms couple
// neighbours).  The pairs touching the chunk are k - cstart in [-1, C-1];
// kRemap as for for_each_seed.
template <typename T, int C, int LIMIT, bool kRemap, bool kSparse = false, typename F>
__device__ __forceinline__ void for_each_pair(const T *__restrict__ xs, int n, int i, int cstart, F &&f)
{
    const SeedK<T> z = seed_constants<T>();
    const int t0 = max(cstart - 1, 0);
    const int t1 = max(t0, min(cstart + C, n - 1));
    auto outside = [&](int k) {
        f(seed_at<T, C, -1>(xs[k], k == i, z), seed_at<T, C, -1>(xs[k + 1], k + 1 == i, z));
    };
    auto touching = [&]() {
        if constexpr (Unroll<C, LIMIT>::value) {
            StaticFor<0, C + 1>::run([&](auto Q) {
                constexpr int t = decltype(Q)::value - 1;
                const int k = cstart + t;
                if (k >= 0 && k + 1 < n)
                    f(seed_at<T, C, t>(xs[k], k == i, z), seed_at<T, C, t + 1>(xs[k + 1], k + 1 == i, z));
            });
        } else {
            for (int k = t0; k < t1; ++k)
                f(seed<T, C>(xs[k], k, i, cstart, z), seed<T, C>(xs[k + 1], k + 1, i, cstart, z));
        }
    };
    if constexpr (kSparse) {
        // Seed-sparse: the pairs touching the chunk, and the pairs (i-1, i),
        // (i, i+1) when they do not touch it.
        touching();
        if (i >= 1 && (i - 1 < t0 || i - 1 >= t1)) outside(i - 1);
        if (i + 1 < n && (i < t0 || i >= t1)) outside(i);
    } else if constexpr (kRemap) {
        const int nout = max(0, n - 1 - (t1 - t0));
        for (int kk = 0; kk < nout; ++kk) outside(kk < t0 ? kk : kk + (t1 - t0));
        touching();
    } else {
        for (int k = 0; k < t0; ++k) outside(k);
        touching();
        for (int k = t1; k < n - 1; ++k) outside(k);
    }
}

// ------------------------------------------------------------------ functions
// Rosenbrock, f = sum_{k<n-1} 100 (x_{k+1} - x_k^2)^2 + (1 - x_k)^2, on hDuals.
template <typename T, int C, bool kRemap, bool kSparse>
__device__ __forceinline__ HD<T, C> rosenbrock_sweep(const T *__restrict__ xs, int n, int i, int cstart)
{
    TermSum<T, C, IsComp<T>::value> acc;
    acc.init();
    for_each_pair<T, C, 8, kRemap, kSparse>(xs, n, i, cstart, [&](const HD<T, C> &y0, const HD<T, C> &y1) {
        const T x0 = y0.v;
        HD<T, C> d = y1;
        sfma_unary<true>(d, T(-1), y0, x0 * x0, T(2) * x0, T(2));  // d = x_{k+1} - x_k^2
        const T dv = d.v, e = T(1) - x0;
        // += 100 d^2 + (1 - x_k)^2, each by the unary rule of its square
        acc.add_unary2(d, T(100) * dv * dv, T(200) * dv, T(200), y0, e * e, T(-2) * e, T(2));
    });
    return acc.value();
}

// One Ackley table entry: x_k and the derivatives of cos(2 pi t) at x_k.
template <typename T>
struct alignas(16) AckEnt {
    T x, d1, d2, pad;
};

// Ackley on hDuals.  S = sum y_k^2 and Cs = sum cos(2 pi y_k) are accumulated
// in the sweep for their derivative components; their value components are
// the per-point FP64 sums from the table.  Each derivative component of S and
// Cs receives at most one nonzero term under CHUNK-INIT seeding (y_k carries
// a nonzero d/dx only for k == i or k in the chunk), so these sums are exact
// up to that term's own rounding and need no compensation.
template <typename T, int C, bool kRemap, bool kSparse>
__device__ __forceinline__ HD<T, C> ackley_sweep(const AckEnt<T> *__restrict__ tab, const T *__restrict__ sc, int n,
                                                 int i, int cstart)
{
    const SeedK<T> z = seed_constants<T>();
    HD<T, C> Sh = hzero<T, C>();  // S / 2: derivative components of sum y_k^2 / 2
    HD<T, C> Cs = hzero<T, C>();
    // y^2 / 2 by the unary rule (phi' = y, phi'' = 1), doubled once after the
    // sweep (exact); cos(2 pi t): phi' = -2 pi sin(2 pi t), phi'' = -4 pi^2 cos(2 pi t)
    auto term = [&](const AckEnt<T> &e, const HD<T, C> &y) {
        add_unary<false>(Sh, y, T(0), y.v, T(1));
        add_unary<false>(Cs, y, T(0), e.d1, e.d2);
    };
    const int lo = min(cstart, n), hi = min(cstart + C, n);
    if constexpr (kSparse) {
        // Seed-sparse: besides the chunk (below) only y_i has a nonzero
        // derivative part.
        if (i < lo || i >= hi) {
            const AckEnt<T> e = tab[i];
            term(e, seed_at<T, C, -1>(e.x, true, z));
        }
    } else if constexpr (kRemap) {
        // The variables after the chunk, then (wrapping, on the table's second
        // copy) those before it: one pointer, uniform trip count n - C.
        const AckEnt<T> *p = tab + hi;
        const AckEnt<T> *prow = tab + (i >= hi ? i : i + n);
        const int nout = n - (hi - lo);
#pragma unroll 4
        for (int kk = 0; kk < nout; ++kk, ++p) {
            const AckEnt<T> e = *p;
            term(e, seed_at<T, C, -1>(e.x, p == prow, z));
        }
    } else {
        for (int k = 0; k < lo; ++k) {
            const AckEnt<T> e = tab[k];
            term(e, seed_at<T, C, -1>(e.x, k == i, z));
        }
        for (int k = hi; k < n; ++k) {
            const AckEnt<T> e = tab[k];
            term(e, seed_at<T, C, -1>(e.x, k == i, z));
        }
    }
    if constexpr (Unroll<C, 16>::value) {
        StaticFor<0, C>::run([&](auto P) {
            const int k = cstart + P.value;
            if (k < n) {
                const AckEnt<T> e = tab[k];
                term(e, seed_at<T, C, P.value>(e.x, k == i, z));
            }
        });
    } else {
        for (int k = lo; k < hi; ++k) {
            const AckEnt<T> e = tab[k];
            term(e, seed<T, C>(e.x, k, i, cstart, z));
        }
    }
    // The tail, each step one unary rule with the constant factors folded
    // into phi' and phi'' (the per-point values come from the FP64 island
    // sums: sc[3] = sqrt(S/n) with its derivatives sc[4], sc[5]; sc[6] =
    // exp(-0.2 sqrt(S/n)); sc[7] = exp(Cs/n)):
    //   r  = sqrt(S/n) as a function of Sh = S/2: phi' = (2/n) sc[4], phi'' = (2/n)^2 sc[5]
    //   f  = -20 exp(-0.2 r) as a function of r:  phi' = 4 sc[6], phi'' = -0.8 sc[6]
    //   f += -exp(Cs/n) as a function of Cs:      phi' = -sc[7]/n, phi'' = -sc[7]/n^2
    const T inv_n = sc[2];
    const T k2 = T(2) * inv_n;
    const HD<T, C> r = unary(Sh, sc[3], k2 * sc[4], (k2 * k2) * sc[5]);
    const T e1 = sc[6], e2 = sc[7];
    HD<T, C> f = unary(r, T(-20) * e1, T(4) * e1, T(-0.8) * e1);
    add_unary<true>(f, Cs, -e2, -inv_n * e2, -(inv_n * inv_n) * e2);
    f.v = f.v + T(20) + T(2.718281828459045);
    return f;
}

// ------------------------------------------------------------------ block work
// A block-uniform unit of work: the rows [row0, row0 + blockDim/tpr) of a
// point-major row space (row = point * n + i) over `npoints` points of one
// function and one n.  Point addressing is a policy: a contiguous batch, or a
// list of requests with their own offsets (the uneven batch).
struct Job {
    const void *x;
    const void *v;
    void *out;
    const double *A;
    const double *B;
    long long npoints;
    long long row0;
    int n, nch, tpr, maxpts, mt, ld;
};

// Points p = 0 .. batch-1 of a [batch][n] array; one E for all points.
struct ContigPoints {
    const double *E;
    int n;
    __device__ __forceinline__ long long off(long long p) const { return p * n; }
    __device__ __forceinline__ const double *e(long long) const { return E; }
};

// Point p of a request group is request list[p]; its x, v, out start at
// off[list[p]] and its Fletcher-Powell E at Epack + eoff[list[p]].
struct ListPoints {
    const int *list;
    const long long *offs;
    const long long *eoffs;
    const double *Epack;
    __device__ __forceinline__ long long off(long long p) const { return offs[list[p]]; }
    __device__ __forceinline__ const double *e(long long p) const { return Epack + eoffs[list[p]]; }
};

// Copy src[0 .. cnt) (global memory, T-aligned) to dst (shared memory): the
// 16-byte-aligned middle of the range with vector loads (float4 / double2),
// the ragged ends element by element.  Every thread of the block calls it.
template <typename T>
__device__ __forceinline__ void stage_range(T *dst, const T *__restrict__ src, int cnt)
{
    using Vec = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    constexpr int V = (int)(sizeof(Vec) / sizeof(T));
    const int mis = (int)(((16 - ((size_t)src & 15)) & 15) / sizeof(T));
    const int head = mis < cnt ? mis : cnt;
    const int nvec = (cnt - head) / V;
    for (int e = threadIdx.x; e < head; e += blockDim.x) dst[e] = src[e];
    const Vec *sv = reinterpret_cast<const Vec *>(src + head);
    for (int w = threadIdx.x; w < nvec; w += blockDim.x) {
        const Vec q = sv[w];
        T *d = dst + head + w * V;
        if constexpr (V == 2) {
            d[0] = q.x;
            d[1] = q.y;
        } else {
            d[0] = q.x;
            d[1] = q.y;
            d[2] = q.z;
            d[3] = q.w;
        }
    }
    for (int e = head + nvec * V + threadIdx.x; e < cnt; e += blockDim.x) dst[e] = src[e];
}

// Stage the x (and v) of the points p0 .. p0+npts-1 into shared memory and
// build their per-point value tables (the FP64 islands).  Every thread of the
// block calls it; it ends with the block synchronised.
template <typename T, typename IO, int FN, bool HVP, typename PM>
__device__ __forceinline__ void point_prologue(const Job &a, const PM &pm, unsigned char *smem_raw, const Smem<T> &L,
                                               long long p0, int npts)
{
    const int n = a.n;
    const int tid = threadIdx.x;
    T *xs = reinterpret_cast<T *>(smem_raw + L.xs);
    T *vs = reinterpret_cast<T *>(smem_raw + L.vs);
    {
        const IO *X = reinterpret_cast<const IO *>(a.x);
        const IO *V = reinterpret_cast<const IO *>(a.v);
        const int cnt = npts * n;
        if constexpr (std::is_same<PM, ContigPoints>::value && std::is_same<IO, T>::value) {
            // the block's points are one contiguous range of x and v
            stage_range<T>(xs, X + pm.off(p0), cnt);
            if (HVP) stage_range<T>(vs, V + pm.off(p0), cnt);
        } else {
            for (int e = tid; e < cnt; e += blockDim.x) {
                const int q = e / n, k = e - q * n;
                const long long o = pm.off(p0 + q) + k;
                xs[e] = (T)X[o];
                if (HVP) vs[e] = (T)V[o];
            }
        }
    }
    __syncthreads();

    if (FN == FN_ACKLEY) {
        AckEnt<T> *tab = reinterpret_cast<AckEnt<T> *>(smem_raw + L.t1);
        T *sc = reinterpret_cast<T *>(smem_raw + L.sc);
        const int cnt = npts * n;
        for (int e = tid; e < cnt; e += blockDim.x) {
            T s, c;
            if (sizeof(T) == 8) {
                double sd, cd;
                sincospi(2.0 * (double)xs[e], &sd, &cd);
                s = (T)sd;
                c = (T)cd;
            } else {
                float sf, cf;
                sincospif(2.0f * (float)xs[e], &sf, &cf);
                s = (T)sf;
                c = (T)cf;
            }
            AckEnt<T> ent;
            ent.x = xs[e];
            ent.d1 = T(-2.0 * CUDART_PI) * s;
            ent.d2 = T(-4.0 * CUDART_PI * CUDART_PI) * c;
            ent.pad = T(0);
            const int q = e / n, k = e - q * n;
            tab[2 * q * n + k] = ent;
            tab[2 * q * n + n + k] = ent;
        }
        __syncthreads();
        // One warp per point: S = sum x^2 and C = sum cos(2 pi x) in FP64.
        const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
        for (int q = warp; q < npts; q += nw) {
            double S = 0.0, Cv = 0.0;
            for (int k = lane; k < n; k += 32) {
                const double xv = (double)xs[q * n + k];
                S = fma(xv, xv, S);
                Cv += (double)tab[2 * q * n + k].d2 * (-1.0 / (4.0 * CUDART_PI * CUDART_PI));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                S += __shfl_xor_sync(0xffffffffu, S, off);
                Cv += __shfl_xor_sync(0xffffffffu, Cv, off);
            }
            if (lane == 0) {
                T *o = sc + q * kAckScal;
                if (sizeof(T) == 8) {
                    const double nn = (double)n;
                    const double a0 = S / nn;
                    const double sq = sqrt(a0);
                    o[0] = (T)S;
                    o[1] = (T)Cv;
                    o[2] = (T)(1.0 / nn);
                    o[3] = (T)sq;                        // sqrt at S/n
                    o[4] = (T)(0.5 / sq);                // its first derivative
                    o[5] = (T)(-0.25 / (sq * a0));       // its second derivative
                    o[6] = (T)exp(-0.2 * sq);            // exp at -0.2 sqrt(S/n)
                    o[7] = (T)exp(Cv / nn);              // exp at C/n
                } else {
                    // The sums are FP64 (the island); the scalar functions of
                    // them only feed FP32 arithmetic, so they are evaluated in
                    // FP32 from the correctly rounded arguments, off the slow
                    // FP64 pipe.
                    const float a0 = (float)(S / (double)n);
                    const float sq = sqrtf(a0);
                    o[0] = (T)S;
                    o[1] = (T)Cv;
                    o[2] = (T)(1.0f / (float)n);
                    o[3] = (T)sq;
                    o[4] = (T)(0.5f / sq);
                    o[5] = (T)(-0.25f / (sq * a0));
                    o[6] = (T)expf(-0.2f * sq);
                    o[7] = (T)expf((float)(Cv / (double)n));
                }
            }
        }
        __syncthreads();
    } else if (FN == FN_FP) {
        T *ts = reinterpret_cast<T *>(smem_raw + L.t1);
        T *tc = reinterpret_cast<T *>(smem_raw + L.t2);
        T *res = reinterpret_cast<T *>(smem_raw + L.res);
        double *ds = reinterpret_cast<double *>(smem_raw + L.dsin);
        double *dc = reinterpret_cast<double *>(smem_raw + L.dcos);
        const int cnt = npts * n;
        for (int e = tid; e < cnt; e += blockDim.x) {
            double sd, cd;
            sincos((double)xs[e], &sd, &cd);
            ds[e] = sd;
            dc[e] = cd;
            ts[e] = (T)sd;
            tc[e] = (T)cd;
        }
        __syncthreads();
        // r_m = E_m - sum_j (A_mj sin x_j + B_mj cos x_j), FP64, one (point, m)
        // pair per thread.
        for (int e = tid; e < cnt; e += blockDim.x) {
            const int q = e / n, m = e - q * n;
            const double *Ar = a.A + (size_t)m * a.ld;
            const double *Br = a.B + (size_t)m * a.ld;
            const double *sq = ds + q * n;
            const double *cq = dc + q * n;
            double s = 0.0;
            for (int j = 0; j < n; ++j) s = fma(Ar[j], sq[j], fma(Br[j], cq[j], s));
            res[e] = (T)(pm.e(p0 + q)[m] - s);
        }
        __syncthreads();
    }
}

// Fletcher-Powell on hDuals for one (row i, chunk at cstart):
// f = sum_m r_m^2, r_m = E_m - sum_j (A_mj sin y_j + B_mj cos y_j).  A and B
// stream through shared memory in tiles of mt rows, stored transposed
// ([j][m]) so a thread reads MB consecutive rows per j; MB residual hDuals are
// accumulated in registers at once so each seeded y_j serves MB rows.  The
// tile loads are block-wide: every thread of the block makes the same calls
// (threads without a sweep pass has = false); with a single tile the load
// happens only when `reload` is set.
// MB consecutive shared-memory values starting at an element offset that is
// a multiple of MB from a 16-byte-aligned base (the A/B tile rows), read with
// the widest vector loads that alignment allows.
template <typename T, int MB>
__device__ __forceinline__ void load_rows(const T *__restrict__ p, T (&r)[MB])
{
    if constexpr (sizeof(T) == 4 && MB % 4 == 0) {
#pragma unroll
        for (int u = 0; u < MB; u += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(p + u);
            r[u] = q.x;
            r[u + 1] = q.y;
            r[u + 2] = q.z;
            r[u + 3] = q.w;
        }
    } else if constexpr (sizeof(T) == 4 && MB % 2 == 0) {
#pragma unroll
        for (int u = 0; u < MB; u += 2) {
            const float2 q = *reinterpret_cast<const float2 *>(p + u);
            r[u] = q.x;
            r[u + 1] = q.y;
        }
    } else if constexpr (sizeof(T) == 8 && MB % 2 == 0) {
#pragma unroll
        for (int u = 0; u < MB; u += 2) {
            const double2 q = *reinterpret_cast<const double2 *>(p + u);
            r[u] = q.x;
            r[u + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int u = 0; u < MB; ++u) r[u] = p[u];
    }
}

template <typename T, int C, int MB, bool kRemap, bool kSparse>
__device__ __forceinline__ HD<T, C> fp_sweep(const Job &a, unsigned char *smem_raw, const Smem<T> &L, const T *xq,
                                             const T *ts, const T *tc, const T *res, int i, int cstart, bool has,
                                             bool reload)
{
    const int n = a.n;
    const int tid = threadIdx.x;
    T *At = reinterpret_cast<T *>(smem_raw + L.at);
    T *Bt = reinterpret_cast<T *>(smem_raw + L.bt);
    const int mt = a.mt;
    const int ntiles = (n + mt - 1) / mt;
    TermSum<T, C, IsComp<T>::value> acc;
    acc.init();
    for (int tile = 0; tile < ntiles; ++tile) {
        const int m0 = tile * mt;
        if (ntiles > 1 || reload) {
            __syncthreads();
            const int cnt = mt * n;
            for (int e = tid; e < cnt; e += blockDim.x) {
                const int mm = e / n, jj = e - mm * n;
                const int m = m0 + mm;
                T av = T(0), bv = T(0);
                if (m < n) {
                    av = (T)a.A[(size_t)m * a.ld + jj];
                    bv = (T)a.B[(size_t)m * a.ld + jj];
                }
                At[jj * mt + mm] = av;
                Bt[jj * mt + mm] = bv;
            }
            __syncthreads();
        }
        if (!has) continue;
        const int mend = min(m0 + mt, n);
        for (int mb = m0; mb < mend; mb += MB) {
            HD<T, C> s[MB];
#pragma unroll
            for (int u = 0; u < MB; ++u) s[u] = hzero<T, C>();
            for_each_seed<T, C, 16, kRemap, kSparse>(xq, n, i, cstart, [&](int jv, const HD<T, C> &y) {
                const T sj = ts[jv], cj = tc[jv];
                T ar[MB], br[MB];
                load_rows<T, MB>(At + jv * mt + (mb - m0), ar);
                load_rows<T, MB>(Bt + jv * mt + (mb - m0), br);
                // sin(y_j) and cos(y_j) once per j (unary rule), then
                // s_m += A_mj sin(y_j) + B_mj cos(y_j) for the MB rows.
                const HD<T, C> sy = unary(y, sj, cj, -sj);
                const HD<T, C> cy = unary(y, cj, -sj, -cj);
#pragma unroll
                for (int u = 0; u < MB; ++u) {
                    sfma<false>(s[u], ar[u], sy);
                    sfma<false>(s[u], br[u], cy);
                }
            });
#pragma unroll
            for (int u = 0; u < MB; ++u) {
                if (mb + u < mend) {
                    HD<T, C> rr = rsub(T(0), s[u]);
                    rr.v = res[mb + u];  // E_m - sum_j (...)  (FP64 island)
                    acc.add_sq(rr);
                }
            }
        }
    }
    return acc.value();
}

// Per-point table pointers of staged point q.
template <typename T>
struct PointTables {
    const T *x, *v, *t1, *t2, *sc, *res;
    const AckEnt<T> *ack;
    __device__ __forceinline__ PointTables(unsigned char *smem_raw, const Smem<T> &L, int q, int n)
    {
        x = reinterpret_cast<const T *>(smem_raw + L.xs) + q * n;
        v = reinterpret_cast<const T *>(smem_raw + L.vs) + q * n;
        t1 = reinterpret_cast<const T *>(smem_raw + L.t1) + q * n;
        t2 = reinterpret_cast<const T *>(smem_raw + L.t2) + q * n;
        ack = reinterpret_cast<const AckEnt<T> *>(smem_raw + L.t1) + 2 * q * n;
        sc = reinterpret_cast<const T *>(smem_raw + L.sc) + q * kAckScal;
        res = reinterpret_cast<const T *>(smem_raw + L.res) + q * n;
    }
};

// f's hDual for (row i, chunk at cstart) of a staged point.  Rosenbrock and
// Ackley sweeps are per-thread; Fletcher-Powell's is block-uniform (see
// fp_sweep), so every thread calls this with the same trip counts.
template <typename T, int C, int FN, int MB, bool kRemap, bool kSparse = false>
__device__ __forceinline__ HD<T, C> row_chunk(const Job &a, unsigned char *smem_raw, const Smem<T> &L,
                                              const PointTables<T> &pt, int i, int cstart, bool has, bool reload)
{
    if constexpr (FN == FN_ROSENBROCK) {
        if (has) return rosenbrock_sweep<T, C, kRemap, kSparse>(pt.x, a.n, i, cstart);
        return hzero<T, C>();
    } else if constexpr (FN == FN_ACKLEY) {
        if (has) return ackley_sweep<T, C, kRemap, kSparse>(pt.ack, pt.sc, a.n, i, cstart);
        return hzero<T, C>();
    } else {
        return fp_sweep<T, C, MB, kRemap, kSparse>(a, smem_raw, L, pt.x, pt.t1, pt.t2, pt.res, i, cstart, has, reload);
    }
}

// T is the arithmetic type of the sweep, IO the element type of x, v and the
// output (IO = T except for the one-variable compensated-FP32 case, which
// computes in FP64 with float I/O).  Every thread of the block must call it
// (it synchronises the block).  CHESS-VEC / CHUNK-HESS (Alg. 7 / Alg. 5):
// every chunk of every row is evaluated.
template <typename T, typename IO, int C, int FN, bool HVP, int MB, typename PM>
__device__ __forceinline__ void block_sweeps(const Job &a, const PM &pm, unsigned char *smem_raw)
{
    const int n = a.n;
    const Smem<T> L = smem_layout<T>(FN, HVP, n, a.maxpts, a.mt);

    const int rows_per_block = blockDim.x / a.tpr;
    const long long p0 = a.row0 / n;
    long long plast = (a.row0 + rows_per_block - 1) / n;
    if (plast > a.npoints - 1) plast = a.npoints - 1;
    const int npts = (int)(plast - p0 + 1);
    const int tid = threadIdx.x;

    point_prologue<T, IO, FN, HVP>(a, pm, smem_raw, L, p0, npts);

    // ---- this thread's (point, row, lane)
    const long long row = a.row0 + tid / a.tpr;
    const int r = tid % a.tpr;
    const long long p = row / n;
    const int i = (int)(row - p * n);
    const bool active = p < a.npoints;
    const int q = active ? (int)(p - p0) : 0;
    const PointTables<T> pt(smem_raw, L, q, n);

    using Dot = typename std::conditional<IsComp<T>::value, CSum, T>::type;
    Dot dot;
    if constexpr (IsComp<T>::value) {
        dot.s = 0.f;
        dot.e = 0.f;
    } else {
        dot = T(0);
    }

    // Uniform trip count for the block-wide Fletcher-Powell tiles; the other
    // functions simply skip the iterations a lane has no chunk for.
    const int iters = (a.nch + a.tpr - 1) / a.tpr;
    for (int it = 0; it < iters; ++it) {
        const int j = r + it * a.tpr;
        const bool has = j < a.nch;
        if (FN != FN_FP && !has) break;
        const int cstart = j * C;
        // One lane per row: a warp's lanes share the chunk, the three-segment
        // loop is cheapest.  Several lanes per row: lanes differ in chunk,
        // the uniform-trip-count loop keeps them converged.
        const HD<T, C> f = (a.tpr == 1) ? row_chunk<T, C, FN, MB, false>(a, smem_raw, L, pt, i, cstart, has, it == 0)
                                        : row_chunk<T, C, FN, MB, true>(a, smem_raw, L, pt, i, cstart, has, it == 0);
        if (!has) continue;
        if constexpr (HVP) {
#pragma unroll
            for (int l = 0; l < C; ++l) {
                if (cstart + l < n) {
                    if constexpr (IsComp<T>::value) cdot_add(dot, f.h[l], pt.v[cstart + l]);
                    else dot = fma_(f.h[l], pt.v[cstart + l], dot);
                }
            }
        } else if (active) {
            IO *H = reinterpret_cast<IO *>(a.out) + (pm.off(p) + i) * n;
#pragma unroll
            for (int l = 0; l < C; ++l)
                if (cstart + l < n) H[cstart + l] = (IO)f.h[l];
        }
    }

    if constexpr (HVP) {
        // Sum the tpr lanes of the row (aligned groups inside one warp).
        IO *O = reinterpret_cast<IO *>(a.out);
        if constexpr (IsComp<T>::value) {
            for (int off = a.tpr >> 1; off > 0; off >>= 1) {
                CSum o;
                o.s = __shfl_xor_sync(0xffffffffu, dot.s, off);
                o.e = __shfl_xor_sync(0xffffffffu, dot.e, off);
                dot = csum_merge(dot, o);
            }
            if (active && r == 0) O[pm.off(p) + i] = (IO)csum_value(dot);
        } else {
            for (int off = a.tpr >> 1; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
            if (active && r == 0) O[pm.off(p) + i] = (IO)dot;
        }
    }
}

// ------------------------------------------------------------------ kernel
// One launch over a contiguous batch: block b handles rows
// [b * blockDim/tpr, (b+1) * blockDim/tpr) of the batch's row space.
template <typename T, typename IO, int C, int FN, bool HVP, int MB>
__global__ void __launch_bounds__(256, 1) sweep_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Job job;
    job.x = a.x;
    job.v = a.v;
    job.out = a.out;
    job.A = a.A;
    job.B = a.B;
    job.npoints = a.batch;
    job.row0 = (long long)blockIdx.x * (blockDim.x / a.tpr);
    job.n = a.n;
    job.nch = a.nch;
    job.tpr = a.tpr;
    job.maxpts = a.maxpts;
    job.mt = a.mt;
    job.ld = a.ld;
    ContigPoints pm{a.E, a.n};
    block_sweeps<T, IO, C, FN, HVP, MB>(job, pm, smem_raw);
}

// ------------------------------------------------------------------ symmetric
// (items and staging layout: sym_layout.cuh)
template <typename T>
__host__ __device__ inline size_t sym_hs_bytes(int n, int C)
{
    return align_up((size_t)sym_hs_elems(n, C) * sizeof(T), 16);
}

template <typename T, typename IO, int C, int FN, bool HVP, int MB, bool kSparse = false>
__global__ void __launch_bounds__(256, 1) sym_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n;
    const int ppb = a.maxpts;  // points per block
    const int tpp = a.tpp;     // threads per point
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

    const int tid = threadIdx.x;
    const int q = tid / tpp, t = tid - q * tpp;
    const bool active = q < npts;
    const long long p = p0 + (active ? q : 0);
    const PointTables<T> pt(smem_raw, L, active ? q : 0, n);
    T *Hs = reinterpret_cast<T *>(smem_raw + align_up(L.total, 16) + (size_t)(active ? q : 0) * sym_hs_bytes<T>(n, C));
    // Accumulator form of the HVP (points whose chunk matrix does not fit
    // shared memory): one FP64 accumulator per row of each staged point, and
    // a per-iteration stage of every thread's chunk (see below).
    double *accs_all = reinterpret_cast<double *>(smem_raw + align_up(L.total, 16));
    double *accs = accs_all + (size_t)(active ? q : 0) * n;
    const bool acc_form = HVP && a.sym_acc;
    SymStage<T, C> stage(smem_raw + align_up(L.total, 16) + align_up((size_t)ppb * n * sizeof(double), 16),
                         (int)blockDim.x);
    if (acc_form) {
        for (int e = tid; e < npts * n; e += blockDim.x) accs_all[e] = 0.0;
        __syncthreads();
    }

    const int nch = a.nch;
    const int items = C * nch * (nch + 1) / 2;
    const int iters = (items + tpp - 1) / tpp;
    for (int it = 0; it < iters; ++it) {
        const int k = t + it * tpp;
        int i = 0, cn = 0;
        bool has = active && k < items;
        if (has) {
            sym_item(k, C, nch, i, cn);
            has = i < n;
        }
        if (FN != FN_FP && !has && !acc_form) continue;
        const int cstart = cn * C;
        const HD<T, C> f = row_chunk<T, C, FN, MB, true, kSparse>(job, smem_raw, L, pt, i, cstart, has, it == 0);
        if constexpr (HVP) {
            if (acc_form) {
                // Alg. 8's two updates, r_i += sum_l H_il v_l and, off the
                // diagonal chunk, r_l += H_il v_i, made reproducible: every
                // thread stages its chunk and its row dot (FP64; products of
                // two FP32 values are exact there), then each thread adds, for
                // the rows it owns, the staged contributions of its point's
                // threads in thread order.
                double own = 0.0;
                if (has) {
#pragma unroll
                    for (int l = 0; l < C; ++l)
                        if (cstart + l < n) own = fma((double)f.h[l], (double)pt.v[cstart + l], own);
                }
                stage.put(tid, f.h, own, has ? i : -1, cn);
                __syncthreads();
                if (active) {
                    const int t0 = q * tpp;
                    for (int srow = t; srow < n; srow += tpp) {
                        const int scn = srow / C, sl = srow - scn * C;
                        double acc = accs[srow];
                        for (int u = 0; u < tpp; ++u) {
                            const int ui = stage.row(t0 + u);
                            if (ui < 0) continue;
                            if (ui == srow) acc += stage.own(t0 + u);
                            const int ucn = stage.chunk(t0 + u);
                            if (ucn == scn && ucn > ui / C)
                                acc += (double)stage.h(t0 + u, sl) * (double)pt.v[ui];
                        }
                        accs[srow] = acc;
                    }
                }
                __syncthreads();
                continue;
            }
            if (!has) continue;
            T *hrow = Hs + sym_hs_row(i, n, C) - (i / C) * C;
#pragma unroll
            for (int l = 0; l < C; ++l)
                if (cstart + l < n) hrow[cstart + l] = f.h[l];
        } else {
            if (!has) continue;
            IO *H = reinterpret_cast<IO *>(a.out) + (size_t)p * n * n;
            const bool mirror = cn > i / C;
#pragma unroll
            for (int l = 0; l < C; ++l) {
                const int j = cstart + l;
                if (j < n) {
                    H[(size_t)i * n + j] = (IO)f.h[l];
                    if (mirror) H[(size_t)j * n + i] = (IO)f.h[l];
                }
            }
        }
    }

    if constexpr (HVP) {
        // r_s = sum_j H_sj v_j over the staged chunks: entries right of row
        // s's diagonal chunk from row s, entries left of it from column s
        // (H_sj = H_js), so every off-diagonal-chunk entry serves both r_i and
        // r_s as in Alg. 8.
        __syncthreads();
        if (active && acc_form) {
            IO *O = reinterpret_cast<IO *>(a.out) + (size_t)p * n;
            for (int srow = t; srow < n; srow += tpp) O[srow] = (IO)accs[srow];
        } else if (active) {
            const T *Hq = Hs;
            IO *O = reinterpret_cast<IO *>(a.out) + (size_t)p * n;
            for (int srow = t; srow < n; srow += tpp) {
                const int dstart = (srow / C) * C;
                const T *own = Hq + sym_hs_row(srow, n, C) - dstart;  // own[j], j >= dstart
                if constexpr (IsComp<T>::value) {
                    CSum d{0.f, 0.f};
                    for (int j = 0; j < dstart; ++j) cdot_add(d, Hq[sym_hs_row(j, n, C) + srow - (j / C) * C], pt.v[j]);
                    for (int j = dstart; j < n; ++j) cdot_add(d, own[j], pt.v[j]);
                    O[srow] = (IO)csum_value(d);
                } else {
                    T d = T(0);
                    for (int j = 0; j < dstart; ++j) d = fma_(Hq[sym_hs_row(j, n, C) + srow - (j / C) * C], pt.v[j], d);
                    for (int j = dstart; j < n; ++j) d = fma_(own[j], pt.v[j], d);
                    O[srow] = (IO)d;
                }
            }
        }
    }
}

// Host-side launch helpers: compute the layout, opt into large dynamic
// shared memory once per (kernel, device), launch, report the error.  The
// per-device record of the limit already set only grows, and it is read and
// raised under one lock, so launches from several host threads never see the
// limit lowered under them.
inline std::mutex &smem_attr_mutex()
{
    static std::mutex mu;
    return mu;
}

template <typename K>
cudaError_t opt_in_smem(K kern, size_t bytes, std::atomic<int> *configured)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (configured[dev].load(std::memory_order_acquire) >= (int)bytes) return cudaSuccess;
    std::lock_guard<std::mutex> lk(smem_attr_mutex());
    if (configured[dev].load(std::memory_order_relaxed) >= (int)bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) configured[dev].store((int)bytes, std::memory_order_release);
    return e;
}

template <typename T, typename IO, int C, int FN, bool HVP, int MB>
cudaError_t launch_sweep(SweepArgs a, int block_threads, cudaStream_t stream)
{
    const Smem<T> L = smem_layout<T>(FN, HVP, a.n, a.maxpts, a.mt);
    auto kern = sweep_kernel<T, IO, C, FN, HVP, MB>;
    static std::atomic<int> configured[64];
    cudaError_t e = opt_in_smem(kern, L.total, configured);
    if (e != cudaSuccess) return e;
    const long long threads = a.batch * (long long)a.tpp;
    const long long blocks = (threads + block_threads - 1) / block_threads;
    kern<<<(unsigned)blocks, block_threads, L.total, stream>>>(a);
    return cudaGetLastError();
}

// Symmetric launch: a.maxpts = points per block, a.tpp = threads per point.
template <typename T, typename IO, int C, int FN, bool HVP, int MB>
size_t sym_smem_bytes(const SweepArgs &a)
{
    const Smem<T> L = smem_layout<T>(FN, HVP, a.n, a.maxpts, a.mt);
    if (HVP && a.sym_acc)
        return align_up(L.total, 16) + align_up((size_t)a.maxpts * a.n * sizeof(double), 16) +
               (size_t)SymStage<T, C>::bytes(a.maxpts * a.tpp);
    return align_up(L.total, 16) + (HVP ? (size_t)a.maxpts * sym_hs_bytes<T>(a.n, C) : 0);
}

template <typename T, typename IO, int C, int FN, bool HVP, int MB, bool kSparse = false>
cudaError_t launch_sym(SweepArgs a, cudaStream_t stream)
{
    const size_t bytes = sym_smem_bytes<T, IO, C, FN, HVP, MB>(a);
    auto kern = sym_kernel<T, IO, C, FN, HVP, MB, kSparse>;
    static std::atomic<int> configured[64];
    cudaError_t e = opt_in_smem(kern, bytes, configured);
    if (e != cudaSuccess) return e;
    const long long blocks = (a.batch + a.maxpts - 1) / a.maxpts;
    kern<<<(unsigned)blocks, a.maxpts * a.tpp, bytes, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace chessfad
