// sym_layout.cuh -- the symmetric method's work items and the compact
// staging layout of a point's chunk matrix; shared by the built-in sweep
// kernels and the run-time-compiled user-function kernels.
#pragma once

namespace chessfad {

// ------------------------------------------------------------------ symmetric
// SCHUNK-HESS (Alg. 6) and SC-HESS-VEC (Alg. 8): a row evaluates only the
// chunks from its diagonal chunk on.  The items of one point are the pairs
// (row i, chunk cn) with cn >= floor(i/C), enumerated by chunk-block pairs
// (R, cn), R <= cn, in row-major order and within a pair by row offset;
// C * nch (nch + 1) / 2 items per point (rows beyond n in the last chunk row
// are empty items).  A block holds `ppb` points with `tpp` threads each; a
// point's items are dealt round-robin to its threads.
__device__ __forceinline__ void sym_item(int k, int C, int nch, int &i, int &cn)
{
    int b = k / C;
    const int rho = k - b * C;
    int R = 0, cnt = nch;
    while (b >= cnt) {
        b -= cnt;
        ++R;
        --cnt;
    }
    i = R * C + rho;
    cn = R + b;
}

// Staged chunk matrix of one point (HVP), compact: row i (chunk row
// R = i / C, offset rho) keeps columns R*C .. n-1 plus one pad element, so rows
// of a chunk row have an odd-friendly stride n - R*C + 1 and column reads
// across lanes hit distinct banks.
__host__ __device__ inline long long sym_hs_row(int i, int n, int C)
{
    const long long R = i / C, rho = i - R * C;
    return C * (R * (n + 1) - C * R * (R - 1) / 2) + rho * (n - R * C + 1);
}

__host__ __device__ inline long long sym_hs_elems(int n, int C)
{
    const long long nch = (n + C - 1) / C;
    return C * (nch * (n + 1) - C * nch * (nch - 1) / 2);
}

// Per-iteration stage of the symmetric HVP's accumulator form (points whose
// chunk matrix does not fit shared memory).  Alg. 8 lets every entry H_il
// right of row i's diagonal chunk update both r_i and r_l; on the GPU many
// threads produce entries of the same row at once, so, to add them in an
// order that does not depend on timing, every thread stages its chunk
// h[0..C) (component-major: the writes of a warp are conflict-free), its row
// dot sum_l h_l v_(cstart+l) (FP64), its row (-1: no item) and its chunk;
// after a barrier each thread adds, for the rows it owns, the staged
// contributions of its point's threads in thread order.
template <typename T, int C>
struct SymStage {
    unsigned char *base;
    int threads;
    __host__ __device__ static inline unsigned long long hs_bytes(int threads)
    {
        return ((unsigned long long)threads * C * sizeof(T) + 15) / 16 * 16;
    }
    __host__ __device__ static inline unsigned long long bytes(int threads)
    {
        return hs_bytes(threads) + (unsigned long long)threads * (sizeof(double) + 2 * sizeof(int));
    }
    __device__ __forceinline__ SymStage(unsigned char *p, int nthreads) : base(p), threads(nthreads) {}
    __device__ __forceinline__ T *hs() const { return reinterpret_cast<T *>(base); }
    __device__ __forceinline__ double *owns() const { return reinterpret_cast<double *>(base + hs_bytes(threads)); }
    __device__ __forceinline__ int *ids() const { return reinterpret_cast<int *>(owns() + threads); }
    __device__ __forceinline__ void put(int tid, const T *h, double own, int i, int cn) const
    {
#pragma unroll
        for (int l = 0; l < C; ++l) hs()[(unsigned long long)l * threads + tid] = h[l];
        owns()[tid] = own;
        ids()[2 * tid] = i;
        ids()[2 * tid + 1] = cn;
    }
    __device__ __forceinline__ T h(int tid, int l) const { return hs()[(unsigned long long)l * threads + tid]; }
    __device__ __forceinline__ double own(int tid) const { return owns()[tid]; }
    __device__ __forceinline__ int row(int tid) const { return ids()[2 * tid]; }
    __device__ __forceinline__ int chunk(int tid) const { return ids()[2 * tid + 1]; }
};

}  // namespace chessfad
