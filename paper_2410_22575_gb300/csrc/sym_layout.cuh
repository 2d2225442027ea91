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

}  // namespace chessfad
