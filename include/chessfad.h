/*
 * chessfad.h -- C ABI of the GB300 (sm_103a) chunked-hDual Hessian /
 * Hessian-vector-product library.
 *
 * The method is CHESSFAD (Ranjan & Zubair, arXiv:2410.22575): forward-mode
 * AD on "hDual" numbers that carry a value, the derivative with respect to
 * the Hessian row variable x_i, the derivatives with respect to a contiguous
 * chunk of csize variables, and the csize second derivatives
 * d2f/dx_i dx_{cstart+l} (Sec. III-B, Sec. IV / Fig. 1).  One evaluation of f
 * on seeded hDuals (CHUNK-INIT, Alg. 4) yields one chunk of one Hessian row;
 * n * ceil(n/csize) evaluations give the whole Hessian (CHUNK-HESS, Alg. 5),
 * and each chunk, dotted with the matching slice of v and summed over the
 * row, gives (H v)_i (CHESS-VEC, Alg. 7; Sec. III-C).  The library evaluates
 * this at many independent points at once, the paper's L0/L1/L2 parallelism
 * over (point, row, chunk) (Sec. VI, Alg. 9, Alg. 10, Fig. 2).
 *
 * Conventions for every call below:
 *  - Pointers named "device" must point to device memory of the current
 *    device; the caller owns every buffer.  The compute calls allocate no
 *    memory, never synchronise the host, and are ordered on `stream`
 *    (NULL = the legacy default stream).
 *  - Layout is point-major and row-major: x, v, out are [batch][n]; a
 *    Hessian is [batch][n][n].  Outputs are overwritten, never accumulated.
 *  - Precision CHESSFAD_FP64: x, v, out, H are double and all arithmetic is
 *    FP64.  CHESSFAD_FP32_COMP: x, v, out, H are float; the hDual arithmetic
 *    runs in FP32 with FMA, the row-times-v products and the reductions over
 *    a function's terms use error-free transformations (TwoProd by FMA,
 *    TwoSum), and the sums whose cancellation matters -- the Fletcher-Powell
 *    residuals E_m - sum_j(...) and the Ackley sums under sqrt and exp -- are
 *    computed in FP64 once per point.  Fletcher-Powell A, B, E are always
 *    double.
 *  - csize (the chunk size) must be one of 1, 2, 4, 8, 16, 32, or 0 for
 *    "choose for me" (the autotuned table entry for (function, n, precision)
 *    if one exists, else a default).  It need not divide n: the last chunk is
 *    ragged and its positions beyond n are never seeded.
 *  - 1 <= n <= CHESSFAD_MAX_N.  batch == 0 is a valid no-op; batch < 0 is an
 *    error.  NaN and Inf inputs propagate; they are not trapped.  The
 *    Ackley Hessian is undefined where sum x_k^2 == 0 (sqrt at 0); the
 *    library returns whatever the hDual sqrt rule gives there (Inf/NaN).
 *  - Return value: CHESSFAD_SUCCESS (0) or a negative CHESSFAD_ERR_* code;
 *    chessfad_strerror() names it.  Argument errors are detected on the host
 *    before anything is launched.  CHESSFAD_ERR_CUDA reports a launch or
 *    runtime error taken from the CUDA runtime.
 */
#ifndef CHESSFAD_H
#define CHESSFAD_H

#include <stddef.h>

#if defined(__GNUC__)
#define CHESSFAD_API __attribute__((visibility("default")))
#else
#define CHESSFAD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t is `struct CUstream_st *` */
typedef struct CUstream_st *chessfad_stream_t;

/* Test functions (named in Sec. VII of the paper). */
#define CHESSFAD_ROSENBROCK 0      /* f = sum_{k<n-1} 100(x_{k+1}-x_k^2)^2 + (1-x_k)^2 */
#define CHESSFAD_ACKLEY 1          /* f = -20 exp(-0.2 sqrt(sum x^2/n)) - exp(sum cos(2 pi x)/n) + 20 + e */
#define CHESSFAD_FLETCHER_POWELL 2 /* f = sum_m (E_m - sum_j (A_mj sin x_j + B_mj cos x_j))^2 */

/* Precisions. */
#define CHESSFAD_FP64 0
#define CHESSFAD_FP32_COMP 1

#define CHESSFAD_MAX_N 512

/* Status codes. */
#define CHESSFAD_SUCCESS 0
#define CHESSFAD_ERR_FUNCTION (-1)  /* unknown function id */
#define CHESSFAD_ERR_SIZE (-2)      /* n < 1 or n > CHESSFAD_MAX_N */
#define CHESSFAD_ERR_BATCH (-3)     /* batch < 0, or a batch whose launch grid would exceed 2^31 - 1 blocks */
#define CHESSFAD_ERR_CHUNK (-4)     /* csize not in {0,1,2,4,8,16,32} */
#define CHESSFAD_ERR_NULL (-5)      /* a required pointer is NULL */
#define CHESSFAD_ERR_PARAMS (-6)    /* Fletcher-Powell parameters missing or ld < n */
#define CHESSFAD_ERR_PRECISION (-7) /* unknown precision */
#define CHESSFAD_ERR_WORKSPACE (-8) /* workspace missing or too small */
#define CHESSFAD_ERR_CONFIG (-9)    /* launch configuration out of range */
#define CHESSFAD_ERR_CUDA (-10)     /* CUDA runtime / launch error */
#define CHESSFAD_ERR_PLAN (-11)     /* ragged plan invalid or built for another precision */
#define CHESSFAD_ERR_JIT (-12)      /* user function: NVRTC unavailable or the source did not compile */

/* Fletcher-Powell parameters, shared by the whole batch.  A, B: device,
 * double, row-major with leading dimension ld >= n; the leading n x n block
 * is used.  E: device, double, n entries.  Passed by host pointer. */
typedef struct {
    const double *A;
    const double *B;
    const double *E;
    int ld;
} chessfad_fp_params;

/* Methods. */
#define CHESSFAD_METHOD_PLAIN 0     /* every chunk of every row: CHUNK-HESS (Alg. 5), CHESS-VEC (Alg. 7) */
#define CHESSFAD_METHOD_SYMMETRIC 1 /* only chunks from the row's diagonal chunk on: SCHUNK-HESS (Alg. 6),
                                       SC-HESS-VEC (Alg. 8); about half the evaluations of f (Sec. V) */
#define CHESSFAD_METHOD_SYMMETRIC_SPARSE 2 /* the symmetric method with seed-sparse propagation: an
                                       evaluation of f visits only the variables whose CHUNK-INIT seed
                                       has a nonzero derivative part (x_i and the chunk; for
                                       Rosenbrock the terms touching them).  The others add to
                                       value components only, which are per-point constants.  This
                                       departs from the paper's dense arithmetic: the result equals
                                       the dense one for finite inputs, but NaN/Inf in the skipped
                                       variables does not reach the derivatives.  csize 4, 8 or 16;
                                       never chosen by the autotuner. */
#define CHESSFAD_METHOD_POINT 3     /* the L0 decomposition (L0-HESS-VEC, Alg. 9): one thread per
                                       point sweeps every chunk of every row (CHESS-VEC, Alg. 7 /
                                       CHUNK-HESS, Alg. 5); block_threads points per CTA; csize
                                       1..16; the same arithmetic, in the same order per row, as
                                       the plain method with one thread per row, so the results
                                       are identical.  Never chosen by the autotuner. */

/* Launch configuration of the (point, row, chunk) decomposition.
 *   csize             chunk size, 1..32 power of two
 *   threads_per_row   plain method: lanes sharing one Hessian row (power of
 *                     two, 1..32); lane r of a row evaluates chunks r, r+tpr,
 *                     ... and the row sum is finished by warp shuffles
 *                     (Sec. VI, Fig. 2 does this through shared memory)
 *   method            CHESSFAD_METHOD_PLAIN, _SYMMETRIC, _SYMMETRIC_SPARSE or _POINT
 *   block_threads     plain method: CTA size, multiple of 32, 32..256;
 *                     symmetric method: the CTA holds
 *                     block_threads / threads_per_point points (at least
 *                     one; fewer when the staged chunks of an HVP do not fit
 *                     shared memory)
 *   threads_per_point symmetric method: threads sharing one point's
 *                     (row, chunk) items, 8..256 power of two (below 32 a
 *                     warp serves several points)
 * Zero in any field means "default".  With csize 0, method 0 means the
 * default method (the tuned one, else chessfad_default_config's), not
 * necessarily the plain method, and the chunk size follows the method: the
 * tuned or default configuration's for that method, else the Sec. V optimum
 * c = sqrt(n/2) (rounded up to a power of two) for the symmetric methods and
 * the largest register-resident chunk for the plain and one-thread-per-point
 * methods; with csize != 0, method 0 is the plain method.  Default
 * threads_per_point never exceeds the point's (row, chunk) item count
 * C nch (nch + 1) / 2 rounded up to a power of two (at least 8).  The
 * symmetric HVP stages a point's chunks on and above the diagonal chunks in
 * shared memory (about n (n + C) / 2 values per point) and sums whole rows,
 * reproducibly, for n up to about 280 (FP32) / 200 (FP64); beyond, it sums
 * each row in an FP64 shared-memory accumulator (the two updates of Alg. 8),
 * adding each iteration's staged chunks in thread order, so results are
 * bitwise reproducible at every n.  The symmetric Hessian writes chunks and
 * their mirror images directly, at any n. */
typedef struct {
    int csize;
    int threads_per_row;
    int block_threads;
    int method;
    int threads_per_point;
} chessfad_config;

/* out[p][i] = sum_j H(x_p)[i][j] v[p][j] for p < batch (CHESS-VEC, Alg. 7,
 * evaluated per point with the L2 decomposition of Sec. VI).
 *   fn      CHESSFAD_ROSENBROCK / _ACKLEY / _FLETCHER_POWELL
 *   n       number of variables
 *   batch   number of points
 *   csize   chunk size (see conventions), 0 = tuned/default
 *   x, v    device, [batch][n], double (FP64) or float (FP32_COMP)
 *   out     device, [batch][n], same type; must not overlap x or v
 *   params  host pointer to device Fletcher-Powell parameters; required for
 *           CHESSFAD_FLETCHER_POWELL, ignored otherwise
 *   prec    CHESSFAD_FP64 or CHESSFAD_FP32_COMP
 *   stream  CUDA stream */
CHESSFAD_API int chessfad_hvp(int fn, int n, long long batch, int csize, const void *x, const void *v, void *out,
                 const chessfad_fp_params *params, int prec, chessfad_stream_t stream);

/* H[p][i][j] = d2f/dx_i dx_j at x_p, both triangles, every entry computed
 * (CHUNK-HESS, Alg. 5).  H: device, [batch][n][n], double or float by prec;
 * other arguments as chessfad_hvp. */
CHESSFAD_API int chessfad_hessian(int fn, int n, long long batch, int csize, const void *x, void *H,
                     const chessfad_fp_params *params, int prec, chessfad_stream_t stream);

/* As chessfad_hvp / chessfad_hessian with an explicit launch configuration
 * (cfg may be NULL = defaults). */
CHESSFAD_API int chessfad_hvp_config(int fn, int n, long long batch, const chessfad_config *cfg, const void *x,
                        const void *v, void *out, const chessfad_fp_params *params, int prec,
                        chessfad_stream_t stream);
CHESSFAD_API int chessfad_hessian_config(int fn, int n, long long batch, const chessfad_config *cfg, const void *x,
                            void *H, const chessfad_fp_params *params, int prec, chessfad_stream_t stream);

/* chessfad_hvp for x, v and out in HOST memory, end to end: the batch is cut
 * into `slices` contiguous parts (0 = 8; at most 64; at most batch); part k's
 * x and v are copied host -> device, its HVPs computed (as chessfad_hvp with
 * csize) and its out copied device -> host, with part k's sweep overlapping
 * the copies of its neighbours (internal copy and compute streams of the
 * current device, created on first use and kept until exit, joined to
 * `stream` by events: the call is one stream-ordered operation on `stream`
 * and can be captured into a CUDA graph from it).  Points are independent
 * (Sec. VI, L0), so slicing changes no result beyond the launch
 * configuration chessfad_hvp picks for the part's size.
 *   x_host, v_host  host, [batch][n], double or float by prec; page-locked
 *                   memory lets the copies overlap (pageable memory works
 *                   but serialises them)
 *   out_host        host, [batch][n]; valid once `stream` reaches this point
 *   x_dev, v_dev, out_dev  device buffers of the whole batch (caller-owned
 *                   staging; their contents are overwritten)
 * Other arguments and errors as chessfad_hvp; slices out of range is
 * CHESSFAD_ERR_CONFIG.  Concurrent calls for one device are serialised on a
 * per-device lock while they enqueue.  Allocates no device memory. */
CHESSFAD_API int chessfad_hvp_host(int fn, int n, long long batch, int csize, const void *x_host,
                                   const void *v_host, void *out_host, void *x_dev, void *v_dev, void *out_dev,
                                   const chessfad_fp_params *params, int prec, int slices, chessfad_stream_t stream);

/* The configuration chessfad_hvp would use for csize = 0: the tuned entry if
 * present, else the default (n >= 4: the symmetric method at the Sec. V
 * optimum csize = sqrt(n/2) rounded up to a power of two; n < 4: the plain
 * method).  A call with csize != 0 and no configuration uses the plain method
 * with that chunk size.  Host only; launches nothing. */
CHESSFAD_API int chessfad_default_config(int fn, int n, long long batch, int prec, chessfad_config *cfg);

/* The configuration chessfad_hvp_config (hvp != 0) or
 * chessfad_hessian_config (hvp == 0) would use for (fn, n, batch, prec, cfg)
 * (cfg may be NULL), with every default filled in, or the error it would
 * return for cfg.  Host only; launches nothing. */
CHESSFAD_API int chessfad_resolve_config(int fn, int n, long long batch, int prec, int hvp,
                                         const chessfad_config *cfg, chessfad_config *out);

/* Autotune the HVP launch configuration for (fn, n, prec) by timing the
 * candidates on the caller's buffers (x, v, out as for chessfad_hvp; out is
 * overwritten): for every chunk size (largest first, following the Sec. V
 * operation-count model) the plain method over (threads_per_row,
 * block_threads) and the symmetric method over (threads_per_point 8..256,
 * block_threads), discarding chunk sizes whose kernels spill registers.  The
 * seed-sparse and one-thread-per-point methods are never candidates.  The
 * winner is stored in the process-wide table used by
 * csize = 0 (chessfad_hvp) and returned in *best (may be NULL).
 * Synchronises `stream`.  Allocates no device memory. */
CHESSFAD_API int chessfad_autotune_hvp(int fn, int n, long long batch, const void *x, const void *v, void *out,
                          const chessfad_fp_params *params, int prec, chessfad_stream_t stream,
                          chessfad_config *best);

/* Autotune the Hessian launch configuration for (fn, n, prec) as
 * chessfad_autotune_hvp does for the HVP (the same candidates, timed as
 * Hessian launches on a prefix of the caller's x and H, which is
 * overwritten).  The winner is stored in the process-wide Hessian table used
 * by chessfad_hessian with csize = 0 and returned in *best (may be NULL).
 * Synchronises `stream`; allocates no device memory. */
CHESSFAD_API int chessfad_autotune_hessian(int fn, int n, long long batch, const void *x, void *H,
                                           const chessfad_fp_params *params, int prec, chessfad_stream_t stream,
                                           chessfad_config *best);

/* Peak CUDA-core throughput measured on the current device by an
 * independent-chain FMA microbenchmark over all SMs: FP32 FFMA for CHESSFAD_FP32_COMP,
 * FP64 DFMA for CHESSFAD_FP64, counting one FMA as two flops.  Synchronises
 * the device; allocates no device memory. */
CHESSFAD_API int chessfad_peak_flops(int prec, double *flops_per_s);

/* chessfad_peak_flops, plus the SM clock (MHz) the fastest run saw, read
 * from the SM cycle counter against the GPU's nanosecond timer inside the
 * kernel (sm_mhz may be NULL).  The FP32 shapes timed are 8 chains x 8 CTAs
 * and 16 chains x 4 CTAs of 256 threads per SM; FP64 adds 16 and 32 chains,
 * at 8 and 4 CTAs per SM; both also run with a multiplier and an addend per
 * chain instead of shared ones, and as accumulation chains acc[l] = fma(s,
 * v[l], acc[l]) (17 or 9 accumulators, one scalar per step); the best is
 * reported. */
CHESSFAD_API int chessfad_peak_info(int prec, double *flops_per_s, double *sm_mhz);

/* The accumulation-chain shape of chessfad_peak_info (17 accumulators,
 * acc[l] = fma(s, v[l], acc[l])) timed twice: with the multipliers v[l] in
 * general registers (*register_flops) and as literals, which the compiler
 * turns into constant operands (*literal_flops).  It shows how the FMA pipe's
 * rate depends on where one operand comes from: on GB300 the literal form
 * runs at about 0.85 of the register form in FP64 and at the same rate in
 * FP32.  Flop/s, one FMA = two flops.  Synchronises the device;
 * allocates no device memory.  CHESSFAD_ERR_NULL for a NULL output,
 * CHESSFAD_ERR_PRECISION for an unknown prec. */
CHESSFAD_API int chessfad_peak_operand_rates(int prec, double *register_flops, double *literal_flops);

/* ---------------------------------------------------------------------------
 * Compensated-FP32 primitives.  The paper computes in FP64 (Sec. IV); the
 * CHESSFAD_FP32_COMP precision rests on error-free transformations and
 * compensated sums from the literature, and these two calls run the very
 * device routines the sweep kernels use over caller arrays, so that their
 * defining properties can be checked directly.  All pointers device, float,
 * caller-owned; stream-ordered; no allocation, no host synchronisation.
 * ------------------------------------------------------------------------- */

/* Elementwise over k < count:
 *   TwoSum (Knuth, TAOCP vol. 2):  s[k] = fl(a[k] + b[k]) and e[k] with
 *                                  s[k] + e[k] == a[k] + b[k] exactly;
 *   TwoProd (by FMA):              p[k] = fl(a[k] * b[k]) and q[k] =
 *                                  fma(a[k], b[k], -p[k]), so p[k] + q[k] ==
 *                                  a[k] * b[k] exactly unless q underflows.
 * Any of s, e, p, q may be NULL (that output is skipped).  count == 0 is a
 * no-op; CHESSFAD_ERR_BATCH for count < 0, CHESSFAD_ERR_NULL for a NULL a
 * or b. */
CHESSFAD_API int chessfad_eft(const float *a, const float *b, long long count, float *s, float *e, float *p,
                              float *q, chessfad_stream_t stream);

/* Compensated sums of the rows of a ([rows][len], row-major): Dot2 of a's
 * and b's rows (b != NULL) or Sum2 of a's rows (b == NULL), both from Ogita,
 * Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6),
 * 2005 (each rounding error, found by TwoSum and TwoProd, is added into a
 * second accumulator, and the two are added once at the end), in the order
 * of the compensated-FP32 row-times-v reduction of the HVP kernels: `lanes`
 * (1, 2, 4, 8, 16 or 32) lanes per row, lane r taking the blocks r, r +
 * lanes, r + 2 lanes, ... of `chunk` consecutive elements in ascending
 * order, then the lanes merged pairwise at distances lanes/2, ..., 1 (the
 * lanes' sums added by TwoSum, their error terms added plainly).  out[r]
 * receives row r's result (rows floats).  rows == 0 is a no-op; len == 0
 * gives zeros.  CHESSFAD_ERR_BATCH for rows < 0, len < 0 or rows * len
 * beyond 64 bits, CHESSFAD_ERR_CONFIG for a bad lanes or chunk < 1,
 * CHESSFAD_ERR_NULL for a NULL out (or a NULL a with len > 0). */
CHESSFAD_API int chessfad_compensated_rows(const float *a, const float *b, long long rows, int len, int lanes,
                                           int chunk, float *out, chessfad_stream_t stream);

/* ---------------------------------------------------------------------------
 * Uneven batches: requests of different functions and sizes in one launch.
 *
 * Request q evaluates out[off .. off+n) = H_fn(x[off .. off+n)) v[off .. off+n)
 * on the packed arrays xpack, vpack, outpack (element offsets, any order, the
 * caller keeps different requests' ranges disjoint).  A Fletcher-Powell
 * request uses the leading n x n block of the shared A, B and the n-vector
 * E = params->E + eoff.  The paper's workload is many independent instances
 * (Sec. VI, L0); this entry serves instances of uneven cost in one persistent
 * launch: the host plan cuts every (function, n) group into CTA-sized tiles of
 * the (point, row, lane) decomposition and sorts them by estimated cost, and
 * the kernel's CTAs pull tiles from a device queue counter.
 * ------------------------------------------------------------------------- */
typedef struct {
    int fn;         /* CHESSFAD_ROSENBROCK / _ACKLEY / _FLETCHER_POWELL */
    int n;          /* 1 .. CHESSFAD_MAX_N */
    long long off;  /* element offset of x, v, out in the packed arrays */
    long long eoff; /* Fletcher-Powell: element offset of E; ignored otherwise */
} chessfad_request;

typedef struct chessfad_ragged_plan_s *chessfad_ragged_plan;

/* Build a plan (host memory, owned by the caller until
 * chessfad_ragged_plan_destroy) from a host array of nreq requests for
 * precision prec.  csize 8 or 16: every (function, n) group uses that chunk
 * size and the default lanes per row; csize 0: each group takes the chunk
 * size and lanes per row that chessfad_ragged_autotune stored for its
 * (precision, function, n range), else the defaults (chunk 16 for compensated
 * FP32, 8 for FP64; lanes per row min(32, pow2_floor(ceil(n/C) / 8))).  The
 * n ranges are the powers of two, 2^b <= n < 2^(b+1) (n = 512 with 256..511).
 * Validates every request: CHESSFAD_ERR_FUNCTION / _SIZE for a bad fn or n,
 * CHESSFAD_ERR_PLAN for a negative offset.  Launches nothing. */
CHESSFAD_API int chessfad_ragged_plan_create(const chessfad_request *reqs, long long nreq, int prec, int csize,
                                             chessfad_ragged_plan *plan);
CHESSFAD_API int chessfad_ragged_plan_destroy(chessfad_ragged_plan plan);

/* Device workspace bytes the plan needs (tile table, request list, offsets,
 * the queue counter, a tile counter per request and, for the Fletcher-Powell
 * requests with n >= 128, one FP64 partial row vector per tile), the number
 * of tiles and the dynamic shared memory per CTA.  Any pointer may be NULL. */
CHESSFAD_API int chessfad_ragged_plan_info(chessfad_ragged_plan plan, size_t *workspace_bytes, long long *ntiles,
                                           size_t *smem_bytes);

/* The chunk size, lanes per row and Fletcher-Powell A/B tile height (rows of
 * A and B staged per shared-memory tile; 8 for the other functions) the plan
 * uses for requests of function fn and size n (CHESSFAD_ERR_SIZE if it holds
 * no such request).  Any output pointer may be NULL.  Host only. */
CHESSFAD_API int chessfad_ragged_plan_group_config(chessfad_ragged_plan plan, int fn, int n, int *csize,
                                                   int *threads_per_row, int *tile_rows);

/* Autotune the uneven batch: for every (function, n range) group of the
 * requests (ranges as for chessfad_ragged_plan_create), run the persistent
 * kernel on a sample of the group's requests (in table order, enough rows to
 * fill the GPU about four times) for every chunk size (16, 8), lanes per
 * row (1 .. 32; for the symmetric Fletcher-Powell tiles, whose (row, chunk)
 * items are dealt to all 256 threads, this sets the rows per tile, 256 /
 * lanes) and,
 * for Fletcher-Powell, shared-memory budget of the A/B row tiles (48 or 144
 * KiB, where they differ in tile height),
 * measuring the SM cycles its tiles take, summed over the CTAs (the group's
 * throughput inside a large mixed run, free of the small sample's own tail),
 * and store the cheapest per (prec, function, n range) in the process-wide
 * table
 * that chessfad_ragged_plan_create(..., csize = 0, ...) reads.  xpack, vpack,
 * outpack, params as for chessfad_hvp_ragged (outpack of the sampled requests
 * is overwritten); workspace: device scratch of workspace_bytes (candidates
 * whose trial plan needs more, plus 256 bytes for the cycle counter, are
 * skipped; the workspace of a plan of all the requests is usually enough).  *groups_tuned (may be NULL) receives the number
 * of groups stored.  Synchronises `stream`; allocates no device memory. */
CHESSFAD_API int chessfad_ragged_autotune(const chessfad_request *reqs, long long nreq, int prec, const void *xpack,
                                          const void *vpack, void *outpack, const chessfad_fp_params *params,
                                          void *workspace, size_t workspace_bytes, chessfad_stream_t stream,
                                          long long *groups_tuned);

/* The tuned (chunk size, lanes per row, A/B tile budget in KiB) of (prec,
 * fn, n's range), or CHESSFAD_ERR_CONFIG if that group has not been tuned.
 * Any output pointer may be NULL.  Host only. */
CHESSFAD_API int chessfad_ragged_tuned_config(int prec, int fn, int n, int *csize, int *threads_per_row,
                                              int *ab_kib);

/* Copy the plan's tables into a caller-allocated device workspace of at least
 * workspace_bytes (cudaMemcpyAsync on stream from the plan's host memory;
 * synchronise the stream before destroying the plan).  Once per workspace. */
CHESSFAD_API int chessfad_ragged_plan_upload(chessfad_ragged_plan plan, void *workspace, size_t workspace_bytes,
                                             chessfad_stream_t stream);

/* Run the plan: reset the queue counter and the per-request tile counters in
 * the workspace (one cudaMemsetAsync) and launch one persistent kernel, both
 * on stream; no host synchronisation, no allocation, so the call can be
 * captured into a CUDA graph and replayed.  Fletcher-Powell requests with
 * n >= 128 use the symmetric method (SC-HESS-VEC, Alg. 8; about half the
 * evaluations): each entry right of a row's diagonal chunk also updates the
 * row it mirrors, usually in another tile; every tile adds its rows'
 * contributions in a fixed order into a partial row vector of its own (FP64)
 * and the tile that completes a request adds the request's partial vectors
 * in tile order, so every result is bitwise reproducible from run to run.
 * xpack, vpack, outpack: device, float (FP32_COMP) or double (FP64) by the
 * plan's precision.  params: required when the plan holds Fletcher-Powell
 * requests (ld >= their largest n).  Runs that share a workspace must not
 * overlap on the GPU. */
CHESSFAD_API int chessfad_hvp_ragged(chessfad_ragged_plan plan, const void *xpack, const void *vpack, void *outpack,
                                     const chessfad_fp_params *params, void *workspace, size_t workspace_bytes,
                                     chessfad_stream_t stream);

/* No-allocation variant of chessfad_hvp_ragged, for callers that cannot call
 * cudaMalloc: a host framework that owns device memory through its own pool,
 * a plugin or callback that must not allocate or implicitly synchronise the
 * device, or real-time code with no room for allocation latency.  The paper
 * has no counterpart; it is a deployment convenience.
 *
 * The scratch (the plan's tables, counters and partial row vectors) lives in a
 * static device array of CHESSFAD_RAGGED_STATIC_BYTES that every GPU which
 * loads the library holds until the process exits.  Each call copies the
 * plan's tables into it from the plan's host memory (cudaMemcpyAsync on
 * stream), zeroes the counters (cudaMemsetAsync) and
 * launches the persistent kernel; it allocates nothing and calls no
 * allocating routine.  Keep the plan alive for as long as any work issued by
 * a call with it may still run.
 * The first call on a device also looks up the array's device address on
 * that device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array, so calls whose work overlaps on
 * the GPU (other streams, other host threads) race; serialise them.
 * Returns CHESSFAD_ERR_WORKSPACE if the plan's workspace exceeds
 * CHESSFAD_RAGGED_STATIC_BYTES (chessfad_ragged_plan_info reports the
 * size); other arguments and errors as chessfad_hvp_ragged. */
#define CHESSFAD_RAGGED_STATIC_BYTES (32u << 20)
CHESSFAD_API int chessfad_hvp_ragged_noalloc(chessfad_ragged_plan plan, const void *xpack, const void *vpack,
                                             void *outpack, const chessfad_fp_params *params,
                                             chessfad_stream_t stream);

/* Registers per thread and local-memory (spill) bytes per thread of the
 * HVP (hvp != 0) or Hessian kernel for (fn, prec, csize), as compiled for
 * the current device.  Host only; launches nothing. */
CHESSFAD_API int chessfad_kernel_info(int fn, int prec, int csize, int hvp, int *registers, long long *local_bytes);

/* Human-readable name of a status code (static storage). */
CHESSFAD_API const char *chessfad_strerror(int status);

/* Library version, major*10000 + minor*100 + patch. */
CHESSFAD_API int chessfad_version(void);

/* ---------------------------------------------------------------------------
 * User-supplied functions.
 *
 * The paper's premise (Sec. I, Sec. IV) is that the user writes f once,
 * generically, and instantiates it on hDual numbers; a compiled library
 * cannot instantiate the caller's template, so here the caller passes the
 * source text of f and the library compiles it at run time (NVRTC, sm_103a)
 * together with its hDual operators and the CHESS-VEC (Alg. 7) /
 * CHUNK-HESS (Alg. 5) sweep, once per handle.  The source must define
 *
 *     template <class R, class X>
 *     R NAME(const X &x, int n, const double *params)
 *
 * (device code; __device__ may be omitted).  x[k], 0 <= k < n, is variable k
 * as an R; R supports + - * / with R and with double on either side, unary
 * -, += -= *= /=, the comparisons < <= > >= == != (on values, also against
 * double), value(u), and the functions sin cos tan tanh exp log sqrt
 * pow(u, double) abs fabs fmin fmax; a double converts to an R constant.
 * Division, abs and comparisons are among the overloads Sec. IV lists; their
 * rules are the quotient rule (u / w = u * (1/w)), sign(u) u with sign(0) =
 * +1, and a comparison of values (the branch taken is differentiated as it
 * stands).  params is the caller's device pointer, passed through (may be
 * NULL).  The arithmetic of f runs in the handle's precision: FP64, or FP32
 * (CHESSFAD_FP32_COMP: only the row-times-v reduction is compensated; the
 * function's own sums are plain FP32 as written; at n = 1, where the Hessian
 * is one entry whose terms can cancel, the arithmetic is FP64 with float
 * inputs and outputs).
 *
 * Two decompositions, as for the built-in functions: plain (CHESS-VEC,
 * Alg. 7 / CHUNK-HESS, Alg. 5: one thread per (point, Hessian row), sweeping
 * the row's ceil(n/csize) chunks) and symmetric (SC-HESS-VEC, Alg. 8 /
 * SCHUNK-HESS, Alg. 6: threads_per_point threads share a point's (row, chunk
 * >= diagonal chunk) items; the HVP stages a point's chunks in shared memory,
 * or, where they do not fit, sums rows in FP64 shared-memory accumulators
 * fed in a fixed order, bitwise reproducible).  x, v, out, H
 * as for chessfad_hvp / chessfad_hessian, 1 <= n <= CHESSFAD_MAX_N.
 * --------------------------------------------------------------------------- */
typedef struct chessfad_user_fn chessfad_user_fn;

/* Compile `source` for chunk size csize (1, 2, 4, 8, 16 or 32) and precision
 * prec, and load it on the current device.  name: the function template's
 * name (a C identifier).  *fn receives the handle (NULL on failure).  log
 * (may be NULL) receives NVRTC's messages, NUL-terminated, truncated to
 * log_bytes.  Returns CHESSFAD_ERR_JIT if NVRTC is missing or compilation
 * fails, CHESSFAD_ERR_CUDA if the compiled code cannot be loaded (no
 * device); synchronous; allocates host memory and the loaded module only. */
CHESSFAD_API int chessfad_user_fn_create(const char *source, const char *name, int csize, int prec,
                                         chessfad_user_fn **fn, char *log, size_t log_bytes);

/* Unload and free a handle (NULL is a no-op).  No launch using it may still
 * be in flight. */
CHESSFAD_API int chessfad_user_fn_destroy(chessfad_user_fn *fn);

/* The handle's chunk size and precision, and the registers per thread and
 * local (spill/stack) bytes of its plain HVP (hvp != 0) or Hessian kernel.
 * Any output pointer may be NULL. */
CHESSFAD_API int chessfad_user_fn_info(const chessfad_user_fn *fn, int hvp, int *csize, int *prec, int *registers,
                                       int *local_bytes);

/* out[p] = H(x_p) v_p for the user's f, p < batch; types by the handle's
 * precision (double, or float for CHESSFAD_FP32_COMP), by the symmetric
 * method with 32 threads per point.  Asynchronous on `stream`; allocates nothing.  The first symmetric
 * launch on a device that needs more than 48 KiB of shared memory raises the
 * kernel's limit (a host call; make it before capturing a CUDA graph). */
CHESSFAD_API int chessfad_user_hvp(chessfad_user_fn *fn, int n, long long batch, const void *x, const void *v,
                                   void *out, const double *params, chessfad_stream_t stream);

/* H[p] = the Hessian of the user's f at x_p, every entry, [batch][n][n]
 * (symmetric method: chunks on and above the diagonal evaluated, the rest
 * mirrored). */
CHESSFAD_API int chessfad_user_hessian(chessfad_user_fn *fn, int n, long long batch, const void *x, void *H,
                                       const double *params, chessfad_stream_t stream);

/* As chessfad_user_hvp / chessfad_user_hessian with an explicit
 * configuration (cfg may be NULL = the defaults above): csize 0 or the
 * handle's (else CHESSFAD_ERR_CHUNK); method CHESSFAD_METHOD_PLAIN or
 * _SYMMETRIC (else CHESSFAD_ERR_CONFIG); threads_per_row 0 or 1;
 * block_threads 0 (= 256) or 32..256, a multiple of 32; threads_per_point 0
 * (= 32) or 32..256, a power of two. */
CHESSFAD_API int chessfad_user_hvp_config(chessfad_user_fn *fn, int n, long long batch, const chessfad_config *cfg,
                                          const void *x, const void *v, void *out, const double *params,
                                          chessfad_stream_t stream);
CHESSFAD_API int chessfad_user_hessian_config(chessfad_user_fn *fn, int n, long long batch, const chessfad_config *cfg,
                                              const void *x, void *H, const double *params, chessfad_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CHESSFAD_H */
