// hdual.cuh -- register-resident chunked hDual numbers and their rules.
//
// An hDual<T, C> is the chunked number of Sec. III-B / Sec. IV (Fig. 1):
//   v      the value                                   (v[0] in Fig. 1)
//   d1     d/dx_i, i the Hessian row                   (v[1])
//   g[l]   d/dx_{cstart+l}, l < C, the chunk           (v[2 .. C+1])
//   h[l]   d2/dx_i dx_{cstart+l}                       (v[C+2 .. 2C+1])
// C is a template constant so the 2C+2 components live in registers; every
// loop over components is fully unrolled.
//
// The rules are the ones of Sec. III-A generalised to a chunk, as in Fig. 1:
//   product   (u w)      = u w
//             (u w)_k    = u w_k + w u_k                       (first order)
//             (u w)_{il} = u w_{il} + u_i w_l + w_i u_l + w u_{il}
//   unary     phi(u)     = phi(u),  phi(u)_k = phi'(u) u_k,
//             phi(u)_{il} = phi'(u) u_{il} + phi''(u) u_i u_l
//   sums and products with a scalar act componentwise.
// The "fused" forms (acc + u*w, acc + s*phi(u)) apply exactly these rules
// and add the result into an accumulator with FMAs; they reorder rounding,
// not arithmetic, and they keep the FP32/FP64 pipes on FMA instructions.
#pragma once

#include <cuda_runtime.h>

namespace chessfad {

template <typename T, int C>
struct HD {
    T v, d1;
    T g[C];
    T h[C];
};

template <typename T>
__device__ __forceinline__ T fma_(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T, int C>
__device__ __forceinline__ HD<T, C> hzero()
{
    HD<T, C> r;
    r.v = T(0);
    r.d1 = T(0);
#pragma unroll
    for (int l = 0; l < C; ++l) {
        r.g[l] = T(0);
        r.h[l] = T(0);
    }
    return r;
}

// The zero and the one of CHUNK-INIT's seeds.  Neither may be a constant the
// compiler can fold: the seeds keep the dense semantics of the method, every
// product with a seed zero or one is executed (as in a library whose seeds
// are run-time values).  Where the values come from is a matter of the
// pipe: on GB300 a DFMA that takes an operand from the zero register or from
// the constant bank issues at about 84 % of the FP64 pipe's rate, one whose
// operands are all general registers at up to 99 %
// (chessfad_peak_operand_rates), while FFMA is not slowed by constant
// operands.  So FP32 seeds use an opaque move of 0 (which becomes the zero
// register) and a literal one, and FP64 seeds read both from device memory,
// once per sweep.
template <typename T>
struct SeedK {
    T z, one;
};

static __device__ __align__(16) double g_seed_zero_one[2] = {0.0, 1.0};

template <typename T>
__device__ __forceinline__ SeedK<T> seed_constants();
template <>
__device__ __forceinline__ SeedK<float> seed_constants<float>()
{
    SeedK<float> k;
    asm volatile("mov.b32 %0, 0;" : "=f"(k.z));
    k.one = 1.0f;
    return k;
}
template <>
__device__ __forceinline__ SeedK<double> seed_constants<double>()
{
    SeedK<double> k;
    asm("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %2;\n\tld.global.nc.v2.f64 {%0, %1}, [ga];\n\t}"
        : "=d"(k.z), "=d"(k.one)
        : "l"(g_seed_zero_one));
    return k;
}

// CHUNK-INIT (Alg. 4) for one variable k, generated on the fly instead of
// materialising y[n]: <x_k, [k == i], e_{k - cstart} if k is in the chunk, 0>.
template <typename T, int C>
__device__ __forceinline__ HD<T, C> seed(T xk, int k, int i, int cstart, const SeedK<T> &s)
{
    HD<T, C> y;
    y.v = xk;
    y.d1 = (k == i) ? s.one : s.z;
    const int d = k - cstart;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        y.g[l] = (d == l) ? s.one : s.z;
        y.h[l] = s.z;
    }
    return y;
}

// CHUNK-INIT seeds with the chunk position known at compile time: variable
// k with chunk offset P = k - cstart (P outside [0, C) for variables outside
// the chunk).  With P a constant the seed needs no per-component selects, and
// the arithmetic that consumes it is the full dense rule.
template <typename T, int C, int P>
__device__ __forceinline__ HD<T, C> seed_at(T xk, bool is_row, const SeedK<T> &s)
{
    HD<T, C> y;
    y.v = xk;
    y.d1 = is_row ? s.one : s.z;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        y.g[l] = (l == P) ? s.one : s.z;
        y.h[l] = s.z;
    }
    return y;
}

// ------------------------------------------------------------------ components
// The derivative parts g[0..C) and h[0..C) are updated with one scalar factor
// per step.  FP32 with an even C runs the pairs (l, l+1) as one packed
// instruction (__ffma2_rn, __fmul2_rn, __fadd2_rn; sm_100 and later): each
// component rounds exactly as the scalar __fmaf_rn, __fmul_rn or __fadd_rn,
// in half the issued instructions (the FP32 sweeps are bound by instruction
// issue).  The packed products and sums are never contracted into FMAs with
// a later addition, so a user function's FP32 arithmetic follows its source
// operation by operation.

// acc[l] = fma(s, a[l], acc[l])
template <typename T, int C>
__device__ __forceinline__ void vfma(T s, const T (&a)[C], T (&acc)[C])
{
#pragma unroll
    for (int l = 0; l < C; ++l) acc[l] = fma_(s, a[l], acc[l]);
}
template <int C>
__device__ __forceinline__ void vfma(float s, const float (&a)[C], float (&acc)[C])
{
    if constexpr (C % 2 == 0) {
        const float2 s2 = make_float2(s, s);
#pragma unroll
        for (int l = 0; l < C; l += 2) {
            const float2 r = __ffma2_rn(s2, make_float2(a[l], a[l + 1]), make_float2(acc[l], acc[l + 1]));
            acc[l] = r.x;
            acc[l + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int l = 0; l < C; ++l) acc[l] = __fmaf_rn(s, a[l], acc[l]);
    }
}

// r[l] = s * a[l]
template <typename T, int C>
__device__ __forceinline__ void vmul(T s, const T (&a)[C], T (&r)[C])
{
#pragma unroll
    for (int l = 0; l < C; ++l) r[l] = s * a[l];
}
template <int C>
__device__ __forceinline__ void vmul(float s, const float (&a)[C], float (&r)[C])
{
    if constexpr (C % 2 == 0) {
        const float2 s2 = make_float2(s, s);
#pragma unroll
        for (int l = 0; l < C; l += 2) {
            const float2 p = __fmul2_rn(s2, make_float2(a[l], a[l + 1]));
            r[l] = p.x;
            r[l + 1] = p.y;
        }
    } else {
#pragma unroll
        for (int l = 0; l < C; ++l) r[l] = s * a[l];
    }
}

// r[l] = a[l] + b[l]
template <typename T, int C>
__device__ __forceinline__ void vadd(const T (&a)[C], const T (&b)[C], T (&r)[C])
{
#pragma unroll
    for (int l = 0; l < C; ++l) r[l] = a[l] + b[l];
}
template <int C>
__device__ __forceinline__ void vadd(const float (&a)[C], const float (&b)[C], float (&r)[C])
{
    if constexpr (C % 2 == 0) {
#pragma unroll
        for (int l = 0; l < C; l += 2) {
            const float2 t = __fadd2_rn(make_float2(a[l], a[l + 1]), make_float2(b[l], b[l + 1]));
            r[l] = t.x;
            r[l + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int l = 0; l < C; ++l) r[l] = a[l] + b[l];
    }
}

// u * w (Fig. 1).
template <typename T, int C>
__device__ __forceinline__ HD<T, C> hmul(const HD<T, C> &a, const HD<T, C> &b)
{
    HD<T, C> r;
    r.v = a.v * b.v;
    r.d1 = fma_(b.v, a.d1, a.v * b.d1);
    vmul(a.v, b.g, r.g);
    vfma(b.v, a.g, r.g);
    vmul(a.v, b.h, r.h);
    vfma(a.d1, b.g, r.h);
    vfma(b.d1, a.g, r.h);
    vfma(b.v, a.h, r.h);
    return r;
}

// acc + u * w: the product rule, each component's terms added into acc.
template <typename T, int C>
__device__ __forceinline__ HD<T, C> hfma(const HD<T, C> &a, const HD<T, C> &b, const HD<T, C> &acc)
{
    HD<T, C> r = acc;
    r.v = fma_(a.v, b.v, acc.v);
    r.d1 = fma_(b.v, a.d1, fma_(a.v, b.d1, acc.d1));
    vfma(a.v, b.g, r.g);
    vfma(b.v, a.g, r.g);
    vfma(a.v, b.h, r.h);
    vfma(a.d1, b.g, r.h);
    vfma(b.d1, a.g, r.h);
    vfma(b.v, a.h, r.h);
    return r;
}

template <typename T, int C>
__device__ __forceinline__ HD<T, C> hadd(const HD<T, C> &a, const HD<T, C> &b)
{
    HD<T, C> r;
    r.v = a.v + b.v;
    r.d1 = a.d1 + b.d1;
    vadd(a.g, b.g, r.g);
    vadd(a.h, b.h, r.h);
    return r;
}

template <typename T, int C>
__device__ __forceinline__ HD<T, C> hsub(const HD<T, C> &a, const HD<T, C> &b)
{
    HD<T, C> r;
    r.v = a.v - b.v;
    r.d1 = a.d1 - b.d1;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        r.g[l] = a.g[l] - b.g[l];
        r.h[l] = a.h[l] - b.h[l];
    }
    return r;
}

// s * u
template <typename T, int C>
__device__ __forceinline__ HD<T, C> smul(T s, const HD<T, C> &a)
{
    HD<T, C> r;
    r.v = s * a.v;
    r.d1 = s * a.d1;
    vmul(s, a.g, r.g);
    vmul(s, a.h, r.h);
    return r;
}

// s - u
template <typename T, int C>
__device__ __forceinline__ HD<T, C> rsub(T s, const HD<T, C> &a)
{
    HD<T, C> r;
    r.v = s - a.v;
    r.d1 = -a.d1;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        r.g[l] = -a.g[l];
        r.h[l] = -a.h[l];
    }
    return r;
}

// phi(u) with phi, phi', phi'' evaluated at u.v by the caller.
template <typename T, int C>
__device__ __forceinline__ HD<T, C> unary(const HD<T, C> &a, T phi, T dphi, T d2phi)
{
    HD<T, C> r;
    r.v = phi;
    r.d1 = dphi * a.d1;
    const T q = d2phi * a.d1;
    vmul(dphi, a.g, r.g);
    vmul(dphi, a.h, r.h);
    vfma(q, a.g, r.h);
    return r;
}

// acc + s * phi(u): the unary rule scaled by s, added into acc.  The value
// component is skipped when the caller replaces it (kValue == false).
template <bool kValue, typename T, int C>
__device__ __forceinline__ void sfma_unary(HD<T, C> &acc, T s, const HD<T, C> &a, T phi, T dphi, T d2phi)
{
    if (kValue) acc.v = fma_(s, phi, acc.v);
    const T sd = s * dphi;
    const T q = (s * d2phi) * a.d1;
    acc.d1 = fma_(sd, a.d1, acc.d1);
    vfma(sd, a.g, acc.g);
    vfma(q, a.g, acc.h);
    vfma(sd, a.h, acc.h);
}

// acc + s * u, componentwise; the value component only when kValue.
template <bool kValue, typename T, int C>
__device__ __forceinline__ void sfma(HD<T, C> &acc, T s, const HD<T, C> &a)
{
    if (kValue) acc.v = fma_(s, a.v, acc.v);
    acc.d1 = fma_(s, a.d1, acc.d1);
    vfma(s, a.g, acc.g);
    vfma(s, a.h, acc.h);
}

// acc + phi(u) (s = 1 of the above).
template <bool kValue, typename T, int C>
__device__ __forceinline__ void add_unary(HD<T, C> &acc, const HD<T, C> &a, T phi, T dphi, T d2phi)
{
    if (kValue) acc.v += phi;
    const T q = d2phi * a.d1;
    acc.d1 = fma_(dphi, a.d1, acc.d1);
    vfma(dphi, a.g, acc.g);
    vfma(q, a.g, acc.h);
    vfma(dphi, a.h, acc.h);
}

// ---------------------------------------------------------------------------
// Error-free transformations (compensated FP32 path).
//   TwoSum      Knuth (TAOCP vol. 2): s + e == a + b exactly, no ordering
//               precondition, 6 additions.
//   TwoProd     with FMA: p + e == a * b exactly (e = fma(a, b, -p)).
//   Sum2 / Dot2 Ogita, Rump & Oishi, "Accurate sum and dot product", SIAM J.
//               Sci. Comput. 26(6), 2005: cascade the rounding errors of a
//               recursive sum / dot product into a second accumulator and add
//               it once at the end; the result is as accurate as if computed
//               in twice the working precision, then rounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// A compensated scalar: s + e is the running sum, e collects the rounding
// errors (Sum2).
struct CSum {
    float s, e;
};

__device__ __forceinline__ void csum_add(CSum &acc, float x)
{
    float t;
    two_sum(acc.s, x, acc.s, t);
    acc.e = __fadd_rn(acc.e, t);
}

// acc += a * b with TwoProd + TwoSum (one Dot2 step).
__device__ __forceinline__ void cdot_add(CSum &acc, float a, float b)
{
    float p, pe, t;
    two_prod(a, b, p, pe);
    two_sum(acc.s, p, acc.s, t);
    acc.e = __fadd_rn(acc.e, __fadd_rn(t, pe));
}

// Merge two compensated partial sums (used across shuffle lanes).
__device__ __forceinline__ CSum csum_merge(CSum a, CSum b)
{
    CSum r;
    float t;
    two_sum(a.s, b.s, r.s, t);
    r.e = __fadd_rn(__fadd_rn(a.e, b.e), t);
    return r;
}

__device__ __forceinline__ float csum_value(const CSum &a) { return __fadd_rn(a.s, a.e); }

// A compensated hDual accumulator: Sum2 applied to each component of a sum
// over terms.  Components the caller never reads are dead code and vanish.
template <int C>
struct CHD {
    HD<float, C> s, e;
};

template <int C>
__device__ __forceinline__ void chd_zero(CHD<C> &a)
{
    a.s = hzero<float, C>();
    a.e = hzero<float, C>();
}

template <int C>
__device__ __forceinline__ void chd_add(CHD<C> &a, const HD<float, C> &x)
{
    float t;
    two_sum(a.s.v, x.v, a.s.v, t);
    a.e.v = __fadd_rn(a.e.v, t);
    two_sum(a.s.d1, x.d1, a.s.d1, t);
    a.e.d1 = __fadd_rn(a.e.d1, t);
#pragma unroll
    for (int l = 0; l < C; ++l) {
        two_sum(a.s.g[l], x.g[l], a.s.g[l], t);
        a.e.g[l] = __fadd_rn(a.e.g[l], t);
        two_sum(a.s.h[l], x.h[l], a.s.h[l], t);
        a.e.h[l] = __fadd_rn(a.e.h[l], t);
    }
}

template <int C>
__device__ __forceinline__ HD<float, C> chd_value(const CHD<C> &a)
{
    return hadd(a.s, a.e);
}

}  // namespace chessfad
