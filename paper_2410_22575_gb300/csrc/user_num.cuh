// user_num.cuh -- the number type on which a user-supplied function is
// evaluated, and its operator set.  Compiled at run time (NVRTC) together
// with the user's source; see user_kernel.cuh and user.cu.
//
// Num<T, C> wraps one chunked hDual (hdual.cuh).  The user writes f once as a
// template on the number type (the library's premise, Sec. I and Sec. IV:
// f is overloaded on hDual so that one evaluation yields one chunk of one
// Hessian row).  The operators are the Fig. 1 rules and the unary chain rule
//   phi(u) = <phi(u), phi'(u) u_k, phi'(u) u_il + phi''(u) u_i u_l>
// with, per function:
//   sin    cos u, -sin u            cos   -sin u, -cos u
//   tan    1 + t^2, 2t(1 + t^2)     tanh  1 - t^2, -2t(1 - t^2)
//   exp    e^u, e^u                 log   1/u, -1/u^2
//   sqrt   1/(2 sqrt u), -1/(4 u^{3/2})
//   u^p    p u^{p-1}, p(p-1) u^{p-2} (p a real constant)
//   1/u    -1/u^2, 2/u^3            u / w = u * (1/w)
//   |u|    sign(u) u componentwise, sign(0) = +1
// Comparisons (Sec. IV lists them among the overloads) compare values;
// fmin / fmax return the operand the value comparison selects.
#pragma once

#include "hdual.cuh"

namespace chessfad {
namespace user {

// Scalar math by precision (distinct names, so the Num overloads below never
// hide the scalar ones inside this namespace).
__device__ __forceinline__ float m_sin(float x) { return sinf(x); }
__device__ __forceinline__ double m_sin(double x) { return sin(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ float m_tan(float x) { return tanf(x); }
__device__ __forceinline__ double m_tan(double x) { return tan(x); }
__device__ __forceinline__ float m_tanh(float x) { return tanhf(x); }
__device__ __forceinline__ double m_tanh(double x) { return tanh(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_pow(float x, float p) { return powf(x, p); }
__device__ __forceinline__ double m_pow(double x, double p) { return pow(x, p); }

template <typename T, int C>
struct Num {
    HD<T, C> a;

    __device__ __forceinline__ Num() : a(hzero<T, C>()) {}
    // A constant: value s, every derivative component zero.
    __device__ __forceinline__ Num(double s) : a(hzero<T, C>()) { a.v = T(s); }
    __device__ __forceinline__ explicit Num(const HD<T, C> &h) : a(h) {}

    __device__ __forceinline__ T value() const { return a.v; }

    __device__ __forceinline__ Num &operator+=(const Num &w) { a = hadd(a, w.a); return *this; }
    __device__ __forceinline__ Num &operator-=(const Num &w) { a = hsub(a, w.a); return *this; }
    __device__ __forceinline__ Num &operator*=(const Num &w) { a = hmul(a, w.a); return *this; }
    __device__ __forceinline__ Num &operator+=(double s) { a.v += T(s); return *this; }
    __device__ __forceinline__ Num &operator-=(double s) { a.v -= T(s); return *this; }
    __device__ __forceinline__ Num &operator*=(double s) { a = smul(T(s), a); return *this; }
    __device__ __forceinline__ Num &operator/=(const Num &w);
    __device__ __forceinline__ Num &operator/=(double s);
};

template <typename T, int C>
__device__ __forceinline__ T value(const Num<T, C> &u) { return u.a.v; }

// ---- arithmetic (Fig. 1)
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator+(const Num<T, C> &u, const Num<T, C> &w) { return Num<T, C>(hadd(u.a, w.a)); }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator-(const Num<T, C> &u, const Num<T, C> &w) { return Num<T, C>(hsub(u.a, w.a)); }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator*(const Num<T, C> &u, const Num<T, C> &w) { return Num<T, C>(hmul(u.a, w.a)); }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator-(const Num<T, C> &u) { return Num<T, C>(rsub(T(0), u.a)); }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator+(const Num<T, C> &u) { return u; }

template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator+(const Num<T, C> &u, double s) { Num<T, C> r = u; r.a.v += T(s); return r; }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator+(double s, const Num<T, C> &u) { Num<T, C> r = u; r.a.v = T(s) + r.a.v; return r; }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator-(const Num<T, C> &u, double s) { Num<T, C> r = u; r.a.v -= T(s); return r; }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator-(double s, const Num<T, C> &u) { return Num<T, C>(rsub(T(s), u.a)); }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator*(const Num<T, C> &u, double s) { return Num<T, C>(smul(T(s), u.a)); }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator*(double s, const Num<T, C> &u) { return Num<T, C>(smul(T(s), u.a)); }

// phi(u) from phi, phi', phi'' at the value.
template <typename T, int C>
__device__ __forceinline__ Num<T, C> apply(const Num<T, C> &u, T phi, T d1, T d2) { return Num<T, C>(unary(u.a, phi, d1, d2)); }

template <typename T, int C>
__device__ __forceinline__ Num<T, C> recip(const Num<T, C> &u)
{
    const T r = T(1) / u.a.v;
    return apply(u, r, -r * r, T(2) * r * r * r);
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator/(const Num<T, C> &u, const Num<T, C> &w) { return u * recip(w); }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator/(double s, const Num<T, C> &w) { return s * recip(w); }
// u / s divides every component (correctly rounded per component).
template <typename T, int C>
__device__ __forceinline__ Num<T, C> operator/(const Num<T, C> &u, double s)
{
    const T d = T(s);
    Num<T, C> r = u;
    r.a.v /= d;
    r.a.d1 /= d;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        r.a.g[l] /= d;
        r.a.h[l] /= d;
    }
    return r;
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> &Num<T, C>::operator/=(const Num<T, C> &w) { *this = *this / w; return *this; }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> &Num<T, C>::operator/=(double s) { *this = *this / s; return *this; }

// ---- elementary functions
template <typename T, int C>
__device__ __forceinline__ Num<T, C> sin(const Num<T, C> &u)
{
    const T s = m_sin(u.a.v), c = m_cos(u.a.v);
    return apply(u, s, c, -s);
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> cos(const Num<T, C> &u)
{
    const T s = m_sin(u.a.v), c = m_cos(u.a.v);
    return apply(u, c, -s, -c);
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> tan(const Num<T, C> &u)
{
    const T t = m_tan(u.a.v), d = T(1) + t * t;
    return apply(u, t, d, T(2) * t * d);
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> tanh(const Num<T, C> &u)
{
    const T t = m_tanh(u.a.v), d = T(1) - t * t;
    return apply(u, t, d, T(-2) * t * d);
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> exp(const Num<T, C> &u)
{
    const T e = m_exp(u.a.v);
    return apply(u, e, e, e);
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> log(const Num<T, C> &u)
{
    const T r = T(1) / u.a.v;
    return apply(u, m_log(u.a.v), r, -r * r);
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> sqrt(const Num<T, C> &u)
{
    const T s = m_sqrt(u.a.v), d = T(0.5) / s;
    return apply(u, s, d, -d / (T(2) * u.a.v));
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> pow(const Num<T, C> &u, double p)
{
    const T q = T(p);
    return apply(u, m_pow(u.a.v, q), q * m_pow(u.a.v, q - T(1)), q * (q - T(1)) * m_pow(u.a.v, q - T(2)));
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> abs(const Num<T, C> &u)
{
    return u.a.v < T(0) ? -u : u;
}
template <typename T, int C>
__device__ __forceinline__ Num<T, C> fabs(const Num<T, C> &u) { return abs(u); }

// ---- comparisons on values
#define CHESSFAD_USER_CMP(op)                                                                               \
    template <typename T, int C>                                                                           \
    __device__ __forceinline__ bool operator op(const Num<T, C> &u, const Num<T, C> &w) { return u.a.v op w.a.v; } \
    template <typename T, int C>                                                                           \
    __device__ __forceinline__ bool operator op(const Num<T, C> &u, double s) { return u.a.v op T(s); }    \
    template <typename T, int C>                                                                           \
    __device__ __forceinline__ bool operator op(double s, const Num<T, C> &u) { return T(s) op u.a.v; }
CHESSFAD_USER_CMP(<)
CHESSFAD_USER_CMP(<=)
CHESSFAD_USER_CMP(>)
CHESSFAD_USER_CMP(>=)
CHESSFAD_USER_CMP(==)
CHESSFAD_USER_CMP(!=)
#undef CHESSFAD_USER_CMP

template <typename T, int C>
__device__ __forceinline__ Num<T, C> fmin(const Num<T, C> &u, const Num<T, C> &w) { return w.a.v < u.a.v ? w : u; }
template <typename T, int C>
__device__ __forceinline__ Num<T, C> fmax(const Num<T, C> &u, const Num<T, C> &w) { return w.a.v > u.a.v ? w : u; }

// The variables x_0 .. x_{n-1} of one evaluation: x[k] is the CHUNK-INIT
// seed of variable k (Alg. 4) for Hessian row i and the chunk starting at
// cstart, generated on the fly; its zeros are opaque (dense arithmetic).
template <typename T, int C>
struct Vars {
    const T *x;
    int i, cstart;
    SeedK<T> z;
    __device__ __forceinline__ Num<T, C> operator[](int k) const { return Num<T, C>(seed<T, C>(x[k], k, i, cstart, z)); }
};

}  // namespace user
}  // namespace chessfad
