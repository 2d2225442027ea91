/*
 * oracle.c -- plain, slow FP64 CPU oracle for CHESSFAD (Ranjan & Zubair,
 * "An AD based library for Efficient Hessian and Hessian-Vector Product
 * Computation on GPU", arXiv:2410.22575).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * of the package entry module and the CPU-baseline leg of the benchmark may
 * load this library.  It shares no code, header, table or helper with the CUDA
 * library; the only thing both sides share is the seeded input generator,
 * which holds none of the method's arithmetic.
 *
 * Two independent implementations of the same mathematics:
 *
 *  O1  Closed forms.  Every chunked method of the paper reaches the dense
 *      Hessian exactly, up to rounding (Sec. III-B: each call of f computes
 *      csize entries of one Hessian row; Alg. 5 assembles all of them).  So
 *      the reference result is the plain definition: H(x) from its analytic
 *      formula, then r = H v by ascending-j summation.  The three test
 *      functions are only named in the paper (Sec. VII); their definitions
 *      are the standard ones (Rosenbrock; Ackley with a=20, b=0.2, c=2*pi;
 *      Fletcher-Powell with A, B, E shared by the whole batch) and the
 *      derivatives below are derived by hand from them.
 *
 *  O2  The paper's own algorithm, written out step by step in the paper's
 *      order and notation: the hDual<csize> number type of Sec. IV (Fig. 1)
 *      with the second-order rules of Sec. III-A generalised to chunks, the
 *      seeding CHUNK-INIT (Alg. 4), CHUNK-HESS (Alg. 5), SCHUNK-HESS (Alg. 6),
 *      CHESS-VEC (Alg. 7) and SC-HESS-VEC (Alg. 8), with the test functions
 *      written once, generically, on hDuals.  O2 also carries the operation
 *      counters used to check the Sec. V analysis.
 *
 * Readings of the paper taken here:
 *  - csize need not divide n: nchunk = ceil(n/csize); the last chunk covers
 *    [cstart, n) and its seeds beyond n are zero (Sec. III-B assumes
 *    divisibility).
 *  - Alg. 7 and Alg. 10 pass the chunk number j where CHUNK-INIT expects
 *    cstart; the chunk start j*csize is passed.
 *  - Alg. 8 loops l = csize+2 .. 2*csize-1; the full chunk l = csize+2 ..
 *    2*csize+1 is used.  Alg. 6 copies j = 0..endindex inclusive; exclusive
 *    is used (the inclusive copy rewrites an equal, already computed entry).
 *  - sqrt at 0 (Ackley at the origin) is not differentiable; the closed-form
 *    gradient takes the subgradient 0 for the first Ackley term there, and
 *    the Hessian at S == 0 is undefined (not used as a reference).
 *
 * Precision: double throughout; cos(2*pi*x) is evaluated as cos(2.0*M_PI*x).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_ROSENBROCK = 0, ORC_ACKLEY = 1, ORC_FLETCHER_POWELL = 2, ORC_MIX = 3 };

/* Fletcher-Powell parameters: A, B are row-major with leading dimension ld,
 * of which the leading n x n block is used; E has n entries. */
typedef struct {
    const double *A, *B, *E;
    int ld;
} orc_fp;

/* ======================================================================
 * O1 -- function values, gradients and Hessians in closed form
 * ====================================================================== */

/* Rosenbrock: f = sum_{k=0}^{n-2} [100 (x_{k+1} - x_k^2)^2 + (1 - x_k)^2]. */
static double rosen_f(int n, const double *x)
{
    double f = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
        double d = x[k + 1] - x[k] * x[k];
        double e = 1.0 - x[k];
        f += 100.0 * d * d + e * e;
    }
    return f;
}

/* g_k = [k<n-1] (-400 x_k (x_{k+1}-x_k^2) - 2 (1-x_k)) + [k>0] 200 (x_k - x_{k-1}^2) */
static void rosen_g(int n, const double *x, double *g)
{
    for (int k = 0; k < n; ++k) {
        double gk = 0.0;
        if (k + 1 < n) gk += -400.0 * x[k] * (x[k + 1] - x[k] * x[k]) - 2.0 * (1.0 - x[k]);
        if (k > 0) gk += 200.0 * (x[k] - x[k - 1] * x[k - 1]);
        g[k] = gk;
    }
}

/* Tridiagonal: H_kk = [k<n-1](1200 x_k^2 - 400 x_{k+1} + 2) + [k>0] 200,
 *              H_{k,k+1} = H_{k+1,k} = -400 x_k. */
static void rosen_h(int n, const double *x, double *H)
{
    memset(H, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int k = 0; k < n; ++k) {
        double hk = 0.0;
        if (k + 1 < n) hk += 1200.0 * x[k] * x[k] - 400.0 * x[k + 1] + 2.0;
        if (k > 0) hk += 200.0;
        H[(size_t)k * n + k] = hk;
        if (k + 1 < n) {
            H[(size_t)k * n + k + 1] = -400.0 * x[k];
            H[(size_t)(k + 1) * n + k] = -400.0 * x[k];
        }
    }
}

/* Ackley: f = -20 exp(-0.2 sqrt(S/n)) - exp(C/n) + 20 + e,
 *         S = sum x_k^2, C = sum cos(2 pi x_k). */
static double ackley_f(int n, const double *x)
{
    double S = 0.0, C = 0.0;
    for (int k = 0; k < n; ++k) {
        S += x[k] * x[k];
        C += cos(2.0 * M_PI * x[k]);
    }
    return -20.0 * exp(-0.2 * sqrt(S / n)) - exp(C / n) + 20.0 + exp(1.0);
}

/* With r = sqrt(S/n), E1 = exp(-0.2 r), E2 = exp(C/n), s_k = sin(2 pi x_k):
 *   g_k = 4 E1 x_k / (n r) + (2 pi / n) E2 s_k,
 * where the first term is taken as 0 when S == 0 (subgradient at the kink). */
static void ackley_g(int n, const double *x, double *g)
{
    double S = 0.0, C = 0.0;
    for (int k = 0; k < n; ++k) {
        S += x[k] * x[k];
        C += cos(2.0 * M_PI * x[k]);
    }
    double r = sqrt(S / n), E1 = exp(-0.2 * r), E2 = exp(C / n);
    for (int k = 0; k < n; ++k) {
        double t1 = (S == 0.0) ? 0.0 : 4.0 * E1 * x[k] / (n * r);
        g[k] = t1 + (2.0 * M_PI / n) * E2 * sin(2.0 * M_PI * x[k]);
    }
}

/* H = 4 E1/(n r) I - E1 (0.8/(n^2 r^2) + 4/(n^2 r^3)) x x^T
 *     + (4 pi^2 / n) E2 (diag(cos 2 pi x) - s s^T / n). */
static void ackley_h(int n, const double *x, double *H)
{
    double S = 0.0, C = 0.0;
    for (int k = 0; k < n; ++k) {
        S += x[k] * x[k];
        C += cos(2.0 * M_PI * x[k]);
    }
    double r = sqrt(S / n), E1 = exp(-0.2 * r), E2 = exp(C / n);
    double nn = (double)n;
    double a = 4.0 * E1 / (nn * r);
    double b = E1 * (0.8 / (nn * nn * r * r) + 4.0 / (nn * nn * r * r * r));
    double q = 4.0 * M_PI * M_PI / nn * E2;
    for (int k = 0; k < n; ++k) {
        double sk = sin(2.0 * M_PI * x[k]);
        for (int l = 0; l < n; ++l) {
            double sl = sin(2.0 * M_PI * x[l]);
            double h = -b * x[k] * x[l] - q * sk * sl / nn;
            if (k == l) h += a + q * cos(2.0 * M_PI * x[k]);
            H[(size_t)k * n + l] = h;
        }
    }
}

/* Fletcher-Powell: f = sum_m r_m^2,  r_m = E_m - sum_j P_mj,
 *   P_mj = A_mj sin x_j + B_mj cos x_j,  J_mj = A_mj cos x_j - B_mj sin x_j. */
static void fp_residual(int n, const double *x, const orc_fp *p, double *r)
{
    for (int m = 0; m < n; ++m) {
        double s = 0.0;
        for (int j = 0; j < n; ++j)
            s += p->A[(size_t)m * p->ld + j] * sin(x[j]) + p->B[(size_t)m * p->ld + j] * cos(x[j]);
        r[m] = p->E[m] - s;
    }
}

static double fp_f(int n, const double *x, const orc_fp *p)
{
    double *r = (double *)malloc(sizeof(double) * n);
    fp_residual(n, x, p, r);
    double f = 0.0;
    for (int m = 0; m < n; ++m) f += r[m] * r[m];
    free(r);
    return f;
}

/* g_j = -2 sum_m r_m J_mj */
static void fp_g(int n, const double *x, const orc_fp *p, double *g)
{
    double *r = (double *)malloc(sizeof(double) * n);
    fp_residual(n, x, p, r);
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int m = 0; m < n; ++m) {
            double J = p->A[(size_t)m * p->ld + j] * cos(x[j]) - p->B[(size_t)m * p->ld + j] * sin(x[j]);
            s += r[m] * J;
        }
        g[j] = -2.0 * s;
    }
    free(r);
}

/* H_jk = 2 sum_m J_mj J_mk + 2 delta_jk sum_m r_m P_mj */
static void fp_h(int n, const double *x, const orc_fp *p, double *H)
{
    double *r = (double *)malloc(sizeof(double) * n);
    double *J = (double *)malloc(sizeof(double) * (size_t)n * n);
    fp_residual(n, x, p, r);
    for (int m = 0; m < n; ++m)
        for (int j = 0; j < n; ++j)
            J[(size_t)m * n + j] = p->A[(size_t)m * p->ld + j] * cos(x[j]) - p->B[(size_t)m * p->ld + j] * sin(x[j]);
    for (int j = 0; j < n; ++j) {
        for (int k = 0; k < n; ++k) {
            double s = 0.0;
            for (int m = 0; m < n; ++m) s += J[(size_t)m * n + j] * J[(size_t)m * n + k];
            H[(size_t)j * n + k] = 2.0 * s;
        }
        double d = 0.0;
        for (int m = 0; m < n; ++m)
            d += r[m] * (p->A[(size_t)m * p->ld + j] * sin(x[j]) + p->B[(size_t)m * p->ld + j] * cos(x[j]));
        H[(size_t)j * n + j] += 2.0 * d;
    }
    free(J);
    free(r);
}

/* Fletcher-Powell Hessian-vector product without forming H, from the same
 * closed form H = 2 J^T J + 2 diag(P^T r):
 *   (H v)_j = 2 sum_m J_mj (sum_k J_mk v_k) + 2 v_j sum_m r_m P_mj,
 * O(n^2) per point.  When hnorm is not NULL it also returns ||H||_F, from
 * G = J^T J (accumulated row by row of J, upper triangle) and D_j =
 * sum_m r_m P_mj:  ||H||_F^2 = 4 (sum_jk G_jk^2 + 2 sum_j G_jj D_j +
 * sum_j D_j^2). */
static int fp_hvp(int n, const double *x, const double *v, const orc_fp *p, double *out, double *hnorm)
{
    double *sn = (double *)malloc(sizeof(double) * n);
    double *cs = (double *)malloc(sizeof(double) * n);
    double *J = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *r = (double *)malloc(sizeof(double) * n);
    double *Jv = (double *)malloc(sizeof(double) * n);
    double *D = (double *)malloc(sizeof(double) * n);
    if (!sn || !cs || !J || !r || !Jv || !D) {
        free(sn); free(cs); free(J); free(r); free(Jv); free(D);
        return -1;
    }
    for (int j = 0; j < n; ++j) {
        sn[j] = sin(x[j]);
        cs[j] = cos(x[j]);
        D[j] = 0.0;
        out[j] = 0.0;
    }
    for (int m = 0; m < n; ++m) {
        const double *Am = p->A + (size_t)m * p->ld, *Bm = p->B + (size_t)m * p->ld;
        double *Jm = J + (size_t)m * n;
        double s = 0.0, jv = 0.0;
        for (int j = 0; j < n; ++j) {
            s += Am[j] * sn[j] + Bm[j] * cs[j];
            Jm[j] = Am[j] * cs[j] - Bm[j] * sn[j];
            jv += Jm[j] * v[j];
        }
        r[m] = p->E[m] - s;
        Jv[m] = jv;
    }
    for (int m = 0; m < n; ++m) {
        const double *Am = p->A + (size_t)m * p->ld, *Bm = p->B + (size_t)m * p->ld;
        const double *Jm = J + (size_t)m * n;
        for (int j = 0; j < n; ++j) {
            out[j] += Jm[j] * Jv[m];
            D[j] += r[m] * (Am[j] * sn[j] + Bm[j] * cs[j]);
        }
    }
    for (int j = 0; j < n; ++j) out[j] = 2.0 * out[j] + 2.0 * D[j] * v[j];
    int rc = 0;
    if (hnorm) {
        double *G = (double *)calloc((size_t)n * n, sizeof(double));
        if (!G) {
            rc = -1;
        } else {
            for (int m = 0; m < n; ++m) {
                const double *Jm = J + (size_t)m * n;
                for (int j = 0; j < n; ++j) {
                    const double a = Jm[j];
                    double *Gj = G + (size_t)j * n;
                    for (int k = j; k < n; ++k) Gj[k] += a * Jm[k];
                }
            }
            double off = 0.0, diag = 0.0;
            for (int j = 0; j < n; ++j) {
                const double *Gj = G + (size_t)j * n;
                for (int k = j + 1; k < n; ++k) off += Gj[k] * Gj[k];
                diag += Gj[j] * Gj[j] + 2.0 * Gj[j] * D[j] + D[j] * D[j];
            }
            *hnorm = 2.0 * sqrt(2.0 * off + diag);
            free(G);
        }
    }
    free(sn); free(cs); free(J); free(r); free(Jv); free(D);
    return rc;
}

/* Test function of the extended operator set.  Sec. IV lists division, abs
 * and comparisons among the overloaded operators, but none of the paper's
 * three test functions uses them; this function does (it is defined here,
 * not in the paper):
 *   f = sum_{k<n-1} [ (x_{k+1} - x_k)^2 / (1 + x_k^2) + |x_k| x_{k+1}
 *                     + tanh(x_k x_{k+1}) ]
 *     + sum_k [ log(1 + x_k^2) + 0.1 (2 + x_k^2)^{3/2} + tan(0.3 x_k) ]
 *     + (x_0 > x_{n-1} ? x_0 x_{n-1} : -x_0^2)
 * |x| is differentiated as sign(x) x with sign(0) = +1; the branch is taken
 * on values, and each branch is differentiated as it stands. */
static double mix_f(int n, const double *x)
{
    double f = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
        double d = x[k + 1] - x[k];
        f += d * d / (1.0 + x[k] * x[k]) + fabs(x[k]) * x[k + 1] + tanh(x[k] * x[k + 1]);
    }
    for (int k = 0; k < n; ++k)
        f += log(1.0 + x[k] * x[k]) + 0.1 * pow(2.0 + x[k] * x[k], 1.5) + tan(0.3 * x[k]);
    f += (x[0] > x[n - 1]) ? x[0] * x[n - 1] : -x[0] * x[0];
    return f;
}

static double sign1(double a) { return a < 0.0 ? -1.0 : 1.0; }

/* Gradient, term by term (d = x_{k+1} - x_k, q = 1 + x_k^2, t = tanh(x_k x_{k+1})):
 *   d/dx_k     [d^2/q] = -2d/q - 2 x_k d^2/q^2,  d/dx_{k+1} [d^2/q] = 2d/q
 *   d/dx_k     [|x_k| x_{k+1}] = sign(x_k) x_{k+1},  d/dx_{k+1} = |x_k|
 *   d/dx_k     [tanh] = (1 - t^2) x_{k+1},  d/dx_{k+1} = (1 - t^2) x_k
 *   d/dx [log(1+x^2)] = 2x/(1+x^2);  d/dx [0.1 s^{3/2}] = 0.3 x s^{1/2} (s = 2+x^2);
 *   d/dx [tan(0.3x)] = 0.3 (1 + tan^2(0.3x)). */
static void mix_g(int n, const double *x, double *g)
{
    for (int k = 0; k < n; ++k) {
        double s = 2.0 + x[k] * x[k], tau = tan(0.3 * x[k]);
        g[k] = 2.0 * x[k] / (1.0 + x[k] * x[k]) + 0.3 * x[k] * sqrt(s) + 0.3 * (1.0 + tau * tau);
    }
    for (int k = 0; k + 1 < n; ++k) {
        double d = x[k + 1] - x[k], q = 1.0 + x[k] * x[k], t = tanh(x[k] * x[k + 1]);
        g[k] += -2.0 * d / q - 2.0 * x[k] * d * d / (q * q) + sign1(x[k]) * x[k + 1] + (1.0 - t * t) * x[k + 1];
        g[k + 1] += 2.0 * d / q + fabs(x[k]) + (1.0 - t * t) * x[k];
    }
    if (x[0] > x[n - 1]) {
        g[0] += x[n - 1];
        g[n - 1] += x[0];
    } else {
        g[0] += -2.0 * x[0];
    }
}

/* Hessian, term by term (a = x_k, d, q, t as above, T'' = -2t(1 - t^2)):
 *   [d^2/q]:  H_kk += 2/q + 8ad/q^2 - 2d^2/q^2 + 8a^2 d^2/q^3,
 *             H_{k,k+1} += -2/q - 4ad/q^2,  H_{k+1,k+1} += 2/q
 *   [|x_k| x_{k+1}]:  H_{k,k+1} += sign(x_k)
 *   [tanh]:  H_kk += T'' x_{k+1}^2,  H_{k+1,k+1} += T'' x_k^2,
 *            H_{k,k+1} += T'' x_k x_{k+1} + (1 - t^2)
 *   per variable:  (2 - 2x^2)/(1+x^2)^2 + 0.3 s^{1/2} + 0.3 x^2 s^{-1/2}
 *                  + 0.18 tau (1 + tau^2),  tau = tan(0.3x)
 *   branch:  x_0 > x_{n-1}: H_{0,n-1} = H_{n-1,0} += 1;  else H_00 += -2. */
static void mix_h(int n, const double *x, double *H)
{
    memset(H, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int k = 0; k < n; ++k) {
        double xx = x[k] * x[k], s = 2.0 + xx, tau = tan(0.3 * x[k]);
        H[(size_t)k * n + k] = (2.0 - 2.0 * xx) / ((1.0 + xx) * (1.0 + xx)) + 0.3 * sqrt(s) + 0.3 * xx / sqrt(s) +
                               0.18 * tau * (1.0 + tau * tau);
    }
    for (int k = 0; k + 1 < n; ++k) {
        double a = x[k], b = x[k + 1], d = b - a, q = 1.0 + a * a, t = tanh(a * b);
        double t2 = -2.0 * t * (1.0 - t * t);
        H[(size_t)k * n + k] += 2.0 / q + 8.0 * a * d / (q * q) - 2.0 * d * d / (q * q) + 8.0 * a * a * d * d / (q * q * q) +
                                t2 * b * b;
        H[(size_t)(k + 1) * n + k + 1] += 2.0 / q + t2 * a * a;
        double off = -2.0 / q - 4.0 * a * d / (q * q) + sign1(a) + t2 * a * b + (1.0 - t * t);
        H[(size_t)k * n + k + 1] += off;
        H[(size_t)(k + 1) * n + k] += off;
    }
    if (x[0] > x[n - 1]) {
        H[n - 1] += 1.0;
        H[(size_t)(n - 1) * n] += 1.0;
    } else {
        H[0] += -2.0;
    }
}

double orc_value(int fn, int n, const double *x, const orc_fp *p)
{
    switch (fn) {
    case ORC_ROSENBROCK: return rosen_f(n, x);
    case ORC_ACKLEY: return ackley_f(n, x);
    case ORC_FLETCHER_POWELL: return fp_f(n, x, p);
    case ORC_MIX: return mix_f(n, x);
    }
    return NAN;
}

int orc_gradient(int fn, int n, const double *x, const orc_fp *p, double *g)
{
    switch (fn) {
    case ORC_ROSENBROCK: rosen_g(n, x, g); return 0;
    case ORC_ACKLEY: ackley_g(n, x, g); return 0;
    case ORC_FLETCHER_POWELL: fp_g(n, x, p, g); return 0;
    case ORC_MIX: mix_g(n, x, g); return 0;
    }
    return -1;
}

int orc_hessian(int fn, int n, const double *x, const orc_fp *p, double *H)
{
    switch (fn) {
    case ORC_ROSENBROCK: rosen_h(n, x, H); return 0;
    case ORC_ACKLEY: ackley_h(n, x, H); return 0;
    case ORC_FLETCHER_POWELL: fp_h(n, x, p, H); return 0;
    case ORC_MIX: mix_h(n, x, H); return 0;
    }
    return -1;
}

/* Batched reference HVP: out_p = H(x_p) v_p (plain ascending-j sums), and,
 * when hnorm is not NULL, hnorm_p = ||H(x_p)||_F for the error metric.
 * x, v, out are [batch][n] row-major. */
int orc_hvp_batch(int fn, int n, long long batch, const double *x, const double *v,
                  const orc_fp *p, double *out, double *hnorm)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long long q = 0; q < batch; ++q) {
        double *H = (double *)malloc(sizeof(double) * (size_t)n * n);
        if (!H) { bad |= 1; continue; }
        bad |= (orc_hessian(fn, n, x + q * n, p, H) != 0);
        double fro = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) {
                s += H[(size_t)i * n + j] * v[q * n + j];
                fro += H[(size_t)i * n + j] * H[(size_t)i * n + j];
            }
            out[q * n + i] = s;
        }
        if (hnorm) hnorm[q] = sqrt(fro);
        free(H);
    }
    return bad ? -1 : 0;
}

/* Batched reference Hessians, H is [batch][n][n]. */
int orc_hessian_batch(int fn, int n, long long batch, const double *x, const orc_fp *p, double *H)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long long q = 0; q < batch; ++q)
        bad |= (orc_hessian(fn, n, x + q * n, p, H + q * (long long)n * n) != 0);
    return bad ? -1 : 0;
}

/* Ragged reference HVPs: request q has function fn[q], size nv[q], and its
 * x, v, out start at off[q] in the packed arrays; Fletcher-Powell request q
 * uses E = Epack + eoff[q] with the shared A, B (leading dimension ld) and is
 * evaluated by fp_hvp (O(n^2) without forming H; O(n^3) for its norm). */
int orc_hvp_ragged(long long nreq, const int *fn, const int *nv, const long long *off,
                   const long long *eoff, const double *xpack, const double *vpack,
                   const double *A, const double *B, const double *Epack, int ld,
                   double *outpack, double *hnorm)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (long long q = 0; q < nreq; ++q) {
        int n = nv[q];
        orc_fp p = { A, B, Epack ? Epack + (eoff ? eoff[q] : 0) : NULL, ld };
        if (fn[q] == ORC_FLETCHER_POWELL) {
            bad |= (fp_hvp(n, xpack + off[q], vpack + off[q], &p, outpack + off[q], hnorm ? hnorm + q : NULL) != 0);
            continue;
        }
        double *H = (double *)malloc(sizeof(double) * (size_t)n * n);
        if (!H) { bad |= 1; continue; }
        bad |= (orc_hessian(fn[q], n, xpack + off[q], &p, H) != 0);
        double fro = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) {
                s += H[(size_t)i * n + j] * vpack[off[q] + j];
                fro += H[(size_t)i * n + j] * H[(size_t)i * n + j];
            }
            outpack[off[q] + i] = s;
        }
        if (hnorm) hnorm[q] = sqrt(fro);
        free(H);
    }
    return bad ? -1 : 0;
}

/* ======================================================================
 * O2 -- the paper's chunked hDual forward mode, step by step
 * ====================================================================== */

/* An hDual<csize> is an array of K = 2*csize + 2 doubles (Sec. IV):
 *   v[0]                 value
 *   v[1]                 d/dx_i            (i = the Hessian row)
 *   v[2 .. csize+1]      d/dx_{cstart+l}   (the chunk's variables)
 *   v[csize+2 .. 2csize+1]  d2/dx_i dx_{cstart+l}
 * Operation counters follow Sec. V: scalar multiplications and additions
 * (a subtraction counts as an addition). */
static _Thread_local long long cnt_mul, cnt_add;

/* Fletcher-Powell H v (and ||H||_F when hnorm is not NULL) without forming
 * H; exported for the pins against H from fp_h times v. */
int orc_fp_hvp(int n, const double *x, const double *v, const orc_fp *p, double *out, double *hnorm)
{
    return fp_hvp(n, x, v, p, out, hnorm);
}

void orc_count_reset(void) { cnt_mul = 0; cnt_add = 0; }
void orc_count_get(long long *mul, long long *add) { *mul = cnt_mul; *add = cnt_add; }

#define HK(c) (2 * (c) + 2)

/* op1 + op2, componentwise (Fig. 1). */
static void hd_add(int c, double *r, const double *a, const double *b)
{
    for (int t = 0; t < HK(c); ++t) r[t] = a[t] + b[t];
    cnt_add += HK(c);
}

/* op1 - op2, componentwise (the rule of + with the sign of op2 flipped). */
static void hd_sub(int c, double *r, const double *a, const double *b)
{
    for (int t = 0; t < HK(c); ++t) r[t] = a[t] - b[t];
    cnt_add += HK(c);
}

/* s + op: only the value changes (Fig. 1, double + hDual). */
static void hd_sadd(int c, double *r, double s, const double *a)
{
    r[0] = s + a[0];
    for (int t = 1; t < HK(c); ++t) r[t] = a[t];
    cnt_add += 1;
}

/* s * op, componentwise (Fig. 1, double * hDual). */
static void hd_smul(int c, double *r, double s, const double *a)
{
    for (int t = 0; t < HK(c); ++t) r[t] = s * a[t];
    cnt_mul += HK(c);
}

/* op1 * op2 (Fig. 1): product rule for the value and the first derivatives,
 * and for each chunk entry the second-order rule of Sec. III-A,
 *   (uw)_{i,l} = u w_{i,l} + u_i w_l + w_i u_l + w u_{i,l}.
 * r must not alias a or b. */
static void hd_mul(int c, double *r, const double *a, const double *b)
{
    r[0] = a[0] * b[0];
    cnt_mul += 1;
    for (int t = 1; t <= c + 1; ++t) {
        r[t] = a[0] * b[t] + b[0] * a[t];
        cnt_mul += 2;
        cnt_add += 1;
    }
    for (int l = 2; l <= c + 1; ++l) {
        r[c + l] = a[0] * b[c + l] + a[1] * b[l] + b[1] * a[l] + b[0] * a[c + l];
        cnt_mul += 4;
        cnt_add += 3;
    }
}

/* phi(op) for a scalar function phi with derivatives d1 = phi'(u), d2 =
 * phi''(u) at the value u (the chain rule of Sec. III-A, written for sin
 * there, for a general phi):
 *   value  phi(u)
 *   first  phi'(u) u_k
 *   second phi'(u) u_{i,l} + phi''(u) u_i u_l
 * r must not alias a. */
static void hd_unary(int c, double *r, const double *a, double phi, double d1, double d2)
{
    r[0] = phi;
    for (int t = 1; t <= c + 1; ++t) r[t] = d1 * a[t];
    cnt_mul += c + 1;
    for (int l = 2; l <= c + 1; ++l) r[c + l] = d1 * a[c + l] + d2 * a[1] * a[l];
    cnt_mul += 3 * c;
    cnt_add += c;
}

static void hd_sin(int c, double *r, const double *a) { hd_unary(c, r, a, sin(a[0]), cos(a[0]), -sin(a[0])); }
static void hd_cos(int c, double *r, const double *a) { hd_unary(c, r, a, cos(a[0]), -sin(a[0]), -cos(a[0])); }
static void hd_exp(int c, double *r, const double *a) { double e = exp(a[0]); hd_unary(c, r, a, e, e, e); }

/* sqrt: phi' = 1/(2 sqrt u), phi'' = -1/(4 u^{3/2}).  At u == 0 the
 * derivatives are infinite; they are returned as such (NaN/Inf propagate),
 * which is why the Ackley Hessian at the origin is excluded from parity. */
static void hd_sqrt(int c, double *r, const double *a)
{
    double s = sqrt(a[0]);
    hd_unary(c, r, a, s, 0.5 / s, -0.25 / (s * a[0]));
}

/* The extended operator set, each through the unary rule above:
 *   log u:      phi' = 1/u,         phi'' = -1/u^2
 *   tanh u:     phi' = 1 - t^2,     phi'' = -2t (1 - t^2),   t = tanh u
 *   tan u:      phi' = 1 + t^2,     phi'' = 2t (1 + t^2),    t = tan u
 *   u^p:        phi' = p u^{p-1},   phi'' = p (p-1) u^{p-2}
 *   1/u:        phi' = -1/u^2,      phi'' = 2/u^3
 *   u / w = u * (1/w) by the product rule;
 *   |u| = sign(u0) u componentwise, sign(0) = +1. */
static void hd_log(int c, double *r, const double *a) { hd_unary(c, r, a, log(a[0]), 1.0 / a[0], -1.0 / (a[0] * a[0])); }
static void hd_tanh(int c, double *r, const double *a)
{
    double t = tanh(a[0]);
    hd_unary(c, r, a, t, 1.0 - t * t, -2.0 * t * (1.0 - t * t));
}
static void hd_tan(int c, double *r, const double *a)
{
    double t = tan(a[0]);
    hd_unary(c, r, a, t, 1.0 + t * t, 2.0 * t * (1.0 + t * t));
}
static void hd_pow(int c, double *r, const double *a, double p)
{
    hd_unary(c, r, a, pow(a[0], p), p * pow(a[0], p - 1.0), p * (p - 1.0) * pow(a[0], p - 2.0));
}
static void hd_recip(int c, double *r, const double *a)
{
    hd_unary(c, r, a, 1.0 / a[0], -1.0 / (a[0] * a[0]), 2.0 / (a[0] * a[0] * a[0]));
}
static void hd_div(int c, double *r, const double *a, const double *b)
{
    double *w = (double *)malloc(sizeof(double) * HK(c));
    hd_recip(c, w, b);
    hd_mul(c, r, a, w);
    free(w);
}
static void hd_abs(int c, double *r, const double *a)
{
    double s = a[0] < 0.0 ? -1.0 : 1.0;
    for (int t = 0; t < HK(c); ++t) r[t] = s * a[t];
}

static void hd_zero(int c, double *r) { memset(r, 0, sizeof(double) * HK(c)); }
static void hd_copy(int c, double *r, const double *a) { memcpy(r, a, sizeof(double) * HK(c)); }

/* ---- the test functions, written once on hDuals (as a user would template
 * f on the number type, Sec. I).  y holds n hDuals, contiguous. ---- */

static void rosen_hd(int c, int n, const double *y, double *out)
{
    int K = HK(c);
    double *acc = (double *)calloc(7 * (size_t)K, sizeof(double));
    double *sq = acc + K, *d = sq + K, *d2 = d + K, *a = d2 + K, *e = a + K, *e2 = e + K;
    for (int k = 0; k + 1 < n; ++k) {
        const double *yk = y + (size_t)k * K, *yk1 = y + (size_t)(k + 1) * K;
        hd_mul(c, sq, yk, yk);          /* x_k^2 */
        hd_sub(c, d, yk1, sq);          /* x_{k+1} - x_k^2 */
        hd_mul(c, d2, d, d);            /* (.)^2 */
        hd_smul(c, a, 100.0, d2);       /* 100 (.)^2 */
        hd_smul(c, e, -1.0, yk);        /* 1 - x_k as (-1) x_k + 1 */
        hd_sadd(c, e, 1.0, e);
        hd_mul(c, e2, e, e);            /* (1 - x_k)^2 */
        hd_add(c, sq, acc, a);          /* acc + 100 (.)^2 + (1 - x_k)^2 */
        hd_add(c, acc, sq, e2);
    }
    hd_copy(c, out, acc);
    free(acc);
}

static void ackley_hd(int c, int n, const double *y, double *out)
{
    int K = HK(c);
    double *S = (double *)calloc(8 * (size_t)K, sizeof(double));
    double *C = S + K, *t = C + K, *u = t + K, *w = u + K, *r = w + K, *t1 = r + K, *t2 = t1 + K;
    for (int k = 0; k < n; ++k) {
        const double *yk = y + (size_t)k * K;
        hd_mul(c, t, yk, yk);           /* S += x_k^2 */
        hd_add(c, u, S, t);
        hd_copy(c, S, u);
        hd_smul(c, t, 2.0 * M_PI, yk);  /* C += cos(2 pi x_k) */
        hd_cos(c, u, t);
        hd_add(c, w, C, u);
        hd_copy(c, C, w);
    }
    hd_smul(c, t, 1.0 / n, S);          /* sqrt(S/n) */
    hd_sqrt(c, r, t);
    hd_smul(c, t, -0.2, r);             /* -20 exp(-0.2 sqrt(S/n)) */
    hd_exp(c, u, t);
    hd_smul(c, t1, -20.0, u);
    hd_smul(c, t, 1.0 / n, C);          /* - exp(C/n) */
    hd_exp(c, u, t);
    hd_smul(c, t2, -1.0, u);
    hd_add(c, w, t1, t2);               /* + 20 + e */
    hd_sadd(c, out, 20.0 + exp(1.0), w);
    free(S);
}

static void fp_hd(int c, int n, const double *y, const orc_fp *p, double *out)
{
    int K = HK(c);
    double *sy = (double *)calloc((2 * (size_t)n + 6) * K, sizeof(double));
    double *cy = sy + (size_t)n * K;
    double *f = cy + (size_t)n * K, *s = f + K, *t = s + K, *u = t + K, *r = u + K, *q = r + K;
    for (int j = 0; j < n; ++j) {
        hd_sin(c, sy + (size_t)j * K, y + (size_t)j * K);
        hd_cos(c, cy + (size_t)j * K, y + (size_t)j * K);
    }
    for (int m = 0; m < n; ++m) {
        hd_zero(c, s);
        for (int j = 0; j < n; ++j) {
            hd_smul(c, t, p->A[(size_t)m * p->ld + j], sy + (size_t)j * K);
            hd_add(c, u, s, t);
            hd_smul(c, t, p->B[(size_t)m * p->ld + j], cy + (size_t)j * K);
            hd_add(c, s, u, t);
        }
        hd_smul(c, t, -1.0, s);         /* r = E_m - s */
        hd_sadd(c, r, p->E[m], t);
        hd_mul(c, q, r, r);             /* f += r^2 */
        hd_add(c, t, f, q);
        hd_copy(c, f, t);
    }
    hd_copy(c, out, f);
    free(sy);
}

/* The extended-operator test function on hDuals, in the order of its
 * definition above. */
static void mix_hd(int c, int n, const double *y, double *out)
{
    int K = HK(c);
    double *acc = (double *)calloc(8 * (size_t)K, sizeof(double));
    double *t1 = acc + K, *t2 = t1 + K, *t3 = t2 + K, *t4 = t3 + K, *t5 = t4 + K, *t6 = t5 + K, *t7 = t6 + K;
    for (int k = 0; k + 1 < n; ++k) {
        const double *yk = y + (size_t)k * K, *yk1 = y + (size_t)(k + 1) * K;
        hd_sub(c, t1, yk1, yk);         /* d = x_{k+1} - x_k */
        hd_mul(c, t2, t1, t1);          /* d^2 */
        hd_mul(c, t3, yk, yk);          /* 1 + x_k^2 */
        hd_sadd(c, t3, 1.0, t3);
        hd_div(c, t4, t2, t3);          /* d^2 / (1 + x_k^2) */
        hd_add(c, t5, acc, t4);
        hd_abs(c, t1, yk);              /* |x_k| x_{k+1} */
        hd_mul(c, t2, t1, yk1);
        hd_add(c, t6, t5, t2);
        hd_mul(c, t1, yk, yk1);         /* tanh(x_k x_{k+1}) */
        hd_tanh(c, t2, t1);
        hd_add(c, acc, t6, t2);
    }
    for (int k = 0; k < n; ++k) {
        const double *yk = y + (size_t)k * K;
        hd_mul(c, t1, yk, yk);          /* log(1 + x_k^2) */
        hd_sadd(c, t2, 1.0, t1);
        hd_log(c, t3, t2);
        hd_add(c, t4, acc, t3);
        hd_sadd(c, t2, 2.0, t1);        /* 0.1 (2 + x_k^2)^{3/2} */
        hd_pow(c, t3, t2, 1.5);
        hd_smul(c, t5, 0.1, t3);
        hd_add(c, t6, t4, t5);
        hd_smul(c, t1, 0.3, yk);        /* tan(0.3 x_k) */
        hd_tan(c, t2, t1);
        hd_add(c, acc, t6, t2);
    }
    const double *y0 = y, *yl = y + (size_t)(n - 1) * K;
    if (y0[0] > yl[0]) {                /* comparison on values */
        hd_mul(c, t1, y0, yl);
    } else {
        hd_mul(c, t2, y0, y0);
        hd_smul(c, t1, -1.0, t2);
    }
    hd_add(c, t7, acc, t1);
    hd_copy(c, out, t7);
    free(acc);
}

static void eval_hd(int fn, int c, int n, const double *y, const orc_fp *p, double *out)
{
    switch (fn) {
    case ORC_ROSENBROCK: rosen_hd(c, n, y, out); break;
    case ORC_ACKLEY: ackley_hd(c, n, y, out); break;
    case ORC_FLETCHER_POWELL: fp_hd(c, n, y, p, out); break;
    case ORC_MIX: mix_hd(c, n, y, out); break;
    }
}

/* CHUNK-INIT (Alg. 4): y[k] = <a_k, [k == i], e_{k - cstart} if k is in the
 * chunk, 0 ...>.  Chunk positions at or beyond n stay zero. */
static void chunk_init(int n, double *y, const double *a, int i, int cstart, int c)
{
    int K = HK(c);
    for (int k = 0; k < n; ++k) {
        double *yk = y + (size_t)k * K;
        yk[0] = a[k];
        yk[1] = 0.0;
        if (k == i) yk[1] = 1.0;
        for (int l = 2; l <= c + 1; ++l) yk[l] = 0.0;
        if (k >= cstart && k < cstart + c) yk[k - cstart + 2] = 1.0;
        for (int l = c + 2; l <= 2 * c + 1; ++l) yk[l] = 0.0;
    }
}

/* CHUNK-INIT exported for the seeding pin. */
void orc_chunk_init(int n, double *y, const double *a, int i, int cstart, int c)
{
    chunk_init(n, y, a, i, cstart, c);
}

/* CHUNK-HESS (Alg. 5): n * nchunk calls of f; chunk l of row i goes to
 * H[i][cstart + l]. */
int orc_chunk_hess(int fn, int n, int c, const double *a, const orc_fp *p, double *H)
{
    int K = HK(c), nchunk = (n + c - 1) / c;
    double *y = (double *)malloc(sizeof(double) * ((size_t)n + 1) * K);
    if (!y) return -1;
    double *temp = y + (size_t)n * K;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < nchunk; ++j) {
            int cstart = j * c;
            chunk_init(n, y, a, i, cstart, c);
            eval_hd(fn, c, n, y, p, temp);
            for (int l = 0; l < c && cstart + l < n; ++l) H[(size_t)i * n + cstart + l] = temp[c + 2 + l];
        }
    free(y);
    return 0;
}

/* SCHUNK-HESS (Alg. 6): only chunks on or above the diagonal chunk are
 * evaluated; the strictly lower part left of the diagonal chunk is then
 * mirrored from the upper triangle. */
int orc_schunk_hess(int fn, int n, int c, const double *a, const orc_fp *p, double *H)
{
    int K = HK(c), nchunk = (n + c - 1) / c;
    double *y = (double *)malloc(sizeof(double) * ((size_t)n + 1) * K);
    if (!y) return -1;
    double *temp = y + (size_t)n * K;
    for (int i = 0; i < n; ++i) {
        int startchunk = i / c;
        for (int j = startchunk; j < nchunk; ++j) {
            int cstart = j * c;
            chunk_init(n, y, a, i, cstart, c);
            eval_hd(fn, c, n, y, p, temp);
            for (int l = 0; l < c && cstart + l < n; ++l) H[(size_t)i * n + cstart + l] = temp[c + 2 + l];
        }
    }
    for (int i = c; i < n; ++i) {
        int endindex = (i / c) * c;
        for (int j = 0; j < endindex; ++j) H[(size_t)i * n + j] = H[(size_t)j * n + i];
    }
    free(y);
    return 0;
}

/* CHESS-VEC (Alg. 7): for each row i, res = sum over chunks of
 * sum_l temp.v[csize+2+l] * in[cstart+l]; out[i] = res. */
int orc_chess_vec(int fn, int n, int c, const double *a, const double *in, const orc_fp *p, double *out)
{
    int K = HK(c), nchunk = (n + c - 1) / c;
    double *y = (double *)malloc(sizeof(double) * ((size_t)n + 1) * K);
    if (!y) return -1;
    double *temp = y + (size_t)n * K;
    for (int i = 0; i < n; ++i) {
        double res = 0.0;
        for (int j = 0; j < nchunk; ++j) {
            int cstart = j * c;
            chunk_init(n, y, a, i, cstart, c);
            eval_hd(fn, c, n, y, p, temp);
            for (int l = 0; l < c && cstart + l < n; ++l) res += temp[c + 2 + l] * in[cstart + l];
        }
        out[i] = res;
    }
    free(y);
    return 0;
}

/* SC-HESS-VEC (Alg. 8, Sec. III-C): rows only evaluate chunks from their
 * diagonal chunk on; an off-diagonal-chunk entry H(i,s) adds H(i,s) in[s]
 * to res[i] and H(i,s) in[i] to res[s]. */
int orc_sc_hess_vec(int fn, int n, int c, const double *a, const double *in, const orc_fp *p, double *out)
{
    int K = HK(c), nchunk = (n + c - 1) / c;
    double *y = (double *)malloc(sizeof(double) * ((size_t)n + 1) * K);
    if (!y) return -1;
    double *temp = y + (size_t)n * K;
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (int i = 0; i < n; ++i) {
        int scn = i / c;
        for (int cn = scn; cn < nchunk; ++cn) {
            int cstart = cn * c;
            chunk_init(n, y, a, i, cstart, c);
            eval_hd(fn, c, n, y, p, temp);
            for (int l = 0; l < c && cstart + l < n; ++l) {
                int s = cstart + l;
                out[i] += temp[c + 2 + l] * in[s];
                if (cn > scn) out[s] += temp[c + 2 + l] * in[i];
            }
        }
    }
    free(y);
    return 0;
}

/* Batched CHESS-VEC over points (the sequential method of Alg. 7 applied to
 * every point, OpenMP across points). */
int orc_chess_vec_batch(int fn, int n, int c, long long batch, const double *x, const double *v,
                        const orc_fp *p, double *out)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (long long q = 0; q < batch; ++q)
        bad |= (orc_chess_vec(fn, n, c, x + q * n, v + q * n, p, out + q * n) != 0);
    return bad ? -1 : 0;
}

/* Exported single hDual operations, for the rule pins. */
void orc_hd_mul(int c, double *r, const double *a, const double *b) { hd_mul(c, r, a, b); }
void orc_hd_add(int c, double *r, const double *a, const double *b) { hd_add(c, r, a, b); }
void orc_hd_sin(int c, double *r, const double *a) { hd_sin(c, r, a); }
void orc_hd_cos(int c, double *r, const double *a) { hd_cos(c, r, a); }
void orc_hd_exp(int c, double *r, const double *a) { hd_exp(c, r, a); }
void orc_hd_sqrt(int c, double *r, const double *a) { hd_sqrt(c, r, a); }
void orc_hd_log(int c, double *r, const double *a) { hd_log(c, r, a); }
void orc_hd_tanh(int c, double *r, const double *a) { hd_tanh(c, r, a); }
void orc_hd_tan(int c, double *r, const double *a) { hd_tan(c, r, a); }
void orc_hd_recip(int c, double *r, const double *a) { hd_recip(c, r, a); }
void orc_hd_abs(int c, double *r, const double *a) { hd_abs(c, r, a); }
void orc_hd_pow(int c, double *r, const double *a, double p) { hd_pow(c, r, a, p); }
void orc_hd_div(int c, double *r, const double *a, const double *b) { hd_div(c, r, a, b); }

/* Evaluate f on a caller-seeded hDual array y (n hDuals of size 2c+2). */
void orc_eval_hd(int fn, int c, int n, const double *y, const orc_fp *p, double *out)
{
    eval_hd(fn, c, n, y, p, out);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the OpenMP loops of the next calls use (from the calling thread);
 * returns the previous setting. */
int orc_set_num_threads(int t)
{
#ifdef _OPENMP
    const int old = omp_get_max_threads();
    if (t > 0) omp_set_num_threads(t);
    return old;
#else
    (void)t;
    return 1;
#endif
}
