"""Source text of the test functions as user-supplied functions (the form a
user of chessfad_user_fn_create writes): the paper's three test functions
(Sec. VII) and the extended-operator function of the oracle, each written
once as a template on the number type.  Fletcher-Powell reads A, B (row-major
n x n) and E from params, concatenated."""

ROSENBROCK = r"""
template <class R, class X>
R rosenbrock(const X &x, int n, const double *params)
{
    R f = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
        R a = x[k];
        R d = x[k + 1] - a * a;
        R e = 1.0 - a;
        f += 100.0 * d * d + e * e;
    }
    return f;
}
"""

ACKLEY = r"""
template <class R, class X>
R ackley(const X &x, int n, const double *params)
{
    R s = 0.0, c = 0.0;
    for (int k = 0; k < n; ++k) {
        R a = x[k];
        s += a * a;
        c += cos(6.283185307179586 * a);
    }
    return -20.0 * exp(-0.2 * sqrt(s / double(n))) - exp(c / double(n)) + 20.0 + 2.718281828459045;
}
"""

FLETCHER_POWELL = r"""
template <class R, class X>
R fletcher_powell(const X &x, int n, const double *params)
{
    const double *A = params, *B = params + n * n, *E = params + 2 * n * n;
    R f = 0.0;
    for (int m = 0; m < n; ++m) {
        R r = E[m];
        for (int j = 0; j < n; ++j) {
            R xj = x[j];
            r -= A[m * n + j] * sin(xj) + B[m * n + j] * cos(xj);
        }
        f += r * r;
    }
    return f;
}
"""

MIX = r"""
template <class R, class X>
R mix(const X &x, int n, const double *params)
{
    R f = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
        R a = x[k], b = x[k + 1];
        R d = b - a;
        f += d * d / (1.0 + a * a) + abs(a) * b + tanh(a * b);
    }
    for (int k = 0; k < n; ++k) {
        R a = x[k];
        f += log(1.0 + a * a) + 0.1 * pow(2.0 + a * a, 1.5) + tan(0.3 * a);
    }
    R x0 = x[0], xl = x[n - 1];
    if (x0 > xl)
        f += x0 * xl;
    else
        f -= x0 * x0;
    return f;
}
"""

SOURCES = {0: (ROSENBROCK, "rosenbrock"), 1: (ACKLEY, "ackley"), 2: (FLETCHER_POWELL, "fletcher_powell"),
           3: (MIX, "mix")}
