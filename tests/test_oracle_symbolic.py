"""The oracle's closed forms (O1) against symbolic differentiation.

SymPy differentiates each test function, written here from its definition
(Sec. VII names the three functions; their formulas are the standard ones, and
the extended-operator function is this project's own), and the derivatives are
evaluated in 40-digit arithmetic at the oracle's inputs.  Finite differences pin
the closed forms to about 1e-6; this pin holds them to the FP64 rounding of the
formulas (1e-12 of the Hessian's Frobenius norm), so even a small term that is
wrong or missing shows.  Where a function is not smooth (|x|, a branch), the
expression on the side of the kink that the point lies on is differentiated."""
import math

import numpy as np
import pytest

from paper_2410_22575_gb300 import workloads as W

sympy = pytest.importorskip("sympy")
mpmath = pytest.importorskip("mpmath")

R, A, F, M = W.ROSENBROCK, W.ACKLEY, W.FLETCHER_POWELL, W.MIX
DPS = 40


def _exact(v):
    return sympy.Float(float(v), DPS)  # the double's exact binary value


def _function(fn, x, xs, inst):
    n = len(xs)
    if fn == R:
        return sum(100 * (xs[k + 1] - xs[k] ** 2) ** 2 + (1 - xs[k]) ** 2 for k in range(n - 1))
    if fn == A:
        S = sum(t ** 2 for t in xs)
        C = sum(sympy.cos(2 * sympy.pi * t) for t in xs)
        return -20 * sympy.exp(-sympy.Rational(1, 5) * sympy.sqrt(S / n)) - sympy.exp(C / n) + 20 + sympy.E
    if fn == F:
        f = 0
        for m in range(n):
            r = _exact(inst.E[m]) - sum(_exact(inst.A[m, j]) * sympy.sin(xs[j]) +
                                        _exact(inst.B[m, j]) * sympy.cos(xs[j]) for j in range(n))
            f += r ** 2
        return f
    # the extended-operator function; |x_k| = sign(x_k) x_k and the branch
    # taken at the point
    f = 0
    for k in range(n - 1):
        f += (xs[k + 1] - xs[k]) ** 2 / (1 + xs[k] ** 2) + math.copysign(1.0, x[k]) * xs[k] * xs[k + 1] \
             + sympy.tanh(xs[k] * xs[k + 1])
    for k in range(n):
        f += sympy.log(1 + xs[k] ** 2) + sympy.Rational(1, 10) * (2 + xs[k] ** 2) ** sympy.Rational(3, 2) \
             + sympy.tan(sympy.Rational(3, 10) * xs[k])
    f += xs[0] * xs[n - 1] if x[0] > x[n - 1] else -xs[0] ** 2
    return f


def _symbolic(fn, x, inst):
    n = len(x)
    xs = sympy.symbols(f"x0:{n}")
    f = _function(fn, x, xs, inst)
    g = [sympy.diff(f, t) for t in xs]
    H = [[sympy.diff(gi, t) for t in xs] for gi in g]
    pt = {t: _exact(v) for t, v in zip(xs, x)}
    ev = lambda e: float(sympy.N(sympy.sympify(e).subs(pt), DPS))
    return ev(f), np.array([ev(e) for e in g]), np.array([[ev(e) for e in row] for row in H])


@pytest.mark.parametrize("fn", [R, A, F, M])
@pytest.mark.parametrize("n", [1, 2, 4])
def test_closed_forms_equal_symbolic_derivatives(orc, fn, n):
    inst = W.draw_fp_instance(np.random.Generator(np.random.PCG64(17)), n) if fn == F else None
    p = orc.FPParams(inst.A, inst.B, inst.E) if fn == F else None
    lo, hi = W.X_RANGE[fn]
    for seed in range(2):
        x = np.random.Generator(np.random.PCG64(900 + 10 * n + seed)).uniform(lo, hi, n)
        f, g, H = _symbolic(fn, x, inst)
        Ho = orc.hessian(fn, x, p)
        go = orc.gradient(fn, x, p)
        assert np.linalg.norm(Ho - H) <= 1e-12 * max(np.linalg.norm(H), 1e-300), (fn, n, seed)
        assert np.linalg.norm(go - g) <= 1e-12 * max(np.linalg.norm(g), 1.0), (fn, n, seed)
        assert abs(orc.value(fn, x, p) - f) <= 1e-12 * max(abs(f), 1.0), (fn, n, seed)
        # and H v through the batched entry point
        v = np.random.Generator(np.random.PCG64(950 + seed)).uniform(-1, 1, n)
        r = orc.hvp(fn, x[None], v[None], p)[0]
        assert np.linalg.norm(r - H @ v) <= 1e-12 * max(np.linalg.norm(H) * np.linalg.norm(v), 1e-300)
