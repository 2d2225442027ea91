"""Pins for the FP64 oracle against facts other than the oracle itself.

Each test checks the oracle against something the mathematics or the paper
fixes: hand-derived closed-form values, central finite differences, symmetry,
the four-component rules printed in Sec. III-A, the Sec. V operation counts,
and agreement of its two independent implementations (closed forms O1 and the
chunked hDual algorithms O2).  A dropped term, a wrong sign or index, or a
transposed operand in either implementation fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2410_22575_gb300 import workloads as W

R, A, F, M = W.ROSENBROCK, W.ACKLEY, W.FLETCHER_POWELL, W.MIX
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fp(n, seed=7):
    return W.draw_fp_instance(np.random.Generator(np.random.PCG64(seed)), n)


def _params(orc, fn, n, seed=7):
    if fn != F:
        return None
    inst = _fp(n, seed)
    return orc.FPParams(inst.A, inst.B, inst.E)


def _rand_x(fn, n, seed):
    lo, hi = W.X_RANGE[fn]
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, n)


# ------------------------------------------------------------------ special values
def _read_matrices(path):
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, mat = (s.strip() for s in line.split(";", 1))
        n = int(key.split("=")[1])
        rows = [[float(t) for t in r.split(",")] for r in mat.split(";")]
        out[n] = np.array(rows)
        assert out[n].shape == (n, n)
    return out


def test_rosenbrock_minimizer(orc):
    for n, H in _read_matrices(os.path.join(GOLDEN, "rosenbrock_minimizer.txt")).items():
        x = np.ones(n)
        assert orc.value(R, x) == 0.0
        assert np.all(orc.gradient(R, x) == 0.0)
        np.testing.assert_array_equal(orc.hessian(R, x), H)
    for n in (5, 9):
        H = orc.hessian(R, np.ones(n))
        assert H[0, 0] == 802 and H[n - 1, n - 1] == 200
        assert np.all(np.diag(H)[1:-1] == 1002)
        assert np.all(np.diag(H, 1) == -400) and np.all(np.diag(H, -1) == -400)
        assert np.count_nonzero(H) == 3 * n - 2


def test_rosenbrock_n1_is_zero_function(orc):
    x = np.array([0.7])
    assert orc.value(R, x) == 0.0
    assert orc.hessian(R, x)[0, 0] == 0.0
    assert orc.chunk_hess(R, x, 1)[0, 0] == 0.0


def test_ackley_origin(orc):
    for n in (1, 2, 7):
        x = np.zeros(n)
        # -20 e^0 - e^{n/n} + 20 + e = 0
        assert abs(orc.value(A, x)) < 1e-14
        # sin(0) = 0 and the subgradient convention at S == 0
        assert np.all(orc.gradient(A, x) == 0.0)


@pytest.mark.parametrize("n", [1, 3, 8])
def test_ackley_half_point(orc, n):
    # x_k = 1/2: S = n/4, r = 1/2, E1 = e^{-0.1}, cos(pi) = -1 so C = -n,
    # E2 = e^{-1}, sin(pi) = 0.  Then
    # H = (8 E1/n - 4 pi^2/(e n)) I - (8.8 E1/n^2) 1 1^T.
    x = np.full(n, 0.5)
    E1 = math.exp(-0.1)
    Hx = (8 * E1 / n - 4 * math.pi ** 2 / (math.e * n)) * np.eye(n) - 8.8 * E1 / n ** 2 * np.ones((n, n))
    np.testing.assert_allclose(orc.hessian(A, x), Hx, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n", [1, 4, 6])
def test_ackley_quarter_point(orc, n):
    # x_k = 1/4: S = n/16, r = 1/4, E1 = e^{-0.05}, cos(pi/2) = 0 so C = 0,
    # E2 = 1, sin(pi/2) = 1.  Then
    # H = (16 E1/n) I - ((16.8 E1 + 4 pi^2)/n^2) 1 1^T.
    x = np.full(n, 0.25)
    E1 = math.exp(-0.05)
    Hx = (16 * E1 / n) * np.eye(n) - (16.8 * E1 + 4 * math.pi ** 2) / n ** 2 * np.ones((n, n))
    np.testing.assert_allclose(orc.hessian(A, x), Hx, rtol=1e-12, atol=1e-12)


def test_fletcher_powell_one_variable(orc):
    x = np.array([0.37])
    # A=1, B=0, E=0: f = sin^2 x, f'' = 2 cos 2x
    p = orc.FPParams([[1.0]], [[0.0]], [0.0])
    assert abs(orc.value(F, x, p) - math.sin(0.37) ** 2) < 1e-15
    assert abs(orc.hessian(F, x, p)[0, 0] - 2 * math.cos(0.74)) < 1e-14
    # A=0, B=1, E=1: f = (1 - cos x)^2, f'' = 2 cos x - 2 cos 2x
    p = orc.FPParams([[0.0]], [[1.0]], [1.0])
    assert abs(orc.hessian(F, x, p)[0, 0] - (2 * math.cos(0.37) - 2 * math.cos(0.74))) < 1e-14
    for c in (1, 2):
        assert abs(orc.chunk_hess(F, x, c, p)[0, 0] - (2 * math.cos(0.37) - 2 * math.cos(0.74))) < 1e-14


@pytest.mark.parametrize("n", [2, 5, 32])
def test_fletcher_powell_at_solution(orc, n):
    inst = _fp(n, seed=n)
    p = orc.FPParams(inst.A, inst.B, inst.E)
    x = inst.alpha
    scale = np.abs(inst.A).sum() + np.abs(inst.B).sum()
    assert orc.value(F, x, p) < (1e-13 * scale) ** 2 * n
    assert np.max(np.abs(orc.gradient(F, x, p))) < 1e-9 * scale
    H = orc.hessian(F, x, p)
    w = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert w.min() > -1e-10 * np.abs(w).max()  # 2 J^T J is positive semidefinite


# ------------------------------------------------------------------ finite differences
def _fd_grad(orc, fn, x, p, h):
    g = np.empty_like(x)
    for k in range(len(x)):
        e = np.zeros_like(x)
        e[k] = h * max(1.0, abs(x[k]))
        g[k] = (orc.value(fn, x + e, p) - orc.value(fn, x - e, p)) / (2 * e[k])
    return g


def _fd_hess(orc, fn, x, p, h):
    n = len(x)
    H = np.empty((n, n))
    for k in range(n):
        e = np.zeros_like(x)
        e[k] = h * max(1.0, abs(x[k]))
        H[:, k] = (orc.gradient(fn, x + e, p) - orc.gradient(fn, x - e, p)) / (2 * e[k])
    return H


@pytest.mark.parametrize("fn", [R, A, F, M])
@pytest.mark.parametrize("n", [1, 2, 3, 6])
def test_gradient_vs_finite_differences(orc, fn, n):
    p = _params(orc, fn, n)
    for seed in range(3):
        x = _rand_x(fn, n, 100 + seed)
        g = orc.gradient(fn, x, p)
        gfd = _fd_grad(orc, fn, x, p, 1e-5)
        assert np.max(np.abs(g - gfd)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


@pytest.mark.parametrize("fn", [R, A, F, M])
@pytest.mark.parametrize("n", [1, 2, 3, 6])
def test_hessian_vs_finite_differences(orc, fn, n):
    p = _params(orc, fn, n)
    for seed in range(3):
        x = _rand_x(fn, n, 200 + seed)
        H = orc.hessian(fn, x, p)
        Hfd = _fd_hess(orc, fn, x, p, 1e-6)
        assert np.max(np.abs(H - Hfd)) <= 1e-6 * max(1.0, np.max(np.abs(H)))


@pytest.mark.parametrize("fn", [R, A, F, M])
def test_hvp_vs_directional_difference(orc, fn):
    n = 5
    p = _params(orc, fn, n)
    rng = np.random.Generator(np.random.PCG64(3))
    for seed in range(3):
        x = _rand_x(fn, n, 300 + seed)
        v = rng.uniform(-1, 1, n)
        h = 1e-6
        d = (orc.gradient(fn, x + h * v, p) - orc.gradient(fn, x - h * v, p)) / (2 * h)
        r = orc.hvp(fn, x[None], v[None], p)[0]
        assert np.max(np.abs(r - d)) <= 1e-6 * max(1.0, np.max(np.abs(r)))


@pytest.mark.parametrize("fn", [R, A, F, M])
def test_hessian_symmetric(orc, fn):
    for n in (2, 7, 33):
        p = _params(orc, fn, n)
        H = orc.hessian(fn, _rand_x(fn, n, n), p)
        assert np.max(np.abs(H - H.T)) <= 1e-15 * np.max(np.abs(H))


# ------------------------------------------------------------------ hDual rules
def _parse_vec(s):
    return np.array([float(t) for t in s.split(",")])


def _golden_examples():
    rows = []
    for line in open(os.path.join(GOLDEN, "hdual_worked_examples.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([t.strip() for t in line.split(";")])
    return rows


@pytest.mark.parametrize("row", _golden_examples(), ids=lambda r: r[0])
def test_hdual_worked_examples(orc, row):
    name, c, expr, ins, want = row
    c = int(c)
    env = {}
    for item in ins.split():
        k, vals = item.split("=")
        env[k] = _parse_vec(vals)

    def mul(a, b):
        return orc.hd_op("mul", c, a, b)

    def add(a, b):
        return orc.hd_op("add", c, a, b)

    got = eval(expr, {"mul": mul, "add": add}, env)
    np.testing.assert_array_equal(got, _parse_vec(want))


def test_four_component_rules(orc):
    """c = 1 reproduces the four-component rules printed in Sec. III-A:
    u+v, u*v = <u0 v0, u0 v1 + v0 u1, u0 v2 + v0 u2, u0 v3 + u1 v2 + u2 v1 + u3 v0>,
    sin u = <sin u0, cos u0 u1, cos u0 u2, cos u0 u3 - sin u0 u1 u2>."""
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(20):
        u = rng.uniform(-2, 2, 4)
        v = rng.uniform(-2, 2, 4)
        np.testing.assert_allclose(orc.hd_op("add", 1, u, v), u + v, rtol=0, atol=0)
        want = [u[0] * v[0], u[0] * v[1] + v[0] * u[1], u[0] * v[2] + v[0] * u[2],
                u[0] * v[3] + u[1] * v[2] + u[2] * v[1] + u[3] * v[0]]
        np.testing.assert_allclose(orc.hd_op("mul", 1, u, v), want, rtol=1e-15, atol=1e-15)
        want = [math.sin(u[0]), math.cos(u[0]) * u[1], math.cos(u[0]) * u[2],
                math.cos(u[0]) * u[3] - math.sin(u[0]) * u[1] * u[2]]
        np.testing.assert_allclose(orc.hd_op("sin", 1, u), want, rtol=1e-15, atol=1e-15)


def test_unary_rules_against_calculus(orc):
    """cos, exp, sqrt of g(x, y) = x*y (x seeded as x_i, y as x_j), whose
    second mixed derivative is phi'(xy) + phi''(xy) x y."""
    x, y = 1.3, 0.8
    u = orc.hd_op("mul", 1, [x, 1, 0, 0], [y, 0, 1, 0])
    t = x * y
    cases = {
        "cos": (math.cos(t), -math.sin(t), -math.cos(t)),
        "exp": (math.exp(t), math.exp(t), math.exp(t)),
        "sqrt": (math.sqrt(t), 0.5 / math.sqrt(t), -0.25 * t ** -1.5),
        "sin": (math.sin(t), math.cos(t), -math.sin(t)),
    }
    for op, (f0, f1, f2) in cases.items():
        want = [f0, f1 * y, f1 * x, f1 + f2 * x * y]
        np.testing.assert_allclose(orc.hd_op(op, 1, u), want, rtol=1e-14, atol=1e-14)


def test_extended_unary_rules_against_calculus(orc):
    """log, tanh, tan, 1/u, u^p of g(x, y) = x*y: the mixed second derivative
    is phi'(xy) + phi''(xy) x y, with phi', phi'' from calculus."""
    x, y = 1.3, 0.8
    u = orc.hd_op("mul", 1, [x, 1, 0, 0], [y, 0, 1, 0])
    t = x * y
    th, tn = math.tanh(t), math.tan(t)
    cases = {
        "log": (math.log(t), 1 / t, -1 / t ** 2),
        "tanh": (th, 1 / math.cosh(t) ** 2, -2 * th / math.cosh(t) ** 2),
        "tan": (tn, 1 / math.cos(t) ** 2, 2 * tn / math.cos(t) ** 2),
        "recip": (1 / t, -1 / t ** 2, 2 / t ** 3),
    }
    for op, (f0, f1, f2) in cases.items():
        want = [f0, f1 * y, f1 * x, f1 + f2 * x * y]
        np.testing.assert_allclose(orc.hd_op(op, 1, u), want, rtol=1e-14, atol=1e-14)
    for p in (1.5, -0.5, 3.0):
        want = [t ** p, p * t ** (p - 1) * y, p * t ** (p - 1) * x, p * t ** (p - 1) + p * (p - 1) * t ** (p - 2) * x * y]
        np.testing.assert_allclose(orc.hd_op("pow", 1, u, p), want, rtol=1e-14, atol=1e-14)


def test_division_and_abs_rules(orc):
    """x / y with x seeded as x_i, y as x_j: d/dx = 1/y, d/dy = -x/y^2,
    d2/dxdy = -1/y^2 (quotient rule).  |x*y|: sign(xy) times every component,
    sign(0) = +1."""
    x, y = 1.7, -0.6
    q = orc.hd_op("div", 1, [x, 1, 0, 0], [y, 0, 1, 0])
    np.testing.assert_allclose(q, [x / y, 1 / y, -x / y ** 2, -1 / y ** 2], rtol=1e-15, atol=1e-15)
    # x_i = x_j = x (one variable): d/dx (x / x^2) = -1/x^2, d2/dx2 = 2/x^3
    xx = orc.hd_op("mul", 1, [x, 1, 1, 0], [x, 1, 1, 0])
    q = orc.hd_op("div", 1, [x, 1, 1, 0], xx)
    np.testing.assert_allclose(q, [1 / x, -1 / x ** 2, -1 / x ** 2, 2 / x ** 3], rtol=1e-14, atol=1e-14)
    u = orc.hd_op("mul", 1, [x, 1, 0, 0], [y, 0, 1, 0])
    np.testing.assert_array_equal(orc.hd_op("abs", 1, u), -u)
    np.testing.assert_array_equal(orc.hd_op("abs", 1, -u), -u)
    z = np.array([0.0, 2.0, -3.0, 4.0])
    np.testing.assert_array_equal(orc.hd_op("abs", 1, z), z)


def test_mix_hand_values(orc):
    """The extended-operator function at hand-computed points.  n = 1:
    f = log(1+x^2) + 0.1 (2+x^2)^{3/2} + tan(0.3x) - x^2 (the comparison
    x_0 > x_0 is false).  n = 2 at x = (1, 0): d = -1, q = 2, the branch
    takes x_0 x_1 (1 > 0)."""
    for x0 in (0.0, 0.5, -1.2):
        f = math.log(1 + x0 * x0) + 0.1 * (2 + x0 * x0) ** 1.5 + math.tan(0.3 * x0) - x0 * x0
        assert abs(orc.value(M, np.array([x0])) - f) <= 1e-15 * max(1, abs(f))
    x = np.array([1.0, 0.0])
    f = 1 / 2 + 0 + 0 + (math.log(2) + 0.1 * 3 ** 1.5 + math.tan(0.3)) + (0.1 * 2 ** 1.5) + 0
    assert abs(orc.value(M, x) - f) <= 1e-14
    H = orc.hessian(M, x)
    # H_01: -2/q - 4ad/q^2 + sign(1) + tanh'(0) + T''(0)*0 + branch 1 = -1 + 1 + 1 + 1 + 1
    assert abs(H[0, 1] - 3.0) <= 1e-14 and H[1, 0] == H[0, 1]
    # H_11: 2/q + T''(0) x_0^2 + log'' (2) + 0.3 sqrt(2) + 0 + 0
    assert abs(H[1, 1] - (1.0 + 2.0 + 0.3 * math.sqrt(2))) <= 1e-14


def test_mix_abs_sign_at_zero(orc):
    """|x_k| x_{k+1} at x_k = 0 contributes sign(0) = +1 to H_{k,k+1} in both
    implementations (the convention, not a derivative)."""
    x = np.array([0.0, 0.7, -0.4])
    H = orc.hessian(M, x)
    for c in (1, 2, 3):
        np.testing.assert_allclose(orc.chunk_hess(M, x, c), H, rtol=0, atol=1e-14)
    x2 = x.copy()
    x2[0] = -1e-300  # sign flips to -1
    assert abs((orc.hessian(M, x) - orc.hessian(M, x2))[0, 1] - 2.0) <= 1e-12


def test_chunk_init_seeding(orc):
    """Alg. 4: v[0] = a_k, v[1] = [k == i], v[k - cstart + 2] = 1 for k in the
    chunk, all else 0 -- including the case where row i lies in the chunk."""
    a = np.arange(1.0, 8.0)
    n, c = 7, 3
    for i in range(n):
        for cstart in (0, 3, 6):
            y = orc.chunk_init(a, i, cstart, c)
            assert y.shape == (n, 2 * c + 2)
            np.testing.assert_array_equal(y[:, 0], a)
            np.testing.assert_array_equal(y[:, 1], (np.arange(n) == i).astype(float))
            for k in range(n):
                g = np.zeros(c)
                if cstart <= k < cstart + c:
                    g[k - cstart] = 1.0
                np.testing.assert_array_equal(y[k, 2:c + 2], g)
            assert np.all(y[:, c + 2:] == 0.0)


# ------------------------------------------------------------------ O1 == O2
@pytest.mark.parametrize("fn", [R, A, F, M])
@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_chunk_hess_equals_closed_form(orc, fn, n):
    p = _params(orc, fn, n)
    x = _rand_x(fn, n, 400 + n)
    H = orc.hessian(fn, x, p)
    scale = np.linalg.norm(H) + 1e-300
    for c in sorted({1, 2, 3, 4, 8, 16, 32, n}):
        Hc = orc.chunk_hess(fn, x, c, p)
        assert np.linalg.norm(Hc - H) <= 1e-13 * scale, (c, np.linalg.norm(Hc - H) / scale)


@pytest.mark.parametrize("fn", [R, A, F, M])
@pytest.mark.parametrize("n", [3, 10])
def test_schunk_hess_equals_chunk_hess(orc, fn, n):
    p = _params(orc, fn, n)
    x = _rand_x(fn, n, 500 + n)
    for c in (1, 2, 4, n):
        H1 = orc.chunk_hess(fn, x, c, p)
        H2 = orc.schunk_hess(fn, x, c, p)
        assert np.linalg.norm(H1 - H2) <= 1e-13 * np.linalg.norm(H1)


@pytest.mark.parametrize("fn", [R, A, F, M])
@pytest.mark.parametrize("n", [1, 4, 11])
def test_chess_vec_and_sc_hess_vec(orc, fn, n):
    p = _params(orc, fn, n)
    x = _rand_x(fn, n, 600 + n)
    v = np.random.Generator(np.random.PCG64(n)).uniform(-1, 1, n)
    r, hn = orc.hvp(fn, x[None], v[None], p, with_norm=True)
    den = hn[0] * np.linalg.norm(v)
    for c in (1, 2, 4, 8):
        assert np.linalg.norm(orc.chess_vec(fn, x, v, c, p) - r[0]) <= 1e-13 * den
        assert np.linalg.norm(orc.sc_hess_vec(fn, x, v, c, p) - r[0]) <= 1e-13 * den


def test_batch_permutation(orc):
    b = W.make_batch(A, 9, 40, seed=5)
    r = orc.hvp(A, b.x, b.v)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(40)
    np.testing.assert_array_equal(orc.hvp(A, b.x[perm], b.v[perm]), r[perm])
    rc = orc.chess_vec(A, b.x, b.v, 4)
    np.testing.assert_array_equal(orc.chess_vec(A, b.x[perm], b.v[perm], 4), rc[perm])


def test_ragged_equals_dense(orc):
    rg = W.make_ragged(nreq=60, seed=9, nmax=40)
    out, hn = orc.hvp_ragged(rg.fns, rg.ns, rg.offs, rg.eoffs, rg.xpack, rg.vpack, rg.fp.A, rg.fp.B,
                             rg.Epack, rg.ld)
    for q in range(rg.nreq):
        fn, n, o = int(rg.fns[q]), int(rg.ns[q]), int(rg.offs[q])
        p = None
        if fn == F:
            inst = rg.fp.leading(n)
            p = orc.FPParams(inst.A, inst.B, inst.E)
            np.testing.assert_allclose(rg.Epack[rg.eoffs[q]:rg.eoffs[q] + n], inst.E, rtol=1e-15, atol=1e-12)
        v = rg.vpack[o:o + n]
        r, h = orc.hvp(fn, rg.xpack[o:o + n][None], v[None], p, with_norm=True)
        if fn == F:
            # evaluated without forming H (fp_hvp): the same values up to the
            # summation order
            assert np.linalg.norm(out[o:o + n] - r[0]) <= 1e-14 * h[0] * np.linalg.norm(v)
        else:
            np.testing.assert_allclose(out[o:o + n], r[0], rtol=1e-13, atol=1e-9)
        assert abs(hn[q] - h[0]) <= 1e-13 * h[0]


def test_fp_hvp_without_forming_h(orc):
    """(H v)_j = 2 sum_m J_mj (J v)_m + 2 v_j (P^T r)_j equals the closed-form
    Hessian times v, and its norm the Frobenius norm of that Hessian; at
    n = 1 with A = 1, B = 0, E = 0 (f = sin^2 x) it is 2 cos(2x) v."""
    x = np.array([0.37])
    p = orc.FPParams([[1.0]], [[0.0]], [0.0])
    r, h = orc.fp_hvp(x, np.array([0.5]), p)
    assert abs(r[0] - math.cos(0.74)) < 1e-15 and abs(h - 2 * abs(math.cos(0.74))) < 1e-15
    p = orc.FPParams([[0.0]], [[1.0]], [1.0])  # f = (1 - cos x)^2
    r, h = orc.fp_hvp(x, np.array([-2.0]), p)
    assert abs(r[0] + 2 * (2 * math.cos(0.37) - 2 * math.cos(0.74))) < 1e-14
    for n in (2, 3, 5, 33, 100):
        inst = _fp(n, seed=40 + n)
        p = orc.FPParams(inst.A, inst.B, inst.E)
        rng = np.random.Generator(np.random.PCG64(n))
        for k in range(3):
            x = rng.uniform(-math.pi, math.pi, n) if k else inst.alpha  # at the solution r = 0
            v = rng.uniform(-1, 1, n)
            H = orc.hessian(F, x, p)
            r, h = orc.fp_hvp(x, v, p)
            assert np.linalg.norm(r - H @ v) <= 1e-14 * np.linalg.norm(H) * np.linalg.norm(v), (n, k)
            assert abs(h - np.linalg.norm(H)) <= 1e-13 * np.linalg.norm(H), (n, k)


# ------------------------------------------------------------------ Sec. V counts
@pytest.mark.parametrize("c", [1, 2, 4, 8, 32])
def test_operation_counts(orc, c):
    a = np.ones(2 * c + 2)
    _, m, ad = orc.count_ops(orc.hd_op, "mul", c, a, a)
    # Sec. V states 6c+3 multiplications and 4c additions for one hDual
    # product; the Fig. 1 loops perform 4c+1 additions ((c+1) in the first-
    # derivative loop plus 3c in the second), which is the reading used.
    assert (m, ad) == (6 * c + 3, 4 * c + 1)
    _, m, ad = orc.count_ops(orc.hd_op, "add", c, a, a)
    assert (m, ad) == (0, 2 * c + 2)


def test_chunk_hess_call_counts(orc):
    """CHUNK-HESS calls f n*n/c times; SCHUNK-HESS n(n/c+1)/2 times (Sec. V).
    A call's cost is fixed by c and n, so the ratio of counted multiplications
    equals the ratio of calls."""
    n = 12
    x = _rand_x(R, n, 1)
    for c in (1, 2, 3, 4, 6, 12):
        _, m_full, _ = orc.count_ops(orc.chunk_hess, R, x, c)
        _, m_sym, _ = orc.count_ops(orc.schunk_hess, R, x, c)
        y = orc.chunk_init(x, 0, 0, c)
        _, m_one, _ = orc.count_ops(orc.eval_hd, R, c, y)
        assert m_full == m_one * n * n // c
        assert m_sym == m_one * n * (n // c + 1) // 2
    # Sec. V: the symmetric multiplication count (3/2) n (2n + 2c + n/c + 1) M
    # is smallest at c = sqrt(n/2); for n = 2^{2k+1} that is 2^k.
    for k in range(1, 5):
        nn = 2 ** (2 * k + 1)
        cs = [2 ** e for e in range(0, 2 * k + 2)]
        cost = [1.5 * nn * (2 * nn + 2 * c + nn / c + 1) for c in cs]
        assert cs[int(np.argmin(cost))] == 2 ** k


def test_oracle_thread_count_control(orc):
    """set_num_threads (the bench's single-thread CPU figure) changes the
    OpenMP thread count of later calls and returns the previous one; results
    do not depend on it."""
    b = W.make_batch(A, 12, 30, seed=3)
    want = orc.chess_vec(A, b.x, b.v, 4)
    prev = orc.set_num_threads(1)
    try:
        assert orc.num_threads() == 1
        np.testing.assert_array_equal(orc.chess_vec(A, b.x, b.v, 4), want)
    finally:
        orc.set_num_threads(prev)
    assert orc.num_threads() == prev
