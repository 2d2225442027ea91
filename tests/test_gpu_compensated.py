"""The compensated-FP32 primitives on the device, through the C ABI
(chessfad_eft, chessfad_compensated_rows), against what their published
definitions fix:

* TwoSum (Knuth): s = fl(a + b) and s + e == a + b exactly, for any finite
  pair without overflow, subnormals included.
* TwoProd by FMA: p = fl(a * b) and p + q == a * b exactly when q does not
  underflow.
* Dot2 and Sum2 (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26(6), 2005):
  |res - x^T y| <= u |x^T y| + gamma^2 sum |x_i y_i| (Sum2: sum |a_i|), a
  bound that a plain FP32 recursive dot product breaks on ill-conditioned rows
  (checked below, so the bound has teeth).  The lane-split order of the
  kernels' row reduction adds at most 2 lanes terms to the error sum, hence
  gamma_{2 len + 2 lanes} (twice, for the final rounding).
* Bit for bit, the result of the same published algorithms restated here in
  numpy float32 (round to nearest, as the device's __fadd_rn / __fmaf_rn), in
  the kernels' lane order: lane r takes the blocks r, r + lanes, ... of
  `chunk` elements, and the lanes merge at xor distances lanes/2 .. 1.

Exact references come from math.fsum (the correctly rounded sum of exactly
represented doubles: a sum is zero exactly when fsum returns 0) and from
float64 products of two floats, which are exact."""
import math

import numpy as np
import pytest

import paper_2410_22575_gb300 as cf

pytestmark = pytest.mark.gpu

U = 2.0 ** -24  # unit roundoff of FP32, round to nearest
F32 = np.float32


def gamma(k: int) -> float:
    return k * U / (1.0 - k * U)


def wide_floats(rng, count, emin, emax):
    """sign * m * 2^E with a random 24-bit significand m and E uniform in
    [emin, emax] (exactly representable floats over many binades)."""
    m = 1.0 + rng.integers(0, 2 ** 23, count) / 2.0 ** 23
    e = rng.integers(emin, emax + 1, count)
    s = rng.choice([-1.0, 1.0], count)
    return (s * np.ldexp(m, e)).astype(F32)


def to_dev(a):
    import torch

    return torch.tensor(np.ascontiguousarray(a, dtype=F32), device="cuda")


def run_eft(a, b):
    import torch

    da, db = to_dev(a), to_dev(b)
    outs = [torch.full_like(da, float("nan")) for _ in range(4)]
    assert cf.chessfad_eft(da, db, a.size, *outs) == 0
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def run_rows(a, b, lanes, chunk):
    import torch

    rows, length = a.shape
    da = to_dev(a)
    db = to_dev(b) if b is not None else None
    out = torch.full((rows,), float("nan"), dtype=torch.float32, device="cuda")
    assert cf.chessfad_compensated_rows(da, db, rows, length, lanes, chunk, out) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


# ------------------------------------------------------------ TwoSum, TwoProd
def _sum_pairs(rng):
    n = 1 << 15
    a = wide_floats(rng, n, -140, 120)
    b = np.concatenate([
        wide_floats(rng, n // 4, -140, 120),                         # unrelated magnitudes
        (-a[n // 4: n // 2] * (1 + wide_floats(rng, n // 4, -24, -1))).astype(F32),  # cancellation
        a[n // 2: 3 * n // 4],                                       # doubling
        (a[3 * n // 4:] * wide_floats(rng, n - 3 * n // 4, -30, -20)).astype(F32),  # far apart
    ])
    special = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -149, -(2.0 ** -149), 2.0 ** -126, 3.0, 2.0 ** 100],
                       dtype=F32)
    sa = np.repeat(special, special.size)
    sb = np.tile(special, special.size)
    return np.concatenate([a, sa]), np.concatenate([b, sb])


def test_two_sum_is_error_free():
    a, b = _sum_pairs(np.random.Generator(np.random.PCG64(301)))
    s, e, _, _ = run_eft(a, b)
    # s is the rounded sum (numpy float32 addition rounds to nearest)
    assert np.array_equal((a + b).view(np.uint32), s.view(np.uint32))
    # s + e == a + b exactly, element by element
    bad = [k for k in range(a.size) if math.fsum([float(a[k]), float(b[k]), -float(s[k]), -float(e[k])]) != 0.0]
    assert not bad, (len(bad), bad[:5])
    # and e is the rounding error of s, at most half an ulp of s
    ulp = np.spacing(np.abs(s))
    assert np.all(np.abs(e.astype(np.float64)) <= 0.5 * ulp.astype(np.float64))


def test_two_prod_is_error_free():
    rng = np.random.Generator(np.random.PCG64(302))
    n = 1 << 15
    a = wide_floats(rng, n, -40, 40)
    b = wide_floats(rng, n, -40, 40)
    b[:64] = 1.0  # exact products: the error term is zero
    a[64:128] = F32(2.0 ** 23 + 1)
    b[64:128] = F32(2.0 ** 23 - 1)  # 2^46 - 1 needs 46 bits: the error term is -1
    _, _, p, q = run_eft(a, b)
    assert np.array_equal((a * b).view(np.uint32), p.view(np.uint32))
    exact = a.astype(np.float64) * b.astype(np.float64)  # exact: 48 significant bits at most
    assert np.array_equal(p.astype(np.float64) + q.astype(np.float64), exact)
    assert np.all(q[:64] == 0.0)
    assert np.all(q[64:128] == -1.0)


def test_eft_outputs_are_optional_and_empty_is_a_no_op():
    import torch

    a = to_dev(np.array([1.0, 2.0 ** -30], F32))
    b = to_dev(np.array([2.0 ** -30, 3.0], F32))
    e = torch.full_like(a, 7.0)
    assert cf.chessfad_eft(a, b, 2, None, e, None, None) == 0
    assert cf.chessfad_eft(a, b, 0, None, e, None, None) == 0
    torch.cuda.synchronize()
    assert e.cpu().tolist() == [2.0 ** -30, 2.0 ** -30]


# ------------------------------------------------------------ Dot2, Sum2
def restated_rows(a, b, lanes, chunk):
    """Dot2 (b given) or Sum2 (b None) of Ogita, Rump & Oishi, per lane over
    its blocks, lanes merged pairwise at xor distances lanes/2 .. 1, every
    operation a float32 operation rounded to nearest."""

    def two_sum(x, y):
        s = (x + y).astype(F32)
        bb = (s - x).astype(F32)
        return s, ((x - (s - bb)).astype(F32) + (y - bb).astype(F32)).astype(F32)

    def two_prod(x, y):
        p = (x * y).astype(F32)
        q = (x.astype(np.float64) * y.astype(np.float64) - p.astype(np.float64)).astype(F32)
        return p, q

    rows, length = a.shape
    S = np.zeros((lanes, rows), F32)
    E = np.zeros((lanes, rows), F32)
    for r in range(lanes):
        for blk in range(r, (length + chunk - 1) // chunk, lanes):
            for j in range(blk * chunk, min(length, (blk + 1) * chunk)):
                if b is None:
                    S[r], t = two_sum(S[r], a[:, j])
                    E[r] = (E[r] + t).astype(F32)
                else:
                    p, q = two_prod(a[:, j], b[:, j])
                    S[r], t = two_sum(S[r], p)
                    E[r] = (E[r] + (t + q).astype(F32)).astype(F32)
    off = lanes // 2
    while off:
        S2, E2 = S.copy(), E.copy()
        for r in range(lanes):
            o = r ^ off
            S2[r], t = two_sum(S[r], S[o])
            E2[r] = ((E[r] + E[o]).astype(F32) + t).astype(F32)
        S, E = S2, E2
        off //= 2
    return (S[0] + E[0]).astype(F32)


def dot_rows(rng, rows, length, cond):
    """Rows of x, y: well conditioned (cond False) or with pairs of nearly
    cancelling products spread over the row (condition numbers up to ~1e7)."""
    x = wide_floats(rng, rows * length, -8, 8).reshape(rows, length)
    y = wide_floats(rng, rows * length, -8, 8).reshape(rows, length)
    if cond and length >= 2:
        h = length // 2
        d = wide_floats(rng, rows * h, -24, -12).reshape(rows, h)
        x[:, h:2 * h] = x[:, :h]
        y[:, h:2 * h] = (-y[:, :h] * (1 + d)).astype(F32)
        for r in range(rows):
            perm = rng.permutation(length)
            x[r], y[r] = x[r, perm], y[r, perm]
    return x, y


def exact_rows(x, y):
    prods = x.astype(np.float64) * (y.astype(np.float64) if y is not None else 1.0)
    return np.array([math.fsum(r) for r in prods]), np.abs(prods).sum(axis=1)


def plain_rows(x, y):
    acc = np.zeros(x.shape[0], F32)
    for j in range(x.shape[1]):
        acc = (acc + ((x[:, j] * y[:, j]).astype(F32) if y is not None else x[:, j])).astype(F32)
    return acc


CASES = [(1, 1, 1), (7, 2, 1), (64, 4, 16), (300, 8, 8), (512, 32, 32), (512, 1, 1), (130, 16, 4)]


@pytest.mark.parametrize("length,lanes,chunk", CASES)
@pytest.mark.parametrize("dot", [True, False])
def test_rows_within_the_published_bound_and_bitwise_restated(length, lanes, chunk, dot):
    rng = np.random.Generator(np.random.PCG64(400 + length + lanes + chunk + dot))
    rows = 37  # not a multiple of the rows a warp serves: a ragged last group
    x1, y1 = dot_rows(rng, rows, length, cond=False)
    x2, y2 = dot_rows(rng, rows, length, cond=True)
    x, y = np.concatenate([x1, x2]), np.concatenate([y1, y2])
    if not dot:
        x = (x * y).astype(F32)  # ill-conditioned sums from the cancelling products
        y = None
    got = run_rows(x, y, lanes, chunk)
    exact, absum = exact_rows(x, y)
    n_err = 2 * length + 2 * lanes
    bound = U * np.abs(exact) + 2.0 * gamma(n_err) ** 2 * absum + 2.0 ** -52 * np.abs(exact)
    err = np.abs(got.astype(np.float64) - exact)
    assert np.all(err <= bound), (float(np.max(err / np.maximum(bound, 1e-300))),)
    assert np.array_equal(got.view(np.uint32), restated_rows(x, y, lanes, chunk).view(np.uint32))
    if length >= 64:
        # the bound separates compensated from plain FP32 on the cancelling rows
        perr = np.abs(plain_rows(x, y).astype(np.float64) - exact)
        assert np.mean(perr[rows:] > bound[rows:]) > 0.5


def test_rows_empty_and_zero_length():
    import torch

    out = torch.full((5,), 7.0, device="cuda")
    assert cf.chessfad_compensated_rows(None, None, 0, 4, 4, 1, out) == 0
    assert cf.chessfad_compensated_rows(None, None, 5, 0, 4, 1, out) == 0
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0] * 5


def test_rows_reproducible_and_independent_of_other_rows():
    rng = np.random.Generator(np.random.PCG64(450))
    x, y = dot_rows(rng, 300, 256, cond=True)
    a = run_rows(x, y, 8, 8)
    assert np.array_equal(a.view(np.uint32), run_rows(x, y, 8, 8).view(np.uint32))
    perm = rng.permutation(300)
    assert np.array_equal(a[perm].view(np.uint32), run_rows(x[perm], y[perm], 8, 8).view(np.uint32))
