"""The seeded inputs follow the recipe the design states, draw for draw:
numpy.random.Generator(PCG64(seed)), uniform draws in a fixed order.  Each
named workload is regenerated here from that recipe alone and compared bit
for bit, so a change of order, range or seed in the generator cannot pass
unnoticed (the benchmark's inputs and the tests' inputs are these draws)."""
import math

import numpy as np
import pytest

from paper_2410_22575_gb300 import workloads as W


def _gen(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("name,lo,hi,n,batch,seed", [
    ("rosenbrock_n16", -2.0, 2.0, 16, 4096, 0),
    ("ackley_n64", -5.0, 5.0, 64, 65536, 1),
    ("rosenbrock_n256", -2.0, 2.0, 256, 1024, 3),
])
def test_dense_workloads_follow_the_recipe(name, lo, hi, n, batch, seed):
    rng = _gen(seed)
    x = rng.uniform(lo, hi, (batch, n))
    v = rng.uniform(-1.0, 1.0, (batch, n))
    b = W.workload(name)
    assert (b.n, b.batch) == (n, batch)
    np.testing.assert_array_equal(b.x, x)
    np.testing.assert_array_equal(b.v, v)
    assert b.fp is None


def test_fletcher_powell_workload_follows_the_recipe():
    rng = _gen(2)
    alpha = rng.uniform(-math.pi, math.pi, 32)
    A = rng.uniform(-100.0, 100.0, (32, 32))
    B = rng.uniform(-100.0, 100.0, (32, 32))
    x = rng.uniform(-math.pi, math.pi, (16384, 32))
    v = rng.uniform(-1.0, 1.0, (16384, 32))
    b = W.workload("fletcher_powell_n32")
    np.testing.assert_array_equal(b.fp.alpha, alpha)
    np.testing.assert_array_equal(b.fp.A, A)
    np.testing.assert_array_equal(b.fp.B, B)
    np.testing.assert_array_equal(b.x, x)
    np.testing.assert_array_equal(b.v, v)
    # E_m = sum_j A_mj sin(alpha_j) + B_mj cos(alpha_j): alpha zeroes every residual
    E = np.array([math.fsum(A[m] * np.sin(alpha)) + math.fsum(B[m] * np.cos(alpha)) for m in range(32)])
    np.testing.assert_allclose(b.fp.E, E, rtol=0, atol=1e-11)


def test_uneven_batch_follows_the_recipe():
    rng = _gen(4)
    nreq = 100000
    fns = rng.integers(0, 3, size=nreq)
    ns = np.clip(np.rint(np.exp(rng.uniform(math.log(2.0), math.log(512.0), size=nreq))), 2, 512).astype(int)
    alpha = rng.uniform(-math.pi, math.pi, 512)
    A = rng.uniform(-100.0, 100.0, (512, 512))
    B = rng.uniform(-100.0, 100.0, (512, 512))
    total = int(ns.sum())
    u = rng.uniform(0.0, 1.0, total)
    v = rng.uniform(-1.0, 1.0, total)
    rg = W.make_ragged()
    np.testing.assert_array_equal(rg.fns, fns)
    np.testing.assert_array_equal(rg.ns, ns)
    np.testing.assert_array_equal(rg.fp.A, A)
    np.testing.assert_array_equal(rg.fp.B, B)
    np.testing.assert_array_equal(rg.vpack, v)
    # x: each request's uniforms scaled to its function's range, packed in request order
    assert rg.offs[0] == 0 and np.array_equal(np.diff(rg.offs), ns[:-1])
    ranges = {0: (-2.0, 2.0), 1: (-5.0, 5.0), 2: (-math.pi, math.pi)}
    for q in np.random.Generator(np.random.PCG64(0)).choice(nreq, 300, replace=False):
        lo, hi = ranges[int(fns[q])]
        o, n = int(rg.offs[q]), int(ns[q])
        np.testing.assert_array_equal(rg.xpack[o:o + n], lo + (hi - lo) * u[o:o + n])
        if fns[q] == 2:  # E of size n from the leading n x n block and alpha[:n]
            E = A[:n, :n] @ np.sin(alpha[:n]) + B[:n, :n] @ np.cos(alpha[:n])
            np.testing.assert_allclose(rg.Epack[rg.eoffs[q]:rg.eoffs[q] + n], E, rtol=0, atol=1e-9)
    # log-uniform sizes over [2, 512]: the mean of ln n sits at the middle of the range
    assert ns.min() == 2 and ns.max() == 512
    assert abs(np.mean(np.log(ns)) - 0.5 * (math.log(2) + math.log(512))) < 0.02
