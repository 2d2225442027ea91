"""Parity of the CUDA path with the FP64 oracle, element by element, through
the C ABI.  Bounds (per point, normalised by ||H||_F ||v||_2, or ||H||_F for a
Hessian): 1e-12 for FP64 and 1e-5 for compensated FP32.  For FP32 the oracle
receives the same float-rounded inputs the device holds."""
import math

import numpy as np
import pytest

import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import workloads as W

from gpu_helpers import BOUND, Dev, hessian_err, hvp_err

pytestmark = pytest.mark.gpu

FNS = [W.ROSENBROCK, W.ACKLEY, W.FLETCHER_POWELL]
PRECS = [cf.FP64, cf.FP32_COMP]
CHUNKS = [1, 2, 4, 8, 16, 32]


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("c", CHUNKS)
def test_hvp_and_hessian_every_chunk(fn, prec, c):
    # n = 19: ragged last chunk for every c > 1, rows spanning several lanes;
    # 150 points: several CTAs and a partial last CTA.
    d = Dev(W.make_batch(fn, 19, 150, seed=10 + c), prec)
    e = hvp_err(d, d.hvp(csize=c))
    assert e.max() <= BOUND[prec], (e.max(), np.median(e))
    e = hessian_err(d, d.hessian(csize=c))
    assert e.max() <= BOUND[prec], (e.max(), np.median(e))


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 31, 64])
def test_sizes(fn, prec, n):
    d = Dev(W.make_batch(fn, n, 97, seed=100 + n), prec)
    for c in (1, 4, 16):
        e = hvp_err(d, d.hvp(csize=c))
        assert e.max() <= BOUND[prec], (c, e.max())


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
def test_launch_configurations(fn, prec):
    d = Dev(W.make_batch(fn, 24, 70, seed=7), prec)
    ref = None
    for c in (2, 8):
        nch = -(-24 // c)
        for tpr in (1, 2, 4, 8, 16, 32):
            for bt in (32, 96, 256):
                cfg = cf.Config(c, tpr, bt)
                out = d.hvp(cfg=cfg)
                e = hvp_err(d, out)
                assert e.max() <= BOUND[prec], (c, tpr, bt, e.max())
        H = d.hessian(cfg=cf.Config(c, 4, 64))
        assert hessian_err(d, H).max() <= BOUND[prec]


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
def test_max_size(fn, prec):
    # n = CHESSFAD_MAX_N at a few points; FP at this size streams A/B tiles.
    d = Dev(W.make_batch(fn, 512, 2 if fn == W.FLETCHER_POWELL else 3, seed=5), prec)
    c = 32 if prec == cf.FP32_COMP else 16
    e = hvp_err(d, d.hvp(csize=c))
    assert e.max() <= BOUND[prec], e.max()


@pytest.mark.parametrize("prec", PRECS)
def test_fletcher_powell_tiled_rows(prec):
    # n = 300 does not fit one shared-memory tile of A and B; also ld > n.
    rng = np.random.Generator(np.random.PCG64(3))
    inst = W.draw_fp_instance(rng, 320).leading(300)
    A = np.zeros((300, 320)); A[:, :300] = inst.A
    B = np.zeros((300, 320)); B[:, :300] = inst.B
    b = W.Batch("fp300", W.FLETCHER_POWELL, 300, rng.uniform(-math.pi, math.pi, (3, 300)),
                rng.uniform(-1, 1, (3, 300)), W.FPInstance(inst.alpha, A, B, inst.E))
    d = Dev(b, prec)
    for c in (4, 8):
        e = hvp_err(d, d.hvp(csize=c))
        assert e.max() <= BOUND[prec], (c, e.max())


def test_batch_zero_and_nan_propagation():
    import torch

    b = W.make_batch(W.ACKLEY, 9, 20, seed=1)
    b.x[3, 2] = np.nan
    d = Dev(b, cf.FP64)
    out = d.hvp(csize=4)
    assert np.all(np.isnan(out[3]))
    ok = np.ones(20, bool)
    ok[3] = False
    assert np.all(np.isfinite(out[ok]))
    z = torch.zeros((0, 9), dtype=torch.float64, device="cuda:0")
    assert cf.chessfad_hvp(W.ACKLEY, 9, 0, 4, z, z, z, None, cf.FP64) == 0


def test_fp64_bitwise_deterministic_and_point_independent():
    d = Dev(W.make_batch(W.FLETCHER_POWELL, 17, 64, seed=2), cf.FP64)
    a = d.hvp(csize=4)
    b = d.hvp(csize=4)
    assert np.array_equal(a, b)
    # permuting the batch permutes the outputs bit for bit (points are independent)
    perm = np.random.Generator(np.random.PCG64(0)).permutation(64)
    bp = W.Batch("p", d.b.fn, d.b.n, d.b.x[perm], d.b.v[perm], d.b.fp)
    dp = Dev(bp, cf.FP64)
    assert np.array_equal(dp.hvp(csize=4), a[perm])


def test_side_stream():
    import torch

    d = Dev(W.make_batch(W.ROSENBROCK, 16, 50, seed=4), cf.FP32_COMP)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = cf.hvp(W.ROSENBROCK, d.x, d.v, csize=4, prec=cf.FP32_COMP, stream=s)
    s.synchronize()
    e = hvp_err(d, out.double().cpu().numpy())
    assert e.max() <= BOUND[cf.FP32_COMP]


def test_hessian_symmetry_within_bound():
    for prec in PRECS:
        d = Dev(W.make_batch(W.ACKLEY, 20, 10, seed=8), prec)
        H = d.hessian(csize=8)
        asym = np.linalg.norm(H - np.swapaxes(H, 1, 2), axis=(1, 2)) / np.linalg.norm(H, axis=(1, 2))
        assert asym.max() <= 2 * BOUND[prec]


def test_kernel_info_and_peak():
    info = cf.chessfad_kernel_info(W.ACKLEY, cf.FP32_COMP, 8, True)
    assert 16 <= info["registers"] <= 255 and info["local_bytes"] >= 0
    f32 = cf.chessfad_peak_flops(cf.FP32_COMP)
    f64 = cf.chessfad_peak_flops(cf.FP64)
    assert 1e13 < f32 < 2e14
    assert 1e11 < f64 < f32
    for prec in (cf.FP32_COMP, cf.FP64):
        reg, lit = cf.chessfad_peak_operand_rates(prec)
        assert 1e11 < reg < 2e14 and 1e11 < lit < 2e14


# ------------------------------------------------------------------ symmetric method
@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("c", CHUNKS)
def test_symmetric_every_chunk(fn, prec, c):
    """SC-HESS-VEC (Alg. 8) and SCHUNK-HESS (Alg. 6) against the oracle, n = 19
    (ragged last chunk and last chunk row)."""
    d = Dev(W.make_batch(fn, 19, 75, seed=300 + c), prec)
    for tpp in (8, 16, 32, 64):
        cfg = cf.Config(c, 0, 0, cf.SYMMETRIC, tpp)
        e = hvp_err(d, d.hvp(cfg=cfg))
        assert e.max() <= BOUND[prec], (tpp, e.max())
        e = hessian_err(d, d.hessian(cfg=cfg))
        assert e.max() <= BOUND[prec], (tpp, e.max())


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [1, 2, 3, 16, 64, 128])
def test_symmetric_sizes(fn, prec, n):
    batch = 40 if n <= 64 else 6
    d = Dev(W.make_batch(fn, n, batch, seed=400 + n), prec)
    for c in (4, 16):
        cfg = cf.Config(c, 0, 0, cf.SYMMETRIC, 0)
        assert hvp_err(d, d.hvp(cfg=cfg)).max() <= BOUND[prec], c
        assert hessian_err(d, d.hessian(cfg=cfg)).max() <= BOUND[prec], c


def test_symmetric_limits():
    # symmetric Hessian at n = 300 (no staging); symmetric HVP beyond the
    # staging limit (FP64 n > ~200, FP32 n > ~280) sums rows in FP64
    # shared-memory accumulators
    d = Dev(W.make_batch(W.ROSENBROCK, 300, 2, seed=1), cf.FP64)
    cfg = cf.Config(16, 0, 0, cf.SYMMETRIC, 128)
    assert hessian_err(d, d.hessian(cfg=cfg)).max() <= BOUND[cf.FP64]
    assert hvp_err(d, d.hvp(cfg=cfg)).max() <= BOUND[cf.FP64]
    d32 = Dev(W.make_batch(W.ACKLEY, 200, 3, seed=2), cf.FP32_COMP)
    assert hvp_err(d32, d32.hvp(cfg=cf.Config(8, 0, 0, cf.SYMMETRIC, 64))).max() <= BOUND[cf.FP32_COMP]


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
def test_symmetric_hvp_accumulator_form(fn, prec):
    """n = 512 and 300: the chunk matrix of a point exceeds shared memory, the
    symmetric HVP accumulates rows in FP64 (both updates of Alg. 8)."""
    for n, batch in ((300, 5), (512, 3)):
        if fn == W.FLETCHER_POWELL and n == 512:
            batch = 2
        d = Dev(W.make_batch(fn, n, batch, seed=60 + n), prec)
        for c, tpp in ((8, 64), (16, 128)):
            cfg = cf.Config(c, 0, 0, cf.SYMMETRIC, tpp)
            first = d.hvp(cfg=cfg)
            e = hvp_err(d, first)
            assert e.max() <= BOUND[prec], (n, c, e.max())
            # the accumulators add the staged contributions in thread order:
            # bitwise reproducible
            assert np.array_equal(first, d.hvp(cfg=cfg)), (n, c)
        e = hvp_err(d, d.hvp(cfg=cf.Config(8, 0, 0, cf.SYMMETRIC_SPARSE, 64)))
        assert e.max() <= BOUND[prec], (n, "sparse", e.max())


def test_symmetric_deterministic_and_equal_to_plain_within_bound():
    d = Dev(W.make_batch(W.ACKLEY, 64, 300, seed=6), cf.FP64)
    cfg = cf.Config(8, 0, 0, cf.SYMMETRIC, 32)
    a = d.hvp(cfg=cfg)
    b = d.hvp(cfg=cfg)
    assert np.array_equal(a, b)
    p = d.hvp(cfg=cf.Config(8, 1, 256))
    ref, hn = d.ref_hvp()
    assert np.max(np.linalg.norm(a - p, axis=1) / (hn * np.linalg.norm(d.vh, axis=1))) <= 2e-12


# ------------------------------------------------------------------ seed-sparse symmetric method
SPARSE_CHUNKS = [4, 8, 16]


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("c", SPARSE_CHUNKS)
def test_symmetric_sparse_every_chunk(fn, prec, c):
    """The seed-sparse symmetric kernels against the oracle: n = 19 and 37
    (ragged last chunk; variables on both sides of the seeded chunk)."""
    for n, seed in ((19, 500 + c), (37, 600 + c)):
        d = Dev(W.make_batch(fn, n, 61, seed=seed), prec)
        for tpp in (32, 64):
            cfg = cf.Config(c, 0, 0, cf.SYMMETRIC_SPARSE, tpp)
            e = hvp_err(d, d.hvp(cfg=cfg))
            assert e.max() <= BOUND[prec], (n, tpp, e.max())
            e = hessian_err(d, d.hessian(cfg=cfg))
            assert e.max() <= BOUND[prec], (n, tpp, e.max())


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 64, 128])
def test_symmetric_sparse_sizes(fn, prec, n):
    batch = 40 if n <= 64 else 6
    d = Dev(W.make_batch(fn, n, batch, seed=700 + n), prec)
    for c in SPARSE_CHUNKS:
        cfg = cf.Config(c, 0, 0, cf.SYMMETRIC_SPARSE, 0)
        assert hvp_err(d, d.hvp(cfg=cfg)).max() <= BOUND[prec], c
        assert hessian_err(d, d.hessian(cfg=cfg)).max() <= BOUND[prec], c


def test_symmetric_sparse_matches_dense_and_is_deterministic():
    for fn in FNS:
        d = Dev(W.make_batch(fn, 48, 200, seed=9), cf.FP64)
        sp = cf.Config(8, 0, 0, cf.SYMMETRIC_SPARSE, 32)
        a = d.hvp(cfg=sp)
        assert np.array_equal(a, d.hvp(cfg=sp))
        dense = d.hvp(cfg=cf.Config(8, 0, 0, cf.SYMMETRIC, 32))
        ref, hn = d.ref_hvp()
        assert np.max(np.linalg.norm(a - dense, axis=1) / (hn * np.linalg.norm(d.vh, axis=1))) <= 2e-12


def test_symmetric_sparse_chunk_auto_and_nan_point():
    """csize = 0 with the seed-sparse method picks one of its chunk sizes; a
    NaN input reaches its own point's output and no other point's."""
    b = W.make_batch(W.ROSENBROCK, 21, 30, seed=11)
    b.x[4, 7] = np.nan
    d = Dev(b, cf.FP64)
    out = d.hvp(cfg=cf.Config(0, 0, 0, cf.SYMMETRIC_SPARSE, 32))
    assert np.any(np.isnan(out[4]))
    ok = np.ones(30, bool)
    ok[4] = False
    assert np.all(np.isfinite(out[ok]))
    e = hvp_err(d, out)
    assert e[ok].max() <= BOUND[cf.FP64]


# ------------------------------------------------------------------ L0 / L1 / L2
@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", PRECS)
def test_decompositions_l0_l1_l2(fn, prec):
    """The paper's three GPU decompositions (Sec. VI) compute the same HVP:
    L0 (one thread per point, Alg. 9) and L1 (one thread per row, Alg. 10)
    evaluate the same chunks in the same order per row, so their results are
    identical; L2 (a row's chunks over lanes, Fig. 2) sums in another order and
    agrees within the bound.  n = 21: ragged last chunk; 300 points: several
    CTAs and a partial one."""
    d = Dev(W.make_batch(fn, 21, 300, seed=70), prec)
    for c in (1, 4, 8, 16):
        nch = -(-21 // c)
        l0 = d.hvp(cfg=cf.Config(c, 0, 64, cf.POINT, 0))
        l1 = d.hvp(cfg=cf.Config(c, 1, 256))
        l2 = d.hvp(cfg=cf.Config(c, min(32, 1 << (nch - 1).bit_length()), 256))
        assert np.array_equal(l0, l1), c
        assert hvp_err(d, l0).max() <= BOUND[prec], c
        assert hvp_err(d, l2).max() <= BOUND[prec], c
        H0 = d.hessian(cfg=cf.Config(c, 0, 32, cf.POINT, 0))
        assert hessian_err(d, H0).max() <= BOUND[prec], c
