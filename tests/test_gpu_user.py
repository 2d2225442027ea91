"""User-supplied functions (compiled at run time) against the FP64 oracle:
the paper's three test functions written as user sources, and the
extended-operator function (division, abs, log, tanh, tan, pow, a
comparison), HVP and Hessian, element by element.

Bounds, per point, normalised by ||H||_F ||v||_2 (||H||_F for a Hessian):
1e-12 in FP64 and 1e-5 in FP32, for every function and n.  In FP32 the
function's own arithmetic is plain FP32, as the user wrote it (only the
row-times-v sum is compensated): its n-term sums (Ackley's Sum x^2 and
Sum cos 2 pi x, the Fletcher-Powell residuals) carry a relative error up to
about n u = 64 * 6e-8 = 4e-6 at the sizes tested, inside 1e-5.  At n = 1 the
Hessian is one entry, a sum of terms that can cancel far below their size,
and an FP32 handle evaluates it in FP64 (float in and out)."""
import numpy as np
import pytest

import oracle
import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import metrics, workloads as W

from user_sources import SOURCES

pytestmark = pytest.mark.gpu

FNS = [W.ROSENBROCK, W.ACKLEY, W.FLETCHER_POWELL, W.MIX]
BOUND = {
    cf.FP64: {f: 1e-12 for f in FNS},
    cf.FP32_COMP: {f: 1e-5 for f in FNS},
}


_cache = {}


def user_fn(fn, c, prec):
    key = (fn, c, prec)
    if key not in _cache:
        src, name = SOURCES[fn]
        _cache[key] = cf.UserFunction(src, name, c, prec)
    return _cache[key]


class Case:
    def __init__(self, fn, n, batch, seed, prec):
        import torch

        self.b = W.make_batch(fn, n, batch, seed)
        self.fn, self.n, self.prec = fn, n, prec
        dt = torch.float64 if prec == cf.FP64 else torch.float32
        self.x = torch.tensor(self.b.x, dtype=dt, device="cuda")
        self.v = torch.tensor(self.b.v, dtype=dt, device="cuda")
        self.xh = self.x.double().cpu().numpy()
        self.vh = self.v.double().cpu().numpy()
        self.params = None
        self.oparams = None
        if fn == W.FLETCHER_POWELL:
            A, B, E = self.b.fp.A[:n, :n], self.b.fp.B[:n, :n], self.b.fp.E
            self.params = torch.tensor(np.concatenate([A.ravel(), B.ravel(), E]), dtype=torch.float64,
                                       device="cuda")
            self.oparams = oracle.FPParams(A, B, E)

    def hvp_err(self, out):
        ref, hn = oracle.hvp(self.fn, self.xh, self.vh, self.oparams, with_norm=True)
        return metrics.hvp_errors(out.double().cpu().numpy(), ref, hn, self.vh)

    def hess_err(self, H):
        return metrics.hessian_errors(H.double().cpu().numpy(), oracle.hessian_batch(self.fn, self.xh, self.oparams))


PLAIN = cf.Config(0, 1, 256, cf.PLAIN, 0)
SYM = cf.Config(0, 0, 0, cf.SYMMETRIC, 32)


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("prec", [cf.FP64, cf.FP32_COMP])
@pytest.mark.parametrize("c", [1, 4, 8, 16])
def test_user_hvp_and_hessian(fn, prec, c):
    """n = 19: ragged last chunk; 70 points: several CTAs and a partial one;
    plain (Alg. 7 / Alg. 5), symmetric (Alg. 8 / Alg. 6) and the default."""
    f = user_fn(fn, c, prec)
    k = Case(fn, 19, 70, 900 + c, prec)
    for cfg in (PLAIN, SYM, cf.Config(0, 0, 128, cf.SYMMETRIC, 64), None):
        e = k.hvp_err(f.hvp(k.x, k.v, k.params, cfg=cfg))
        assert e.max() <= BOUND[prec][fn], (cfg, e.max(), np.median(e))
        e = k.hess_err(f.hessian(k.x, k.params, cfg=cfg))
        assert e.max() <= BOUND[prec][fn], (cfg, e.max(), np.median(e))


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("n", [1, 2, 3, 64, 130])
def test_user_sizes(fn, n):
    for prec in (cf.FP64, cf.FP32_COMP):
        f = user_fn(fn, 8, prec)
        k = Case(fn, n, 37 if n < 100 else 5, 950 + n, prec)
        for cfg in (PLAIN, None):
            e = k.hvp_err(f.hvp(k.x, k.v, k.params, cfg=cfg))
            assert e.max() <= BOUND[prec][fn], (prec, cfg, e.max())


@pytest.mark.parametrize("fn", FNS)
def test_user_fp32_one_variable_many_points(fn):
    """n = 1 in an FP32 handle over 20000 points, HVP and Hessian, both
    methods: within 1e-5 everywhere (an FP32 evaluation of the single entry
    misses it at about 3 % of random Ackley points)."""
    f = user_fn(fn, 8, cf.FP32_COMP)
    k = Case(fn, 1, 20000, 990 + fn, cf.FP32_COMP)
    for cfg in (PLAIN, SYM, None):
        e = k.hvp_err(f.hvp(k.x, k.v, k.params, cfg=cfg))
        assert e.max() <= 1e-5, (cfg, e.max())
        e = k.hess_err(f.hessian(k.x, k.params, cfg=cfg))
        assert e.max() <= 1e-5, (cfg, e.max())


def test_user_equals_builtin_fp64():
    """The user-source Ackley and the built-in Ackley kernel agree to FP64
    rounding (same method, different code)."""
    k = Case(W.ACKLEY, 33, 200, 5, cf.FP64)
    a = user_fn(W.ACKLEY, 8, cf.FP64).hvp(k.x, k.v).double().cpu().numpy()
    b = cf.hvp(W.ACKLEY, k.x, k.v, csize=8, prec=cf.FP64).double().cpu().numpy()
    ref, hn = oracle.hvp(W.ACKLEY, k.xh, k.vh, None, with_norm=True)
    assert np.max(np.linalg.norm(a - b, axis=1) / (hn * np.linalg.norm(k.vh, axis=1))) <= 2e-12


def test_user_misc():
    import torch

    f = user_fn(W.MIX, 4, cf.FP64)
    info = f.info(True)
    assert info["csize"] == 4 and info["prec"] == cf.FP64 and 16 <= info["registers"] <= 255
    # batch 0 is a no-op; bad n is rejected before launch
    z = torch.zeros((0, 5), dtype=torch.float64, device="cuda")
    assert cf.chessfad_user_hvp(f.handle, 5, 0, z, z, z) == 0
    assert cf.chessfad_user_hvp(f.handle, 0, 1, z, z, z) == -2
    assert cf.chessfad_user_hvp(f.handle, 513, 1, z, z, z) == -2
    # NaN reaches its own point only; results are deterministic
    b = W.make_batch(W.MIX, 9, 20, 3)
    b.x[4, 6] = np.nan
    x = torch.tensor(b.x, device="cuda")
    v = torch.tensor(b.v, device="cuda")
    o1 = f.hvp(x, v).cpu().numpy()
    o2 = f.hvp(x, v).cpu().numpy()
    assert np.array_equal(o1, o2, equal_nan=True)
    assert np.all(np.isnan(o1[4]))
    ok = np.ones(20, bool)
    ok[4] = False
    assert np.all(np.isfinite(o1[ok]))
    # side stream
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        o3 = f.hvp(x, v, stream=s)
    s.synchronize()
    assert np.array_equal(o3.cpu().numpy(), o1, equal_nan=True)


def test_user_compile_error_on_device():
    st, handle, log = cf.chessfad_user_fn_create(
        "template <class R, class X> R g(const X &x, int n, const double *p) { return x[0] * ; }", "g", 8, cf.FP64)
    assert st == -12 and handle is None and "error" in log


def test_user_symmetric_limits_and_config_errors():
    import torch

    f = user_fn(W.ROSENBROCK, 8, cf.FP64)
    k = Case(W.ROSENBROCK, 300, 3, 17, cf.FP64)
    out = torch.empty_like(k.x)
    # the symmetric HVP's chunk matrix does not fit shared memory: FP64 row
    # accumulators instead, explicitly and by default
    first = f.hvp(k.x, k.v, cfg=SYM)
    assert k.hvp_err(first).max() <= 1e-12
    # the accumulators add each iteration's staged chunks in thread order
    assert np.array_equal(first.cpu().numpy(), f.hvp(k.x, k.v, cfg=SYM).cpu().numpy())
    assert k.hvp_err(f.hvp(k.x, k.v)).max() <= 1e-12
    k32 = Case(W.MIX, 512, 3, 18, cf.FP32_COMP)
    assert k32.hvp_err(user_fn(W.MIX, 16, cf.FP32_COMP).hvp(k32.x, k32.v, cfg=SYM)).max() <= 1e-5
    # the symmetric Hessian has no staging limit
    assert k.hess_err(f.hessian(k.x, cfg=SYM)).max() <= 1e-12
    for bad, code in ((cf.Config(4, 0, 0, cf.PLAIN, 0), -4), (cf.Config(0, 0, 0, cf.SYMMETRIC_SPARSE, 0), -9),
                      (cf.Config(0, 2, 0, cf.PLAIN, 0), -9), (cf.Config(0, 0, 48, cf.PLAIN, 0), -9),
                      (cf.Config(0, 0, 0, cf.SYMMETRIC, 48), -9)):
        assert cf.chessfad_user_hvp_config(f.handle, 300, 3, bad, k.x, k.v, out) == code, bad


def test_user_symmetric_faster_than_plain_on_ackley():
    """SC-HESS-VEC does about half the evaluations of CHESS-VEC (Sec. V)."""
    import torch

    f = user_fn(W.ACKLEY, 8, cf.FP32_COMP)
    k = Case(W.ACKLEY, 64, 8192, 3, cf.FP32_COMP)
    out = torch.empty_like(k.x)

    def t(cfg):
        f.hvp(k.x, k.v, out=out, cfg=cfg)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            f.hvp(k.x, k.v, out=out, cfg=cfg)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    assert t(SYM) < 0.85 * t(PLAIN)
