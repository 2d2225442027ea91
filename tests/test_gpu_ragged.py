"""The uneven batch (requests of three functions and n in [1, 512] in one
persistent launch) against the FP64 oracle, request by request, and its
CUDA-graph capture."""
import numpy as np
import pytest

import oracle
import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import metrics, workloads as W

from gpu_helpers import BOUND

pytestmark = pytest.mark.gpu


class DevRagged:
    def __init__(self, rg: W.Ragged, prec, csize=0):
        import torch

        self.rg = rg
        self.prec = prec
        dt = torch.float64 if prec == cf.FP64 else torch.float32
        self.x = torch.tensor(rg.xpack, dtype=dt, device="cuda")
        self.v = torch.tensor(rg.vpack, dtype=dt, device="cuda")
        self.out = torch.full_like(self.x, float("nan"))
        self.xh = self.x.double().cpu().numpy()
        self.vh = self.v.double().cpu().numpy()
        self.A = torch.tensor(rg.fp.A, device="cuda")
        self.B = torch.tensor(rg.fp.B, device="cuda")
        self.E = torch.tensor(rg.Epack, device="cuda")
        self.params = cf.fp_params(self.A, self.B, self.E)
        self.plan = cf.RaggedPlan(cf.requests(rg.fns, rg.ns, rg.offs, rg.eoffs), prec, csize)

    def run(self, stream=None):
        import torch

        self.plan.run(self.x, self.v, self.out, self.params, stream)
        torch.cuda.synchronize()
        return self.out.double().cpu().numpy()

    def errors(self, out, idx=None):
        rg = self.rg
        if idx is None:
            idx = np.arange(rg.nreq)
        sub = rg.subset(idx)
        xs = np.concatenate([self.xh[rg.offs[q]:rg.offs[q] + rg.ns[q]] for q in idx])
        vs = np.concatenate([self.vh[rg.offs[q]:rg.offs[q] + rg.ns[q]] for q in idx])
        got = np.concatenate([out[rg.offs[q]:rg.offs[q] + rg.ns[q]] for q in idx])
        ref, hn = oracle.hvp_ragged(sub.fns, sub.ns, sub.offs, sub.eoffs, xs, vs, rg.fp.A, rg.fp.B, rg.Epack, rg.ld)
        return metrics.ragged_hvp_errors(got, ref, hn, vs, sub.ns, sub.offs)


@pytest.mark.parametrize("prec", [cf.FP64, cf.FP32_COMP])
@pytest.mark.parametrize("csize", [8, 16])
def test_small_uneven_batch(prec, csize):
    rg = W.make_ragged(nreq=400, seed=9, nmax=80)
    d = DevRagged(rg, prec, csize)
    out = d.run()
    assert np.all(np.isfinite(out))
    e = d.errors(out)
    assert e.max() <= BOUND[prec], (e.max(), np.median(e))


def test_one_variable_and_mixed_requests():
    rg = W.make_ragged(nreq=300, seed=21, nmax=12)
    # force some one-variable requests
    fns = rg.fns.copy()
    ns = rg.ns.copy()
    ns[::7] = 1
    offs = np.zeros(len(ns), dtype=np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    rng = np.random.Generator(np.random.PCG64(2))
    xp = np.concatenate([rng.uniform(*W.X_RANGE[int(f)], int(n)) for f, n in zip(fns, ns)])
    vp = rng.uniform(-1, 1, int(ns.sum()))
    eoffs = np.array([rg.e_of_n.get(int(n), 0) if f == W.FLETCHER_POWELL else 0 for f, n in zip(fns, ns)])
    # E for every FP size present (including 1)
    Epack, e_of_n, pos = [], {}, 0
    for n in sorted(set(int(n) for f, n in zip(fns, ns) if f == W.FLETCHER_POWELL)):
        e = W.fp_rhs(rg.fp.A[:n, :n], rg.fp.B[:n, :n], rg.fp.alpha[:n])
        e_of_n[n] = pos
        Epack.append(e)
        pos += n
    eoffs = np.array([e_of_n.get(int(n), 0) if f == W.FLETCHER_POWELL else 0 for f, n in zip(fns, ns)])
    rg2 = W.Ragged(fns, ns, offs, xp, vp, rg.fp, np.concatenate(Epack), eoffs, e_of_n)
    for prec in (cf.FP64, cf.FP32_COMP):
        d = DevRagged(rg2, prec)
        e = d.errors(d.run())
        assert e.max() <= BOUND[prec], (prec, e.max())


def test_graph_capture_and_replay_are_deterministic():
    import torch

    rg = W.make_ragged(nreq=500, seed=3, nmax=64)
    d = DevRagged(rg, cf.FP32_COMP)
    direct = d.run()  # also performs the one-time per-device set-up
    d.out.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        d.plan.run(d.x, d.v, d.out, d.params)
    for _ in range(2):
        d.out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(d.out.double().cpu().numpy(), direct)
    e = d.errors(direct)
    assert e.max() <= BOUND[cf.FP32_COMP]


def test_full_ragged_workload_sampled():
    """All 100000 requests in one persistent launch (compensated FP32); a
    sample of 600 requests, including the 60 most expensive, is compared with
    the oracle, and every output is finite."""
    rg = W.make_ragged()
    d = DevRagged(rg, cf.FP32_COMP)
    out = d.run()
    assert np.all(np.isfinite(out))
    cost = np.where(rg.fns == W.FLETCHER_POWELL, rg.ns.astype(float) ** 4, rg.ns.astype(float) ** 3)
    big = np.argsort(-cost)[:60]
    rnd = np.random.Generator(np.random.PCG64(0)).choice(rg.nreq, 540, replace=False)
    idx = np.unique(np.concatenate([big, rnd]))
    e = d.errors(out, idx)
    assert e.max() <= BOUND[cf.FP32_COMP], (e.max(), np.median(e))


def _ragged_from(fns, ns, seed, nmax=320):
    """An uneven batch with the given functions and sizes (inputs drawn as in
    the named workloads; A, B shared, E per Fletcher-Powell size)."""
    base = W.make_ragged(nreq=1, seed=seed, nmax=nmax)
    fns = np.asarray(fns, np.int32)
    ns = np.asarray(ns, np.int32)
    offs = np.zeros(len(ns), dtype=np.int64)
    offs[1:] = np.cumsum(ns[:-1])
    rng = np.random.Generator(np.random.PCG64(seed))
    xp = np.concatenate([rng.uniform(*W.X_RANGE[int(f)], int(n)) for f, n in zip(fns, ns)])
    vp = rng.uniform(-1, 1, int(ns.sum()))
    Epack, e_of_n, pos = [], {}, 0
    for n in sorted(set(int(n) for f, n in zip(fns, ns) if f == W.FLETCHER_POWELL)):
        Epack.append(W.fp_rhs(base.fp.A[:n, :n], base.fp.B[:n, :n], base.fp.alpha[:n]))
        e_of_n[n] = pos
        pos += n
    eoffs = np.array([e_of_n.get(int(n), 0) if f == W.FLETCHER_POWELL else 0 for f, n in zip(fns, ns)])
    return W.Ragged(fns, ns, offs, xp, vp, base.fp, np.concatenate(Epack), eoffs, e_of_n)


@pytest.mark.parametrize("prec", [cf.FP64, cf.FP32_COMP])
@pytest.mark.parametrize("csize", [8, 16])
def test_symmetric_fletcher_powell_requests(prec, csize):
    """Fletcher-Powell requests with n >= 128 run SC-HESS-VEC (Alg. 8), each
    tile adding its rows' contributions into a partial row vector and the
    last tile of a request summing them in tile order: sizes on and off tile
    and chunk boundaries, two requests of one size, mixed with small requests
    of every function; every request against the oracle, and a second run
    bit for bit equal to the first."""
    F, R, A = W.FLETCHER_POWELL, W.ROSENBROCK, W.ACKLEY
    fns = [F, R, F, A, F, F, R, F, A, F]
    ns = [128, 7, 131, 30, 200, 256, 300, 256, 150, 320]
    rg = _ragged_from(fns, ns, seed=40 + csize)
    d = DevRagged(rg, prec, csize)
    first = d.run()
    e = d.errors(first)
    assert e.max() <= BOUND[prec], (e.max(), np.median(e))
    d.out.fill_(float("nan"))
    second = d.run()
    assert np.array_equal(first, second)


def test_ragged_autotune_then_plan_parity():
    """chessfad_ragged_autotune stores a (chunk size, lanes per row) per
    (function, n range); a plan built with csize 0 uses them, and its results
    meet the bounds against the oracle (every request)."""
    import torch

    F, R, A = W.FLETCHER_POWELL, W.ROSENBROCK, W.ACKLEY
    rg = W.make_ragged(nreq=900, seed=31, nmax=200)
    for prec in (cf.FP32_COMP, cf.FP64):
        d = DevRagged(rg, prec, 16)
        reqs = cf.requests(rg.fns, rg.ns, rg.offs, rg.eoffs)
        ws = d.plan.workspace
        tuned = cf.chessfad_ragged_autotune(reqs, prec, d.x, d.v, d.out, d.params, ws, ws.numel())
        assert tuned >= 9, tuned
        plan = cf.RaggedPlan(reqs, prec, 0)
        for f, n in ((R, 5), (A, 40), (F, 150), (F, 33)):
            tc = cf.chessfad_ragged_tuned_config(prec, f, n)
            assert tc is not None and tc[0] in (8, 16) and 1 <= tc[1] <= 32 and tc[2] in (48, 144)
            if (f, n) in set(zip(rg.fns.tolist(), rg.ns.tolist())):
                c, t, mt = cf.chessfad_ragged_plan_group_config(plan.handle, f, n)
                assert c == tc[0] and mt >= 8
        d.out.fill_(float("nan"))
        plan.run(d.x, d.v, d.out, d.params)
        torch.cuda.synchronize()
        out = d.out.double().cpu().numpy()
        assert np.all(np.isfinite(out))
        e = d.errors(out)
        assert e.max() <= BOUND[prec], (prec, e.max())
        plan.close()
