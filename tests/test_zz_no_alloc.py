"""The no-allocation uneven-batch entry point, chessfad_hvp_ragged_noalloc.

It serves callers that cannot call cudaMalloc (a framework that owns device
memory through its own pool, a plugin that must not allocate or synchronise,
real-time code); its scratch is the library's static device array instead of a
caller workspace.  This file is collected last so that a run stopping at the
first failure has already run every other test; it passes on its own in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import metrics, workloads as W

pytestmark = pytest.mark.gpu

TOL = {cf.FP64: metrics.FP64_BOUND, cf.FP32_COMP: metrics.FP32_COMP_BOUND}


def _device_batch(rg, prec):
    import torch

    dt = torch.float64 if prec == cf.FP64 else torch.float32
    x = torch.tensor(rg.xpack, dtype=dt, device="cuda")
    v = torch.tensor(rg.vpack, dtype=dt, device="cuda")
    A = torch.tensor(rg.fp.A, device="cuda")
    B = torch.tensor(rg.fp.B, device="cuda")
    E = torch.tensor(rg.Epack, device="cuda")
    return x, v, (A, B, E), cf.fp_params(A, B, E)


@pytest.mark.parametrize("prec", [cf.FP32_COMP, cf.FP64])
def test_noalloc_matches_oracle_and_workspace_entry_point_on_two_calls(prec):
    import torch

    rg = W.make_ragged(nreq=600, seed=11, nmax=96)
    other = W.make_ragged(nreq=50, seed=12, nmax=40)
    x, v, keep, params = _device_batch(rg, prec)
    reqs = cf.requests(rg.fns, rg.ns, rg.offs, rg.eoffs)

    # the oracle's HVPs and norms on the exact values the device holds
    xh = x.double().cpu().numpy()
    vh = v.double().cpu().numpy()
    want, hn = oracle.hvp_ragged(rg.fns, rg.ns, rg.offs, rg.eoffs, xh, vh, rg.fp.A, rg.fp.B, rg.Epack, rg.ld)

    # the existing entry point, with a caller-allocated workspace
    ref_plan = cf.RaggedPlan(reqs, prec)
    ref = torch.full_like(x, float("nan"))
    ref_plan.run(x, v, ref, params)
    torch.cuda.synchronize()
    ref = ref.double().cpu().numpy()
    assert metrics.ragged_hvp_errors(ref, want, hn, vh, rg.ns, rg.offs).max() <= TOL[prec]

    # a different plan first, so the shared scratch holds stale tables
    xo, vo, keep_o, params_o = _device_batch(other, prec)
    oplan = cf.chessfad_ragged_plan_create(cf.requests(other.fns, other.ns, other.offs, other.eoffs), prec)
    oo = torch.empty_like(xo)
    assert cf.chessfad_hvp_ragged_noalloc(oplan, xo, vo, oo, params_o) == 0

    plan = cf.chessfad_ragged_plan_create(reqs, prec)
    for call in range(2):
        out = torch.full_like(x, float("nan"))
        assert cf.chessfad_hvp_ragged_noalloc(plan, x, v, out, params) == 0
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert np.all(np.isfinite(got)), call
        e = metrics.ragged_hvp_errors(got, want, hn, vh, rg.ns, rg.offs)
        assert e.max() <= TOL[prec], (call, "oracle", e.max())
        e = metrics.ragged_hvp_errors(got, ref, hn, vh, rg.ns, rg.offs)
        assert e.max() <= TOL[prec], (call, "workspace entry point", e.max())
    cf.chessfad_ragged_plan_destroy(plan)
    cf.chessfad_ragged_plan_destroy(oplan)
    del keep, keep_o


def test_noalloc_rejects_tables_beyond_the_static_scratch():
    # 1500000 two-variable Rosenbrock requests need more table space than the
    # static scratch holds; the call is rejected before anything is launched.
    # The buffers are real device allocations of the packed size, so even a
    # launch would stay in bounds.
    import torch

    n = 1500000
    reqs = cf.requests(np.zeros(n, np.int32), np.full(n, 2, np.int32), 2 * np.arange(n, dtype=np.int64))
    plan = cf.chessfad_ragged_plan_create(reqs, cf.FP32_COMP)
    assert cf.chessfad_ragged_plan_info(plan)["workspace_bytes"] > 32 * 1024 * 1024
    x = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    out = torch.full_like(x, 7.0)
    assert cf.chessfad_hvp_ragged_noalloc(plan, x, v, out, None) == -8
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())  # nothing was written
    cf.chessfad_ragged_plan_destroy(plan)
