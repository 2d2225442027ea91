"""chessfad_hvp_host: host-resident x, v, out with overlapped copies and
sweeps, against the FP64 oracle; slicing, pageable memory, stream order and
CUDA-graph capture."""
import numpy as np
import pytest

import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import workloads as W

from gpu_helpers import BOUND, Dev, hvp_err

pytestmark = pytest.mark.gpu


def _host(d, pinned=True):
    import torch

    xh = d.x.cpu()
    vh = d.v.cpu()
    oh = torch.empty_like(xh)
    if pinned:
        xh, vh, oh = xh.pin_memory(), vh.pin_memory(), oh.pin_memory()
    return xh, vh, oh


@pytest.mark.parametrize("prec", [cf.FP32_COMP, cf.FP64])
@pytest.mark.parametrize("slices", [0, 1, 3, 16])
def test_host_pipeline_matches_oracle(prec, slices):
    import torch

    d = Dev(W.make_batch(W.ACKLEY, 40, 3001, seed=21), prec)
    xh, vh, oh = _host(d)
    xd, vd, od = torch.empty_like(d.x), torch.empty_like(d.v), torch.empty_like(d.x)
    st = cf.chessfad_hvp_host(W.ACKLEY, 40, 3001, 8, xh, vh, oh, xd, vd, od, None, prec, slices)
    assert st == 0
    torch.cuda.current_stream().synchronize()
    e = hvp_err(d, oh.double().numpy())
    assert e.max() <= BOUND[prec], e.max()
    # the device staging buffers hold the same result
    assert np.array_equal(od.cpu().numpy(), oh.numpy())


def test_host_pipeline_fletcher_powell_pageable_and_small_batch():
    import torch

    d = Dev(W.make_batch(W.FLETCHER_POWELL, 17, 5, seed=4), cf.FP64)
    xh, vh, oh = _host(d, pinned=False)
    xd, vd, od = torch.empty_like(d.x), torch.empty_like(d.v), torch.empty_like(d.x)
    # more slices than points: one point per slice
    assert cf.chessfad_hvp_host(W.FLETCHER_POWELL, 17, 5, 4, xh, vh, oh, xd, vd, od, d.params, cf.FP64, 9) == 0
    torch.cuda.current_stream().synchronize()
    assert hvp_err(d, oh.numpy()).max() <= BOUND[cf.FP64]
    assert cf.chessfad_hvp_host(W.FLETCHER_POWELL, 17, 0, 4, xh, vh, oh, xd, vd, od, d.params, cf.FP64, 9) == 0
    assert cf.chessfad_hvp_host(W.FLETCHER_POWELL, 17, 5, 4, xh, vh, oh, xd, vd, od, d.params, cf.FP64, 65) == -9


def test_host_pipeline_side_stream_and_graph():
    import torch

    d = Dev(W.make_batch(W.ROSENBROCK, 24, 2000, seed=8), cf.FP32_COMP)
    xh, vh, oh = _host(d)
    xd, vd, od = torch.empty_like(d.x), torch.empty_like(d.v), torch.empty_like(d.x)
    s = torch.cuda.Stream()
    assert cf.chessfad_hvp_host(W.ROSENBROCK, 24, 2000, 8, xh, vh, oh, xd, vd, od, None, cf.FP32_COMP, 4, s) == 0
    s.synchronize()
    ref = oh.numpy().copy()
    assert hvp_err(d, ref.astype(np.float64)).max() <= BOUND[cf.FP32_COMP]
    # captured once (after the first call created the per-device streams), replayed
    oh.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = cf.chessfad_hvp_host(W.ROSENBROCK, 24, 2000, 8, xh, vh, oh, xd, vd, od, None, cf.FP32_COMP, 4)
    assert st == 0
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(oh.numpy(), ref)
