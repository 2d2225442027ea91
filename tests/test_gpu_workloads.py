"""Parity at the full sizes of the named workloads, in the launch
configurations the benchmark times, compared with the oracle point by point
(the oracle's closed forms finish every point in seconds)."""
import numpy as np
import pytest

import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import workloads as W

from gpu_helpers import BOUND, Dev, hessian_err, hvp_err

pytestmark = pytest.mark.gpu


def test_rosenbrock_n16_fp64_c4_hvp_and_hessian():
    d = Dev(W.workload("rosenbrock_n16"), cf.FP64)
    e = hvp_err(d, d.hvp(csize=4))
    assert e.max() <= BOUND[cf.FP64]
    e = hessian_err(d, d.hessian(csize=4))
    assert e.max() <= BOUND[cf.FP64]


@pytest.mark.parametrize("prec", [cf.FP64, cf.FP32_COMP])
@pytest.mark.parametrize("c", [4, 8, 16, 32])
def test_ackley_n64_chunk_sweep(prec, c):
    if prec == cf.FP64 and c == 32:
        pytest.skip("FP64 c=32 spills registers; covered at small sizes")
    d = Dev(W.workload("ackley_n64"), prec)
    e = hvp_err(d, d.hvp(csize=c))
    assert e.max() <= BOUND[prec], (e.max(), np.median(e))


@pytest.mark.parametrize("prec", [cf.FP64, cf.FP32_COMP])
def test_fletcher_powell_n32(prec):
    d = Dev(W.workload("fletcher_powell_n32"), prec)
    e = hvp_err(d, d.hvp())
    assert e.max() <= BOUND[prec], (e.max(), np.median(e))


@pytest.mark.parametrize("prec", [cf.FP64, cf.FP32_COMP])
def test_rosenbrock_n256_hessian_and_hvp(prec):
    d = Dev(W.workload("rosenbrock_n256"), prec)
    e = hvp_err(d, d.hvp())
    assert e.max() <= BOUND[prec]
    H = d.hessian()
    for lo in range(0, 1024, 128):  # bounded host memory for the reference
        rows = slice(lo, lo + 128)
        assert hessian_err(d, H, rows).max() <= BOUND[prec]


@pytest.mark.parametrize("prec", [cf.FP32_COMP, cf.FP64])
def test_ackley_n64_autotuned_launch(prec):
    """The launch configuration the benchmark times: autotune (both methods),
    then csize = 0, at the full size of the headline workload."""
    import torch

    d = Dev(W.workload("ackley_n64"), prec)
    out = torch.empty_like(d.x)
    cfg = cf.chessfad_autotune_hvp(W.ACKLEY, 64, d.x.shape[0], d.x, d.v, out, None, prec)
    assert cfg.csize in (1, 2, 4, 8, 16, 32)
    e = hvp_err(d, d.hvp(csize=0))
    assert e.max() <= BOUND[prec], (cfg.as_dict(), e.max())
    # the symmetric configuration the benchmark reports, explicitly
    e = hvp_err(d, d.hvp(cfg=cf.Config(8, 0, 0, cf.SYMMETRIC, 64)))
    assert e.max() <= BOUND[prec]


@pytest.mark.parametrize("prec", [cf.FP32_COMP, cf.FP64])
def test_symmetric_full_workloads(prec):
    for name in ("rosenbrock_n16", "fletcher_powell_n32"):
        d = Dev(W.workload(name), prec)
        e = hvp_err(d, d.hvp(cfg=cf.Config(4, 0, 0, cf.SYMMETRIC, 32)))
        assert e.max() <= BOUND[prec], (name, e.max())


def test_error_report_every_workload():
    """Max / median normalised error of every named workload in both
    precisions, in the autotuned configuration (both methods searched); the
    bounds are asserted, and the table is written to the file named by
    CHESSFAD_ERROR_REPORT when that variable is set."""
    import json
    import os

    import torch

    rows = []
    for name in ("rosenbrock_n16", "ackley_n64", "fletcher_powell_n32", "rosenbrock_n256"):
        for prec in (cf.FP32_COMP, cf.FP64):
            d = Dev(W.workload(name), prec)
            out = torch.empty_like(d.x)
            cfg = cf.chessfad_autotune_hvp(d.b.fn, d.b.n, d.b.batch, d.x, d.v, out, d.params, prec)
            e = hvp_err(d, d.hvp(csize=0))
            assert e.max() <= BOUND[prec], (name, prec, e.max())
            rows.append({"workload": name, "precision": "fp64" if prec == cf.FP64 else "fp32_comp",
                         "config": cfg.as_dict(), "max": float(e.max()), "median": float(np.median(e))})
    path = os.environ.get("CHESSFAD_ERROR_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(rows, f, indent=1)


@pytest.mark.parametrize("prec", [cf.FP32_COMP, cf.FP64])
def test_symmetric_sparse_full_workloads(prec):
    """The seed-sparse symmetric method at the full sizes of every named
    workload, in the configuration the benchmark reports for it."""
    for name, c in (("rosenbrock_n16", 4), ("ackley_n64", 8), ("fletcher_powell_n32", 8), ("rosenbrock_n256", 16)):
        d = Dev(W.workload(name), prec)
        cfg = cf.Config(c, 0, 0, cf.SYMMETRIC_SPARSE, 32)
        if name == "rosenbrock_n256" and prec == cf.FP64:
            # FP64 symmetric HVP stages at most n ~ 200 in shared memory: Hessian
            rows = slice(0, 128)
            assert hessian_err(d, d.hessian(cfg=cfg), rows).max() <= BOUND[prec]
            continue
        e = hvp_err(d, d.hvp(cfg=cfg))
        assert e.max() <= BOUND[prec], (name, e.max())
