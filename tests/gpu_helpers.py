"""Shared helpers of the GPU tests: device copies of a seeded batch, calls
through the C ABI binding, and the oracle reference on the same inputs."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2410_22575_gb300 as cf
from paper_2410_22575_gb300 import metrics, workloads as W

BOUND = {cf.FP64: metrics.FP64_BOUND, cf.FP32_COMP: metrics.FP32_COMP_BOUND}


def torch_dtype(prec):
    import torch

    return torch.float64 if prec == cf.FP64 else torch.float32


class Dev:
    """A batch on the device in the precision's dtype, plus the exact values
    the device holds (as float64) for the oracle."""

    def __init__(self, b: W.Batch, prec: int, device="cuda:0"):
        import torch

        self.b = b
        self.prec = prec
        dt = torch_dtype(prec)
        self.x = torch.tensor(b.x, dtype=dt, device=device)
        self.v = torch.tensor(b.v, dtype=dt, device=device)
        self.xh = self.x.double().cpu().numpy()
        self.vh = self.v.double().cpu().numpy()
        self.params = None
        self.oparams = None
        self._keep = []
        if b.fn == W.FLETCHER_POWELL:
            A = torch.tensor(b.fp.A, dtype=torch.float64, device=device)
            B = torch.tensor(b.fp.B, dtype=torch.float64, device=device)
            E = torch.tensor(b.fp.E, dtype=torch.float64, device=device)
            self._keep = [A, B, E]
            self.params = cf.fp_params(A, B, E)
            self.oparams = oracle.FPParams(b.fp.A, b.fp.B, b.fp.E)

    def hvp(self, csize=0, cfg=None, stream=None):
        import torch

        out = cf.hvp(self.b.fn, self.x, self.v, csize=csize, params=self.params, prec=self.prec, cfg=cfg,
                     stream=stream)
        torch.cuda.synchronize()
        return out.double().cpu().numpy()

    def hessian(self, csize=0, cfg=None):
        import torch

        H = cf.hessian(self.b.fn, self.x, csize=csize, params=self.params, prec=self.prec, cfg=cfg)
        torch.cuda.synchronize()
        return H.double().cpu().numpy()

    def ref_hvp(self, rows=None):
        sl = slice(None) if rows is None else rows
        return oracle.hvp(self.b.fn, self.xh[sl], self.vh[sl], self.oparams, with_norm=True)

    def ref_hessian(self, rows=None):
        sl = slice(None) if rows is None else rows
        return oracle.hessian_batch(self.b.fn, self.xh[sl], self.oparams)


def hvp_err(dev: Dev, out, rows=None):
    ref, hn = dev.ref_hvp(rows)
    sl = slice(None) if rows is None else rows
    return metrics.hvp_errors(out[sl], ref, hn, dev.vh[sl])


def hessian_err(dev: Dev, H, rows=None):
    sl = slice(None) if rows is None else rows
    return metrics.hessian_errors(H[sl], dev.ref_hessian(rows))
