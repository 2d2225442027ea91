#!/usr/bin/env python3
"""Benchmark: Hessian-vector products per second on one GB300 (and N GPUs).

Workload: Ackley, n = 64, 65536 points, x ~ U[-5,5], v ~ U[-1,1], seed 1
(PCG64), the configuration the headline metric is quoted on.  One step is one
``chessfad_hvp`` call over the whole batch: seeding, chunked-hDual propagation,
row-times-v products and the in-kernel row reduction, all in the library's
sweep kernel.  The headline ``value`` is the FP64 rate (the paper's precision,
Sec. IV) with inputs resident in HBM; the compensated-FP32 rate is reported
beside it as a complete block (``fp32_comp``: rate, roofline, end-to-end rate,
error), so "FP32-comp vs FP64" is one line.  ``workloads`` holds the other
named workloads (Rosenbrock n=16 and n=256 with Hessians, Fletcher-Powell
n=32) in both precisions, ``ragged_100k`` the 100000-request uneven batch.

Roofline: the sweep kernels are bound by CUDA-core arithmetic (FP64 DFMA or
FP32 FFMA pipe).  ``achieved`` = FP instructions the kernel executes per launch
(ncu thread-instruction counts, FMA = 2 flops, a packed FP32 instruction
twice, recorded in ``profiles/counts.json`` per point and keyed by a hash of
the kernel sources' code; null when that code changed since) / the launch's
CUDA-event time; ``peak`` = SMs x FMA lanes x 2 x the maximum SM clock (the
unit-count figure); ``peak_measured`` = the library's FMA microbenchmark
(``chessfad_peak_info``, the best of several chain shapes) measured in the
same run on the same GPU, reported beside it.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream, with a 256 MiB buffer written between steps to flush
the 129 MB L2 (outside the events).  Barrier + synchronize on both sides, max
over ranks.  Under torchrun every rank runs the same per-GPU batch (weak
scaling; points are independent, there is no collective on the data path).

``--impl reference`` times the FP64 CPU oracle (the paper's sequential
CHESS-VEC, Alg. 7, OpenMP over points) on the host cores instead.
``--profile-kernels`` launches every kernel of ``profiles/counts.json`` once
(the command ncu captures); ``--ingest-ncu CSV`` turns that capture into
``profiles/counts.json``.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hessian-vector products/sec per function and n, FP32-comp vs FP64, 1 GB300"
WORKLOAD = "ackley_n64"
WORKLOAD_DESC = "Ackley n=64, 65536 points, x~U[-5,5], v~U[-1,1], seed 1 (PCG64)"
# CUDA-core lanes per SM of sm_103 (GB300): 128 FP32 FMA lanes, and FP64 at
# 1/64 of that (2 DFMA per clock per SM; GB300's nominal FP64 rate).  The SM
# count and the clock come from the device at run time.
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2
COUNTS_FILE = os.path.join(ROOT, "profiles", "counts.json")
PREC_NAME = {0: "fp64", 1: "fp32_comp"}


def sym_items(n: int, c: int) -> int:
    """Evaluations of f per point by the symmetric method (Alg. 6 / Alg. 8):
    rows i with the chunks from their diagonal chunk on, n(n/c+1)/2 when c
    divides n (Sec. V)."""
    nch = -(-n // c)
    return sum(min(c, n - R * c) * (nch - R) for R in range(nch))


def model_flops_eval(fn: int, n: int, c: int) -> float:
    """Model flops of one evaluation of f on hDual<c>: every component
    operation of each function's op list as the kernels state it, zeros of
    the seeds included (dense), FMA = 2.  Operation costs on K = 2c+2
    components: a unary-rule accumulation acc += phi(u) 6c+3 (6c+4 with its
    value); scalar-times-hDual accumulation 4c+2; a unary rule 4c+2; a
    componentwise add, negation or scaling 2c+1 or 2c+2.
      Rosenbrock (n-1)(18c+15): per term d = x_{k+1} - x_k^2 (6c+7), then
        100 d^2 and (1-x_k)^2 accumulated (2 x (6c+4));
      Ackley n(12c+5) + 14c+17: per variable y_k^2/2 and cos(2 pi y_k), each
        accumulated by the unary rule; then the tail, three unary rules with
        the constant factors folded into phi' and phi'' (sqrt(S/n) of S/2,
        -20 exp(-0.2 r), -exp(C/n) accumulated);
      Fletcher-Powell n^2(8c+4) + n(16c+10): per (m, j) two scalar-times-hDual
        accumulations, per j sin(y_j) and cos(y_j) (once), per m the residual
        negated and its square accumulated."""
    if fn == 0:
        return max(0, n - 1) * (18 * c + 15)
    if fn == 1:
        return n * (12 * c + 5) + 14 * c + 17
    return n * n * (8 * c + 4) + n * (16 * c + 10)


def model_flops_hvp(fn: int, n: int, c: int, symmetric: bool = False) -> float:
    """Model flops of one HVP by the dense chunked-hDual method: n*nch
    evaluations (plain, Alg. 7) or sym_items(n, c) (symmetric, Alg. 8), plus
    2n^2 for the row dots."""
    nch = -(-n // c)
    sweeps = sym_items(n, c) if symmetric else n * nch
    return sweeps * model_flops_eval(fn, n, c) + 2 * n * n


def model_flops_hessian(fn: int, n: int, c: int, symmetric: bool = False) -> float:
    """Model flops of one Hessian: the HVP's evaluations without the dots."""
    nch = -(-n // c)
    sweeps = sym_items(n, c) if symmetric else n * nch
    return sweeps * model_flops_eval(fn, n, c)


def model_flops_ackley(n: int, c: int, symmetric: bool = False) -> float:
    return model_flops_hvp(1, n, c, symmetric)


def algorithmic_bytes(n: int, prec: int, kind: str) -> int:
    """HBM bytes one point needs by definition: x, v, out (HVP) or x, H
    (Hessian), s = 8 (FP64) or 4 (compensated FP32)."""
    s = 8 if prec == 0 else 4
    return 3 * n * s if kind == "hvp" else (n + n * n) * s


# Sources that define the batched sweep kernels: the executed-instruction
# counts and DRAM traffic in profiles/counts.json are used only while the code
# of these files (comments and whitespace aside) is unchanged since the capture.
KERNEL_SOURCES = ("hdual.cuh", "sym_layout.cuh", "sweep.cuh", "dispatch.h", "point.cuh", "instances.cu")


def code_tokens(text: str) -> str:
    """C++/CUDA source without its comments, whitespace runs collapsed.  The
    kernel sources hold no comment markers inside string literals."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(csrc: str | None = None) -> str:
    import glob

    h = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_2410_22575_gb300", "csrc")
    for pat in KERNEL_SOURCES:
        for p in sorted(glob.glob(os.path.join(csrc, pat))):
            h.update(os.path.basename(p).encode())
            h.update(code_tokens(open(p, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def load_counts() -> dict:
    """Executed FP instructions and DRAM bytes per point, per kernel key, from
    the ncu capture of ``--profile-kernels``; entries whose sources changed
    since the capture are dropped."""
    if not os.path.exists(COUNTS_FILE):
        return {}
    tj = json.load(open(COUNTS_FILE))
    h = kernel_source_hash()
    return {k: v for k, v in tj.get("kernels", {}).items() if tj.get("source_hash") == h}


def count_key(workload: str, prec: int, kind: str, method: str, c: int) -> str:
    return f"{workload}/{PREC_NAME[prec]}/{kind}/{method}/c{c}"


def device_peaks(cf, dev_index: int) -> dict:
    """FMA peaks of this GPU: the library's microbenchmark (measured now, with
    the SM clock it saw) and the unit-count figure SMs x lanes x 2 x max SM
    clock (SM count from the device, max clock from nvidia-smi)."""
    import torch

    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    max_mhz = None
    try:
        q = subprocess.run(["nvidia-smi", f"--id={dev_index}", "--query-gpu=clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        max_mhz = float(q.stdout.strip().splitlines()[0])
    except Exception:
        max_mhz = None
    out = {"sms": sms, "sm_max_mhz": max_mhz}
    for prec, lanes in ((0, FP64_LANES_PER_SM), (1, FP32_LANES_PER_SM)):
        try:
            f, mhz = cf.chessfad_peak_info(prec)
        except Exception as e:  # report, do not hide
            print(f"peak microbenchmark failed: {e}", file=sys.stderr)
            f, mhz = None, None
        try:
            reg, lit = cf.chessfad_peak_operand_rates(prec)
            operands = {"register": reg, "literal": lit, "literal_over_register": lit / reg}
        except Exception as e:
            print(f"operand microbenchmark failed: {e}", file=sys.stderr)
            operands = None
        out[PREC_NAME[prec]] = {
            "microbench": f, "microbench_sm_mhz": mhz,
            "axpy_operands": operands,
            "derived": None if max_mhz is None else sms * lanes * 2 * max_mhz * 1e6,
            "derived_note": f"{sms} SMs x {lanes} {'DFMA' if prec == 0 else 'FFMA'} lanes x 2 flop x "
                            f"{max_mhz} MHz (max SM clock)"}
    return out


def roofline_entry(counts: dict, key: str, units: int, ms: float, prec: int, peaks: dict, n: int, kind: str,
                   model_flops_per_unit: float, kernel: str) -> dict:
    """The ALU roofline of one kernel launch of `units` points taking `ms`."""
    p = peaks[PREC_NAME[prec]]
    ent = counts.get(key)
    executed = None if ent is None else ent["executed_flops_per_unit"] * units
    traffic = None if ent is None or ent.get("dram_bytes_per_unit") is None else ent["dram_bytes_per_unit"] * units
    achieved = None if executed is None else executed / (ms * 1e-3)
    model = model_flops_per_unit * units
    algo = algorithmic_bytes(n, prec, kind) * units
    return {
        "bound": "alu", "unit": "TFLOP/s", "kernel": kernel,
        "achieved": None if achieved is None else achieved / 1e12,
        "peak": None if p["derived"] is None else p["derived"] / 1e12,
        "frac": None if achieved is None or p["derived"] is None else achieved / p["derived"],
        "peak_source": f"derived from unit counts and clock: {p['derived_note']}",
        "peak_measured": None if p["microbench"] is None else p["microbench"] / 1e12,
        "frac_of_measured": None if achieved is None or p["microbench"] is None else achieved / p["microbench"],
        "peak_measured_source": f"chessfad_peak_info({PREC_NAME[prec]}) FMA microbenchmark in this run, "
                                f"SM clock {p['microbench_sm_mhz'] and round(p['microbench_sm_mhz'])} MHz",
        "executed_flops_per_launch": executed,
        "model_flops_per_launch": model,
        "model_over_executed": None if executed is None else model / executed,
        "traffic": traffic,
        "algorithmic_bytes_per_launch": algo,
        "dram_gbs_algorithmic": algo / (ms * 1e-3) / 1e9,
        "dram_gbs_measured_traffic": None if traffic is None else traffic / (ms * 1e-3) / 1e9,
        "issue_active_pct_ncu": None if ent is None else ent.get("issue_active_pct"),
        "counts_key": key, "counts_present": ent is not None,
    }


def kernel_name(method: str, prec: int, c: int, fn: int, kind: str) -> str:
    t = "double" if prec == 0 else "float"
    f = {0: "ROSENBROCK", 1: "ACKLEY", 2: "FP"}[fn]
    k = "HVP" if kind == "hvp" else "HESSIAN"
    base = "sym_kernel" if method in ("symmetric", "symmetric_sparse") else (
        "point_kernel" if method == "point" else "sweep_kernel")
    return f"{base}<{t},{c},{f},{k}>"

# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = [s for s in sm if s > 0.5 * (max(mx) if mx else 0)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("CHESSFAD_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value: float, device) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ GPU arm
def timed_steps(fn_step, steps, warmup, stream, flush_buf):
    """Per-step CUDA-event durations (ms) of fn_step, L2 flushed in between."""
    import torch

    for _ in range(warmup):
        fn_step()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush_buf.add_(1)  # 256 MiB write, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn_step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _checked(st, what):
    import paper_2410_22575_gb300 as cf

    if st != 0:
        raise cf.ChessfadError(st, what)


def headline_arm(cf, b, prec, args, world, dev, stream, flush, peaks, counts):
    """The named workload in one precision: autotuned HVP config, K timed
    steps (clocks sampled), then the same through host buffers (e2e)."""
    import torch

    dt = torch.float64 if prec == cf.FP64 else torch.float32
    fn, n, batch = b.fn, b.n, b.batch
    x = torch.tensor(b.x, dtype=dt, device=dev)
    v = torch.tensor(b.v, dtype=dt, device=dev)
    out = torch.empty_like(x)
    cfg = cf.chessfad_autotune_hvp(fn, n, batch, x, v, out, None, prec, stream)

    def step():
        _checked(cf.chessfad_hvp(fn, n, batch, 0, x, v, out, None, prec, stream), "chessfad_hvp")

    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        ms = timed_steps(step, args.steps, args.warmup, stream, flush)
    clocks = clk.summary()
    torch.cuda.synchronize()
    barrier(world)
    tot = max_over_ranks(world, sum(ms), dev)
    per = tot / len(ms)
    cd = cfg.as_dict()
    sym = cd["method"] == "symmetric"
    key = count_key(WORKLOAD, prec, "hvp", cd["method"], cfg.csize)
    roof = roofline_entry(counts, key, batch, sum(ms) / len(ms), prec, peaks, n, "hvp",
                          model_flops_hvp(fn, n, cfg.csize, sym), kernel_name(cd["method"], prec, cfg.csize, fn, "hvp"))
    res = {"value": world * batch / (per * 1e-3), "unit": "HVP/s", "steps": len(ms), "ms_per_step": per,
           "config": cd, "roofline": roof, "clocks": clocks, "_out": out.double().cpu().numpy(),
           "_x": x.double().cpu().numpy(), "_v": v.double().cpu().numpy()}

    # chunk-size sweep (shorter), same precision, both methods
    sweep = {}
    for c in (4, 8, 16, 32):
        info = cf.chessfad_kernel_info(fn, prec, c, True)
        if info["local_bytes"] > 48:
            sweep[str(c)] = {"skipped": "spills registers", **info}
            continue
        ent = dict(info)
        for mname, ccfg in (("plain", cf.Config(c, 1, 256)), ("symmetric", cf.Config(c, 0, 0, cf.SYMMETRIC, 64))):
            def stc(ccfg=ccfg):
                _checked(cf.chessfad_hvp_config(fn, n, batch, ccfg, x, v, out, None, prec, stream), "chessfad_hvp")

            k = max(1, min(3, args.steps))
            m = timed_steps(stc, k, 1, stream, flush)
            t = max_over_ranks(world, sum(m), dev) / k
            ent[mname] = {"hvp_per_s": world * batch / (t * 1e-3), "ms": t}
        sweep[str(c)] = ent
    res["chunk_sweep"] = sweep

    # seed-sparse symmetric method (a different arithmetic: reported beside
    # the headline, never as it)
    sparse = {}
    for c in (4, 8):
        scfg = cf.Config(c, 0, 128, cf.SYMMETRIC_SPARSE, 64)

        def sts(scfg=scfg):
            _checked(cf.chessfad_hvp_config(fn, n, batch, scfg, x, v, out, None, prec, stream), "chessfad_hvp")

        k = max(1, min(3, args.steps))
        m = timed_steps(sts, k, 1, stream, flush)
        t = max_over_ranks(world, sum(m), dev) / k
        sparse[str(c)] = {**scfg.as_dict(), "hvp_per_s": world * batch / (t * 1e-3), "ms": t}
    res["seed_sparse"] = sparse
    del x, v, out

    # end to end through the public host-buffer call: pinned host x, v ->
    # device -> sweeps -> host out, copies of consecutive slices overlapping
    # the sweeps, all inside the events
    xh = torch.tensor(b.x, dtype=dt).pin_memory()
    vh = torch.tensor(b.v, dtype=dt).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(xh, device=dev)
    vd = torch.empty_like(vh, device=dev)
    od = torch.empty_like(xh, device=dev)

    def e2e_step():
        _checked(cf.chessfad_hvp_host(fn, n, batch, 0, xh, vh, oh, xd, vd, od, None, prec, args.e2e_slices, stream),
                 "chessfad_hvp_host")

    barrier(world)
    ms_e2e = timed_steps(e2e_step, args.steps, args.warmup, stream, flush)
    torch.cuda.synchronize()
    barrier(world)
    tot_e2e = max_over_ranks(world, sum(ms_e2e), dev)
    s = 8 if prec == cf.FP64 else 4
    res["e2e"] = {"value": world * batch * len(ms_e2e) / (tot_e2e * 1e-3), "unit": "HVP/s",
                  "h2d_bytes_per_step": 2 * batch * n * s, "d2h_bytes_per_step": batch * n * s,
                  "api": "chessfad_hvp_host (pinned host buffers)", "slices": args.e2e_slices,
                  "ms_per_step": tot_e2e / len(ms_e2e)}
    return res


# The other named workloads and what is measured on each.  C1 (Rosenbrock
# n=16) is quoted in FP64 with c=4 by the plain method, HVP and Hessian; C3
# (Fletcher-Powell n=32) in FP64 and in compensated FP32 (FP64 residuals);
# C4 (Rosenbrock n=256) HVP and Hessian, autotuned, in both precisions.
WORKLOAD_ROWS = (
    ("rosenbrock_n16", "hvp", "stated", 0),
    ("rosenbrock_n16", "hessian", "stated", 0),
    ("rosenbrock_n16", "hvp", "tuned", 0),
    ("rosenbrock_n16", "hessian", "tuned", 0),
    ("rosenbrock_n16", "hvp", "tuned", 1),
    ("rosenbrock_n16", "hessian", "tuned", 1),
    ("fletcher_powell_n32", "hvp", "tuned", 0),
    ("fletcher_powell_n32", "hvp", "tuned", 1),
    ("rosenbrock_n256", "hvp", "tuned", 0),
    ("rosenbrock_n256", "hessian", "tuned", 0),
    ("rosenbrock_n256", "hvp", "tuned", 1),
    ("rosenbrock_n256", "hessian", "tuned", 1),
)


def workloads_arm(cf, args, world, dev, stream, flush, peaks, counts):
    """Every row of WORKLOAD_ROWS: rate, roofline (executed flops when the
    counts are current), DRAM GB/s; the outputs are kept for the oracle leg."""
    import torch
    from paper_2410_22575_gb300 import workloads as W

    rows = {}
    for name, kind, how, prec in WORKLOAD_ROWS:
        b = W.workload(name)
        dt = torch.float64 if prec == cf.FP64 else torch.float32
        keep, params = [], None
        if b.fn == W.FLETCHER_POWELL:
            keep = [torch.tensor(a, dtype=torch.float64, device=dev) for a in (b.fp.A, b.fp.B, b.fp.E)]
            params = cf.fp_params(*keep)
        x = torch.tensor(b.x, dtype=dt, device=dev)
        v = torch.tensor(b.v, dtype=dt, device=dev)
        if kind == "hvp":
            out = torch.empty_like(x)
            if how == "stated":
                cfg = cf.Config(4, 1, 256, cf.PLAIN, 0)
            else:
                cfg = cf.chessfad_autotune_hvp(b.fn, b.n, b.batch, x, v, out, params, prec, stream)

            def step(cfg=cfg):
                _checked(cf.chessfad_hvp_config(b.fn, b.n, b.batch, cfg, x, v, out, params, prec, stream),
                         "chessfad_hvp_config")
        else:
            out = torch.empty((b.batch, b.n, b.n), dtype=dt, device=dev)
            if how == "stated":
                cfg = cf.Config(4, 1, 256, cf.PLAIN, 0)
            else:
                cfg = cf.chessfad_autotune_hessian(b.fn, b.n, b.batch, x, out, params, prec, stream)

            def step(cfg=cfg):
                _checked(cf.chessfad_hessian_config(b.fn, b.n, b.batch, cfg, x, out, params, prec, stream),
                         "chessfad_hessian_config")
        cfg = cf.chessfad_resolve_config(b.fn, b.n, b.batch, prec, cfg, hvp=(kind == "hvp"))
        cd = cfg.as_dict()
        k = max(1, min(args.steps, args.workload_steps))
        barrier(world)
        ms = timed_steps(step, k, 2, stream, flush)
        tot = max_over_ranks(world, sum(ms), dev)
        per = tot / len(ms)
        sym = cd["method"] == "symmetric"
        mf = (model_flops_hvp if kind == "hvp" else model_flops_hessian)(b.fn, b.n, cfg.csize, sym)
        key = count_key(name, prec, kind, cd["method"], cfg.csize)
        roof = roofline_entry(counts, key, b.batch, sum(ms) / len(ms), prec, peaks, b.n, kind, mf,
                              kernel_name(cd["method"], prec, cfg.csize, b.fn, kind))
        rate = world * b.batch / (per * 1e-3)
        row = {"workload": name, "function": W.FN_NAMES[b.fn], "n": b.n, "batch": b.batch,
               "precision": PREC_NAME[prec], "kind": kind, "configuration": how, "config": cd,
               ("hvp_per_s" if kind == "hvp" else "hessians_per_s"): rate, "ms": per, "steps": len(ms),
               "roofline": roof}
        row["_out"] = out.double().cpu().numpy() if kind == "hvp" else out.cpu().numpy()
        row["_x"] = x.double().cpu().numpy()
        row["_v"] = v.double().cpu().numpy()
        row["_b"] = b
        rows[f"{name}/{PREC_NAME[prec]}/{kind}/{how}"] = row
        print(json.dumps({k2: v2 for k2, v2 in row.items() if not k2.startswith("_")}), file=sys.stderr, flush=True)
        del x, v, out, keep
    return rows


def gpu_arm(args):
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cf.load()
    b = W.workload(WORKLOAD)
    fn, n, batch = b.fn, b.n, b.batch
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = device_peaks(cf, local)
    counts = load_counts()

    f64 = headline_arm(cf, b, cf.FP64, args, world, dev, stream, flush, peaks, counts)
    f32 = headline_arm(cf, b, cf.FP32_COMP, args, world, dev, stream, flush, peaks, counts)
    rows = {} if args.no_workloads else workloads_arm(cf, args, world, dev, stream, flush, peaks, counts)
    ragged = None if args.no_ragged else ragged_arm(args, world, dev, stream, flush)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    config = headline_config(batch, world)
    pub = lambda d: {k: v for k, v in d.items() if not k.startswith("_")}
    line = {
        "metric": METRIC,
        "value": f64["value"],
        "unit": "HVP/s",
        "n_gpus": world,
        "steps": f64["steps"],
        "warmup": args.warmup,
        "ms_per_step": f64["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded PCG64 draws of the workload's distributions)",
        "config": config,
        "launch": f64["config"],
        "roofline": f64["roofline"],
        "e2e": f64["e2e"],
        "gpu_launches": f64["steps"],
        "clocks": f64["clocks"],
        "fp32_comp": {"value": f32["value"], "unit": "HVP/s", "dtype": "f32",
                      "precision": "FP32 hDual arithmetic with compensated sums and dots, FP64 islands",
                      "steps": f32["steps"], "ms_per_step": f32["ms_per_step"], "launch": f32["config"],
                      "roofline": f32["roofline"], "e2e": f32["e2e"], "clocks": f32["clocks"]},
        "fp32_over_fp64": f32["value"] / f64["value"],
        "chunk_sweep": {"fp64": f64["chunk_sweep"], "fp32_comp": f32["chunk_sweep"]},
        "seed_sparse": {"fp64": f64["seed_sparse"], "fp32_comp": f32["seed_sparse"],
                        "method": "symmetric, seed-sparse propagation (skips variables whose seed has no "
                                  "derivative part); equal to the dense result for finite inputs"},
        "peaks": {k: v for k, v in peaks.items()},
        "counts_source_hash": kernel_source_hash(),
        "counts_current": bool(counts),
    }
    if rows:
        line["workloads"] = {k: pub(r) for k, r in rows.items()}
    if ragged is not None:
        line["ragged_100k"] = pub(ragged)
    if world == 1 and not args.no_cpu_baseline:
        # The oracle leg: CPU baselines and every error against the oracle.
        line["cpu_baseline"] = cpu_baseline(b, 8, args)
        line["error_vs_oracle"] = headline_error(f64, 0)
        line["fp32_comp"]["error_vs_oracle"] = headline_error(f32, 1)
        for k, r in rows.items():
            line["workloads"][k]["error_vs_oracle"] = workload_error(r)
        if ragged is not None:
            e, t_all = ragged_error_all(ragged)
            line["ragged_100k"]["error_vs_oracle"] = e
            line["ragged_100k"]["cpu_baseline"] = ragged_cpu_baseline(ragged, t_all, args)
    try:
        line["summary"] = compact_summary(line)
    except Exception as exc:  # the summary repeats figures; it must never cost the line
        line["summary"] = {"error": repr(exc)}
    print(json.dumps(line))


def _sig(x, digits: int = 3):
    return None if x is None else float(f"{x:.{digits}g}")


def compact_summary(line: dict) -> dict:
    """The line's figures in a few hundred characters, printed as its last
    key so that the end of the output carries every workload's numbers:
    per entry [rate, roofline frac (executed flops / unit-count peak), e2e
    rate or null, max error against the oracle or null]."""
    def err(d):
        return _sig((d.get("error_vs_oracle") or {}).get("max"), 2)

    def frac(d):
        return _sig((d.get("roofline") or {}).get("frac"))

    out = {"fields": "rate, frac, e2e rate, max err",
           "fp64": [_sig(line["value"], 4), frac(line), _sig(line["e2e"]["value"], 4), err(line)]}
    f32 = line.get("fp32_comp")
    if f32:
        out["fp32_comp"] = [_sig(f32["value"], 4), frac(f32), _sig(f32["e2e"]["value"], 4), err(f32)]
    for k, r in (line.get("workloads") or {}).items():
        rate = r.get("hvp_per_s", r.get("hessians_per_s"))
        out[k] = [_sig(rate), frac(r), None, err(r)]
    rg = line.get("ragged_100k")
    if rg:
        untuned = rg.get("untuned_ms_per_step")
        out["ragged_100k"] = {"s_per_step": _sig(rg["ms_per_step"] / 1e3), "hvp_per_s": _sig(rg["value"]),
                              "untuned_s": None if untuned is None else _sig(untuned / 1e3),
                              "max_err": err(rg),
                              "requests_checked": (rg.get("error_vs_oracle") or {}).get("requests"),
                              "cpu_hvp_per_s": _sig((rg.get("cpu_baseline") or {}).get("value"))}
    cb = line.get("cpu_baseline")
    if cb:
        out["cpu_oracle_hvp_per_s"] = [_sig(cb["value"]), cb["cores"]]
    return out


def headline_config(batch: int, world: int) -> dict:
    """The workload description both arms print (the GPU launch configuration
    is reported separately under "launch")."""
    return {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}", "function": "ackley", "n": 64, "batch": batch,
            "precision": "fp64", "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas x{world} (points independent, no collective)"}


# ------------------------------------------------------------------ uneven batch
RAGGED_SYM_MIN_N = 128  # Fletcher-Powell requests this large run the symmetric method


def model_flops_request(fn: int, n: int, c: int) -> float:
    """Model flops of one HVP of the uneven batch: the symmetric method for
    Fletcher-Powell requests with n >= 128, the plain method otherwise."""
    return model_flops_hvp(fn, n, c, fn == 2 and n >= RAGGED_SYM_MIN_N)


def ragged_arm(args, world, dev, stream, flush):
    """The 100000-request uneven batch (three functions, n log-uniform in
    [2, 512], seed 4) in compensated FP32: the library's uneven-batch
    autotuner picks (chunk size, lanes per row) per (function, n range), then
    one persistent launch per step, replayed from a captured CUDA graph.  The
    default (untuned) plan is timed once beside it."""
    import numpy as np
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    rg = W.make_ragged()
    reqs = cf.requests(rg.fns, rg.ns, rg.offs, rg.eoffs)
    x = torch.tensor(rg.xpack, dtype=torch.float32, device=dev)
    v = torch.tensor(rg.vpack, dtype=torch.float32, device=dev)
    out = torch.empty_like(x)
    A = torch.tensor(rg.fp.A, device=dev)
    B = torch.tensor(rg.fp.B, device=dev)
    E = torch.tensor(rg.Epack, device=dev)
    params = cf.fp_params(A, B, E)

    def time_plan(plan, steps):
        plan.run(x, v, out, params)  # per-device set-up, outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.run(x, v, out, params)
        barrier(world)
        ms = timed_steps(g.replay, steps, 0, stream, flush)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(world, sum(ms), dev), len(ms)

    default_plan = cf.RaggedPlan(reqs, cf.FP32_COMP, 16)
    t_default, _ = (None, 0) if args.no_ragged_default else time_plan(default_plan, 1)
    ws = default_plan.workspace
    t0 = time.perf_counter()
    ngroups = cf.chessfad_ragged_autotune(reqs, cf.FP32_COMP, x, v, out, params, ws, ws.numel())
    t_tune = time.perf_counter() - t0
    del default_plan, ws
    t0 = time.perf_counter()
    plan = cf.RaggedPlan(reqs, cf.FP32_COMP, 0)
    t_plan = time.perf_counter() - t0
    tot, steps = time_plan(plan, args.ragged_steps)
    groups = {}
    flops = 0.0
    for f in (0, 1, 2):
        for b in range(1, 9):
            lo, hi = 1 << b, min(512, (2 << b) - 1) if b < 8 else 512
            sel = (rg.fns == f) & (rg.ns >= lo) & (rg.ns <= hi)
            if not sel.any():
                continue
            c, tpr, mt = cf.chessfad_ragged_plan_group_config(plan.handle, f, int(rg.ns[sel][0]))
            groups[f"{W.FN_NAMES[f]}/n{lo}-{hi}"] = {"csize": c, "threads_per_row": tpr, "requests": int(sel.sum()),
                                                    **({"ab_tile_rows_at_n": [int(rg.ns[sel][0]), mt]}
                                                       if f == 2 else {})}
            flops += sum(model_flops_request(f, int(n), c) for n in rg.ns[sel])
    per = tot / steps
    return {"value": world * rg.nreq * steps / (tot * 1e-3), "unit": "HVP/s", "requests": rg.nreq,
            "steps": steps, "warmup": 1, "ms_per_step": per, "precision": "fp32_comp",
            "launch": "one persistent kernel per step, CUDA graph replay", "tiles": plan.info["ntiles"],
            "method": "plain; symmetric (SC-HESS-VEC) for Fletcher-Powell n >= 128",
            "tuned_groups": groups, "autotune_seconds": t_tune, "groups_tuned": ngroups,
            "untuned_ms_per_step": t_default, "untuned_config": "csize 16, default lanes per row",
            "workspace_bytes": plan.info["workspace_bytes"], "plan_seconds": t_plan,
            "model_tflops": flops / (per * 1e-3) / 1e12,
            "_out": out.double().cpu().numpy(), "_x": x.double().cpu().numpy(), "_v": v.double().cpu().numpy(),
            "_rg": rg, "_c": 16}  # the oracle's CHESS-VEC chunk size for the CPU baseline


# ------------------------------------------------------------------ oracle leg
# Everything below runs the oracle (test infrastructure): the CPU baselines and
# the errors of the GPU outputs against it.  It runs on rank 0 at N = 1 only.
def headline_error(res, prec):
    """Per-point normalised error of the headline outputs over the whole
    batch (the oracle is given the values the device held)."""
    import oracle
    from paper_2410_22575_gb300 import metrics

    ref, hn = oracle.hvp(1, res["_x"], res["_v"], with_norm=True)
    e = metrics.hvp_errors(res["_out"], ref, hn, res["_v"])
    bound = metrics.FP64_BOUND if prec == 0 else metrics.FP32_COMP_BOUND
    # the spectral-norm normalisation as well (n <= 64), on the first 4096 points
    k = min(4096, len(e))
    es = metrics.hvp_errors_spectral(res["_out"][:k], ref[:k], oracle.hessian_batch(1, res["_x"][:k]),
                                     res["_v"][:k])
    return {**metrics.summary(e), "points": int(len(e)), "bound": bound, "within_bound": bool(e.max() <= bound),
            "max_spectral": float(es.max()), "spectral_points": int(k)}


def workload_error(row):
    import oracle
    from paper_2410_22575_gb300 import metrics, workloads as W

    b = row["_b"]
    p = None if b.fp is None else oracle.FPParams(b.fp.A, b.fp.B, b.fp.E)
    extra = {}
    if row["kind"] == "hvp":
        ref, hn = oracle.hvp(b.fn, row["_x"], row["_v"], p, with_norm=True)
        e = metrics.hvp_errors(row["_out"], ref, hn, row["_v"])
        if b.n <= 64:
            es = metrics.hvp_errors_spectral(row["_out"], ref, oracle.hessian_batch(b.fn, row["_x"], p), row["_v"])
            extra = {"max_spectral": float(es.max())}
    else:
        e = metrics.hessian_errors(row["_out"], oracle.hessian_batch(b.fn, row["_x"], p))
    bound = metrics.FP64_BOUND if row["precision"] == "fp64" else metrics.FP32_COMP_BOUND
    return {**metrics.summary(e), "points": int(len(e)), "bound": bound, "within_bound": bool(e.max() <= bound),
            **extra}


def ragged_error_all(r):
    """Error of every one of the 100000 requests against the oracle (closed
    forms, O1); also returns the oracle's wall time on all of them."""
    import oracle
    from paper_2410_22575_gb300 import metrics

    rg = r["_rg"]
    t0 = time.perf_counter()
    ref, hn = oracle.hvp_ragged(rg.fns, rg.ns, rg.offs, rg.eoffs, r["_x"], r["_v"], rg.fp.A, rg.fp.B, rg.Epack,
                                rg.ld)
    t_all = time.perf_counter() - t0
    e = metrics.ragged_hvp_errors(r["_out"], ref, hn, r["_v"], rg.ns, rg.offs)
    per_fn = {}
    for f, name in ((0, "rosenbrock"), (1, "ackley"), (2, "fletcher_powell")):
        sel = rg.fns == f
        per_fn[name] = metrics.summary(e[sel])
    return {**metrics.summary(e), "requests": int(len(e)), "bound": metrics.FP32_COMP_BOUND,
            "within_bound": bool(e.max() <= metrics.FP32_COMP_BOUND), "per_function": per_fn}, t_all


def ragged_cpu_baseline(r, t_closed_form_all, args):
    """The oracle's CHESS-VEC (Alg. 7, FP64, the plan's chunk size) on a random
    sample of the 100000 requests whose model cost is bounded, run on all host
    cores (one request per thread), extrapolated to all requests by the model
    flops of each request; and the closed-form oracle on all of them."""
    import concurrent.futures as futures

    import numpy as np

    import oracle

    rg = r["_rg"]
    c = r["_c"]
    oracle.build()
    cost = np.array([model_flops_hvp(int(f), int(n), c) for f, n in zip(rg.fns, rg.ns)])
    rng = np.random.Generator(np.random.PCG64(5))
    cap = args.ragged_cpu_cap
    cand = np.nonzero(cost <= cap)[0]
    order = rng.permutation(cand)
    cores = oracle.num_threads()
    budget = args.cpu_seconds

    def one(q):
        o, n = int(rg.offs[q]), int(rg.ns[q])
        pe = oracle.FPParams(rg.fp.A[:n, :n], rg.fp.B[:n, :n], rg.Epack[rg.eoffs[q]:rg.eoffs[q] + n]) \
            if rg.fns[q] == 2 else None
        oracle.chess_vec(int(rg.fns[q]), r["_x"][o:o + n], r["_v"][o:o + n], c, pe)

    # grow the sample in rounds until the budget is spent
    done = 0
    t_run = 0.0
    with futures.ThreadPoolExecutor(cores) as ex:
        while done < len(order) and t_run < budget:
            take = order[done:done + max(cores * 8, 64)]
            t0 = time.perf_counter()
            list(ex.map(one, take))
            t_run += time.perf_counter() - t0
            done += len(take)
    sample = order[:done]
    frac_flops = cost.sum() / cost[sample].sum()
    t_all_est = t_run * frac_flops
    return {"value": rg.nreq / t_all_est, "unit": "HVP/s", "cores": cores, "kind": "oracle",
            "extrapolated": True,
            "sample": (f"CHESS-VEC (Alg. 7) FP64 c={c} on {len(sample)} random requests with model cost <= "
                       f"{cap:.0e} flops ({cost[sample].sum() / cost.sum() * 100:.3f} % of the batch's model "
                       f"flops), {t_run:.1f} s on {cores} threads; scaled to all {rg.nreq} requests by model "
                       f"flops"),
            "sample_requests": int(len(sample)), "sample_seconds": t_run,
            "closed_form_all_requests_seconds": t_closed_form_all,
            "closed_form_hvp_per_s": rg.nreq / t_closed_form_all}


def cpu_sample_time(b, c, target_s):
    """Time the oracle's CHESS-VEC (Alg. 7, FP64, OpenMP over points) on a
    prefix of the batch sized for about target_s seconds; return
    (hvp_per_s, sample_points, seconds, outputs)."""
    import oracle

    oracle.build()
    probe = 64
    t0 = time.perf_counter()
    oracle.chess_vec(b.fn, b.x[:probe], b.v[:probe], c)
    dt = time.perf_counter() - t0
    m = int(min(b.batch, max(probe, probe * target_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    out = oracle.chess_vec(b.fn, b.x[:m], b.v[:m], c)
    dt = time.perf_counter() - t0
    return m / dt, m, dt, out


def cpu_baseline(b, c, args):
    """The oracle's CHESS-VEC (FP64, chunk c) on a timed prefix of the
    headline batch, and the closed-form oracle on the same prefix."""
    import oracle

    rate, m, dt, _ = cpu_sample_time(b, c, args.cpu_seconds)
    t0 = time.perf_counter()
    oracle.hvp(b.fn, b.x[:m], b.v[:m])
    t_cf = time.perf_counter() - t0
    # one thread, as the paper's sequential CPU runs (Sec. VII)
    cores = oracle.num_threads()
    prev = oracle.set_num_threads(1)
    try:
        rate1, m1, dt1, _ = cpu_sample_time(b, c, max(1.0, args.cpu_seconds / 4))
    finally:
        oracle.set_num_threads(prev)
    return {"value": rate, "unit": "HVP/s", "cores": cores, "kind": "oracle",
            "sample": f"first {m} of {b.batch} points, CHESS-VEC (Alg. 7) FP64 with c={c}, {dt:.1f} s",
            "closed_form_hvp_per_s": m / t_cf,
            "single_thread": {"value": rate1, "unit": "HVP/s", "cores": 1,
                              "sample": f"first {m1} points, CHESS-VEC (Alg. 7) FP64 with c={c}, {dt1:.1f} s"}}


def reference_arm(args):
    """The oracle's CHESS-VEC (Alg. 7, FP64, c = 8) on the host cores: each
    step a prefix of the headline batch sized to the step budget; ms_per_step
    is the measured time of that step."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2410_22575_gb300 import workloads as W

    b = W.workload(WORKLOAD)
    c = 8
    per = max(0.5, min(20.0, args.ref_budget / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_sample_time(b, c, per / 4)
    rates, secs, pts = [], [], []
    for _ in range(args.steps):
        r, m, dt, _ = cpu_sample_time(b, c, per)
        rates.append(r)
        secs.append(dt)
        pts.append(m)
    value = sum(pts) / sum(secs)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "HVP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64 draws of the workload's distributions)",
        "config": headline_config(b.batch, world),
        "launch": {"oracle": "CHESS-VEC (Alg. 7)", "csize": c, "points_per_step": int(statistics.median(pts))},
        "cpu_baseline": {"value": value, "unit": "HVP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: the first {int(statistics.median(pts))} of {b.batch} points "
                                   f"(about {per:.1f} s of work), CHESS-VEC (Alg. 7) FP64, c={c}"},
        "e2e": {"value": value, "unit": "HVP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ executed-instruction counts
# The kernels whose executed FP instructions (and DRAM bytes) the roofline
# reports: for each named workload and precision both methods at every chunk
# size the autotuner may pick (profile_set).  Counts are
# per point: the per-point work of these kernels does not depend on the number
# of points, threads per point or points per CTA, so a capture on a prefix of
# the batch scales to the full batch by the number of points.
PROFILE_BATCH = {("ackley_n64", 0): 16384, ("ackley_n64", 1): 16384, ("rosenbrock_n16", 0): 4096,
                 ("rosenbrock_n16", 1): 4096, ("fletcher_powell_n32", 0): 2048, ("fletcher_powell_n32", 1): 8192,
                 ("rosenbrock_n256", 0): 128, ("rosenbrock_n256", 1): 512}


def profile_set():
    """Every (workload, precision, kind, method, chunk size) the bench's
    autotuned or stated configurations can land on: both methods, chunk sizes
    2..32 up to the next power of two of n (spilling kernels are skipped at
    run time), HVPs everywhere and Hessians of the Rosenbrock workloads."""
    from paper_2410_22575_gb300 import workloads as W

    out = []
    for name in ("ackley_n64", "rosenbrock_n16", "fletcher_powell_n32", "rosenbrock_n256"):
        fn, n, _, _ = W.WORKLOADS[name]
        kinds = ("hvp", "hessian") if name in ("rosenbrock_n16", "rosenbrock_n256") else ("hvp",)
        for prec in (0, 1):
            cs = [c for c in (2, 4, 8, 16, 32) if c <= max(1, 1 << (n - 1).bit_length())]
            for kind in kinds:
                for method in ("symmetric", "plain"):
                    for c in cs:
                        out.append((name, prec, kind, method, c))
    return out


def profile_kernels(args):
    """Launch every kernel of profile_set() once on a prefix of its workload
    (after one untimed warm-up launch of the library's FMA microbenchmark,
    which no kernel filter matches).  Writes the launch order to
    --profile-keys so --ingest-ncu can name the captured launches."""
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    cf.load()
    keys = []
    for name, prec, kind, method, c in profile_set():
        b = W.workload(name, batch=PROFILE_BATCH[(name, prec)])
        dt = torch.float64 if prec == 0 else torch.float32
        if cf.chessfad_kernel_info(b.fn, prec, c, kind == "hvp")["local_bytes"] > 48:
            continue
        keep, params = [], None
        if b.fn == W.FLETCHER_POWELL:
            keep = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (b.fp.A, b.fp.B, b.fp.E)]
            params = cf.fp_params(*keep)
        x = torch.tensor(b.x, dtype=dt, device="cuda")
        v = torch.tensor(b.v, dtype=dt, device="cuda")
        cfg = cf.Config(c, 1, 256, cf.PLAIN, 0) if method == "plain" else cf.Config(c, 0, 0, cf.SYMMETRIC, 0)
        cfg = cf.chessfad_resolve_config(b.fn, b.n, b.batch, prec, cfg, hvp=(kind == "hvp"))
        if kind == "hvp":
            out = torch.empty_like(x)
            st = cf.chessfad_hvp_config(b.fn, b.n, b.batch, cfg, x, v, out, params, prec)
        else:
            out = torch.empty((b.batch, b.n, b.n), dtype=dt, device="cuda")
            st = cf.chessfad_hessian_config(b.fn, b.n, b.batch, cfg, x, out, params, prec)
        torch.cuda.synchronize()
        if st != 0:
            raise cf.ChessfadError(st, f"profile launch {name} {prec} {kind} {method} {c}")
        keys.append({"key": count_key(name, prec, kind, method, c), "batch": b.batch, "fn": b.fn, "prec": prec,
                     "c": c, "kind": kind, "method": method, "config": cfg.as_dict()})
        del x, v, out, keep
    with open(args.profile_keys, "w") as f:
        json.dump({"source_hash": kernel_source_hash(), "launches": keys}, f, indent=1)
    print(json.dumps({"mode": "profile-kernels", "launches": len(keys)}))


NCU_METRICS = ("gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum,"
               "smsp__issue_active.avg.pct_of_peak_sustained_active,smsp__inst_executed.sum,"
               "smsp__sass_thread_inst_executed_op_ffma_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_fadd_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_fmul_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_ffma2_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_fadd2_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_fmul2_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_dfma_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_dadd_pred_on.sum,"
               "smsp__sass_thread_inst_executed_op_dmul_pred_on.sum")


def _num(s: str) -> float:
    s = s.strip().replace(",", "")
    return float(s) if s not in ("", "n/a") else float("nan")


def read_ncu_csv(path: str) -> list[dict]:
    """Launches of an ncu --csv capture (the details page, one row per
    metric, or the raw page, one row per launch), in capture order."""
    rows = list(csv.reader(open(path)))
    hdr_i = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hdr_i]
    body = rows[hdr_i + 1:]
    launches: dict[str, dict] = {}
    order = []
    if "Metric Name" in hdr:
        ci, ck, cm, cv, cu = (hdr.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Value",
                                                     "Metric Unit"))
        for r in body:
            if len(r) <= cv:
                continue
            lid = r[ci]
            if lid not in launches:
                launches[lid] = {"name": r[ck]}
                order.append(lid)
            val = _num(r[cv])
            unit = r[cu].strip().lower()
            scale = {"kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "usecond": 1e3, "msecond": 1e6,
                     "nsecond": 1.0, "second": 1e9}.get(unit, 1.0)
            launches[lid][r[cm]] = val * scale
    else:
        ci, ck = hdr.index("ID"), hdr.index("Kernel Name")
        for r in body:
            if len(r) != len(hdr) or not r[ci].strip().isdigit():
                continue
            d = {"name": r[ck]}
            for j, h in enumerate(hdr):
                if "__" in h:
                    d[h] = _num(r[j])
            launches[r[ci]] = d
            order.append(r[ci])
    return [launches[i] for i in order]


def ingest_ncu(args):
    """profiles/counts.json from an ncu capture of --profile-kernels: per
    kernel key, executed FP flops per point (2 x FMA + ADD + MUL thread
    instructions, FP32 and FP64; a packed FP32 instruction, FFMA2, FADD2 or
    FMUL2, does two of them) and DRAM bytes per point."""
    keys = json.load(open(args.profile_keys))
    launches = [l for l in read_ncu_csv(args.ingest_ncu) if "sym_kernel" in l["name"] or "sweep_kernel" in l["name"]]
    if len(launches) != len(keys["launches"]):
        raise SystemExit(f"ncu captured {len(launches)} sweep launches, the profile run made {len(keys['launches'])}")
    kernels = {}
    for l, k in zip(launches, keys["launches"]):
        nm = l["name"]
        want_t = "double" if k["prec"] == 0 else "float"
        base = "sweep_kernel" if k["method"] == "plain" else "sym_kernel"
        targs = nm[nm.index("<") + 1:nm.index(">")].split(",")
        targs = [t.strip() for t in targs]
        if base not in nm or targs[0] != want_t or int(targs[2]) != k["c"] or int(targs[3]) != k["fn"] or \
                int(targs[4]) != (1 if k["kind"] == "hvp" else 0):
            raise SystemExit(f"launch {nm} does not match {k['key']}")
        g = lambda m: l.get(f"smsp__sass_thread_inst_executed_op_{m}_pred_on.sum", 0.0)
        fp32 = 2 * g("ffma") + g("fadd") + g("fmul") + 2 * (2 * g("ffma2") + g("fadd2") + g("fmul2"))
        fp64 = 2 * g("dfma") + g("dadd") + g("dmul")
        fl = fp32 + fp64
        dram = l.get("dram__bytes_read.sum", float("nan")) + l.get("dram__bytes_write.sum", float("nan"))
        u = k["batch"]
        kernels[k["key"]] = {
            "kernel": nm, "config": k["config"], "points_captured": u,
            "executed_flops_per_unit": fl / u,
            "fp32_flops_per_unit": fp32 / u,
            "fp64_flops_per_unit": fp64 / u,
            "fp32_packed_share": (2 * (g("ffma2") + g("fadd2") + g("fmul2")) /
                                  (g("ffma") + g("fadd") + g("fmul") + 2 * (g("ffma2") + g("fadd2") + g("fmul2")))
                                  if fp32 else 0.0),
            "dram_bytes_per_unit": None if math.isnan(dram) else dram / u,
            "duration_ns_captured": l.get("gpu__time_duration.sum"),
            "issue_active_pct": l.get("smsp__issue_active.avg.pct_of_peak_sustained_active"),
            "warp_instructions_per_unit": l.get("smsp__inst_executed.sum", float("nan")) / u,
        }
    doc = {"source_hash": keys["source_hash"],
           "note": ("per point ('unit'): executed flops = 2 x FMA + ADD + MUL thread instructions (FP32 and "
                    "FP64, predicated on; a packed FP32 FFMA2 / FADD2 / FMUL2 counts twice), "
                    "fp32_packed_share = share of the FP32 operations done by packed instructions, DRAM bytes = dram__bytes_read.sum + dram__bytes_write.sum, from one "
                    "ncu capture per kernel on a prefix of the workload (points_captured), divided by the points"),
           "command": args.ncu_command, "kernels": kernels}
    if keys["source_hash"] != kernel_source_hash():
        raise SystemExit("the kernel sources changed since the capture")
    out_path = args.counts_out or COUNTS_FILE
    with open(out_path, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
    print(f"{len(kernels)} kernels -> {out_path}")
    # a markdown table of the capture (executed against model flops, DRAM
    # bytes against algorithmic bytes, per point)
    from paper_2410_22575_gb300 import workloads as W

    print("| kernel key | kernel | executed flop/pt | model / executed | issue active % | DRAM B/pt | "
          "algorithmic B/pt | ncu time (ms) |")
    print("|---|---|---|---|---|---|---|---|")
    for key in sorted(kernels):
        e = kernels[key]
        name, prec_s, kind, method, c = key.split("/")
        fn, n, _, _ = W.WORKLOADS[name]
        prec = 0 if prec_s == "fp64" else 1
        c = int(c[1:])
        sym = method == "symmetric"
        mf = (model_flops_hvp if kind == "hvp" else model_flops_hessian)(fn, n, c, sym)
        kn = kernel_name(method, prec, c, fn, kind)
        dram = e["dram_bytes_per_unit"]
        ia = e.get("issue_active_pct")
        print(f"| {key} | {kn} | {e['executed_flops_per_unit']:.4g} | {mf / e['executed_flops_per_unit']:.2f} | "
              f"{'-' if ia is None else f'{ia:.1f}'} | "
              f"{'-' if dram is None else f'{dram:.0f}'} | {algorithmic_bytes(n, prec, kind)} | "
              f"{(e['duration_ns_captured'] or 0) / 1e6:.2f} |")


def kernel_only(args):
    """Run only the sweep kernel of the workload in a fixed configuration
    (W + K launches, no autotune): the command profiled with ncu."""
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    if args.fn is not None:
        b = W.make_batch(args.fn, args.n, args.batch or 1024, args.seed)
    else:
        b = W.workload(args.workload, batch=args.batch)
    prec = cf.FP64 if args.prec == "fp64" else cf.FP32_COMP
    dt = torch.float64 if prec == cf.FP64 else torch.float32
    x = torch.tensor(b.x, dtype=dt, device="cuda")
    v = torch.tensor(b.v, dtype=dt, device="cuda")
    out = torch.empty_like(x)
    keep, params = [], None
    if b.fn == W.FLETCHER_POWELL:
        keep = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (b.fp.A, b.fp.B, b.fp.E)]
        params = cf.fp_params(*keep)
    if args.method in ("symmetric", "symmetric_sparse"):
        m = cf.SYMMETRIC if args.method == "symmetric" else cf.SYMMETRIC_SPARSE
        cfg = cf.Config(args.csize, 0, args.block, m, args.tpp)
    else:
        cfg = cf.Config(args.csize, args.tpr, args.block)
    stream = torch.cuda.current_stream()
    ms = []
    for k in range(args.warmup + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = cf.chessfad_hvp_config(b.fn, b.n, b.batch, cfg, x, v, out, params, prec, stream)
        e1.record(stream)
        if st != 0:
            raise cf.ChessfadError(st, "chessfad_hvp_config")
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    print(json.dumps({"mode": "kernel-only", "workload": args.workload, "batch": b.batch, "prec": args.prec,
                      **cfg.as_dict(), "ms": ms, "hvp_per_s": b.batch / (min(ms) * 1e-3)}))


def ragged_only(args):
    """Run only the uneven-batch kernel on a subset of the 100000-request
    workload (the requests of one function with n in [--ragged-min-n,
    --ragged-max-n], the first --ragged-count of them): W + K launches, the
    command the ncu summary of the persistent kernel captures."""
    import numpy as np
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    rg = W.make_ragged()
    idx = np.nonzero((rg.fns == args.ragged_fn) & (rg.ns >= args.ragged_min_n) & (rg.ns <= args.ragged_max_n))[0]
    sub = rg.subset(idx[: args.ragged_count])
    prec = cf.FP64 if args.prec == "fp64" else cf.FP32_COMP
    dt = torch.float64 if prec == cf.FP64 else torch.float32
    plan = cf.RaggedPlan(cf.requests(sub.fns, sub.ns, sub.offs, sub.eoffs), prec, args.csize)
    x = torch.tensor(sub.xpack, dtype=dt, device="cuda")
    v = torch.tensor(sub.vpack, dtype=dt, device="cuda")
    out = torch.empty_like(x)
    keep = [torch.tensor(a, device="cuda") for a in (sub.fp.A, sub.fp.B, sub.Epack)]
    params = cf.fp_params(*keep)
    ms = []
    for k in range(args.warmup + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.run(x, v, out, params)
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    print(json.dumps({"mode": "ragged-only", "requests": len(sub.fns), "fn": args.ragged_fn,
                      "n_range": [int(sub.ns.min()), int(sub.ns.max())], "prec": args.prec, "csize": args.csize, "plan": plan.info,
                      "ms": ms, "hvp_per_s": len(sub.fns) / (min(ms) * 1e-3)}))


def graph_timed(fn_call, reps: int) -> float:
    """Device time per call in ms: reps calls captured in one CUDA graph and
    replayed between two events (best of two replays), so host-side call
    overhead (tens of microseconds through the binding) never leaves the GPU
    idle inside the timed region -- it would dominate the small workloads."""
    import torch

    fn_call()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            fn_call()
    g.replay()
    torch.cuda.synchronize()
    best = None
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        best = t if best is None else min(best, t)
    return best


def sparse_study(args):
    """Seed-sparse symmetric method against the tuned dense method, every
    named workload in both precisions: the dense rate is the HVP autotuner's
    pick; the seed-sparse rate is the best over c in {4, 8, 16}, threads per
    point in {32, 64, 128} and CTAs of 128 or 256 threads (kernel time, CUDA
    graph replay).  The seed-sparse method skips variables whose seed has no
    derivative part, which the paper's dense arithmetic does not."""
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    rows = []
    for name in ("rosenbrock_n16", "ackley_n64", "fletcher_powell_n32", "rosenbrock_n256"):
        b = W.workload(name)
        keep, params = [], None
        if b.fn == W.FLETCHER_POWELL:
            keep = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (b.fp.A, b.fp.B, b.fp.E)]
            params = cf.fp_params(*keep)
        for prec, dt in ((cf.FP64, torch.float64), (cf.FP32_COMP, torch.float32)):
            x = torch.tensor(b.x, dtype=dt, device="cuda")
            v = torch.tensor(b.v, dtype=dt, device="cuda")
            out = torch.empty_like(x)
            reps = 5 if prec == cf.FP32_COMP else 2
            cfg = cf.chessfad_autotune_hvp(b.fn, b.n, b.batch, x, v, out, params, prec)
            t_dense = graph_timed(lambda: cf.chessfad_hvp(b.fn, b.n, b.batch, 0, x, v, out, params, prec), reps)
            best = None
            for c in (4, 8, 16):
                for tpp in (32, 64, 128):
                    for block in (128, 256):
                        if block < tpp:
                            continue
                        sc = cf.Config(c, 0, block, cf.SYMMETRIC_SPARSE, tpp)
                        t = graph_timed(lambda: cf.chessfad_hvp_config(b.fn, b.n, b.batch, sc, x, v, out, params,
                                                                       prec), reps)
                        if best is None or t < best[0]:
                            best = (t, sc.as_dict())
            row = {"workload": name, "precision": PREC_NAME[0 if prec == cf.FP64 else 1],
                   "dense": {"config": cfg.as_dict(), "hvp_per_s": b.batch / (t_dense * 1e-3)},
                   "seed_sparse": {"config": best[1], "hvp_per_s": b.batch / (best[0] * 1e-3)},
                   "ratio": t_dense / best[0]}
            rows.append(row)
            print(json.dumps(row), flush=True)
            del x, v, out
    return rows


def report(args):
    """Per-workload table: HVP/s (and Hessians/s) for every
    named workload in both precisions, autotuned over both methods, plus the
    plain method at the workload's stated chunk size."""
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    rows = []
    peaks = device_peaks(cf, 0)
    timed = graph_timed

    for name in ("rosenbrock_n16", "ackley_n64", "fletcher_powell_n32", "rosenbrock_n256"):
        b = W.workload(name)
        keep, params = [], None
        if b.fn == W.FLETCHER_POWELL:
            keep = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (b.fp.A, b.fp.B, b.fp.E)]
            params = cf.fp_params(*keep)
        for prec, dt in ((cf.FP32_COMP, torch.float32), (cf.FP64, torch.float64)):
            x = torch.tensor(b.x, dtype=dt, device="cuda")
            v = torch.tensor(b.v, dtype=dt, device="cuda")
            out = torch.empty_like(x)
            reps = 5 if prec == cf.FP32_COMP else 2
            cfg = cf.chessfad_autotune_hvp(b.fn, b.n, b.batch, x, v, out, params, prec)
            t = timed(lambda: cf.chessfad_hvp(b.fn, b.n, b.batch, 0, x, v, out, params, prec), reps)
            row = {"workload": name, "precision": "fp64" if prec == cf.FP64 else "fp32_comp",
                   "tuned": cfg.as_dict(), "hvp_per_s": b.batch / (t * 1e-3), "ms": t}
            mf = model_flops_hvp(b.fn, b.n, cfg.csize, cfg.method == cf.SYMMETRIC)
            row["model_tflops"] = mf * b.batch / (t * 1e-3) / 1e12
            peak = peaks[PREC_NAME[prec]]["microbench"]
            row["model_frac_of_microbench"] = None if not peak else mf * b.batch / (t * 1e-3) / peak
            c0 = 4 if name == "rosenbrock_n16" else cfg.csize
            plain = cf.Config(c0, 1, 256)
            t = timed(lambda: cf.chessfad_hvp_config(b.fn, b.n, b.batch, plain, x, v, out, params, prec), reps)
            row["plain_c%d_hvp_per_s" % c0] = b.batch / (t * 1e-3)
            if name in ("rosenbrock_n16", "rosenbrock_n256"):
                H = torch.empty((b.batch, b.n, b.n), dtype=dt, device="cuda")
                best = None
                for hc in (cf.Config(c0, 1, 256), cf.Config(c0, 0, 256, cf.SYMMETRIC, 64)):
                    t = timed(lambda: cf.chessfad_hessian_config(b.fn, b.n, b.batch, hc, x, H, params, prec), reps)
                    if best is None or t < best[0]:
                        best = (t, hc.as_dict())
                row["hessians_per_s"] = b.batch / (best[0] * 1e-3)
                row["hessian_cfg"] = best[1]
                del H
            rows.append(row)
            print(json.dumps(row), flush=True)
    return rows


def cpu_baseline_report(args):
    """The CPU-baseline leg for every named workload: the oracle's CHESS-VEC
    (Alg. 7, FP64, OpenMP over points) on a timed prefix of the batch and the
    closed-form oracle on the whole batch, on this host's cores."""
    import oracle
    from paper_2410_22575_gb300 import workloads as W

    oracle.build()
    for name, c in (("rosenbrock_n16", 4), ("ackley_n64", 8), ("fletcher_powell_n32", 4), ("rosenbrock_n256", 16)):
        b = W.workload(name)
        p = None if b.fp is None else oracle.FPParams(b.fp.A, b.fp.B, b.fp.E)
        probe = 8
        t0 = time.perf_counter()
        oracle.chess_vec(b.fn, b.x[:probe], b.v[:probe], c, p)
        dt = time.perf_counter() - t0
        m = int(min(b.batch, max(probe, probe * args.cpu_seconds / 3 / max(dt, 1e-6))))
        t0 = time.perf_counter()
        oracle.chess_vec(b.fn, b.x[:m], b.v[:m], c, p)
        t_cv = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.hvp(b.fn, b.x, b.v, p)
        t_cf = time.perf_counter() - t0
        print(json.dumps({"workload": name, "cores": oracle.num_threads(), "chess_vec_c": c,
                          "chess_vec_hvp_per_s": m / t_cv, "chess_vec_sample": m,
                          "closed_form_hvp_per_s": b.batch / t_cf}), flush=True)


def chunk_study(args):
    """Measured best chunk size per (function, n, method) in compensated FP32
    against the Sec. V operation-count model: for the plain method the
    multiplication count (6 + 3/c) n^2 M falls with c (largest c best); for
    the symmetric method (3/2) n (2n + 2c + n/c + 1) M is smallest at
    c = sqrt(n/2)."""
    import math

    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    for fn in (W.ROSENBROCK, W.ACKLEY, W.FLETCHER_POWELL):
        for n in (8, 16, 32, 64, 128):
            budget = 2.0e11 if fn != W.FLETCHER_POWELL else 6.0e11
            cost = n ** 3 if fn != W.FLETCHER_POWELL else n ** 4
            batch = int(max(256, min(65536, budget / (20 * cost))))
            b = W.make_batch(fn, n, batch, seed=100 + n)
            keep, params = [], None
            if fn == W.FLETCHER_POWELL:
                keep = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (b.fp.A, b.fp.B, b.fp.E)]
                params = cf.fp_params(*keep)
            x = torch.tensor(b.x, dtype=torch.float32, device="cuda")
            v = torch.tensor(b.v, dtype=torch.float32, device="cuda")
            out = torch.empty_like(x)
            res = {}
            for method in ("plain", "symmetric"):
                for c in (1, 2, 4, 8, 16, 32):
                    if c > max(1, 1 << (n - 1).bit_length()):
                        continue
                    cfg = (cf.Config(c, 1, 256) if method == "plain"
                           else cf.Config(c, 0, 128, cf.SYMMETRIC, 32))
                    if cf.chessfad_hvp_config(fn, n, batch, cfg, x, v, out, params, cf.FP32_COMP) != 0:
                        continue
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(3):
                        cf.chessfad_hvp_config(fn, n, batch, cfg, x, v, out, params, cf.FP32_COMP)
                    e1.record()
                    torch.cuda.synchronize()
                    res[(method, c)] = 3 * batch / (e0.elapsed_time(e1) * 1e-3)
            for method in ("plain", "symmetric"):
                cs = {c: r for (m, c), r in res.items() if m == method}
                if not cs:
                    continue
                best = max(cs, key=cs.get)
                print(json.dumps({"function": W.FN_NAMES[fn], "n": n, "method": method, "best_c": best,
                                  "model_c": (max(cs) if method == "plain" else math.sqrt(n / 2)),
                                  "hvp_per_s": {str(c): round(r) for c, r in sorted(cs.items())}}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["chessfad", "reference"], default="chessfad")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ragged", action="store_true", help="skip the 100000-request uneven batch")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other named workloads")
    ap.add_argument("--workload-steps", type=int, default=5, help="timed steps per row of the workloads block")
    ap.add_argument("--ragged-steps", type=int, default=1)
    ap.add_argument("--no-ragged-default", action="store_true", help="skip timing the untuned uneven-batch plan")
    ap.add_argument("--ragged-cpu-cap", type=float, default=3e9,
                    help="uneven-batch CPU baseline: model-flop cap of the sampled requests")
    ap.add_argument("--kernel-only", action="store_true", help="run only the sweep kernel (for ncu)")
    ap.add_argument("--ragged-only", action="store_true",
                    help="run only the uneven-batch kernel on a subset of the 100000-request workload (for ncu)")
    ap.add_argument("--ragged-fn", type=int, default=2)
    ap.add_argument("--ragged-min-n", type=int, default=256)
    ap.add_argument("--ragged-max-n", type=int, default=512)
    ap.add_argument("--ragged-count", type=int, default=32)
    ap.add_argument("--report", action="store_true", help="per-workload table (all named workloads)")
    ap.add_argument("--chunk-study", action="store_true", help="measured best chunk size vs the Sec. V model")
    ap.add_argument("--sparse-study", action="store_true", help="seed-sparse vs tuned dense method, every workload")
    ap.add_argument("--cpu-report", action="store_true", help="CPU-baseline leg for every named workload")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="launch each kernel of the executed-count set once (the command ncu captures)")
    ap.add_argument("--profile-keys", default="profile_keys.json",
                    help="where --profile-kernels writes, and --ingest-ncu reads, the launch order")
    ap.add_argument("--ingest-ncu", default=None, help="ncu CSV of --profile-kernels -> profiles/counts.json")
    ap.add_argument("--ncu-command", default="", help="the ncu command recorded in profiles/counts.json")
    ap.add_argument("--counts-out", default=None, help="--ingest-ncu: output file (default profiles/counts.json)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fn", type=int, default=None, help="kernel-only: function id instead of a named workload")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--prec", choices=["fp32_comp", "fp64"], default="fp32_comp")
    ap.add_argument("--csize", type=int, default=32)
    ap.add_argument("--tpr", type=int, default=1)
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--ref-budget", type=float, default=100.0,
                    help="reference arm: seconds of oracle work over all steps (bounded per step)")
    ap.add_argument("--e2e-slices", type=int, default=16,
                    help="slices of the end-to-end call (copies of one overlap the sweep of the next)")
    ap.add_argument("--method", choices=["plain", "symmetric", "symmetric_sparse"], default="plain")
    ap.add_argument("--tpp", type=int, default=64, help="kernel-only, symmetric: threads per point")
    args = ap.parse_args()
    if args.warmup < 3 and not (args.kernel_only or args.profile_kernels or args.ragged_only):
        args.warmup = 3
    if args.ingest_ncu:
        ingest_ncu(args)
    elif args.profile_kernels:
        profile_kernels(args)
    elif args.cpu_report:
        cpu_baseline_report(args)
    elif args.chunk_study:
        chunk_study(args)
    elif args.report:
        report(args)
    elif args.sparse_study:
        sparse_study(args)
    elif args.kernel_only:
        kernel_only(args)
    elif args.ragged_only:
        ragged_only(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
