#!/usr/bin/env python3
"""Benchmark: Hessian-vector products per second on one GB300 (and N GPUs).

Workload: Ackley, n = 64, 65536 points, x ~ U[-5,5], v ~ U[-1,1], seed 1
(PCG64), the configuration the headline metric is quoted on.  One step is one
``chessfad_hvp`` call over the whole batch: seeding, chunked-hDual propagation,
row-times-v products and the in-kernel row reduction, all in the library's
sweep kernel.  The headline ``value`` is compensated-FP32 HVP/s with inputs
resident in HBM; the FP64 rate, a chunk-size sweep and the end-to-end rate
through host buffers are reported beside it.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream, with a 256 MiB buffer written between steps to flush
the 129 MB L2 (outside the events).  Barrier + synchronize on both sides, max
over ranks.  Under torchrun every rank runs the same per-GPU batch (weak
scaling; points are independent, there is no collective on the data path).

``--impl reference`` times the FP64 CPU oracle (the paper's sequential
CHESS-VEC, Alg. 7, OpenMP over points) on the host cores instead.
"""
from __future__ import annotations

import argparse
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
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# FP64 DFMA lanes per SM: GB300's nominal 1.25 TFLOP/s FP64 at 2070 MHz over
# 152 SMs is 3.97 flop/clk/SM, i.e. 2 DFMA per clock per SM.
FP64_LANES_PER_SM = 2


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


def model_flops_ackley(n: int, c: int, symmetric: bool = False) -> float:
    return model_flops_hvp(1, n, c, symmetric)


# Sources that define the headline sweep kernel (the ncu traffic figure is
# reported only while these are unchanged since the capture).
KERNEL_SOURCES = ("hdual.cuh", "sym_layout.cuh", "sweep.cuh", "dispatch.h", "k_ackley_f32c.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2410_22575_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


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


def gpu_arm(args):
    import numpy as np
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

    res = {}
    for prec, dt in ((cf.FP32_COMP, torch.float32), (cf.FP64, torch.float64)):
        x = torch.tensor(b.x, dtype=dt, device=dev)
        v = torch.tensor(b.v, dtype=dt, device=dev)
        out = torch.empty_like(x)
        cfg = cf.chessfad_autotune_hvp(fn, n, batch, x, v, out, None, prec, stream)
        steps = args.steps if prec == cf.FP32_COMP else max(1, min(args.steps, args.fp64_steps))

        def step():
            st = cf.chessfad_hvp(fn, n, batch, 0, x, v, out, None, prec, stream)
            if st != 0:
                raise cf.ChessfadError(st, "chessfad_hvp")

        barrier(world)
        torch.cuda.synchronize()
        if prec == cf.FP32_COMP:
            with ClockSampler(local) as clk:
                ms = timed_steps(step, steps, args.warmup, stream, flush)
            clocks = clk.summary()
        else:
            ms = timed_steps(step, steps, args.warmup, stream, flush)
        torch.cuda.synchronize()
        barrier(world)
        tot = max_over_ranks(world, sum(ms), dev)
        res[prec] = {"cfg": cfg.as_dict(), "ms": ms, "total_ms": tot, "steps": steps,
                     "out_sample": out[:256].double().cpu().numpy(), "x32": x[:256].double().cpu().numpy(),
                     "v32": v[:256].double().cpu().numpy()}
        if prec == cf.FP32_COMP:
            res[prec]["clocks"] = clocks

        # chunk-size sweep (shorter), same precision
        sweep = {}
        for c in (4, 8, 16, 32):
            info = cf.chessfad_kernel_info(fn, prec, c, True)
            if info["local_bytes"] > 48:
                sweep[str(c)] = {"skipped": "spills registers", **info}
                continue
            ent = dict(info)
            for mname, ccfg in (("plain", cf.Config(c, 1, 256)), ("symmetric", cf.Config(c, 0, 0, cf.SYMMETRIC, 64))):
                def stc(ccfg=ccfg):
                    st = cf.chessfad_hvp_config(fn, n, batch, ccfg, x, v, out, None, prec, stream)
                    if st != 0:
                        raise cf.ChessfadError(st, "chessfad_hvp")

                k = max(1, min(5, steps))
                m = timed_steps(stc, k, 1, stream, flush)
                t = max_over_ranks(world, sum(m), dev) / k
                ent[mname] = {"hvp_per_s": world * batch / (t * 1e-3), "ms": t}
            sweep[str(c)] = ent
        res[prec]["sweep"] = sweep

        # seed-sparse symmetric method (a different arithmetic: reported beside
        # the headline, never as it)
        sparse = {}
        for c in (4, 8):
            scfg = cf.Config(c, 0, 128, cf.SYMMETRIC_SPARSE, 64)

            def sts(scfg=scfg):
                st = cf.chessfad_hvp_config(fn, n, batch, scfg, x, v, out, None, prec, stream)
                if st != 0:
                    raise cf.ChessfadError(st, "chessfad_hvp")

            k = max(1, min(5, steps))
            m = timed_steps(sts, k, 1, stream, flush)
            t = max_over_ranks(world, sum(m), dev) / k
            sparse[str(c)] = {**scfg.as_dict(), "hvp_per_s": world * batch / (t * 1e-3), "ms": t}
        res[prec]["sparse"] = sparse
        del x, v, out

    # ---- end to end: pinned host buffers -> device -> hvp -> host, FP32-comp
    xh = torch.tensor(b.x, dtype=torch.float32).pin_memory()
    vh = torch.tensor(b.v, dtype=torch.float32).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(xh, device=dev)
    vd = torch.empty_like(vh, device=dev)
    od = torch.empty_like(xh, device=dev)

    def e2e_step():
        # one C-ABI call: pinned host x, v -> device -> sweeps -> host out,
        # copies of consecutive slices overlapping the sweeps
        st = cf.chessfad_hvp_host(fn, n, batch, 0, xh, vh, oh, xd, vd, od, None, cf.FP32_COMP, args.e2e_slices,
                                  stream)
        if st != 0:
            raise cf.ChessfadError(st, "chessfad_hvp_host")

    barrier(world)
    ms_e2e = timed_steps(e2e_step, args.steps, args.warmup, stream, flush)
    torch.cuda.synchronize()
    barrier(world)
    tot_e2e = max_over_ranks(world, sum(ms_e2e), dev)

    ragged = None if args.no_ragged else ragged_arm(args, world, dev, stream, flush)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    f32 = res[cf.FP32_COMP]
    f64 = res[cf.FP64]
    value = world * batch * f32["steps"] / (f32["total_ms"] * 1e-3)
    v64 = world * batch * f64["steps"] / (f64["total_ms"] * 1e-3)
    c = f32["cfg"]["csize"]
    sym32 = f32["cfg"]["method"] == "symmetric"
    flops_launch = model_flops_ackley(n, c, sym32) * batch
    avg_ms = sum(f32["ms"]) / len(f32["ms"])
    peak_fp32 = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
    peak_fp64 = SM_COUNT * FP64_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
    achieved = flops_launch / (avg_ms * 1e-3)
    try:
        micro32 = cf.chessfad_peak_flops(cf.FP32_COMP)
        micro64 = cf.chessfad_peak_flops(cf.FP64)
    except Exception as e:  # report, do not hide
        micro32 = micro64 = None
        print(f"peak microbenchmark failed: {e}", file=sys.stderr)
    traffic = None
    executed = None  # ncu's executed FP32 flops of the same kernel (FMA = 2), same gating as traffic
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        tj = json.load(open(tfile))
        ent = tj.get(f"{WORKLOAD}/fp32_comp/{f32['cfg']['method']}/c{c}")
        if ent and ent.get("source_hash") == kernel_source_hash():
            traffic = ent.get("dram_bytes_per_launch")
            executed = ent.get("executed_flops_per_launch")
    c64 = f64["cfg"]["csize"]
    sym64 = f64["cfg"]["method"] == "symmetric"
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "HVP/s",
        "n_gpus": world,
        "steps": f32["steps"],
        "warmup": args.warmup,
        "ms_per_step": f32["total_ms"] / f32["steps"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded PCG64 draws of the workload's distributions)",
        "config": {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}", "function": "ackley", "n": n, "batch": batch,
                   "precision": "fp32_comp (FP32 hDual arithmetic with compensated sums and dots, FP64 islands)",
                   **f32["cfg"], "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (points independent, no collective)"},
        "fp64": {"value": v64, "unit": "HVP/s", "steps": f64["steps"], "ms_per_step": f64["total_ms"] / f64["steps"],
                 **{k: v for k, v in f64["cfg"].items()},
                 "model_tflops": model_flops_ackley(n, c64, sym64) * batch / (f64["total_ms"] / f64["steps"] * 1e-3) / 1e12,
                 "peak_tflops_derived": peak_fp64 / 1e12},
        "fp32_over_fp64": value / v64,
        "chunk_sweep": {"fp32_comp": f32["sweep"], "fp64": f64["sweep"]},
        "seed_sparse": {"fp32_comp": f32["sparse"], "fp64": f64["sparse"],
                        "method": "symmetric, seed-sparse propagation (skips variables whose seed has no "
                                  "derivative part); equal to the dense result for finite inputs"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_fp32 / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak_fp32, "traffic": traffic,
                     "flops_per_launch": flops_launch,
                     "executed_flops_per_launch": executed,
                     "frac_executed": None if executed is None else executed / (avg_ms * 1e-3) / peak_fp32,
                     "model_over_executed": None if executed is None else flops_launch / executed,
                     "kernel": ("sym_kernel<float,%d,ACKLEY,HVP>" if sym32 else "sweep_kernel<float,%d,ACKLEY,HVP>") % c,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                     "peak_microbench": None if micro32 is None else micro32 / 1e12,
                     "frac_of_microbench": None if micro32 is None else achieved / micro32,
                     "fp64_peak_microbench": None if micro64 is None else micro64 / 1e12},
        "e2e": {"value": world * batch * args.steps / (tot_e2e * 1e-3), "unit": "HVP/s",
                "h2d_bytes_per_step": 2 * batch * n * 4, "d2h_bytes_per_step": batch * n * 4,
                "api": "chessfad_hvp_host (pinned host buffers)", "slices": args.e2e_slices},
        "gpu_launches": f32["steps"],
        "clocks": f32.get("clocks"),
    }
    if ragged is not None:
        line["ragged_100k"] = {k: v for k, v in ragged.items() if not k.startswith("_")}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(b, c, f32, f64, args)
        if ragged is not None:
            line["ragged_100k"]["error_vs_oracle_sample"] = ragged_error(ragged)
    print(json.dumps(line))


# ------------------------------------------------------------------ uneven batch
RAGGED_SYM_MIN_N = 128  # Fletcher-Powell requests this large run the symmetric method


def model_flops_request(fn: int, n: int, c: int) -> float:
    """Model flops of one HVP of the uneven batch: the symmetric method for
    Fletcher-Powell requests with n >= 128, the plain method otherwise."""
    return model_flops_hvp(fn, n, c, fn == 2 and n >= RAGGED_SYM_MIN_N)


def ragged_arm(args, world, dev, stream, flush):
    """The 100000-request uneven batch (three functions, n log-uniform in
    [2, 512], seed 4) in compensated FP32: one persistent launch per step,
    replayed from a captured CUDA graph."""
    import numpy as np
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    rg = W.make_ragged()
    c = 16  # the plan's default chunk size for compensated FP32
    reqs = cf.requests(rg.fns, rg.ns, rg.offs, rg.eoffs)
    t0 = time.perf_counter()
    plan = cf.RaggedPlan(reqs, cf.FP32_COMP, c)
    t_plan = time.perf_counter() - t0
    x = torch.tensor(rg.xpack, dtype=torch.float32, device=dev)
    v = torch.tensor(rg.vpack, dtype=torch.float32, device=dev)
    out = torch.empty_like(x)
    A = torch.tensor(rg.fp.A, device=dev)
    B = torch.tensor(rg.fp.B, device=dev)
    E = torch.tensor(rg.Epack, device=dev)
    params = cf.fp_params(A, B, E)
    plan.run(x, v, out, params)  # per-device set-up, outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run(x, v, out, params)
    barrier(world)
    ms = timed_steps(g.replay, args.ragged_steps, 0, stream, flush)
    torch.cuda.synchronize()
    barrier(world)
    tot = max_over_ranks(world, sum(ms), dev)
    flops = sum(model_flops_request(int(f), int(n), c) for f, n in zip(rg.fns, rg.ns))
    per = tot / len(ms)
    return {"value": world * rg.nreq * len(ms) / (tot * 1e-3), "unit": "HVP/s", "requests": rg.nreq,
            "steps": len(ms), "warmup": 1, "ms_per_step": per, "precision": "fp32_comp", "csize": c,
            "launch": "one persistent kernel per step, CUDA graph replay", "tiles": plan.info["ntiles"],
            "method": "plain; symmetric (SC-HESS-VEC) for Fletcher-Powell n >= 128",
            "workspace_bytes": plan.info["workspace_bytes"], "plan_seconds": t_plan,
            "model_tflops": flops / (per * 1e-3) / 1e12,
            "_out": out, "_x": x, "_v": v, "_rg": rg}


def ragged_error(r):
    """Oracle check of 200 requests of the uneven batch (cpu_baseline leg)."""
    import numpy as np

    import oracle
    from paper_2410_22575_gb300 import metrics

    rg = r["_rg"]
    idx = np.sort(np.random.Generator(np.random.PCG64(0)).choice(rg.nreq, 200, replace=False))
    sub = rg.subset(idx)
    xh = r["_x"].double().cpu().numpy()
    vh = r["_v"].double().cpu().numpy()
    oh = r["_out"].double().cpu().numpy()
    take = lambda a: np.concatenate([a[rg.offs[q]:rg.offs[q] + rg.ns[q]] for q in idx])
    xs, vs, got = take(xh), take(vh), take(oh)
    ref, hn = oracle.hvp_ragged(sub.fns, sub.ns, sub.offs, sub.eoffs, xs, vs, rg.fp.A, rg.fp.B, rg.Epack, rg.ld)
    e = metrics.ragged_hvp_errors(got, ref, hn, vs, sub.ns, sub.offs)
    return {**metrics.summary(e), "requests": len(idx)}


# ------------------------------------------------------------------ CPU oracle
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


def cpu_baseline(b, c, f32, f64, args):
    import numpy as np

    import oracle
    from paper_2410_22575_gb300 import metrics

    rate, m, dt, _ = cpu_sample_time(b, c, args.cpu_seconds)
    # closed-form oracle (O1) on the same prefix, and the GPU's error against it
    t0 = time.perf_counter()
    oracle.hvp(b.fn, b.x[:m], b.v[:m])
    t_cf = time.perf_counter() - t0
    acc = {}
    for name, r in (("fp32_comp", f32), ("fp64", f64)):
        ref, hn = oracle.hvp(b.fn, r["x32"], r["v32"], with_norm=True)
        e = metrics.hvp_errors(r["out_sample"], ref, hn, r["v32"])
        acc[name] = metrics.summary(e)
    return {"value": rate, "unit": "HVP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {m} of {b.batch} points, CHESS-VEC (Alg. 7) FP64 with c={c}, {dt:.1f} s",
            "closed_form_hvp_per_s": m / t_cf,
            "gpu_error_vs_oracle_first256": acc}


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2410_22575_gb300 import workloads as W

    b = W.workload(WORKLOAD)
    c = 16
    per = max(0.5, min(20.0, args.ref_budget / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_sample_time(b, c, per / 4)
    rates, secs, ms = [], 0.0, []
    sample = 0
    for _ in range(args.steps):
        r, m, dt, _ = cpu_sample_time(b, c, per)
        rates.append(r)
        secs += dt
        sample = m
        ms.append(dt * 1e3 * b.batch / m)
    value = statistics.median(rates)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "HVP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64 draws of the workload's distributions)",
        "config": {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}", "function": "ackley", "n": 64, "batch": b.batch,
                   "precision": "fp64", "csize": c},
        "cpu_baseline": {"value": value, "unit": "HVP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: first {sample} of {b.batch} points, CHESS-VEC (Alg. 7) FP64, c={c}"},
        "e2e": {"value": value, "unit": "HVP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


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


def report(args):
    """Per-workload table: HVP/s (and Hessians/s) for every
    named workload in both precisions, autotuned over both methods, plus the
    plain method at the workload's stated chunk size."""
    import torch

    import paper_2410_22575_gb300 as cf
    from paper_2410_22575_gb300 import workloads as W

    rows = []

    def timed(fn_call, reps):
        # device time per call: reps calls captured in one CUDA graph and
        # replayed between two events, so host-side call overhead (tens of
        # microseconds through the binding) never leaves the GPU idle inside
        # the timed region -- it would dominate the small workloads
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
            peak = SM_COUNT * (FP64_LANES_PER_SM if prec == cf.FP64 else FP32_LANES_PER_SM) * 2 * SM_MAX_MHZ * 1e6
            row["model_tflops"] = mf * b.batch / (t * 1e-3) / 1e12
            row["frac_of_derived_peak"] = mf * b.batch / (t * 1e-3) / peak
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
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--impl", choices=["chessfad", "reference"], default="chessfad")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ragged", action="store_true", help="skip the 100000-request uneven batch")
    ap.add_argument("--ragged-steps", type=int, default=1)
    ap.add_argument("--kernel-only", action="store_true", help="run only the sweep kernel (for ncu)")
    ap.add_argument("--ragged-only", action="store_true",
                    help="run only the uneven-batch kernel on a subset of the 100000-request workload (for ncu)")
    ap.add_argument("--ragged-fn", type=int, default=2)
    ap.add_argument("--ragged-min-n", type=int, default=256)
    ap.add_argument("--ragged-max-n", type=int, default=512)
    ap.add_argument("--ragged-count", type=int, default=32)
    ap.add_argument("--report", action="store_true", help="per-workload table (all named workloads)")
    ap.add_argument("--chunk-study", action="store_true", help="measured best chunk size vs the Sec. V model")
    ap.add_argument("--cpu-report", action="store_true", help="CPU-baseline leg for every named workload")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fn", type=int, default=None, help="kernel-only: function id instead of a named workload")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--prec", choices=["fp32_comp", "fp64"], default="fp32_comp")
    ap.add_argument("--csize", type=int, default=32)
    ap.add_argument("--tpr", type=int, default=1)
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="reference arm: seconds of oracle work over all steps (bounded per step)")
    ap.add_argument("--e2e-slices", type=int, default=16,
                    help="slices of the end-to-end call (copies of one overlap the sweep of the next)")
    ap.add_argument("--method", choices=["plain", "symmetric", "symmetric_sparse"], default="plain")
    ap.add_argument("--tpp", type=int, default=64, help="kernel-only, symmetric: threads per point")
    args = ap.parse_args()
    if args.warmup < 3 and not args.kernel_only:
        args.warmup = 3
    if args.cpu_report:
        cpu_baseline_report(args)
    elif args.chunk_study:
        chunk_study(args)
    elif args.report:
        report(args)
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
