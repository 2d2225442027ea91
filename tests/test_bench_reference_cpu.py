"""The benchmark's reference arm (the oracle timed on the host cores) runs
without a GPU and prints the contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    import time

    t0 = time.perf_counter()
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--ref-budget", "6"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    wall = time.perf_counter() - t0
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "HVP/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]
    # the same workload description as the GPU arm, and measured (not
    # extrapolated) step times that fit inside the run
    import bench

    assert d["config"] == bench.headline_config(65536, 1)
    assert d["dtype"] == "f64"
    assert d["steps"] * d["ms_per_step"] * 1e-3 <= wall
    assert abs(d["cpu_baseline"]["value"] - d["value"]) < 1e-9 * d["value"]


def test_ingest_ncu_counts(tmp_path):
    """--ingest-ncu turns an ncu CSV (one row per metric) into per-point
    executed flops (2 x FMA + ADD + MUL, packed FP32 instructions twice) and
    DRAM bytes, matching launches to the profile run's keys by kernel name."""
    import json

    import bench

    keys = {"source_hash": bench.kernel_source_hash(), "launches": [
        {"key": "ackley_n64/fp64/hvp/symmetric/c4", "batch": 100, "fn": 1, "prec": 0, "c": 4, "kind": "hvp",
         "method": "symmetric", "config": {}},
        {"key": "rosenbrock_n16/fp32_comp/hessian/plain/c8", "batch": 50, "fn": 0, "prec": 1, "c": 8,
         "kind": "hessian", "method": "plain", "config": {}}]}
    kp = tmp_path / "keys.json"
    kp.write_text(json.dumps(keys))
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
           "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    rows = [hdr]
    launches = [("void sym_kernel<double, double, 4, 1, 1, 8, 0>(SweepArgs)",
                 {"smsp__sass_thread_inst_executed_op_dfma_pred_on.sum": "1,000", "dram__bytes_read.sum": "2000",
                  "dram__bytes_write.sum": "0", "smsp__sass_thread_inst_executed_op_dadd_pred_on.sum": "10",
                  "gpu__time_duration.sum": "5000"}),
                ("void sweep_kernel<float, float, 8, 0, 0, 4>(SweepArgs)",
                 {"smsp__sass_thread_inst_executed_op_ffma_pred_on.sum": "500",
                  "smsp__sass_thread_inst_executed_op_fmul_pred_on.sum": "5",
                  "smsp__sass_thread_inst_executed_op_ffma2_pred_on.sum": "200",
                  "smsp__sass_thread_inst_executed_op_fmul2_pred_on.sum": "3",
                  "smsp__sass_thread_inst_executed_op_fadd2_pred_on.sum": "1", "dram__bytes_read.sum": "100",
                  "dram__bytes_write.sum": "50"})]
    for i, (name, mets) in enumerate(launches):
        for m, v in mets.items():
            rows.append([str(i), "1", "python", "h", name, "1", "7", "(256, 1, 1)", "(10, 1, 1)", "0", "10.3",
                         "Command line profiler metrics", m, "", v])
    # an unrelated kernel between them is ignored
    rows.insert(2, ["9", "1", "python", "h", "void fma_peak_kernel<double, 8>(int, double)", "1", "7", "", "", "0",
                    "10.3", "x", "gpu__time_duration.sum", "ns", "1"])
    cp = tmp_path / "counts.csv"
    cp.write_text("==PROF== a header line\n" + "\n".join(",".join(f'"{c}"' for c in r) for r in rows) + "\n")
    out = tmp_path / "counts.json"
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--ingest-ncu", str(cp), "--profile-keys",
                        str(kp), "--counts-out", str(out)], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    doc = json.loads(out.read_text())
    assert doc["source_hash"] == bench.kernel_source_hash()
    a = doc["kernels"]["ackley_n64/fp64/hvp/symmetric/c4"]
    assert a["executed_flops_per_unit"] == (2 * 1000 + 10) / 100 and a["dram_bytes_per_unit"] == 20.0
    r = doc["kernels"]["rosenbrock_n16/fp32_comp/hessian/plain/c8"]
    # a packed FP32 instruction does two operations: FFMA2 = 4 flops, FMUL2 and FADD2 = 2
    assert r["executed_flops_per_unit"] == (2 * 500 + 5 + 4 * 200 + 2 * 3 + 2 * 1) / 50
    assert r["dram_bytes_per_unit"] == 3.0
    assert r["fp32_packed_share"] == 2 * (200 + 3 + 1) / (500 + 5 + 2 * (200 + 3 + 1))
    # a launch that does not match its key is refused
    keys["launches"][0]["c"] = 8
    kp.write_text(json.dumps(keys))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--ingest-ncu", str(cp), "--profile-keys",
                        str(kp), "--counts-out", str(out)], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert p.returncode != 0


def test_kernel_source_hash_ignores_comments_only(tmp_path):
    """The executed counts stay valid through comment and layout edits of the
    kernel sources, and no longer through a change of their code."""
    import shutil

    import bench

    csrc = os.path.join(ROOT, "paper_2410_22575_gb300", "csrc")
    for pat in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(csrc, pat), tmp_path / pat)
    h0 = bench.kernel_source_hash(str(tmp_path))
    assert h0 == bench.kernel_source_hash()
    f = tmp_path / "hdual.cuh"
    text = f.read_text()
    f.write_text("// another comment\n" + text.replace("namespace chessfad {", "namespace chessfad  {  /* x */", 1))
    assert bench.kernel_source_hash(str(tmp_path)) == h0
    f.write_text(text.replace("T v, d1;", "T d1, v;", 1))
    assert bench.kernel_source_hash(str(tmp_path)) != h0


def test_compact_summary_fits_the_end_of_the_output():
    # a line shaped like the GPU arm's, every workload row and the uneven
    # batch included, with long unrounded numbers; the summary is printed as
    # the line's last key and must fit in the last ~1.4 KB of output
    sys.path.insert(0, ROOT)
    import bench

    rnd = 0.123456789123
    roof = {"frac": 0.96912345678}
    err = {"max": 2.512345678e-16, "requests": 100000}
    line = {"value": 641234.56789, "e2e": {"value": 640987.654321}, "roofline": roof, "error_vs_oracle": err,
            "fp32_comp": {"value": 32612345.6789, "e2e": {"value": 31987654.321}, "roofline": roof,
                          "error_vs_oracle": err},
            "workloads": {}, "cpu_baseline": {"value": 7712.3456789, "cores": 16}}
    for name, kind, how, prec in bench.WORKLOAD_ROWS:
        key = f"{name}/{bench.PREC_NAME[prec]}/{kind}/{how}"
        rate = "hvp_per_s" if kind == "hvp" else "hessians_per_s"
        line["workloads"][key] = {rate: 283456789.123 * rnd, "roofline": roof, "error_vs_oracle": err}
    line["ragged_100k"] = {"ms_per_step": 7234.5678, "value": 13823.456, "untuned_ms_per_step": 7512.345,
                           "error_vs_oracle": err, "cpu_baseline": {"value": 2.3456789}}
    s = bench.compact_summary(line)
    text = json.dumps(s)
    assert len(text) <= 1400, len(text)
    assert s["fp64"] == [641200.0, 0.969, 641000.0, 2.5e-16]
    assert len([k for k in s if "/" in k]) == len(bench.WORKLOAD_ROWS)
    assert s["ragged_100k"]["s_per_step"] == 7.23 and s["ragged_100k"]["requests_checked"] == 100000
    assert s["cpu_oracle_hvp_per_s"] == [7710.0, 16]


def test_evaluation_counts_of_the_flop_model_match_the_oracles_algorithms(orc):
    # The bench's model multiplies a per-evaluation cost by the number of
    # evaluations of f per point: n * ceil(n/c) for the plain method (Alg. 5 /
    # Alg. 7) and sym_items(n, c) for the symmetric one (Alg. 6 / Alg. 8).
    # Both counts are read here off the oracle's operation counters (a call's
    # cost is fixed by c and n) and off a brute-force enumeration of the
    # (row, chunk) pairs, ragged last chunks included.
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    for n in (1, 5, 12, 33):
        x = np.random.Generator(np.random.PCG64(n)).uniform(-2, 2, n)
        for c in (1, 2, 4, 8, 16, 32):
            nch = -(-n // c)
            brute = sum(1 for i in range(n) for j in range(nch) if j >= i // c)
            assert bench.sym_items(n, c) == brute, (n, c)
            _, m_one, _ = orc.count_ops(orc.eval_hd, 0, c, orc.chunk_init(x, 0, 0, c))
            _, m_plain, _ = orc.count_ops(orc.chunk_hess, 0, x, c)
            _, m_sym, _ = orc.count_ops(orc.schunk_hess, 0, x, c)
            if m_one:
                assert m_plain == m_one * n * nch, (n, c)
                assert m_sym == m_one * bench.sym_items(n, c), (n, c)
            if n % c == 0:  # Sec. V: n (n/c + 1) / 2 evaluations
                assert bench.sym_items(n, c) == n * (n // c + 1) // 2
