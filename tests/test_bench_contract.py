"""The benchmark's JSON contract, on the CPU: the reference arm (the
oracle timed on the host cores) prints one line with the keys the
contract names, and the byte and operation models behind the GPU arm's
rooflines are the documented formulas."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--cpu-seconds", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert "workload" in d["config"] and "model" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host_cpus"] == os.cpu_count()
    # ms_per_step is the time of what each step ran (a bounded sample of the
    # solve); the extrapolation to a whole solve is its own field
    assert d["ms_per_step"] < d["ms_per_solve_extrapolated"] or d["iters_per_step"] >= d["iters_per_solve"]
    assert abs(d["ms_per_solve_extrapolated"] - 1e3 / d["value"]) <= 1e-6 * d["ms_per_solve_extrapolated"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_roofline_models():
    sys.path.insert(0, ROOT)
    import bench
    n, nnz = 2_097_152, 14_581_760                   # the 128^3 7-point Laplacian
    assert bench.bytes_per_iter_fp64(n, nnz) == 12 * nnz + 108 * n
    assert bench.bytes_per_iter_fp64(n, nnz, 2) == 10 * nnz + 108 * n
    assert bench.stencil_index_bytes(128) == 2 and bench.stencil_index_bytes(464) == 4
    assert bench.ops_per_iter_fp64(n, nnz) == nnz + 6 * n
    assert bench.FP64_NOMINAL_GOPS == 625.0          # 1.25 TFLOP/s in fused multiply-adds
    # standalone MatMult models: values + indices per nonzero, row pointers,
    # the x gather and the y write once per row
    assert bench.bytes_spmv_fp64(n, nnz, 2) == 10 * nnz + 4 * (n + 1) + 16 * n
    assert bench.bytes_spmv_fp32(n, nnz, 2) == 6 * nnz + 4 * (n + 1) + 8 * n
    cfg = bench.config_for(1)
    assert "128^3" in cfg["workload"] and cfg["parallelism"] == "single GPU"
