#!/usr/bin/env python
"""Benchmark of the GB300 Jacobi-PCG solve (one JSON line on stdout).

Headline workload: one Jacobi-preconditioned CG solve per step of the 3D
7-point Dirichlet Laplacian on a 128^3 grid (n = 2,097,152, nnz =
14,581,760), FP64 CSR, x0 = 0, b = A x* with x* uniform[-1,1) (seed 2),
rtol 1e-10 -- solves/s.  Inputs (matrix 175 MB + vectors) exceed the
129 MB L2, so no flush is needed between steps.

Also reported: the roofline of the persistent solve kernel (algorithmic
bytes 12 nnz + 108 n per iteration over its CUDA-event time, against the
measured HBM copy bandwidth), an end-to-end number through the C ABI with
host buffers, the CPU oracle's rate on a bounded sample, SpMV bandwidth,
the 64x64 2D case, mixed precision vs FP64 on the 96^3 27-point case, and
the batched and serving workloads when they are built.

Multi-GPU: every rank solves its own copy of the workload (independent
replicas, no collective on the data path); value = all ranks' solves /
the slowest rank's time ("scaling": "weak").

--impl reference times the CPU oracle (the reference for this path) on the
same workload, each step a bounded sample of iterations.
"""
from __future__ import annotations

import argparse
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

N_GRID = 128
RTOL = 1e-10
MAXIT = 20000


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gbs", "reference"], default="gbs")
    p.add_argument("--no-extras", action="store_true", help="headline line only")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="budget of the bounded oracle sample")
    p.add_argument("--quick", action="store_true",
                   help="device-resident headline solve only (no e2e, extras or CPU baseline)")
    p.add_argument("--maxit", type=int, default=20000,
                   help="iteration cap of the headline solve (profiling runs use a small cap)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def c2_problem():
    from paper_2011_00715_gb300 import inputs as I
    A = I.lap3d7(N_GRID)
    xs = I.xstar(A.n, 2)
    return A, xs


WORKLOAD = (f"3D 7-point Dirichlet Laplacian {N_GRID}^3 (n=2,097,152, nnz=14,581,760), FP64 CSR, "
            "one Jacobi-PCG solve per step, rtol 1e-10 (unpreconditioned ||r||<=rtol||b||), x0=0, "
            "b=A x*, x* uniform[-1,1) seed 2")


def bytes_per_iter_fp64(n, nnz):
    """Fused FP64 PCG iteration: 12 nnz (vals + colidx) + 108 n (rowptr 4n,
    p gather 8n, q write 8n, update phase 64n, p update 24n)."""
    return 12 * nnz + 108 * n


def bytes_per_iter_mixed(n, nnz):
    """FP32 inner iteration: 8 nnz + 56 n."""
    return 8 * nnz + 56 * n


def bytes_spmv_fp64(n, nnz):
    return 12 * nnz + 4 * (n + 1) + 8 * n + 8 * n


# ---------------------------------------------------------------- CPU oracle --

def oracle_rate(A, b, full_iters, budget_s):
    """Time the oracle's FP64 PCG on a bounded number of iterations and
    extrapolate to a full solve of `full_iters` iterations (solves/s)."""
    import oracle
    oracle.build()
    t = time.perf_counter()
    oracle.pcg(A, b, 0.0, 2)
    t2 = time.perf_counter() - t
    per_it = max(t2 / 3.0, 1e-6)          # set-up costs about one iteration
    m = int(max(3, min(full_iters, budget_s / per_it - 1)))
    t = time.perf_counter()
    r = oracle.pcg(A, b, 0.0, m)
    el = time.perf_counter() - t
    per_it = el / (m + 1)
    return {"value": 1.0 / (per_it * (full_iters + 1)), "unit": "solves/s", "cores": 1,
            "kind": "oracle",
            "sample": (f"oracle FP64 Jacobi-PCG (plain C, 1 thread) on the same {N_GRID}^3 system: "
                       f"{m} iterations timed ({el:.1f} s), {per_it*1e3:.1f} ms/iteration, "
                       f"extrapolated to the {full_iters}-iteration solve"),
            "iters_sampled": int(r["iters"]), "seconds": el}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    A, xs = c2_problem()
    b = oracle.spmv(A, xs)
    # one full, untimed oracle solve gives the iteration count that each
    # timed step's bounded sample is extrapolated to
    full = oracle.pcg(A, b, RTOL, MAXIT)
    full_iters = int(full["iters"])
    per_step_budget = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(A, b, full_iters, per_step_budget / 2)
    vals = []
    t0 = time.perf_counter()
    samples = []
    for _ in range(args.steps):
        r = oracle_rate(A, b, full_iters, per_step_budget)
        vals.append(1.0 / r["value"])
        samples.append(r)
    el = time.perf_counter() - t0
    sec_per_solve = statistics.mean(vals)
    value = 1.0 / sec_per_solve
    line = {"impl": "reference", "metric": "Jacobi-PCG solves/s (128^3 7-point, FP64, rtol 1e-10)",
            "value": value, "unit": "solves/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec_per_solve * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": samples[-1]["sample"] + f"; {args.steps} steps in {el:.1f} s"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm --

class Gpu:
    def __init__(self, device):
        import torch
        from paper_2011_00715_gb300 import gbs
        self.torch = torch
        self.gbs = gbs
        torch.cuda.set_device(device)
        self.stream = torch.cuda.current_stream()
        self.ctx = gbs.gbs_ctx_create(device, self.stream.cuda_stream)

    def mat(self, A):
        return self.gbs.gbs_mat_create_aij(self.ctx, A.n, A.n, A.rowptr, A.colidx, A.vals)

    def dvec(self, arr):
        t = self.torch.from_numpy(arr).cuda()
        return self.gbs.gbs_vec_wrap(self.ctx, t), t

    def launches(self):
        return self.gbs.gbs_ctx_launch_count(self.ctx)


def event_time(torch, fn, reps):
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_gbs(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2011_00715_gb300 import gbs
    from paper_2011_00715_gb300 import build as B
    B.build()
    g = Gpu(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    A, xs = c2_problem()
    Ah = g.mat(A)
    xsv, xst = g.dvec(xs)
    bt = torch.empty(A.n, dtype=torch.float64, device="cuda")
    bv = gbs.gbs_vec_wrap(g.ctx, bt)
    gbs.gbs_mat_mult(Ah, xsv, bv)              # b = A x* on the device
    xt = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    xv = gbs.gbs_vec_wrap(g.ctx, xt)
    opts = gbs.gbs_opts_default(mode=gbs.GBS_MODE_FP64, algorithm=gbs.GBS_ALG_PERSISTENT)
    infos = []

    def step():
        gbs.gbs_vec_set(xv, 0.0)
        infos.append(gbs.gbs_ksp_solve_cg_ex(Ah, bv, xv, RTOL, args.maxit, opts))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    infos.clear()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    barrier()
    torch.cuda.synchronize()
    l0 = g.launches()
    el = event_time(torch, step, args.steps)
    l1 = g.launches()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if rank == 0 else None
    el_max = el
    if dist is not None:
        t = torch.tensor([el], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el_max = float(t.item())
    statuses = {i.status for i in infos}
    iters = [i.iters for i in infos]
    dev_ms = statistics.mean(i.device_ms for i in infos)
    value = world * args.steps / el_max
    n, nnz = A.n, A.nnz
    hbm, peak_kind = peaks()
    bpl = iters[0] * bytes_per_iter_fp64(n, nnz)
    achieved = bpl / (dev_ms / 1e3) / 1e9
    # true residual of the last solve, on the device with the library's SpMV
    rt = torch.empty_like(bt)
    rv = gbs.gbs_vec_wrap(g.ctx, rt)
    gbs.gbs_mat_mult(Ah, xv, rv)
    torch.cuda.synchronize()
    true_rel = float(torch.linalg.norm(bt - rt) / torch.linalg.norm(bt))
    err_xs = float(torch.linalg.norm(xt - xst) / torch.linalg.norm(xst))

    line = {"metric": "Jacobi-PCG solves/s (128^3 7-point Laplacian, FP64 CSR, rtol 1e-10)",
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded stencil matrix and manufactured solution)",
            "config": {"workload": WORKLOAD,
                       "l2": "inputs larger than L2 (matrix 175 MB + 5 vectors of 16.8 MB)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "algorithm": "persistent cooperative kernel, 3 grid barriers/iteration"},
            "solve": {"status": sorted(statuses), "iters": iters[0],
                      "true_rel_residual": true_rel, "rel_err_vs_xstar": err_xs,
                      "kernel_ms": dev_ms, "us_per_iter": dev_ms * 1e3 / iters[0]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "kernel": "k_pcg_fp64 (one launch per solve)",
                         "bytes_model": "iters x (12 nnz + 108 n)", "peak_kind": peak_kind},
            "gpu_launches": int(l1 - l0),
            "clocks": clk}
    gbs.gbs_vec_destroy(rv)

    if rank == 0 and world == 1 and not args.quick:
        line["e2e"] = e2e_c2(g, A, xs, args, infos[0].iters)
        if not args.no_extras:
            line["extras"] = extras(g, args, A, Ah, xsv)
        import oracle
        b_host = oracle.spmv(A, xs)
        line["cpu_baseline"] = oracle_rate(A, b_host, iters[0], args.cpu_seconds)
    for v in (xsv, bv, xv):
        gbs.gbs_vec_destroy(v)
    gbs.gbs_mat_destroy(Ah)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def e2e_c2(g, A, xs, args, iters_full):
    """Through the C ABI with host buffers: per step the CSR arrays and b go
    host->device from pinned memory, the solve runs, x comes back."""
    import numpy as np
    import torch
    gbs = g.gbs
    rp = torch.from_numpy(A.rowptr).pin_memory()
    ci = torch.from_numpy(A.colidx).pin_memory()
    va = torch.from_numpy(A.vals).pin_memory()
    import oracle
    bh = torch.from_numpy(oracle.spmv(A, xs)).pin_memory()
    xh = torch.empty(A.n, dtype=torch.float64).pin_memory()
    bt = torch.empty(A.n, dtype=torch.float64, device="cuda")
    xt = torch.empty(A.n, dtype=torch.float64, device="cuda")
    bv = gbs.gbs_vec_wrap(g.ctx, bt)
    xv = gbs.gbs_vec_wrap(g.ctx, xt)
    opts = gbs.gbs_opts_default(mode=gbs.GBS_MODE_FP64)

    def step():
        h = gbs.gbs_mat_create_aij(g.ctx, A.n, A.n, rp, ci, va)
        gbs.gbs_vec_set_values(bv, bh)
        gbs.gbs_vec_set(xv, 0.0)
        info = gbs.gbs_ksp_solve_cg_ex(h, bv, xv, RTOL, MAXIT, opts)
        gbs.gbs_vec_get_values(xv, xh)
        gbs.gbs_mat_destroy(h)
        return info

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        info = step()
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    h2d = A.rowptr.nbytes + A.colidx.nbytes + A.vals.nbytes + A.n * 8
    d2h = A.n * 8
    for v in (bv, xv):
        gbs.gbs_vec_destroy(v)
    return {"value": steps / el, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "status": info.status,
            "path": "gbs_mat_create_aij(host CSR, pinned) + gbs_vec_set_values(b) + "
                    "gbs_ksp_solve_cg_ex + gbs_vec_get_values(x) + gbs_mat_destroy"}


def extras(g, args, A, Ah, xsv):
    import numpy as np
    import torch
    from paper_2011_00715_gb300 import inputs as I
    gbs = g.gbs
    out = {}
    hbm, _ = peaks()
    # --- standalone MatMult on the 128^3 matrix
    yt = torch.empty(A.n, dtype=torch.float64, device="cuda")
    yv = gbs.gbs_vec_wrap(g.ctx, yt)
    for _ in range(3):
        gbs.gbs_mat_mult(Ah, xsv, yv)
    reps = 50
    el = event_time(torch, lambda: gbs.gbs_mat_mult(Ah, xsv, yv), reps)
    bb = bytes_spmv_fp64(A.n, A.nnz)
    out["spmv_c2_fp64"] = {"us": el / reps * 1e6, "GBps": bb / (el / reps) / 1e9,
                           "frac": bb / (el / reps) / 1e9 / hbm,
                           "bytes_model": "12 nnz + 4(n+1) + 8n + 8n"}
    gbs.gbs_vec_destroy(yv)
    # --- C1: 64x64 2D Laplacian, rtol 1e-8
    C1 = I.lap2d5(64)
    h = g.mat(C1)
    xs = I.xstar(C1.n, 1)
    xsv1, _x1 = g.dvec(xs)
    b1 = torch.empty(C1.n, dtype=torch.float64, device="cuda")
    b1v = gbs.gbs_vec_wrap(g.ctx, b1)
    gbs.gbs_mat_mult(h, xsv1, b1v)
    x1 = torch.zeros(C1.n, dtype=torch.float64, device="cuda")
    x1v = gbs.gbs_vec_wrap(g.ctx, x1)
    res = {}
    for name, alg in (("persistent", gbs.GBS_ALG_PERSISTENT), ("perop", gbs.GBS_ALG_PEROP),
                      ("graph", gbs.GBS_ALG_GRAPH)):
        o = gbs.gbs_opts_default(algorithm=alg)
        info = None

        def st():
            nonlocal info
            gbs.gbs_vec_set(x1v, 0.0)
            info = gbs.gbs_ksp_solve_cg_ex(h, b1v, x1v, 1e-8, 10000, o)
        for _ in range(3):
            st()
        n_rep = 20
        el = event_time(torch, st, n_rep)
        res[name] = {"solves_per_s": n_rep / el, "iters": info.iters,
                     "us_per_iter": el / n_rep / info.iters * 1e6, "status": info.status}
    out["c1_lap2d5_64_fp64"] = res
    for v in (xsv1, b1v, x1v):
        gbs.gbs_vec_destroy(v)
    gbs.gbs_mat_destroy(h)
    # --- C3: 96^3 27-point variable coefficient, mixed vs FP64 at rtol 1e-10
    C3 = I.var27(96, seed=3, sigma=1.0)
    h = g.mat(C3)
    xs3 = I.xstar(C3.n, 3)
    xs3v, xs3t = g.dvec(xs3)
    b3 = torch.empty(C3.n, dtype=torch.float64, device="cuda")
    b3v = gbs.gbs_vec_wrap(g.ctx, b3)
    gbs.gbs_mat_mult(h, xs3v, b3v)
    x3 = torch.zeros(C3.n, dtype=torch.float64, device="cuda")
    x3v = gbs.gbs_vec_wrap(g.ctx, x3)
    r3 = torch.empty_like(b3)
    r3v = gbs.gbs_vec_wrap(g.ctx, r3)
    c3 = {}
    sols = {}
    for name, mode in (("fp64", gbs.GBS_MODE_FP64), ("mixed", gbs.GBS_MODE_MIXED)):
        o = gbs.gbs_opts_default(mode=mode)
        info = None

        def st():
            nonlocal info
            gbs.gbs_vec_set(x3v, 0.0)
            info = gbs.gbs_ksp_solve_cg_ex(h, b3v, x3v, 1e-10, MAXIT, o)
        st()
        n_rep = 3
        el = event_time(torch, st, n_rep)
        gbs.gbs_mat_mult(h, x3v, r3v)
        torch.cuda.synchronize()
        sols[name] = x3.clone()
        bpi = (bytes_per_iter_fp64 if name == "fp64" else bytes_per_iter_mixed)(C3.n, C3.nnz)
        c3[name] = {"ms_to_solution": el / n_rep * 1e3, "status": info.status,
                    "iters": info.iters, "outer_iters": info.outer_iters,
                    "true_rel_residual": float(torch.linalg.norm(b3 - r3) / torch.linalg.norm(b3)),
                    "rel_err_vs_xstar": float(torch.linalg.norm(x3 - xs3t) / torch.linalg.norm(xs3t)),
                    "kernel_GBps": info.iters * bpi / (info.device_ms / 1e3) / 1e9}
    c3["mixed_vs_fp64_rel_diff"] = float(torch.linalg.norm(sols["mixed"] - sols["fp64"]) /
                                         torch.linalg.norm(sols["fp64"]))
    c3["speedup_mixed_over_fp64"] = c3["fp64"]["ms_to_solution"] / c3["mixed"]["ms_to_solution"]
    out["c3_var27_96_rtol1e-10"] = c3
    for v in (xs3v, b3v, x3v, r3v):
        gbs.gbs_vec_destroy(v)
    gbs.gbs_mat_destroy(h)
    return out


def main():
    args = parse_args()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_gbs(args, rank, world, local)


if __name__ == "__main__":
    main()
