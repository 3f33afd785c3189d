"""Stored expected values (tests/golden/): the paper's vector-operation cost
model (Sec. 5.1), which the benchmark's byte model must use, and the
oracle's C1 solve, pinned by the CG iteration bound of the closed-form
condition number and kept as a regression fixture for the oracle."""
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_2011_00715_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = v
    return out


def num(v):
    return float.fromhex(v) if "0x" in v else float(v)


def test_benchmark_uses_the_papers_vector_op_model():
    g = read("sec5_1_vector_ops.txt")
    import bench
    assert bench.SWEEP_ACCESSES["VecAXPY"] == int(g["VecAXPY.accesses_per_entry"])
    assert bench.SWEEP_ACCESSES["VecCopy"] == int(g["VecCopy.accesses_per_entry"])
    # the fused iteration's update phase is three AXPY-like passes of 3 accesses
    # plus the Jacobi scaling: x, p, r, q, dinv read and x, r, z written
    n, nnz = 1000, 7000
    assert bench.bytes_per_iter_fp64(n, nnz) == 12 * nnz + 108 * n


def test_c1_golden_respects_the_cg_bound():
    """k <= ceil(ln(2 sqrt(kappa) / rtol) / ln((sqrt(kappa)+1)/(sqrt(kappa)-1)))
    with kappa from the closed-form Laplacian eigenvalues (x0 = 0)."""
    g = read("c1_lap2d5_64_pcg.txt")
    N = 64
    lam = [4 - 2 * math.cos(j * math.pi / (N + 1)) - 2 * math.cos(k * math.pi / (N + 1))
           for j in (1, N) for k in (1, N)]
    kappa = max(lam) / min(lam)
    s = math.sqrt(kappa)
    bound = math.ceil(math.log(2 * s / 1e-8) / math.log((s + 1) / (s - 1)))
    assert bound == 473
    assert int(g["status"]) == 0 and int(g["iters"]) <= bound
    assert num(g["rnorm"]) <= 1e-8 * num(g["bnorm"])
    # the stopping test held first at the last recorded norm
    hist = [num(g[f"rhist[{k}]"]) for k in range(int(g["iters"]) + 1)]
    assert all(h > 1e-8 * num(g["bnorm"]) for h in hist[:-1])


def test_oracle_reproduces_the_c1_golden():
    g = read("c1_lap2d5_64_pcg.txt")
    A = I.lap2d5(64)
    b = orc.spmv(A, I.xstar(A.n, 1))
    r = orc.pcg(A, b, 1e-8, 10000, history=True)
    assert r["status"] == int(g["status"]) and r["iters"] == int(g["iters"])
    hist = np.array([num(g[f"rhist[{k}]"]) for k in range(r["iters"] + 1)])
    np.testing.assert_allclose(r["rhist"], hist, rtol=1e-13, atol=0)
