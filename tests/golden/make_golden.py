"""Writes the stored expected values under tests/golden/ that come from the
oracle (the only source of computed fixtures): run from the repository root
as ``python tests/golden/make_golden.py``.  Calls oracle/ and the seeded
input generators only."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as orc  # noqa: E402
from paper_2011_00715_gb300 import inputs as I  # noqa: E402


def c1():
    A = I.lap2d5(64)
    xs = I.xstar(A.n, 1)
    b = orc.spmv(A, xs)
    r = orc.pcg(A, b, 1e-8, 10000, history=True)
    lines = [
        "# C1: 2D 5-point Dirichlet Laplacian 64x64 (n 4096, nnz 20224), x* uniform[-1,1) seed 1,",
        "# b = A x*, Jacobi-PCG from x0 = 0 to ||r|| <= 1e-8 ||b|| tested before each iteration.",
        "# KSPCG with PCJACOBI (Sec. 5.5, Sec. 5.3); the iteration is textbook PCG (Saad, Alg. 9.1).",
        "# Written by tests/golden/make_golden.py from the oracle; rhist[k] = ||r_k||_2.",
        f"status = {r['status']}",
        f"iters = {r['iters']}",
        f"bnorm = {float(np.linalg.norm(b)).hex()}",
        f"rnorm = {float(r['rnorm']).hex()}",
    ]
    for k, v in enumerate(r["rhist"]):
        lines.append(f"rhist[{k}] = {float(v).hex()}")
    with open(os.path.join(HERE, "c1_lap2d5_64_pcg.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    c1()
