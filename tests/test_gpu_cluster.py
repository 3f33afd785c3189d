"""The one-cluster FP64 Jacobi-PCG (GBS_ALG_CLUSTER, and GBS_ALG_AUTO for
small FP64 systems) against the CPU oracle.

Same bar as the grid solves: iteration counts within +-2 of the oracle,
solutions within 1e-8 relative of the oracle's at rtol 1e-10, the true
residual ||b - A x||_2 (oracle SpMV) within rtol ||b||_2 (1 + 1e-3).
Sizes span one CTA to a full cluster, CTA blocks of 128 to 4096 rows with
ragged last blocks, up to the largest system the path takes; one matrix
couples every block with every other (random far columns).
"""
import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CL = gbs.GBS_ALG_CLUSTER


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


def solve(S, A, b, rtol, maxit, x0=None, **opts):
    h = S.mat(A)
    bv, bt = S.vec(b)
    xv, xt = S.vec(np.zeros(A.n) if x0 is None else x0)
    info = gbs.gbs_ksp_solve_cg_ex(h, bv, xv, rtol, maxit, gbs.gbs_opts_default(**opts))
    x = S.host(xt)
    gbs.gbs_vec_destroy(bv)
    gbs.gbs_vec_destroy(xv)
    gbs.gbs_mat_destroy(h)
    return info, x


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def true_res(orc, A, b, x):
    return np.linalg.norm(b - orc.spmv(A, x))


MAKERS = {
    "lap2d5_64 (4096 rows, C1)": lambda: I.lap2d5(64),
    "lap3d7_17 (4913)": lambda: I.lap3d7(17),
    "var7_17x15x13 (3315)": lambda: I.var7(17, 15, 13, seed=7),
    "var27_12 (1728)": lambda: I.var27(12, seed=3),
    "var7_29x27x25 (19575)": lambda: I.var7(29, 27, 25, seed=5),
    "var5_256x128 (32768, the limit)": lambda: I.var5(256, 128, seed=4),
    "var5_41x25 (1025)": lambda: I.var5(41, 25, seed=2),
    "lap2d5_31x33 (1023)": lambda: I.lap2d5(31, 33),
    "lap2d5_3 (9)": lambda: I.lap2d5(3),
    "random_spd_3000 (far couplings)": lambda: I.random_csr(3000, 3000, 6, seed=8,
                                                            symmetric=True, diag_shift=0.5),
}


@pytest.mark.parametrize("name", sorted(MAKERS))
def test_cluster_matches_oracle(S, orc, name):
    A = MAKERS[name]()
    assert A.n <= gbs.GBS_CLUSTER_MAX_ROWS
    b = orc.spmv(A, I.xstar(A.n, 2))
    ref = orc.pcg(A, b, 1e-10, 20000)
    info, x = solve(S, A, b, 1e-10, 20000, algorithm=CL)
    assert info.status == gbs.GBS_OK, gbs.gbs_status_string(info.status)
    assert abs(info.iters - ref["iters"]) <= 2
    assert rel(x, ref["x"]) <= 1e-8
    nb = np.linalg.norm(b)
    assert true_res(orc, A, b, x) <= 1e-10 * nb * (1 + 1e-3)
    assert abs(info.bnorm - nb) <= 1e-12 * nb
    assert info.rnorm <= 1e-10 * info.bnorm


def test_auto_takes_the_cluster_path_bitwise(S, orc):
    """AUTO routes a small FP64 system to the one-cluster kernel: same bits
    as the explicit choice, and as a second run; the grid kernel reaches
    the same tolerance."""
    A = I.var7(17, 15, 13, seed=7)
    b = orc.spmv(A, I.xstar(A.n, 3))
    i_s, x_s = solve(S, A, b, 1e-10, 20000, algorithm=CL)
    i_a, x_a = solve(S, A, b, 1e-10, 20000)
    i_2, x_2 = solve(S, A, b, 1e-10, 20000, algorithm=CL)
    i_p, x_p = solve(S, A, b, 1e-10, 20000, algorithm=gbs.GBS_ALG_PERSISTENT)
    assert np.array_equal(x_s, x_a) and i_s.iters == i_a.iters and i_s.rnorm == i_a.rnorm
    assert np.array_equal(x_s, x_2) and i_s.rnorm == i_2.rnorm
    assert i_p.status == gbs.GBS_OK and abs(i_p.iters - i_s.iters) <= 2
    assert rel(x_s, x_p) <= 1e-8


def test_c1_stored_golden_cluster(S, orc):
    """The stored C1 fixture (written from the oracle): iteration count
    within 2 and the recurrence residual at the stopping test."""
    import os
    g = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "c1_lap2d5_64_pcg.txt")) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = (t.strip() for t in line.split("=", 1))
                g[k] = v
    A = I.lap2d5(64)
    b = orc.spmv(A, I.xstar(A.n, 1))
    info, _ = solve(S, A, b, 1e-8, 10000, algorithm=CL)
    assert info.status == gbs.GBS_OK
    assert abs(info.iters - int(g["iters"])) <= 2
    assert info.rnorm <= 1e-8 * float.fromhex(g["bnorm"]) * (1 + 1e-12)


def test_cluster_iteration_limits_and_guess(S, orc):
    A = I.var7(12, 11, 10, seed=3)
    b = orc.spmv(A, I.xstar(A.n, 4))
    for k in (0, 1, 5):
        info, x = solve(S, A, b, 1e-14, k, algorithm=CL)
        ref = orc.pcg(A, b, 1e-14, k)
        assert info.status == gbs.GBS_DIVERGED_ITS and info.iters == k
        assert rel(x, ref["x"]) <= 1e-12 if k else np.array_equal(x, ref["x"])
    # a nonzero initial guess: r = b - A x0 in the set-up
    x0 = I.xstar(A.n, 9)
    ref = orc.pcg(A, b, 1e-10, 20000, x0=x0)
    info, x = solve(S, A, b, 1e-10, 20000, x0=x0, algorithm=CL)
    assert info.status == gbs.GBS_OK and abs(info.iters - ref["iters"]) <= 2
    assert rel(x, ref["x"]) <= 1e-8
    # x0 already the solution: no iteration
    xs = I.xstar(A.n, 5)
    bs = orc.spmv(A, xs)
    info, _ = solve(S, A, bs, 1e-8, 100, x0=xs, algorithm=CL)
    assert info.status == gbs.GBS_OK and info.iters == 0


def test_cluster_degenerate_statuses(S, orc):
    A = I.lap2d5(30)
    info, x = solve(S, A, np.zeros(A.n), 1e-8, 100, algorithm=CL)
    assert info.status == gbs.GBS_OK and info.iters == 0 and not x.any()
    b = orc.spmv(A, I.xstar(A.n, 5))
    b[7] = np.nan
    info, _ = solve(S, A, b, 1e-8, 100, algorithm=CL)
    assert info.status == gbs.GBS_ERR_NAN
    B = I.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
              np.array([1.0, 2.0, 2.0, 1.0]))
    info, _ = solve(S, B, np.array([1.0, -1.0]), 1e-10, 10, algorithm=CL)
    assert info.status == gbs.GBS_ERR_INDEFINITE
    one = I.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    info, x = solve(S, one, np.array([2.0]), 1e-12, 10, algorithm=CL)
    assert info.status == gbs.GBS_OK and info.iters == 1 and x[0] == 0.5


def test_cluster_refuses_what_it_cannot_take(S, orc):
    A = I.var5(256, 129, seed=4)          # 33024 rows: past the shared-memory limit
    assert A.n > gbs.GBS_CLUSTER_MAX_ROWS
    b = orc.spmv(A, I.xstar(A.n, 2))
    with pytest.raises(gbs.GbsError) as e:
        solve(S, A, b, 1e-10, 20000, algorithm=CL)
    assert e.value.status == gbs.GBS_ERR_UNSUPPORTED
    info, x = solve(S, A, b, 1e-10, 20000)   # AUTO: the grid kernel
    assert info.status == gbs.GBS_OK
    assert true_res(orc, A, b, x) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-3)
    C = I.lap2d5(20)
    bc = orc.spmv(C, I.xstar(C.n, 1))
    with pytest.raises(gbs.GbsError) as e:
        solve(S, C, bc, 1e-10, 100, algorithm=CL, mode=gbs.GBS_MODE_MIXED)
    assert e.value.status == gbs.GBS_ERR_UNSUPPORTED
