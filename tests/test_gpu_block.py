"""Block Jacobi-PCG (several right-hand sides sharing one search space)
against the oracle's block PCG: block iterations within 2, every column
within 1e-8 of the oracle's FP64 solution at rtol 1e-10 and at its true
residual; one column behaves as the single-vector solve; breakdown and
degenerate cases."""
import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


def rhs(orc, A, k, seed):
    return np.stack([orc.spmv(A, I.xstar(A.n, seed + 17 * j)) for j in range(k)], axis=1)


def block_solve(S, A, B, rtol, maxit):
    k = B.shape[1]
    h = S.mat(A)
    bv, bt = S.vec(B.T.reshape(-1))          # column-major: column j at j * n
    xv, xt = S.zeros(A.n * k)
    info, rn = gbs.gbs_ksp_solve_cg_block(h, k, bv, xv, rtol, maxit)
    X = S.host(xt).reshape(k, A.n).T
    for v in (bv, xv):
        gbs.gbs_vec_destroy(v)
    gbs.gbs_mat_destroy(h)
    return info, rn, X


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("case", ["lap2d5_40", "var7_20x18x16", "var27_14", "lap3d7_30"])
def test_block_cg_matches_oracle(S, orc, case, k):
    A = {"lap2d5_40": lambda: I.lap2d5(40), "var7_20x18x16": lambda: I.var7(20, 18, 16, seed=7),
         "var27_14": lambda: I.var27(14, seed=3), "lap3d7_30": lambda: I.lap3d7(30)}[case]()
    B = rhs(orc, A, k, 3)
    ref = orc.block_pcg(A, B, 1e-10, 5000)
    info, rn, X = block_solve(S, A, B, 1e-10, 5000)
    assert ref["status"] == 0 and info.status == gbs.GBS_OK
    assert abs(info.iters - ref["iters"]) <= 2
    from gpu_util import record
    worst = 0.0
    for j in range(k):
        bn = np.linalg.norm(B[:, j])
        assert np.linalg.norm(B[:, j] - orc.spmv(A, X[:, j])) <= 1e-10 * bn * (1 + 1e-3)
        assert abs(rn[j] - ref["rnorm"][j]) <= 1e-3 * ref["rnorm"][j] + 1e-13 * bn
        e = np.linalg.norm(X[:, j] - ref["x"][:, j]) / np.linalg.norm(ref["x"][:, j])
        worst = max(worst, e)
    record(f"block[{case},k={k}]", "worst_rel_err_vs_oracle", worst, 1e-8)
    assert worst <= 1e-8


def test_block_cg_one_column_is_the_pcg_solve(S, orc):
    A = I.var7(22, 21, 20, seed=4)
    B = rhs(orc, A, 1, 9)
    ref = orc.pcg(A, B[:, 0], 1e-10, 5000)
    info, rn, X = block_solve(S, A, B, 1e-10, 5000)
    assert info.status == gbs.GBS_OK and abs(info.iters - ref["iters"]) <= 2
    assert np.linalg.norm(X[:, 0] - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])


def test_block_cg_fewer_iterations_than_single(S, orc):
    """The shared space: 8 columns of the 2D Laplacian converge in fewer
    block iterations than the slowest column alone (the oracle says so
    too)."""
    A = I.lap2d5(48)
    B = rhs(orc, A, 8, 1)
    info, rn, X = block_solve(S, A, B, 1e-10, 5000)
    single = max(orc.pcg(A, B[:, j], 1e-10, 5000)["iters"] for j in range(8))
    assert info.status == gbs.GBS_OK and info.iters < single


def test_block_cg_degenerate_cases(S, orc):
    A = I.lap2d5(12)
    b = rhs(orc, A, 1, 4)[:, 0]
    info, _, _ = block_solve(S, A, np.stack([b, b], axis=1), 1e-10, 100)
    assert info.status == gbs.GBS_ERR_INDEFINITE
    info, rn, X = block_solve(S, A, np.zeros((A.n, 3)), 1e-10, 100)
    assert info.status == gbs.GBS_OK and info.iters == 0 and not X.any()
    B = rhs(orc, A, 2, 1)
    info, rn, X = block_solve(S, A, B, 1e-14, 2)
    ref = orc.block_pcg(A, B, 1e-14, 2)
    assert info.status == gbs.GBS_DIVERGED_ITS and info.iters == 2
    assert np.linalg.norm(X - ref["x"]) <= 1e-12 * np.linalg.norm(ref["x"])
    # bad arguments: k out of range, sizes that do not match
    h = S.mat(A)
    v9, _ = S.zeros(A.n * 9)
    w9, _ = S.zeros(A.n * 9)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_ksp_solve_cg_block(h, 9, v9, w9, 1e-8, 10)
    v2, _ = S.zeros(A.n * 2)
    w3, _ = S.zeros(A.n * 3)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_ksp_solve_cg_block(h, 2, v2, w3, 1e-8, 10)
    for v in (v9, w9, v2, w3):
        gbs.gbs_vec_destroy(v)
    gbs.gbs_mat_destroy(h)
