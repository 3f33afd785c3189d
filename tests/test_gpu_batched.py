"""Batched multi-system, multi-RHS solves against the oracle (GPU).

Every column is an independent Jacobi-PCG solve.  Checks: status, the true
FP64 residual ||b - A x|| <= rtol ||b|| (recomputed by the oracle's SpMV),
the solution against the oracle's FP64 PCG solution within
max(1e-8, (||r|| + ||r_ref||) / lambda_min) (the guarantee the stopping
rule gives), and isolation: each column's result is bitwise identical
whether its system is solved alone or inside a batch.
"""
import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


def lambda_min(A):
    sp = pytest.importorskip("scipy.sparse")
    sla = pytest.importorskip("scipy.sparse.linalg")
    M = sp.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.n, A.n))
    return float(sla.eigsh(M, k=1, sigma=0, which="LM", return_eigenvectors=False)[0])


def make_batch():
    specs = [("var5", (12, 9), 1), ("var7", (10, 9, 8), 8), ("var5", (40, 37), 3),
             ("var7", (17, 16, 15), 2), ("var5", (70, 65), 5), ("var7", (6, 5, 4), 4),
             ("var5", (3, 2), 2), ("var7", (25, 24, 23), 1),
             ("var5", (150, 130), 2)]          # 610 tiles: several reduction chunks
    mats = []
    for i, (fam, dims, k) in enumerate(specs):
        A = I.family_matrix(fam, dims, seed=500 + i, sigma=0.5)
        mats.append((A, k))
    return mats


def rhs_for(orc, A, k, sysid):
    cols = [orc.spmv(A, I.xstar(A.n, 77, column=c, system=sysid)) for c in range(k)]
    return np.concatenate(cols)          # column-major n x k


def run_batch(S, mats, rhs, mode, rtol=1e-10, maxit=20000):
    hs, bv, xv, keep = [], [], [], []
    for (A, k), b in zip(mats, rhs):
        hs.append(S.mat(A))
        bh, bt = S.vec(b)
        xh, xt = S.vec(np.zeros(A.n * k))
        bv.append(bh); xv.append(xh); keep.append((bt, xt))
    st, its, rns, sts = gbs.gbs_ksp_solve_cg_batched(S.ctx, hs, bv, xv, [k for _, k in mats],
                                                    [rtol] * len(mats), maxit, mode)
    xs = [S.host(xt) for _, xt in keep]
    for h in hs:
        gbs.gbs_mat_destroy(h)
    for v in bv + xv:
        gbs.gbs_vec_destroy(v)
    return st, its, rns, sts, xs


@pytest.mark.parametrize("mode", [gbs.GBS_MODE_MIXED, gbs.GBS_MODE_FP64])
def test_batched_against_oracle(S, orc, mode):
    mats = make_batch()
    rhs = [rhs_for(orc, A, k, i) for i, (A, k) in enumerate(mats)]
    st, its, rns, sts, xs = run_batch(S, mats, rhs, mode)
    assert st == gbs.GBS_OK, (st, sts)
    assert np.all(sts == gbs.GBS_OK)
    from gpu_util import record
    o = 0
    worst = (0.0, 0.0)
    for (A, k), b, x in zip(mats, rhs, xs):
        lmin = lambda_min(A)
        for c in range(k):
            bc = b[c * A.n:(c + 1) * A.n]
            xc = x[c * A.n:(c + 1) * A.n]
            ref = orc.pcg(A, bc, 1e-10, 20000)
            tr = np.linalg.norm(bc - orc.spmv(A, xc))
            assert tr <= 1e-10 * np.linalg.norm(bc), (o, tr)
            trr = np.linalg.norm(bc - orc.spmv(A, ref["x"]))
            tol = max(1e-8, (tr + trr) / (lmin * np.linalg.norm(ref["x"])))
            e = np.linalg.norm(xc - ref["x"]) / np.linalg.norm(ref["x"])
            worst = max(worst, (e, tol))
            assert e <= tol
            assert abs(rns[o] - tr) <= 1e-3 * tr + 1e-14 * np.linalg.norm(bc)
            assert its[o] >= 1
            o += 1
    record(f"batched[{'mixed' if mode == gbs.GBS_MODE_MIXED else 'fp64'}]",
           "worst_rel_err_vs_oracle", worst[0], worst[1])


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_batched_lanes_per_row(orc, lanes):
    """Every lanes-per-row tiling of the SpMV (the autotuner's candidates)
    meets the same bar against the oracle, in both precisions."""
    from gpu_util import Session
    S = Session(gbs.gbs_opts_default(batched_lanes=lanes))
    mats = make_batch()[:8]
    rhs = [rhs_for(orc, A, k, i) for i, (A, k) in enumerate(mats)]
    for mode in (gbs.GBS_MODE_MIXED, gbs.GBS_MODE_FP64):
        st, its, rns, sts, xs = run_batch(S, mats, rhs, mode)
        assert st == gbs.GBS_OK and np.all(sts == gbs.GBS_OK)
        for (A, k), b, x in zip(mats, rhs, xs):
            lmin = lambda_min(A)
            for c in range(k):
                bc, xc = b[c * A.n:(c + 1) * A.n], x[c * A.n:(c + 1) * A.n]
                ref = orc.pcg(A, bc, 1e-10, 20000)
                tr = np.linalg.norm(bc - orc.spmv(A, xc))
                assert tr <= 1e-10 * np.linalg.norm(bc)
                trr = np.linalg.norm(bc - orc.spmv(A, ref["x"]))
                tol = max(1e-8, (tr + trr) / (lmin * np.linalg.norm(ref["x"])))
                assert np.linalg.norm(xc - ref["x"]) <= tol * np.linalg.norm(ref["x"])
    gbs.gbs_ctx_destroy(S.ctx)


def test_batched_isolation_bitwise(S, orc):
    """A system's columns come out bitwise identical alone and in the mix."""
    mats = make_batch()
    rhs = [rhs_for(orc, A, k, i) for i, (A, k) in enumerate(mats)]
    _, _, _, _, xs_all = run_batch(S, mats, rhs, gbs.GBS_MODE_MIXED)
    for i in (1, 4, 7):
        _, _, _, _, xs_one = run_batch(S, [mats[i]], [rhs[i]], gbs.GBS_MODE_MIXED)
        assert np.array_equal(xs_one[0], xs_all[i]), i
    # and in a different batch order
    perm = [7, 3, 1, 0]
    _, _, _, _, xs_p = run_batch(S, [mats[j] for j in perm], [rhs[j] for j in perm],
                                 gbs.GBS_MODE_MIXED)
    for pos, j in enumerate(perm):
        assert np.array_equal(xs_p[pos], xs_all[j]), j


def test_batched_edge_cases(S, orc):
    good = I.var5(20, 18, seed=9)
    bgood = rhs_for(orc, good, 2, 0)
    bad_diag = I.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32),
                     np.array([1.0, -1.0]))
    indef = I.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
                  np.array([1.0, 2.0, 2.0, 1.0]))
    empty = I.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    mats = [(good, 2), (bad_diag, 1), (indef, 1), (empty, 1)]
    rhs = [bgood, np.ones(2), np.array([1.0, -1.0]), np.zeros(0)]
    for mode in (gbs.GBS_MODE_MIXED, gbs.GBS_MODE_FP64):
        st, its, rns, sts, xs = run_batch(S, mats, rhs, mode)
        assert list(sts) == [gbs.GBS_OK, gbs.GBS_OK, gbs.GBS_ERR_DIAG, gbs.GBS_ERR_INDEFINITE,
                             gbs.GBS_OK]
        assert st == gbs.GBS_ERR_DIAG
        for c in range(2):
            bc = bgood[c * good.n:(c + 1) * good.n]
            xc = xs[0][c * good.n:(c + 1) * good.n]
            assert np.linalg.norm(bc - orc.spmv(good, xc)) <= 1e-10 * np.linalg.norm(bc)
    # iteration limit: status DIVERGED_ITS, x still holds an approximation
    st, its, rns, sts, xs = run_batch(S, [(good, 1)], [bgood[:good.n]], gbs.GBS_MODE_MIXED,
                                      rtol=1e-12, maxit=5)
    assert sts[0] == gbs.GBS_DIVERGED_ITS and its[0] <= 6
    assert np.linalg.norm(xs[0]) > 0
    # zero right-hand side: converged at once, x = 0
    st, its, rns, sts, xs = run_batch(S, [(good, 1)], [np.zeros(good.n)], gbs.GBS_MODE_MIXED)
    assert sts[0] == gbs.GBS_OK and its[0] == 0 and not xs[0].any()


def test_batched_matches_single_solves(S, orc):
    A = I.var7(20, 19, 18, seed=21)
    b = rhs_for(orc, A, 1, 3)
    _, its, _, sts, xs = run_batch(S, [(A, 1)], [b], gbs.GBS_MODE_MIXED)
    h = S.mat(A)
    bv, bt = S.vec(b)
    xv, xt = S.vec(np.zeros(A.n))
    info = gbs.gbs_ksp_solve_cg_ex(h, bv, xv, 1e-10, 20000,
                                   gbs.gbs_opts_default(mode=gbs.GBS_MODE_MIXED))
    x1 = S.host(xt)
    assert info.status == gbs.GBS_OK and sts[0] == gbs.GBS_OK
    assert abs(info.outer_iters - 3) <= 1
    assert np.linalg.norm(xs[0] - x1) <= 1e-8 * np.linalg.norm(x1)
    gbs.gbs_mat_destroy(h)


def test_batched_tune_decision_is_cached(S, orc):
    """The autotuner reports one of its candidates, keeps the decision for
    the class (a second system of the class gets it without timing), and a
    fixed option short-cuts it."""
    from gpu_util import Session
    A = I.var5(60, 55, seed=3)
    h = S.mat(A)
    lanes = gbs.gbs_batched_tune(S.ctx, h, 3, gbs.GBS_MODE_MIXED)
    assert lanes in (1, 2, 4)
    B = I.var5(70, 40, seed=4)          # same class: 5-point rows, stride 4, FP32 inner
    hb = S.mat(B)
    assert gbs.gbs_batched_tune(S.ctx, hb, 4, gbs.GBS_MODE_MIXED) == lanes
    gbs.gbs_mat_destroy(h)
    gbs.gbs_mat_destroy(hb)
    F = Session(gbs.gbs_opts_default(batched_lanes=2))
    hf = F.mat(A)
    assert gbs.gbs_batched_tune(F.ctx, hf, 3, gbs.GBS_MODE_FP64) == 2
    gbs.gbs_mat_destroy(hf)
    gbs.gbs_ctx_destroy(F.ctx)


def test_batched_mixes_compressed_and_full_column_indices(S, orc):
    """One batch holding a system whose columns fit 16-bit relative indices
    and one whose columns do not (a coupling between rows 0 and n - 1 with
    n = 40000): both FP32 tile kinds go through the same stage ring."""
    from test_gpu_spmv import far_coupled_chain
    far = far_coupled_chain(40000, 6)
    near = I.var7(20, 18, 16, seed=31)
    mats = [(far, 2), (near, 3)]
    rhs = [rhs_for(orc, A, k, i) for i, (A, k) in enumerate(mats)]
    st, its, rns, sts, xs = run_batch(S, mats, rhs, gbs.GBS_MODE_MIXED)
    assert st == gbs.GBS_OK and np.all(sts == gbs.GBS_OK)
    for (A, k), b, x in zip(mats, rhs, xs):
        for c in range(k):
            bc, xc = b[c * A.n:(c + 1) * A.n], x[c * A.n:(c + 1) * A.n]
            assert np.linalg.norm(bc - orc.spmv(A, xc)) <= 1e-10 * np.linalg.norm(bc)
