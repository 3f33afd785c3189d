"""Jacobi-preconditioned Chebyshev iteration on the GPU against the oracle.

The GPU forms the next direction with one fused multiply-add and sums
||r||^2 in its own order, so its iterates differ from the oracle's by
rounding only: the iteration count must agree within 2, the true FP64
residual must meet the tolerance, and the solution must agree within what
the stopping rule guarantees.
"""
import math

import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


def spectrum_bounds(A):
    """Extreme eigenvalues of D^-1 A (via the symmetric D^-1/2 A D^-1/2)."""
    sp = pytest.importorskip("scipy.sparse")
    sla = pytest.importorskip("scipy.sparse.linalg")
    M = sp.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.n, A.n))
    d = 1 / np.sqrt(M.diagonal())
    B = sp.diags(d) @ M @ sp.diags(d)
    hi = sla.eigsh(B, k=1, which="LA", return_eigenvectors=False)[0]
    lo = sla.eigsh(B, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    return float(lo), float(hi)


def laplacian_bounds(N, dim):
    c = math.cos(math.pi / (N + 1))
    return 1 - c, 1 + c          # D^-1 A of the Dirichlet Laplacian, any dimension


def solve(S, A, b, emin, emax, rtol, maxit):
    h = S.mat(A)
    bv, bt = S.vec(b)
    xv, xt = S.zeros(A.n)
    info = gbs.gbs_ksp_solve_chebyshev(h, bv, xv, emin, emax, rtol, maxit)
    x = S.host(xt)
    gbs.gbs_mat_destroy(h)
    return info, x


@pytest.mark.parametrize("case", ["lap2d5_40", "lap3d7_20", "var7", "var27", "wide",
                                  "lap3d7_56"])
def test_chebyshev_against_oracle(S, orc, case):
    lmin = None
    if case == "lap3d7_56":     # large enough for the 32-warp launch shape
        N = 56
        A, (lo, hi) = I.lap3d7(N), laplacian_bounds(N, 3)
        lmin = 6 * (1 - math.cos(math.pi / (N + 1)))
    elif case == "lap2d5_40":
        A, (lo, hi) = I.lap2d5(40), laplacian_bounds(40, 2)
    elif case == "lap3d7_20":
        A, (lo, hi) = I.lap3d7(20), laplacian_bounds(20, 3)
    elif case == "var7":
        A = I.var7(21, 17, 13, seed=8)
        lo, hi = spectrum_bounds(A)
    elif case == "var27":
        A = I.var27(14, seed=4)
        lo, hi = spectrum_bounds(A)
    else:                       # an interval wider than the spectrum still converges
        A = I.lap2d5(30)
        lo, hi = laplacian_bounds(30, 2)
        lo, hi = 0.8 * lo, 1.1 * hi
    b = orc.spmv(A, I.xstar(A.n, 9))
    ref = orc.chebyshev(A, b, lo, hi, 1e-10, 100000)
    info, x = solve(S, A, b, lo, hi, 1e-10, 100000)
    assert ref["status"] == 0 and info.status == gbs.GBS_OK
    assert abs(info.iters - ref["iters"]) <= 2
    bn = np.linalg.norm(b)
    tr = np.linalg.norm(b - orc.spmv(A, x))
    assert tr <= 1e-10 * bn * (1 + 1e-3)
    assert abs(info.bnorm - bn) <= 1e-12 * bn
    # two vectors with residuals r, r_ref differ by at most (||r|| + ||r_ref||) / lambda_min(A)
    trr = np.linalg.norm(b - orc.spmv(A, ref["x"]))
    if lmin is None:
        sp = pytest.importorskip("scipy.sparse")
        sla = pytest.importorskip("scipy.sparse.linalg")
        M = sp.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.n, A.n))
        lmin = float(sla.eigsh(M, k=1, sigma=0, which="LM", return_eigenvectors=False)[0])
    tol = max(1e-8, (tr + trr) / (lmin * np.linalg.norm(ref["x"])))
    from gpu_util import record
    e = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    record(f"chebyshev[n={A.n}]", "rel_err_vs_oracle", e, tol)
    assert e <= tol


def test_chebyshev_limits_and_errors(S, orc):
    A = I.lap2d5(16)
    lo, hi = laplacian_bounds(16, 2)
    b = orc.spmv(A, I.xstar(A.n, 2))
    for k in (0, 1, 7):
        info, x = solve(S, A, b, lo, hi, 1e-14, k)
        ref = orc.chebyshev(A, b, lo, hi, 1e-14, k)
        assert info.status == gbs.GBS_DIVERGED_ITS and info.iters == k
        assert np.linalg.norm(x - ref["x"]) <= 1e-12 * max(np.linalg.norm(ref["x"]), 1e-300) or k == 0
        if k == 0:
            assert not x.any()
    info, x = solve(S, A, np.zeros(A.n), lo, hi, 1e-8, 10)
    assert info.status == gbs.GBS_OK and info.iters == 0 and not x.any()
    h = S.mat(A)
    bv, _ = S.vec(b)
    xv, _ = S.zeros(A.n)
    for l, u in ((0.0, 1.0), (1.0, 0.5), (-1.0, 2.0), (0.5, math.inf)):
        with pytest.raises(gbs.GbsError):
            gbs.gbs_ksp_solve_chebyshev(h, bv, xv, l, u, 1e-8, 10)
    gbs.gbs_mat_destroy(h)
    bad = I.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    info, _ = solve(S, bad, np.ones(2), 0.5, 2.0, 1e-8, 10)
    assert info.status == gbs.GBS_ERR_DIAG


def test_chebyshev_full_size_c2_against_its_bound(S, orc):
    """The 128^3 Laplacian with the closed-form interval: converges to 1e-10
    within the count the Chebyshev bound implies; true residual checked by
    the oracle's SpMV."""
    N = 128
    A = I.lap3d7(N)
    lo, hi = laplacian_bounds(N, 3)
    b = orc.spmv(A, I.xstar(A.n, 2))
    info, x = solve(S, A, b, lo, hi, 1e-10, 20000)
    assert info.status == gbs.GBS_OK
    sigma = (hi + lo) / (hi - lo)
    kappa = hi / lo
    bound = math.ceil(math.acosh(math.sqrt(kappa) / 1e-10) / math.acosh(sigma))
    assert info.iters <= bound
    bn = np.linalg.norm(b)
    assert np.linalg.norm(b - orc.spmv(A, x)) <= 1e-10 * bn * (1 + 1e-3)
    assert info.model_bytes > 0 and info.device_ms > 0
