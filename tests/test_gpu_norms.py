"""The stopping-test norms (gbs_opts.norm_type) of the FP64 CG solves
against the oracle run with the same norm, on every launch algorithm.

Bar: iteration counts within +-2 of the oracle, solutions within 1e-8
relative at rtol 1e-10, N(b) within 1e-12 relative, the reported N(r) below
rtol N(b), and the chosen norm of the true residual (oracle SpMV) within
rtol N(b) (1 + 1e-3).  With D = 4I the preconditioned and natural norms are
the unpreconditioned one scaled by 1/4 and 1/2 exactly, so the three runs
agree bit for bit wherever the reductions are reproducible (one cluster,
per-op, graph; the grid kernel to the last bits).
"""
import math

import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ALGS = {"cluster": gbs.GBS_ALG_CLUSTER, "persistent": gbs.GBS_ALG_PERSISTENT,
        "perop": gbs.GBS_ALG_PEROP, "graph": gbs.GBS_ALG_GRAPH}
NORMS = {"preconditioned": gbs.GBS_NORM_PRECONDITIONED, "natural": gbs.GBS_NORM_NATURAL,
         "unpreconditioned": gbs.GBS_NORM_UNPRECONDITIONED}


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


def solve(S, A, b, rtol, maxit, **opts):
    h = S.mat(A)
    bv, _ = S.vec(b)
    xv, xt = S.vec(np.zeros(A.n))
    try:
        info = gbs.gbs_ksp_solve_cg_ex(h, bv, xv, rtol, maxit, gbs.gbs_opts_default(**opts))
        x = S.host(xt)
    finally:
        gbs.gbs_vec_destroy(bv)
        gbs.gbs_vec_destroy(xv)
        gbs.gbs_mat_destroy(h)
    return info, x


def norm_of(A, v, m):
    d = np.zeros(A.n)
    for i in range(A.n):
        seg = slice(A.rowptr[i], A.rowptr[i + 1])
        d[i] = A.vals[seg][A.colidx[seg] == i][0]
    if m == gbs.GBS_NORM_UNPRECONDITIONED:
        return float(np.linalg.norm(v))
    if m == gbs.GBS_NORM_PRECONDITIONED:
        return float(np.linalg.norm(v / d))
    return math.sqrt(float(v @ (v / d)))


@pytest.mark.parametrize("alg", sorted(ALGS))
@pytest.mark.parametrize("norm", sorted(NORMS))
def test_norms_match_oracle(S, orc, alg, norm):
    # a system the one-cluster path takes, and a larger one for the others
    A = I.var7(17, 15, 13, seed=7, sigma=1.0) if alg == "cluster" else \
        I.var7(40, 33, 27, seed=7, sigma=1.0)
    m = NORMS[norm]
    b = orc.spmv(A, I.xstar(A.n, 2))
    ref = orc.pcg(A, b, 1e-10, 20000, norm=m)
    info, x = solve(S, A, b, 1e-10, 20000, algorithm=ALGS[alg], norm_type=m)
    assert info.status == gbs.GBS_OK, gbs.gbs_status_string(info.status)
    assert abs(info.iters - ref["iters"]) <= 2
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    assert abs(info.bnorm - ref["bnorm"]) <= 1e-12 * ref["bnorm"]
    assert info.rnorm <= 1e-10 * info.bnorm
    nb = norm_of(A, b, m)
    assert norm_of(A, b - orc.spmv(A, x), m) <= 1e-10 * nb * (1 + 1e-3)


@pytest.mark.parametrize("alg", sorted(ALGS))
def test_norms_scale_exactly_with_constant_diagonal(S, orc, alg):
    A = I.lap2d5(150) if alg == "cluster" else I.lap2d5(210)
    b = orc.spmv(A, I.xstar(A.n, 3))
    runs = [solve(S, A, b, 1e-9, 20000, algorithm=ALGS[alg], norm_type=m)
            for m in (gbs.GBS_NORM_UNPRECONDITIONED, gbs.GBS_NORM_PRECONDITIONED,
                      gbs.GBS_NORM_NATURAL)]
    (iu, xu), (ip, xp), (i_n, xn) = runs
    assert iu.status == ip.status == i_n.status == gbs.GBS_OK
    if alg != "persistent":
        assert iu.iters == ip.iters == i_n.iters
        assert np.array_equal(xu, xp) and np.array_equal(xu, xn)
        assert ip.rnorm == iu.rnorm / 4 and ip.bnorm == iu.bnorm / 4
        assert i_n.rnorm == iu.rnorm / 2 and i_n.bnorm == iu.bnorm / 2
    else:
        # the grid kernel's warps claim tiles dynamically within a CTA, so
        # its sums (and hence the last bits of every run) vary run to run
        assert abs(iu.iters - ip.iters) <= 1 and abs(iu.iters - i_n.iters) <= 1
        for x in (xp, xn):
            assert np.linalg.norm(x - xu) <= 1e-12 * np.linalg.norm(xu)
        assert abs(ip.bnorm - iu.bnorm / 4) <= 1e-14 * ip.bnorm
        assert abs(i_n.bnorm - iu.bnorm / 2) <= 1e-14 * i_n.bnorm
        assert ip.rnorm <= 1e-9 * ip.bnorm and i_n.rnorm <= 1e-9 * i_n.bnorm


def test_norm_options_refused_where_unsupported(S, orc):
    A = I.lap2d5(20)
    b = orc.spmv(A, I.xstar(A.n, 1))
    for bad in ({"norm_type": 3}, {"norm_type": -1},
                {"norm_type": gbs.GBS_NORM_NATURAL, "mode": gbs.GBS_MODE_MIXED}):
        with pytest.raises(gbs.GbsError) as e:
            solve(S, A, b, 1e-8, 100, **bad)
        assert e.value.status == gbs.GBS_ERR_ARG
