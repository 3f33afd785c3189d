"""Device assembly from coordinate triplets against the oracle (GPU).

The assembled CSR must be bitwise the oracle's (same structure, duplicates
summed in triplet order), from host and from device triplets, for short,
medium and long rows; refilled values follow the same rule; a matrix
assembled from the grid's edge contributions is the 7-point Laplacian and
solves bitwise like the one created from CSR."""
import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


def triplets(seed, nrows, ncols, m):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, nrows, m).astype(np.int32)
    j = rng.integers(0, ncols, m).astype(np.int32)
    i[m // 2:] = i[: m - m // 2]          # many repeated pairs
    j[m // 2:] = j[: m - m // 2]
    v = rng.standard_normal(m) * 10.0 ** rng.integers(-10, 11, m)   # order-sensitive sums
    return i, j, v


def assemble(S, nrows, ncols, i, j, v, device):
    if device:
        t = S.torch
        args = [t.from_numpy(np.ascontiguousarray(a)).cuda() for a in (i, j, v)]
    else:
        args = [i, j, v]
    return gbs.gbs_mat_create_coo(S.ctx, nrows, ncols, *args)


@pytest.mark.parametrize("device", [False, True])
@pytest.mark.parametrize("shape", [(40, 50, 600), (3000, 2000, 40000), (1, 1, 1), (5, 7, 0)])
def test_coo_assembly_bitwise(S, orc, shape, device):
    nr, nc, m = shape
    i, j, v = triplets(sum(shape), nr, nc, m)
    h = assemble(S, nr, nc, i, j, v, device)
    rp, ci, vals = gbs.gbs_mat_get_csr(h)
    st, rp0, ci0, v0 = orc.coo_to_csr(nr, nc, i, j, v)
    assert st == 0
    assert np.array_equal(rp, rp0) and np.array_equal(ci, ci0) and np.array_equal(vals, v0)
    gbs.gbs_mat_destroy(h)


def test_coo_medium_and_long_rows(S, orc):
    """Rows of 1, 40, 700, 4096, 4097 and 9000 triplets (warp, CTA and host
    sorting), with repeats."""
    rng = np.random.default_rng(2)
    lens = [1, 40, 700, 4096, 4097, 9000]
    i = np.concatenate([np.full(L, r, np.int32) for r, L in enumerate(lens)])
    j = np.concatenate([rng.integers(0, 6000, L).astype(np.int32) for L in lens])
    v = rng.standard_normal(len(i))
    perm = rng.permutation(len(i))
    i, j, v = i[perm], j[perm], v[perm]
    h = assemble(S, len(lens), 6000, i, j, v, True)
    rp, ci, vals = gbs.gbs_mat_get_csr(h)
    st, rp0, ci0, v0 = orc.coo_to_csr(len(lens), 6000, i, j, v)
    assert np.array_equal(rp, rp0) and np.array_equal(ci, ci0) and np.array_equal(vals, v0)
    gbs.gbs_mat_destroy(h)


def test_coo_refill_and_errors(S, orc):
    i, j, v = triplets(5, 300, 300, 5000)
    h = assemble(S, 300, 300, i, j, v, False)
    v2 = np.random.default_rng(6).standard_normal(len(v))
    gbs.gbs_mat_set_values_coo(h, v2)
    rp, ci, vals = gbs.gbs_mat_get_csr(h)
    _, rp0, ci0, v0 = orc.coo_to_csr(300, 300, i, j, v2)
    assert np.array_equal(ci, ci0) and np.array_equal(vals, v0)
    gbs.gbs_mat_destroy(h)
    with pytest.raises(gbs.GbsError) as e:
        assemble(S, 10, 10, np.array([0, 10], np.int32), np.array([0, 0], np.int32),
                 np.ones(2), False)
    assert e.value.status == gbs.GBS_ERR_CSR
    with pytest.raises(gbs.GbsError):
        assemble(S, 10, 10, np.array([0], np.int32), np.array([-1], np.int32), np.ones(1), True)
    A = I.lap2d5(5)          # not made from triplets
    h = S.mat(A)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_mat_set_values_coo(h, np.ones(10))
    gbs.gbs_mat_destroy(h)


def test_coo_edge_assembly_solves_like_csr(S, orc):
    N = 24
    i, j, v = I.lap3d7_edge_triplets(N, seed=7)
    A = I.lap3d7(N)
    hc = assemble(S, A.n, A.n, i, j, v, True)
    rp, ci, vals = gbs.gbs_mat_get_csr(hc)
    assert np.array_equal(rp, A.rowptr) and np.array_equal(ci, A.colidx) and np.array_equal(vals, A.vals)
    ha = S.mat(A)
    b = orc.spmv(A, I.xstar(A.n, 4))
    xs = []
    for h in (hc, ha):
        bv, _ = S.vec(b)
        xv, xt = S.zeros(A.n)
        info = gbs.gbs_ksp_solve_cg_ex(h, bv, xv, 1e-10, 5000,
                                       gbs.gbs_opts_default(mode=gbs.GBS_MODE_FP64))
        assert info.status == gbs.GBS_OK
        xs.append(S.host(xt))
        gbs.gbs_mat_destroy(h)
    assert np.linalg.norm(xs[0] - xs[1]) <= 1e-12 * np.linalg.norm(xs[1])
