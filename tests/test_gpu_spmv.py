"""MatMult parity: the CUDA CSR SpMV against the CPU oracle.

FP64 rows are accumulated left to right in storage order with fused
multiply-adds: held to ||y - y_orc|| <= 1e-13 ||y_orc|| and, per row, to the
componentwise bound 2 gamma_m (|A||x|)_i (m = nonzeros in the row), and
bitwise on exact inputs.  FP32 rows round each product and sum separately
in the oracle's order with one lane per row, so they are bitwise equal to
the oracle's FP32 product (rows longer than one tile are reduced by a tree
and use the bounds instead).  With 2 or 4 lanes per row (the default for
rows of more than 16 nonzeros) each lane sums a share of the row and the
shares are added by a tree: FP64 and FP32 are then bitwise on exact inputs
and within the componentwise bound gamma_m (|A||x|) of any summation order.
"""
import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


@pytest.fixture(scope="module")
def S1():
    """One lane per row: the FP32 summation order of the oracle."""
    from gpu_util import Session
    return Session(gbs.gbs_opts_default(spmv_lanes=1))


def with_empty_and_long_rows(n=3000, seed=5):
    """Random pattern with empty rows, rows of very different lengths and one
    row longer than a tile (5000 entries)."""
    a = {}
    lens = (I.counter_u64(seed, 30, np.arange(n)) % np.uint64(40)).astype(int)
    lens[::97] = 0
    for i in range(n):
        c = (I.counter_u64(seed, 31 + i % 7, np.arange(lens[i]) + 64 * i) % np.uint64(n)).astype(int)
        v = I.uniform_pm1(seed, 50 + i, lens[i])
        for cc, vv in zip(c.tolist(), v.tolist()):
            a[(i, cc)] = vv
    for j in range(5000):
        a[(17, (j * 7) % n)] = 1.0 / (j + 1)
    return I._from_dict(n, a, {"family": "mixed-lengths"})


def run(S, A, x, dtype=np.float64):
    h = S.mat(A)
    xv, xt = S.vec(x, dtype)
    yv, yt = S.zeros(A.n, dtype)
    gbs.gbs_mat_mult(h, xv, yv)
    y = S.host(yt)
    for v in (xv, yv):
        gbs.gbs_vec_destroy(v)
    gbs.gbs_mat_destroy(h)
    return y


CASES = {
    "lap2d5_64": lambda: I.lap2d5(64),
    "lap3d7_20": lambda: I.lap3d7(20),              # 8000 rows, ragged last tile
    "var27_13": lambda: I.var27(13, seed=3),        # 27 nnz/row: tiles split by nnz
    "random_rect": lambda: I.random_csr(700, 1300, 11, seed=2),
    "tiny": lambda: I.lap2d5(2),
}


def assert_within_bounds(orc, A, x, y, ref):
    rows = np.diff(A.rowptr)
    absA = I.CSR(A.n, A.rowptr, A.colidx, np.abs(A.vals))
    absA.meta["ncols"] = A.meta.get("ncols", A.n)
    g = 2 * rows * U / (1 - 2 * rows * U)
    assert np.all(np.abs(y - ref) <= g * orc.spmv(absA, np.abs(x)))
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", sorted(CASES))
def test_spmv_fp64(S, name, orc):
    A = CASES[name]()
    ncols = A.meta.get("ncols", A.n)
    x = I.uniform_pm1(17, 0, ncols)
    y = run(S, A, x)
    assert_within_bounds(orc, A, x, y, orc.spmv(A, x))


@pytest.mark.parametrize("name", sorted(CASES))
def test_spmv_fp32_bitwise(S1, name, orc):
    A = CASES[name]()
    ncols = A.meta.get("ncols", A.n)
    x = I.uniform_pm1(18, 0, ncols).astype(np.float32)
    y = run(S1, A, x, np.float32)
    ref = orc.spmv_f32(A, x)
    assert np.array_equal(y, ref)


def test_spmv_empty_and_long_rows(S, S1, orc):
    A = with_empty_and_long_rows()
    x = I.uniform_pm1(19, 0, A.n)
    y = run(S, A, x)
    ref = orc.spmv(A, x)
    rows = np.diff(A.rowptr)
    assert np.all(y[rows == 0] == 0.0)
    assert_within_bounds(orc, A, x, y, ref)
    x32 = x.astype(np.float32)
    y32 = run(S1, A, x32, np.float32)
    ref32 = orc.spmv_f32(A, x32)
    short = rows <= 2048
    assert np.array_equal(y32[short], ref32[short])


def test_spmv_exact_inputs(S, orc):
    A = I.exact_csr(5000, 9, seed=4)
    x = I.exact_vector(5000, seed=6)
    assert np.array_equal(run(S, A, x), orc.spmv(A, x))


def test_spmv_device_resident_input_and_set_values(S, orc):
    A = I.var7(30, 20, 10, seed=8)
    h = S.mat(A, device=True)
    x = I.uniform_pm1(3, 0, A.n)
    xv, xt = S.vec(x)
    yv, yt = S.zeros(A.n)
    gbs.gbs_mat_mult(h, xv, yv)
    assert_within_bounds(orc, A, x, S.host(yt), orc.spmv(A, x))
    vals2 = A.vals * 2.0
    gbs.gbs_mat_set_values(h, vals2)
    gbs.gbs_mat_mult(h, xv, yv)
    A2 = I.CSR(A.n, A.rowptr, A.colidx, vals2)
    assert_within_bounds(orc, A2, x, S.host(yt), orc.spmv(A2, x))
    assert gbs.gbs_mat_get_info(h) == (A.n, A.n, A.nnz)
    gbs.gbs_mat_destroy(h)


def test_spmv_argument_errors(S):
    A = I.lap2d5(8)
    h = S.mat(A)
    xv, _xt = S.zeros(A.n)
    yv, _yt = S.zeros(A.n + 1)
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_mat_mult(h, xv, yv)
    assert e.value.status == gbs.GBS_ERR_ARG
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_mat_mult(h, xv, xv)              # aliasing
    assert e.value.status == gbs.GBS_ERR_ARG
    gbs.gbs_mat_destroy(h)


def test_csr_validation_errors(S):
    A = I.lap2d5(6)
    bad = A.colidx.copy(); bad[3] = A.n
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_mat_create_aij(S.ctx, A.n, A.n, A.rowptr, bad, A.vals)
    assert e.value.status == gbs.GBS_ERR_CSR
    uns = A.colidx.copy(); uns[[0, 1]] = uns[[1, 0]]
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_mat_create_aij(S.ctx, A.n, A.n, A.rowptr, uns, A.vals)
    assert e.value.status == gbs.GBS_ERR_CSR
    rp = A.rowptr.copy(); rp[5] = rp[6] + 1
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_mat_create_aij(S.ctx, A.n, A.n, rp, A.colidx, A.vals)
    assert e.value.status == gbs.GBS_ERR_CSR


def test_empty_matrix(S):
    E = I.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    h = S.mat(E)
    xv = gbs.gbs_vec_create(S.ctx, 0)
    yv = gbs.gbs_vec_create(S.ctx, 0)
    gbs.gbs_mat_mult(h, xv, yv)
    assert gbs.gbs_mat_get_info(h) == (0, 0, 0)
    gbs.gbs_mat_destroy(h)


def test_spmv_full_size_3d7_sampled(S, orc):
    """128^3 7-point Laplacian (2,097,152 rows): sampled rows recomputed by
    the oracle one by one."""
    A = I.lap3d7(128)
    x = I.uniform_pm1(2, 0, A.n)
    y = run(S, A, x)
    rows = np.unique((I.counter_u64(9, 0, np.arange(4000)) % np.uint64(A.n)).astype(np.int64))
    rows = np.concatenate([rows, [0, A.n - 1]])
    for i in rows:
        b, e = A.rowptr[i], A.rowptr[i + 1]
        sub = I.CSR(1, np.array([0, e - b], np.int32), A.colidx[b:e].copy(), A.vals[b:e].copy())
        sub.meta["ncols"] = A.n
        ref = orc.spmv(sub, x)[0]
        absd = float(np.abs(A.vals[b:e]) @ np.abs(x[A.colidx[b:e]]))
        m = e - b
        assert abs(y[i] - ref) <= 2 * m * U / (1 - 2 * m * U) * absd
    # a property at full size: A 1 = number of Dirichlet faces per row
    ones = run(S, A, np.ones(A.n))
    c = np.arange(A.n)
    miss = sum((v == 0).astype(int) + (v == 127) for v in (c % 128, (c // 128) % 128, c // 16384))
    assert np.array_equal(ones, miss.astype(float))


def far_coupled_chain(n, seed):
    """SPD chain with one symmetric coupling between rows 0 and n - 1: a
    column more than 32767 away from its row once n > 32768, so the
    compressed 16-bit column indices cannot represent the matrix."""
    rng = np.random.default_rng(seed)
    w = 0.5 + rng.random(n - 1)
    rows, cols, vals = [], [], []
    for i in range(n):
        d = 0.1 + (w[i - 1] if i > 0 else 0.0) + (w[i] if i < n - 1 else 0.0)
        ent = []
        if i == 0:
            d += 0.25
        if i == n - 1:
            d += 0.25
        if i > 0:
            ent.append((i - 1, -w[i - 1]))
        ent.append((i, d))
        if i < n - 1:
            ent.append((i + 1, -w[i]))
        if i == 0:
            ent.append((n - 1, -0.25))
        if i == n - 1:
            ent.insert(0, (0, -0.25))
        for c, v in ent:
            rows.append(i)
            cols.append(c)
            vals.append(v)
    rowptr = np.zeros(n + 1, np.int32)
    np.add.at(rowptr, np.array(rows) + 1, 1)
    return I.CSR(n, np.cumsum(rowptr).astype(np.int32), np.array(cols, np.int32), np.array(vals))


@pytest.mark.parametrize("n", [30000, 40000])
def test_fp32_paths_with_and_without_compressed_indices(S, orc, n):
    """n = 30000 fits 16-bit relative columns, n = 40000 does not: the FP32
    MatMult is bitwise the oracle's either way, and a mixed-precision solve
    converges to the FP64 tolerance."""
    A = far_coupled_chain(n, 5)
    x = I.uniform_pm1(8, 0, n).astype(np.float32)
    assert np.array_equal(run(S, A, x, np.float32), orc.spmv_f32(A, x))
    b = orc.spmv(A, I.xstar(n, 8))
    h = S.mat(A)
    bv, bt = S.vec(b)
    xv, xt = S.zeros(n)
    info = gbs.gbs_ksp_solve_cg_ex(h, bv, xv, 1e-10, 50000, gbs.gbs_opts_default(mode=gbs.GBS_MODE_MIXED))
    assert info.status == gbs.GBS_OK
    xs = S.host(xt)
    assert np.linalg.norm(b - orc.spmv(A, xs)) <= 1e-10 * np.linalg.norm(b)
    gbs.gbs_mat_destroy(h)


@pytest.mark.parametrize("n", [30000, 40000])
def test_fp64_matmult_both_index_widths(S, orc, n):
    """FP64 MatMult streams 16-bit offsets col - row wherever they fit
    (n = 30000) and falls back to the 32-bit indices otherwise (n = 40000):
    bitwise the oracle's product on exact inputs either way, and bitwise the
    same as the 32-bit path (no_rel16) on any input, since the arithmetic
    and its order do not depend on the index width."""
    from gpu_util import Session
    A = far_coupled_chain(n, 5)
    xe = (I.counter_u64(9, 1, np.arange(n)) % np.uint64(17)).astype(np.float64) - 8.0
    Ae = I.CSR(n, A.rowptr, A.colidx, np.round(A.vals * 8.0) / 8.0)
    assert np.array_equal(run(S, Ae, xe), orc.spmv(Ae, xe))
    S32 = Session(gbs.gbs_opts_default(no_rel16=1))
    x = I.uniform_pm1(8, 1, n)
    assert np.array_equal(run(S, A, x), run(S32, A, x))
    assert np.array_equal(run(S32, Ae, xe), orc.spmv(Ae, xe))
    gbs.gbs_ctx_destroy(S32.ctx)


def test_fp64_matmult_index_widths_on_stencils(S, orc):
    """The 7-point and 27-point operators (every offset fits 16 bits): the
    16-bit and 32-bit FP64 MatMult agree bitwise, and both meet the 1e-13
    bound against the oracle."""
    from gpu_util import Session
    S32 = Session(gbs.gbs_opts_default(no_rel16=1))
    for A in (I.lap3d7(40), I.var27(22, seed=3)):
        x = I.uniform_pm1(4, 2, A.n)
        y16, y32 = run(S, A, x), run(S32, A, x)
        assert np.array_equal(y16, y32)
        ref = orc.spmv(A, x)
        assert np.linalg.norm(y16 - ref) <= 1e-13 * np.linalg.norm(ref)
    gbs.gbs_ctx_destroy(S32.ctx)


def exact_version(A, ncols, seed):
    """A copy of A with values on a 1/8 grid in [-64, 64] and an integer x in
    [-8, 8]: every product and partial sum is exact in FP32 and FP64, so any
    summation order gives the oracle's bits."""
    Ae = I.CSR(A.n, A.rowptr, A.colidx, np.round(np.clip(A.vals, -64, 64) * 8.0) / 8.0)
    Ae.meta["ncols"] = ncols
    xe = (I.counter_u64(seed, 3, np.arange(ncols)) % np.uint64(17)).astype(np.float64) - 8.0
    return Ae, xe


LANE_CASES = {
    "var27_13": lambda: I.var27(13, seed=3),
    "lap3d7_20": lambda: I.lap3d7(20),
    "random_rect": lambda: I.random_csr(700, 1300, 11, seed=2),
    "empty_and_long_rows": with_empty_and_long_rows,
}


@pytest.mark.parametrize("lanes", [1, 2, 4])
@pytest.mark.parametrize("name", sorted(LANE_CASES))
def test_spmv_lanes_per_row(orc, name, lanes):
    """Every lanes-per-row tiling of MatMult: bitwise the oracle on exact
    inputs in both precisions; on random inputs FP64 within 2 gamma_m
    (|A||x|) and FP32 within gamma_m (|A32||x32|) (u = 2^-24) of the exact
    product of its FP32 operands."""
    from gpu_util import Session
    S = Session(gbs.gbs_opts_default(spmv_lanes=lanes))
    A = LANE_CASES[name]()
    ncols = A.meta.get("ncols", A.n)
    Ae, xe = exact_version(A, ncols, 5)
    assert np.array_equal(run(S, Ae, xe), orc.spmv(Ae, xe))
    assert np.array_equal(run(S, Ae, xe.astype(np.float32), np.float32),
                          orc.spmv_f32(Ae, xe.astype(np.float32)))
    x = I.uniform_pm1(21, 0, ncols)
    assert_within_bounds(orc, A, x, run(S, A, x), orc.spmv(A, x))
    x32 = x.astype(np.float32)
    y32 = run(S, A, x32, np.float32).astype(np.float64)
    A32 = I.CSR(A.n, A.rowptr, A.colidx, A.vals.astype(np.float32).astype(np.float64))
    A32.meta["ncols"] = ncols
    ref = orc.spmv(A32, x32.astype(np.float64))
    absA = I.CSR(A.n, A.rowptr, A.colidx, np.abs(A32.vals))
    absA.meta["ncols"] = ncols
    m = np.diff(A.rowptr)
    u32 = 2.0 ** -24
    g = m * u32 / (1 - m * u32)
    # the FP64 reference rounds too: 2^-50 of |A||x| covers it
    assert np.all(np.abs(y32 - ref) <= (g + 2.0 ** -50) * orc.spmv(absA, np.abs(x32.astype(np.float64))))
    gbs.gbs_ctx_destroy(S.ctx)


def test_spmv_default_lanes_rule(S, orc):
    """By default rows of more than 16 nonzeros take 2 lanes and shorter rows
    one: the default results are bitwise those of the explicit setting."""
    from gpu_util import Session
    S1_, S2_ = (Session(gbs.gbs_opts_default(spmv_lanes=k)) for k in (1, 2))
    for A, same in ((I.var27(13, seed=3), S2_), (I.lap3d7(20), S1_)):
        x = I.uniform_pm1(22, 0, A.n)
        for dt in (np.float64, np.float32):
            xx = x.astype(dt)
            assert np.array_equal(run(S, A, xx, dt), run(same, A, xx, dt))
    for s_ in (S1_, S2_):
        gbs.gbs_ctx_destroy(s_.ctx)


def test_spmv_lanes_option_refused():
    from gpu_util import Session
    with pytest.raises(Exception):
        Session(gbs.gbs_opts_default(spmv_lanes=3))
