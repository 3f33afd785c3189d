"""Vector operations and the Jacobi apply against the oracle (GPU).

Elementwise operations round each multiply and add separately, as their
definitions do, so they are bitwise equal to the oracle.  Dot products are
reduced by a fixed tree: bitwise on exact inputs, otherwise within Higham's
order-free bound |fl(x.y) - x.y| <= gamma_n |x|.|y|.
"""
import math

import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def S():
    from gpu_util import Session
    return Session()


SIZES = [1, 31, 1000, 65537, 3_000_001]


@pytest.mark.parametrize("n", SIZES)
def test_axpy_aypx_pointwise_copy_set(S, orc, n):
    x = I.uniform_pm1(1, 0, n)
    y = I.uniform_pm1(1, 1, n)
    xv, xt = S.vec(x)
    yv, yt = S.vec(y)
    # one fused multiply-add per entry: bitwise the oracle's fused form
    gbs.gbs_vec_axpy(yv, -0.37, xv)
    assert np.array_equal(S.host(yt), orc.axpy_fused(-0.37, x, y))
    y2 = S.host(yt).copy()
    gbs.gbs_vec_aypx(yv, 1.9, xv)
    assert np.array_equal(S.host(yt), orc.aypx_fused(1.9, x, y2))
    wv, wt = S.zeros(n)
    gbs.gbs_vec_pointwise_mult(wv, xv, yv)
    assert np.array_equal(S.host(wt), x * S.host(yt))
    gbs.gbs_vec_copy(xv, wv)
    assert np.array_equal(S.host(wt), x)
    gbs.gbs_vec_set(wv, 2.5)
    assert np.all(S.host(wt) == 2.5)


@pytest.mark.parametrize("n", SIZES)
def test_dot_norm_fp64(S, orc, n):
    x = I.uniform_pm1(2, 0, n)
    y = I.uniform_pm1(2, 1, n)
    xv, _ = S.vec(x)
    yv, _ = S.vec(y)
    d = gbs.gbs_vec_dot(xv, yv)
    exact = orc.dot2(x, y)
    g = n * U64 / (1 - n * U64)
    assert abs(d - exact) <= g * float(np.abs(x) @ np.abs(y)) + U64 * abs(exact)
    nr = gbs.gbs_vec_norm2(xv)
    assert abs(nr - math.sqrt(orc.dot2(x, x))) <= 2 * g * nr + 1e-300
    # a fixed reduction order: repeated calls give identical bits
    assert gbs.gbs_vec_dot(xv, yv) == d


def test_dot_norm_async_stream_order(S):
    """The asynchronous forms write the same bits as the synchronous ones
    into caller-owned device memory, in stream order: a torch operation
    queued after them on the same stream reads the results."""
    import ctypes
    import torch
    out = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
    res = []
    for k, n in enumerate((31, 65537, 3_000_001)):
        x = I.uniform_pm1(6, k, n)
        y = I.uniform_pm1(6, k + 10, n)
        xv, xt = S.vec(x)
        yv, yt = S.vec(y)
        gbs.gbs_vec_dot_async(xv, yv, out[2 * k:])
        gbs.gbs_vec_norm2_async(xv, out[2 * k + 1:])
        res.append((xv, yv, xt, yt))   # the tensors own the vectors' memory
    doubled = out * 2.0            # queued behind the writes on the same stream
    host = doubled.cpu().numpy() / 2.0
    for k, (xv, yv, _, _) in enumerate(res):
        assert host[2 * k] == gbs.gbs_vec_dot(xv, yv)
        assert host[2 * k + 1] == gbs.gbs_vec_norm2(xv)
    # FP32: the FP32 result widened
    x32 = I.uniform_pm1(7, 0, 100_003).astype(np.float32)
    v32, t32 = S.vec(x32, np.float32)
    gbs.gbs_vec_norm2_async(v32, out[6:])
    gbs.gbs_vec_dot_async(v32, v32, out[7:])
    torch.cuda.current_stream().synchronize()
    assert out[6].item() == gbs.gbs_vec_norm2(v32)
    assert out[7].item() == gbs.gbs_vec_dot(v32, v32)
    # empty vectors give 0; misaligned or missing pointers are refused
    e0 = gbs.gbs_vec_create(S.ctx, 0)
    gbs.gbs_vec_norm2_async(e0, out[0:])
    torch.cuda.current_stream().synchronize()
    assert out[0].item() == 0.0
    assert gbs.lib().gbs_vec_dot_async(res[0][0], res[0][1],
                                       ctypes.c_void_p(out.data_ptr() + 4)) == gbs.GBS_ERR_ARG
    assert gbs.lib().gbs_vec_norm2_async(res[0][0], None) == gbs.GBS_ERR_ARG
    gbs.gbs_vec_destroy(e0)


def test_dot_exact_inputs(S):
    n = 2_000_000
    x = I.exact_vector(n, seed=3)
    y = np.round(I.uniform_pm1(3, 5, n) * 4)
    kx = np.round(x * 2 ** 20).astype(np.int64)
    exact = int(np.sum(kx * y.astype(np.int64))) / 2 ** 20
    xv, _ = S.vec(x)
    yv, _ = S.vec(y)
    assert gbs.gbs_vec_dot(xv, yv) == exact


def test_dot_fp32(S, orc):
    n = 1_000_003
    x = I.uniform_pm1(4, 0, n).astype(np.float32)
    y = I.uniform_pm1(4, 1, n).astype(np.float32)
    xv, _ = S.vec(x, np.float32)
    yv, _ = S.vec(y, np.float32)
    d = gbs.gbs_vec_dot(xv, yv)
    exact = orc.dot2(x.astype(np.float64), y.astype(np.float64))
    # tree accumulation in FP32: depth ~ log2(n) + per-thread chain
    assert abs(d - exact) <= 64 * U32 * float(np.abs(x.astype(np.float64)) @ np.abs(y.astype(np.float64)))


def test_jacobi_apply(S, orc):
    A = I.var7(20, 20, 20, seed=9)
    h = S.mat(A)
    pc = gbs.gbs_pc_jacobi_create(h)
    r = I.uniform_pm1(5, 0, A.n)
    rv, _ = S.vec(r)
    zv, zt = S.zeros(A.n)
    gbs.gbs_pc_apply(pc, rv, zv)
    st, dinv = orc.jacobi_dinv(A)
    assert st == 0 and np.array_equal(S.host(zt), dinv * r)
    gbs.gbs_pc_destroy(pc)
    gbs.gbs_mat_destroy(h)


def test_jacobi_rejects_bad_diagonal(S):
    C = I.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, -2.0]))
    h = S.mat(C)
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_pc_jacobi_create(h)
    assert e.value.status == gbs.GBS_ERR_DIAG
    gbs.gbs_mat_destroy(h)


def test_vector_values_roundtrip_and_errors(S):
    v = gbs.gbs_vec_create(S.ctx, 1000)
    src = I.uniform_pm1(6, 0, 1000)
    gbs.gbs_vec_set_values(v, src)
    out = np.empty(1000)
    gbs.gbs_vec_get_values(v, out)
    assert np.array_equal(out, src)
    assert gbs.gbs_vec_get_info(v)[:2] == (1000, gbs.GBS_F64)
    w = gbs.gbs_vec_create(S.ctx, 999)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_vec_axpy(v, 1.0, w)
    with pytest.raises(gbs.GbsError):
        gbs.gbs_vec_dot(v, w)
    gbs.gbs_vec_destroy(v)
    gbs.gbs_vec_destroy(w)
    e = gbs.gbs_vec_create(S.ctx, 0)
    assert gbs.gbs_vec_dot(e, e) == 0.0
    gbs.gbs_vec_destroy(e)


def test_fp64_rate_probe(S):
    """The FP64 FMA-rate probe (the FP64 roofline's denominator) returns a
    rate between 1/20 and 2x of the nominal 625 G FMA/s of a GB300, scales
    its work with iters, and refuses bad arguments."""
    r1 = gbs.gbs_probe_fp64_rate(S.ctx, 2048)
    r2 = gbs.gbs_probe_fp64_rate(S.ctx, 8192)
    for r in (r1, r2):
        assert 625e9 / 20 < r < 2 * 625e9, r
    assert abs(r1 - r2) <= 0.25 * r2
    assert gbs.lib().gbs_probe_fp64_rate(S.ctx, 0, None) == gbs.GBS_ERR_ARG
    import ctypes
    v = ctypes.c_double()
    assert gbs.lib().gbs_probe_fp64_rate(S.ctx, 0, ctypes.byref(v)) == gbs.GBS_ERR_ARG
    assert gbs.lib().gbs_probe_fp64_rate(S.ctx, (1 << 24) + 1, ctypes.byref(v)) == gbs.GBS_ERR_ARG
