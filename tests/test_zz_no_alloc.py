"""The allocation-free FP64 solve (gbs_ksp_solve_cg_noalloc) gives the same
result as the regular solve entry point, on two calls in a row.

It serves callers that cannot allocate device memory while they solve
(latency-bound loops, where cudaMalloc/cudaFree can synchronise the device,
and processes whose device memory belongs to another allocator's pool).
Its workspace is one fixed array in the library's device image that every
call reuses, so the second call also checks that leftovers of the first
do not leak into the result.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2011_00715_gb300 import gbs
from paper_2011_00715_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NOALLOC_MAX_ROWS = 262144


def test_noalloc_solve_matches_regular_solve_twice(orc):
    import torch
    torch.cuda.set_device(0)
    ctx = gbs.gbs_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    A = I.var7(40, 36, 30, seed=11)                       # 43,200 rows
    xs = I.xstar(A.n, 12)
    b = orc.spmv(A, xs)
    h = gbs.gbs_mat_create_aij(ctx, A.n, A.n, A.rowptr, A.colidx, A.vals)
    bt = torch.from_numpy(b).cuda()
    bv = gbs.gbs_vec_wrap(ctx, bt)
    x_ref_t = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    xv = gbs.gbs_vec_wrap(ctx, x_ref_t)
    ref = gbs.gbs_ksp_solve_cg_ex(h, bv, xv, 1e-10, 20000,
                                  gbs.gbs_opts_default(algorithm=gbs.GBS_ALG_PERSISTENT))
    assert ref.status == gbs.GBS_OK
    x_ref = x_ref_t.cpu().numpy()

    x_t = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    for call in range(2):
        x_t.zero_()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        info = gbs.gbs_ksp_solve_cg_noalloc(h, bt, x_t, 1e-10, 20000)
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the module; the second must not allocate
            assert torch.cuda.mem_get_info()[0] == free_before
        assert info.status == gbs.GBS_OK
        assert abs(info.iters - ref.iters) <= 2
        x = x_t.cpu().numpy()
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
        assert np.linalg.norm(b - orc.spmv(A, x)) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-3)
        assert abs(info.bnorm - np.linalg.norm(b)) <= 1e-12 * np.linalg.norm(b)

    # the binding refuses vectors of the wrong length or on another device
    # before the C entry point (which sees bare pointers) could run past
    # their ends
    short = torch.zeros(A.n - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        gbs.gbs_ksp_solve_cg_noalloc(h, short, x_t, 1e-10, 100)
    with pytest.raises(ValueError):
        gbs.gbs_ksp_solve_cg_noalloc(h, bt, short, 1e-10, 100)
    assert gbs.gbs_mat_get_device(h) == 0
    if torch.cuda.device_count() > 1:
        other = torch.zeros(A.n, dtype=torch.float64, device="cuda:1")
        with pytest.raises(ValueError):
            gbs.gbs_ksp_solve_cg_noalloc(h, other, x_t, 1e-10, 100)
    # the result is the context's last solve as well
    last = gbs.gbs_ksp_last_info(ctx)
    assert last.status == gbs.GBS_OK and last.iters == info.iters

    # sizes beyond the fixed workspace are refused with GBS_ERR_ARG
    big = I.lap3d7(65)                                      # 274,625 rows > 262,144
    hb = gbs.gbs_mat_create_aij(ctx, big.n, big.n, big.rowptr, big.colidx, big.vals)
    tb = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    tx = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_ksp_solve_cg_noalloc(hb, tb, tx, 1e-10, 100)
    assert e.value.status == gbs.GBS_ERR_ARG
    assert big.n > NOALLOC_MAX_ROWS
    gbs.gbs_mat_destroy(hb)
    for v in (bv, xv):
        gbs.gbs_vec_destroy(v)
    gbs.gbs_mat_destroy(h)
    gbs.gbs_ctx_destroy(ctx)
