"""Serving loop (continuous batching) against the oracle (GPU).

Requests are admitted by a device-memory budget and free slots; requests
that arrive while others run join at the next quantum; each result is
checked against the oracle (true FP64 residual, solution within the
stopping rule's guarantee), and a request's result is bitwise the same
alone and in the mix.
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


def request(orc, i, dims, k):
    A = I.var27(*dims, seed=900 + i, sigma=1.0)
    b = np.concatenate([orc.spmv(A, I.xstar(A.n, 31, column=c, system=i)) for c in range(k)])
    return A, b


def submit(srv, A, b, k, rtol=1e-10, maxit=20000):
    return gbs.gbs_server_submit(srv, A.n, A.rowptr, A.colidx, A.vals, k, b, rtol, maxit)


def check(orc, A, b, k, x, sts):
    assert list(sts) == [gbs.GBS_OK] * k
    for c in range(k):
        bc, xc = b[c * A.n:(c + 1) * A.n], x[c * A.n:(c + 1) * A.n]
        assert np.linalg.norm(bc - orc.spmv(A, xc)) <= 1e-10 * np.linalg.norm(bc)
        ref = orc.pcg(A, bc, 1e-10, 20000)
        # lambda_min >= w_min * (14 - 6c - 6c^2 - 2c^3) for the 27-point family
        nx, ny, nz = A.meta["dims"]
        import math
        cs = [math.cos(math.pi / (d + 1)) for d in (nx, ny, nz)]
        lam_unit = (14 - 2 * sum(cs) - 2 * (cs[0] * cs[1] + cs[0] * cs[2] + cs[1] * cs[2])
                    - 2 * cs[0] * cs[1] * cs[2])
        lmin = A.meta["w_min"] * lam_unit
        bound = (np.linalg.norm(bc - orc.spmv(A, xc)) + np.linalg.norm(bc - orc.spmv(A, ref["x"]))) / lmin
        from gpu_util import record
        nr = np.linalg.norm(ref["x"])
        record(f"server[n={A.n},col={c}]", "rel_err_vs_oracle", np.linalg.norm(xc - ref["x"]) / nr,
               max(1e-8, bound / nr))
        assert np.linalg.norm(xc - ref["x"]) <= max(1e-8 * np.linalg.norm(ref["x"]), bound)


def test_server_continuous_batching(S, orc):
    srv = gbs.gbs_server_create(S.ctx, 8 << 30, 0, gbs.GBS_MODE_MIXED)
    # the first request is large enough to need many quanta of the engine,
    # so it is still running when the last two arrive
    reqs = [request(orc, i, d, k) for i, (d, k) in
            enumerate([((34, 32, 30), 2), ((9, 9, 9), 1), ((20, 18, 17), 4), ((6, 7, 5), 3)])]
    tickets = {}
    # the first two arrive, the engine runs, the others arrive while they are on the GPU
    for i in (0, 1):
        A, b = reqs[i]
        tickets[i] = submit(srv, A, b, [2, 1, 4, 3][i])
    gbs.gbs_server_progress(srv)
    q, running, fin, used = gbs.gbs_server_stats(srv)
    assert running >= 1 and used > 0
    for i in (2, 3):
        A, b = reqs[i]
        tickets[i] = submit(srv, A, b, [2, 1, 4, 3][i])
    overlap = False
    for _ in range(100000):
        gbs.gbs_server_progress(srv)
        q, running, fin, used = gbs.gbs_server_stats(srv)
        overlap |= running >= 3
        if fin == 4:
            break
    assert fin == 4 and overlap
    for i, (A, b) in enumerate(reqs):
        k = [2, 1, 4, 3][i]
        assert gbs.gbs_server_poll(srv, tickets[i])
        x, its, rns, sts = gbs.gbs_server_fetch(srv, tickets[i], A.n, k)
        check(orc, A, b, k, x, sts)
    with pytest.raises(gbs.GbsError) as e:
        gbs.gbs_server_fetch(srv, tickets[0], reqs[0][0].n, 2)
    assert e.value.status == gbs.GBS_ERR_NOT_FOUND
    gbs.gbs_server_destroy(srv)


def test_server_result_same_alone_and_in_mix(S, orc):
    A, b = request(orc, 7, (16, 15, 14), 2)
    srv = gbs.gbs_server_create(S.ctx, 8 << 30, 0, gbs.GBS_MODE_MIXED)
    t = submit(srv, A, b, 2)
    gbs.gbs_server_wait(srv, t)
    x_alone = gbs.gbs_server_fetch(srv, t, A.n, 2)[0]
    gbs.gbs_server_destroy(srv)
    srv = gbs.gbs_server_create(S.ctx, 8 << 30, 0, gbs.GBS_MODE_MIXED)
    others = [request(orc, 20 + i, d, 1) for i, d in enumerate([(10, 10, 10), (22, 20, 19)])]
    ts = [submit(srv, Ao, bo, 1) for Ao, bo in others]
    gbs.gbs_server_progress(srv)
    t = submit(srv, A, b, 2)
    gbs.gbs_server_wait(srv, t)
    x_mix = gbs.gbs_server_fetch(srv, t, A.n, 2)[0]
    assert np.array_equal(x_alone, x_mix)
    for tt in ts:
        gbs.gbs_server_wait(srv, tt)
    gbs.gbs_server_destroy(srv)


def test_server_budget_admission(S, orc):
    A, b = request(orc, 3, (12, 12, 12), 1)
    srv = gbs.gbs_server_create(S.ctx, 256 << 10, 0, gbs.GBS_MODE_MIXED)   # 256 KiB
    with pytest.raises(gbs.GbsError) as e:
        submit(srv, A, b, 1)
    assert e.value.status == gbs.GBS_ERR_BUDGET
    gbs.gbs_server_destroy(srv)
    # a budget that holds one request at a time: the second waits in the queue
    one = 0
    srv = gbs.gbs_server_create(S.ctx, 1 << 20, 0, gbs.GBS_MODE_MIXED)    # holds one
    t1 = submit(srv, A, b, 1)
    t2 = submit(srv, A, b, 1)
    gbs.gbs_server_progress(srv)
    q, running, fin, used = gbs.gbs_server_stats(srv)
    assert running + fin >= 1 and used <= 1 << 20
    if fin == 0:
        assert q == 1 and running == 1
        one = 1
    gbs.gbs_server_wait(srv, t1)
    gbs.gbs_server_wait(srv, t2)
    x1 = gbs.gbs_server_fetch(srv, t1, A.n, 1)
    x2 = gbs.gbs_server_fetch(srv, t2, A.n, 1)
    assert np.array_equal(x1[0], x2[0])
    check(orc, A, b, 1, x1[0], x1[3])
    assert one == 1
    gbs.gbs_server_destroy(srv)


def test_server_malformed_and_degenerate_requests(S, orc):
    srv = gbs.gbs_server_create(S.ctx, 1 << 30, 0, gbs.GBS_MODE_MIXED)
    A = I.lap2d5(6)
    bad = A.colidx.copy(); bad[3] = A.n
    t_bad = gbs.gbs_server_submit(srv, A.n, A.rowptr, bad, A.vals, 1, np.ones(A.n), 1e-10, 100)
    C = I.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, -2.0]))
    t_diag = gbs.gbs_server_submit(srv, 2, C.rowptr, C.colidx, C.vals, 1, np.ones(2), 1e-10, 100)
    t_zero = gbs.gbs_server_submit(srv, A.n, A.rowptr, A.colidx, A.vals, 1, np.zeros(A.n),
                                   1e-10, 100)
    for t in (t_bad, t_diag, t_zero):
        gbs.gbs_server_wait(srv, t)
    assert gbs.gbs_server_fetch(srv, t_bad, A.n, 1)[3][0] == gbs.GBS_ERR_CSR
    assert gbs.gbs_server_fetch(srv, t_diag, 2, 1)[3][0] == gbs.GBS_ERR_DIAG
    x, its, rns, sts = gbs.gbs_server_fetch(srv, t_zero, A.n, 1)
    assert sts[0] == gbs.GBS_OK and its[0] == 0 and not x.any()
    q, running, fin, used = gbs.gbs_server_stats(srv)
    assert q == 0 and running == 0 and used == 0
    gbs.gbs_server_destroy(srv)


def test_server_slot_reuse_with_different_sizes(S, orc):
    """One slot: every request lands in the same slot in turn, each with a
    different size, so the engine must rebuild its active lists per request."""
    srv = gbs.gbs_server_create(S.ctx, 1 << 30, 1, gbs.GBS_MODE_MIXED)
    reqs = [request(orc, 40 + i, d, k) for i, (d, k) in
            enumerate([((11, 10, 9), 1), ((5, 5, 4), 2), ((15, 14, 13), 1), ((8, 8, 8), 3)])]
    ks = [1, 2, 1, 3]
    ts = [submit(srv, A, b, k) for (A, b), k in zip(reqs, ks)]
    for t in ts:
        gbs.gbs_server_wait(srv, t)
    for (A, b), k, t in zip(reqs, ks, ts):
        x, its, rns, sts = gbs.gbs_server_fetch(srv, t, A.n, k)
        check(orc, A, b, k, x, sts)
    gbs.gbs_server_destroy(srv)


def test_server_borrowed_submit_matches_copy(S, orc):
    """A borrowed-array request gives bitwise the result of a copied one;
    the engine's time counters add up."""
    A, b = request(orc, 7, (15, 14, 13), 3)
    out = []
    for borrowed in (False, True):
        srv = gbs.gbs_server_create(S.ctx, 8 << 30, 0, gbs.GBS_MODE_MIXED)
        f = gbs.gbs_server_submit_borrowed if borrowed else gbs.gbs_server_submit
        t = f(srv, A.n, A.rowptr, A.colidx, A.vals, 3, b, 1e-10, 20000)
        gbs.gbs_server_wait(srv, t)
        ta, tq, tr, nq = gbs.gbs_server_times(srv)
        assert nq >= 1 and tq > 0.0 and ta > 0.0 and tr >= 0.0
        out.append(gbs.gbs_server_fetch(srv, t, A.n, 3))
        gbs.gbs_server_destroy(srv)
    check(orc, A, b, 3, out[1][0], out[1][3])
    assert np.array_equal(out[0][0], out[1][0])
