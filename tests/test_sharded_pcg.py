"""The sharded single-system PCG (row blocks, halo exchange, two
all-reduces per iteration) run as gloo ranks on CPU, with the oracle's SpMV
as each rank's local product: the partition, the halo plan and the
collective schedule against the single-domain oracle solve."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2011_00715_gb300 import inputs as I
from paper_2011_00715_gb300 import sharded


def test_row_blocks_balance_nonzeros():
    A = I.var27(10, seed=2)
    for world in (1, 2, 3, 7):
        cuts = sharded.row_blocks(A.rowptr, world)
        assert cuts[0] == 0 and cuts[-1] == A.n and all(a <= b for a, b in zip(cuts, cuts[1:]))
        loads = [int(A.rowptr[b] - A.rowptr[a]) for a, b in zip(cuts, cuts[1:])]
        assert max(loads) - min(loads) <= 2 * max(np.diff(A.rowptr))


def test_local_blocks_reassemble_the_matrix():
    A = I.var7(9, 8, 7, seed=3)
    cuts = sharded.row_blocks(A.rowptr, 3)
    dense = np.zeros((A.n, A.n))
    for r in range(3):
        blk = sharded.local_block(A.rowptr, A.colidx, A.vals, cuts, r)
        glob = np.concatenate([np.arange(blk.lo, blk.hi), blk.ghosts])
        for i in range(blk.n_own):
            seg = slice(blk.rowptr[i], blk.rowptr[i + 1])
            dense[blk.lo + i, glob[blk.colidx[seg]]] += blk.vals[seg]
        owners = np.searchsorted(cuts[1:], blk.ghosts, side="right")
        assert not np.any((blk.ghosts >= blk.lo) & (blk.ghosts < blk.hi))
        assert all(np.all(owners[off:off + cnt] == q) for q, (off, cnt) in blk.recv.items())
    ref = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ref[rows, A.colidx] = A.vals
    assert np.array_equal(dense, ref)


def _local_spmv(blk, v):
    import oracle as orc
    return orc.spmv(I.CSR(blk.n_own, blk.rowptr, blk.colidx, blk.vals), v)


class _NoBlockingDotOps(sharded.NumpyOps):
    """The driver must take its dot products through dots() (partials left
    where the all-reduce reads them), never through a blocking dot()."""
    def dot(self, a, b):
        raise AssertionError("blocking dot product in the sharded driver")

    def dots(self, pairs):
        import torch
        return torch.tensor([sharded.NumpyOps.dot(self, a, b) for a, b in pairs],
                            dtype=torch.float64)


def _worker(rank, world, port, out_dir, maker):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = maker()
        cuts = sharded.row_blocks(A.rowptr, world)
        blk = sharded.exchange_plans(sharded.local_block(A.rowptr, A.colidx, A.vals, cuts, rank))
        # the halo brings every ghost's owner value
        v = torch.zeros(blk.ncols, dtype=torch.float64)
        v[: blk.n_own] = torch.arange(blk.lo, blk.hi, dtype=torch.float64)
        sharded.halo_exchange(blk, v)
        assert torch.equal(v[blk.n_own:], torch.as_tensor(blk.ghosts, dtype=torch.float64))
        import oracle as orc
        b = orc.spmv(A, I.xstar(A.n, 21))
        x, st, k, rn, bn = sharded.sharded_pcg(blk, _NoBlockingDotOps(_local_spmv),
                                               b[blk.lo:blk.hi], 1e-10, 20000)
        parts = [None] * world
        dist.all_gather_object(parts, (blk.lo, x.numpy(), st, k, rn, bn))
        if rank == 0:
            full = np.zeros(A.n)
            for lo, xp, *_ in parts:
                full[lo:lo + len(xp)] = xp
            np.savez(os.path.join(out_dir, "res.npz"), x=full,
                     st=np.array([p[2] for p in parts]), k=np.array([p[3] for p in parts]),
                     rn=np.array([p[4] for p in parts]), bn=np.array([p[5] for p in parts]))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _lap():
    return I.lap3d7(14, 12, 10)


def _var():
    return I.var27(11, seed=6)


@pytest.mark.parametrize("world,maker", [(2, _lap), (3, _var)])
def test_sharded_pcg_matches_single_domain(tmp_path, orc, world, maker):
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), maker), nprocs=world, join=True)
    d = np.load(tmp_path / "res.npz")
    A = maker()
    b = orc.spmv(A, I.xstar(A.n, 21))
    ref = orc.pcg(A, b, 1e-10, 20000)
    # every rank ends with the same status, count and norms (all-reduced scalars)
    assert np.all(d["st"] == 0) and len(set(d["k"])) == 1 and len(set(d["rn"])) == 1
    assert abs(int(d["k"][0]) - ref["iters"]) <= 2
    assert np.linalg.norm(b - orc.spmv(A, d["x"])) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
    assert np.linalg.norm(d["x"] - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])


@pytest.mark.gpu
def test_sharded_pcg_library_backend_one_rank(orc):
    """The library backend (local SpMV, Jacobi, AXPY/AYPX and dots in the
    library on the GPU,
    NCCL collectives) on a one-rank group: the same iteration as the
    single-GPU solve, within rounding."""
    import torch
    import torch.distributed as dist
    from paper_2011_00715_gb300 import gbs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        A = I.var7(20, 18, 16, seed=13)
        b = orc.spmv(A, I.xstar(A.n, 3))
        ctx = gbs.gbs_ctx_create(0, torch.cuda.current_stream().cuda_stream)
        blk = sharded.exchange_plans(sharded.local_block(A.rowptr, A.colidx, A.vals,
                                                         sharded.row_blocks(A.rowptr, 1), 0))
        ops = sharded.GbsOps(ctx, blk)
        x, st, k, rn, bn = sharded.sharded_pcg(blk, ops, b, 1e-10, 20000)
        ops.close()
        ref = orc.pcg(A, b, 1e-10, 20000)
        assert st == 0 and abs(k - ref["iters"]) <= 2
        xh = x.cpu().numpy()
        assert np.linalg.norm(b - orc.spmv(A, xh)) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
        assert np.linalg.norm(xh - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
        gbs.gbs_ctx_destroy(ctx)
    finally:
        dist.destroy_process_group()
