"""Multi-rank host logic on CPU (gloo, world size 2): the replica path of
the batched and serving workloads (independent systems assigned to ranks,
results gathered, job throughput = all ranks' units over the slowest rank's
time).  The per-rank solves here are the oracle's, standing in for each
rank's GPU engine; what is tested is that every system is solved exactly
once and the gathered results equal a single-process run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2011_00715_gb300 import inputs as I
from paper_2011_00715_gb300 import shard


def test_lpt_assignment_is_complete_balanced_and_deterministic():
    rng = np.random.default_rng(3)
    costs = list(rng.lognormal(0.0, 1.0, 200))
    for world in (1, 2, 3, 8):
        a = shard.lpt_assign(costs, world)
        assert a == shard.lpt_assign(costs, world)
        assert sorted(set(a)) == list(range(min(world, len(costs))))
        loads = [sum(c for c, r in zip(costs, a) if r == k) for k in range(world)]
        lower = max(sum(costs) / world, max(costs))           # no schedule does better
        assert max(loads) <= (4 / 3 - 1 / (3 * world)) * lower * (1 + 1e-12) or world == 1
        shares = [shard.my_share(costs, k, world) for k in range(world)]
        assert sorted(i for s in shares for i in s) == list(range(len(costs)))
    assert shard.lpt_assign([], 4) == []
    with pytest.raises(ValueError):
        shard.lpt_assign([1.0], 0)


def test_solve_cost_grows_with_size_and_columns():
    assert shard.solve_cost(8000, 56000, 1) < shard.solve_cost(64000, 448000, 1)
    assert shard.solve_cost(8000, 56000, 1) < shard.solve_cost(8000, 56000, 4)


def _systems():
    specs = [("var7", (9, 8, 7)), ("var5", (30, 25)), ("var7", (12, 11, 10)),
             ("var5", (16, 40)), ("var7", (6, 6, 6)), ("var5", (50, 9)), ("var7", (14, 5, 9))]
    out = []
    for i, (fam, dims) in enumerate(specs):
        A = I.family_matrix(fam, dims, seed=70 + i, sigma=0.5)
        out.append(A)
    return out


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        systems = _systems()
        costs = [shard.solve_cost(A.n, A.nnz, 1) for A in systems]
        mine = shard.my_share(costs, rank, world)
        local = {}
        for i in mine:
            A = systems[i]
            b = orc.spmv(A, I.xstar(A.n, 12, system=i))
            r = orc.pcg(A, b, 1e-10, 20000)
            local[i] = (r["status"], r["iters"], r["x"])
        allres = shard.gather_results(local, world)
        thr = shard.job_throughput(len(mine), 1.0 + rank)       # rank r "took" r + 1 seconds
        if rank == 0:
            np.savez(os.path.join(out_dir, "res.npz"),
                     idx=np.array(sorted(allres)), thr=np.array([thr]),
                     **{f"x{i}": allres[i][2] for i in allres},
                     st=np.array([allres[i][0] for i in sorted(allres)]),
                     it=np.array([allres[i][1] for i in sorted(allres)]))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_ranks_solve_every_system_once(tmp_path, orc):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    d = np.load(tmp_path / "res.npz")
    systems = _systems()
    assert list(d["idx"]) == list(range(len(systems)))
    assert float(d["thr"][0]) == pytest.approx(len(systems) / 2.0)
    for i, A in enumerate(systems):
        b = orc.spmv(A, I.xstar(A.n, 12, system=i))
        r = orc.pcg(A, b, 1e-10, 20000)
        assert d["st"][i] == r["status"] == 0 and d["it"][i] == r["iters"]
        assert np.array_equal(d[f"x{i}"], r["x"])
