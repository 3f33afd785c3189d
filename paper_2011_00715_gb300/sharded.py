"""One Jacobi-PCG solve sharded over ranks (row blocks, halo exchange and
two scalar all-reduces per iteration).

The matrix is split into contiguous row blocks balanced by nonzeros (slabs
of a lexicographic grid).  Each rank keeps its rows with their columns
renumbered: its own columns first, then the ghost columns it reads from
other ranks, grouped by owner.  Before each SpMV the owners send the ghost
values of the direction vector (the PetscSF broadcast of Sec. 4 / Response
A4, here point-to-point messages); the dot products are local partials
summed by an all-reduce.  The iteration is the same textbook PCG as the
single-GPU kernels (stopping test before each iteration on the
unpreconditioned residual).

The driver is written once over a small "local operations" interface, so
the partition, the halo plan and the collective schedule are the same code
whether the local work runs in the library on a GPU (GbsOps, NCCL: the
SpMV, Jacobi apply, AXPY/AYPX, copies and dots all in the library's
kernels) or, in the CPU tests, in another implementation (gloo ranks).
The scalar recurrence runs here, on the host, on the all-reduced sums: per
iteration the host waits twice, for the results of the two all-reduces
(the dot products feeding each are left on the device).
"""
from __future__ import annotations

import bisect
from dataclasses import dataclass, field

import numpy as np


def row_blocks(rowptr: np.ndarray, world: int) -> list[int]:
    """Row boundaries r_0 = 0 <= r_1 <= ... <= r_world = n: block k holds
    rows [r_k, r_k+1), cut where the running nonzero count crosses k/world
    of the total (a row is never split)."""
    n = len(rowptr) - 1
    nnz = int(rowptr[-1])
    cuts = [0]
    for k in range(1, world):
        target = nnz * k / world
        r = bisect.bisect_left(rowptr.tolist(), target)
        cuts.append(min(max(r, cuts[-1]), n))
    cuts.append(n)
    return cuts


@dataclass
class LocalBlock:
    """One rank's rows and halo plan."""
    rank: int
    world: int
    lo: int                       # first global row owned
    hi: int                       # one past the last
    rowptr: np.ndarray            # local CSR over columns [own | ghosts]
    colidx: np.ndarray
    vals: np.ndarray
    ghosts: np.ndarray            # global indices of the ghost columns, grouped by owner
    recv: dict = field(default_factory=dict)   # owner -> (offset in the ghost area, count)
    send: dict = field(default_factory=dict)   # peer -> local indices of own rows to send

    @property
    def n_own(self) -> int:
        return self.hi - self.lo

    @property
    def ncols(self) -> int:
        return self.n_own + len(self.ghosts)


def local_block(rowptr, colidx, vals, cuts, rank) -> LocalBlock:
    """The rows of `rank` with columns renumbered to [own | ghosts]; the
    receive plan (which ghosts come from which owner).  The send plan is
    filled in by exchange_plans."""
    world = len(cuts) - 1
    lo, hi = cuts[rank], cuts[rank + 1]
    a, b = int(rowptr[lo]), int(rowptr[hi])
    cols = np.asarray(colidx[a:b], dtype=np.int64)
    own = (cols >= lo) & (cols < hi)
    ghosts = np.unique(cols[~own])                    # sorted, hence grouped by owner
    owner = np.searchsorted(np.asarray(cuts[1:]), ghosts, side="right")
    lcol = np.empty(len(cols), dtype=np.int32)
    lcol[own] = (cols[own] - lo).astype(np.int32)
    lcol[~own] = (hi - lo + np.searchsorted(ghosts, cols[~own])).astype(np.int32)
    recv = {}
    for q in range(world):
        idx = np.nonzero(owner == q)[0]
        if len(idx):
            recv[q] = (int(idx[0]), int(len(idx)))
    lrp = (np.asarray(rowptr[lo:hi + 1], dtype=np.int64) - a).astype(np.int32)
    return LocalBlock(rank, world, lo, hi, lrp, lcol, np.asarray(vals[a:b], dtype=np.float64),
                      ghosts, recv)


def exchange_plans(blk: LocalBlock, group=None) -> LocalBlock:
    """Every rank tells each owner which of its rows it needs (gathered
    lists); the owner's send plan is the list of those rows, in the order
    the requester stores them."""
    import torch.distributed as dist
    mine = {q: blk.ghosts[off:off + cnt].tolist() for q, (off, cnt) in blk.recv.items()}
    allreq = [None] * blk.world
    dist.all_gather_object(allreq, mine, group=group)
    send = {}
    for p, req in enumerate(allreq):
        if p != blk.rank and blk.rank in req:
            send[p] = np.asarray(req[blk.rank], dtype=np.int64) - blk.lo
    blk.send = send
    return blk


class NumpyOps:
    """Local operations on host arrays (CPU tensors); `spmv(blk, v)` must be
    given (the tests pass the oracle's)."""
    def __init__(self, spmv):
        self._spmv = spmv
        self.device = "cpu"
        self._dinv = None

    def setup(self, blk):
        diag = np.zeros(blk.n_own)
        for i in range(blk.n_own):
            seg = slice(blk.rowptr[i], blk.rowptr[i + 1])
            hit = np.nonzero(blk.colidx[seg] == i)[0]
            diag[i] = blk.vals[seg][hit[0]] if len(hit) else 0.0
        if np.any(diag <= 0.0):
            raise ValueError("Jacobi needs a positive diagonal")
        self._dinv = self.vec(1.0 / diag)

    def vec(self, a):
        import torch
        return torch.from_numpy(np.array(a, dtype=np.float64))

    def spmv(self, blk, v, out):
        import torch
        out.copy_(torch.from_numpy(np.asarray(self._spmv(blk, v.numpy()), dtype=np.float64)))

    def dot(self, a, b):
        return float(a[: len(b)].numpy() @ b.numpy())

    def dots(self, pairs):
        """Local partial sums a . b of every pair, as a tensor (the input of
        one all-reduce)."""
        import torch
        return torch.tensor([self.dot(a, b) for a, b in pairs], dtype=torch.float64)

    def axpy(self, y, alpha, x):       # y <- alpha x + y
        y += alpha * x

    def aypx(self, y, beta, x):        # y <- x + beta y
        y.mul_(beta).add_(x)

    def jacobi(self, r, z):            # z <- D^-1 r
        z.copy_(self._dinv * r)

    def copy(self, x, y):              # y <- x
        y.copy_(x)


class GbsOps:
    """Local operations in the library on this rank's GPU: the local block as
    a gbs matrix over [own | ghosts] columns (its Jacobi inverse diagonal made
    at creation), vectors as CUDA tensors; every vector operation runs in the
    library's kernels.  Each tensor (or slice) is wrapped once and its handle
    kept until close(), and the dot products of one reduction point are
    written in stream order into a device buffer that the all-reduce then
    sums, so no host synchronisation happens before the all-reduce."""
    def __init__(self, ctx, blk: LocalBlock):
        import torch
        from . import gbs
        self.gbs = gbs
        self.ctx = ctx
        self.device = "cuda"
        self.torch = torch
        self.A = gbs.gbs_mat_create_aij(ctx, blk.n_own, blk.ncols, blk.rowptr, blk.colidx, blk.vals)
        self.pc = None
        self._handles = {}
        self._keep = []

    def setup(self, blk):
        self.pc = self.gbs.gbs_pc_jacobi_create(self.A)   # GBS_ERR_DIAG -> GbsError

    def vec(self, a):
        return self.torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")

    def _h(self, t):
        key = (t.data_ptr(), t.numel())
        h = self._handles.get(key)
        if h is None:
            h = self.gbs.gbs_vec_wrap(self.ctx, t)
            self._handles[key] = h
            self._keep.append(t)   # the wrapped memory stays alive with its handle
        return h

    def spmv(self, blk, v, out):
        self.gbs.gbs_mat_mult(self.A, self._h(v), self._h(out))

    def dot(self, a, b):
        return self.gbs.gbs_vec_dot(self._h(a[: len(b)]), self._h(b))

    def dots(self, pairs):
        out = self.torch.empty(len(pairs), dtype=self.torch.float64, device="cuda")
        for j, (a, b) in enumerate(pairs):
            self.gbs.gbs_vec_dot_async(self._h(a[: len(b)]), self._h(b), out[j:j + 1])
        return out

    def axpy(self, y, alpha, x):
        self.gbs.gbs_vec_axpy(self._h(y), alpha, self._h(x))

    def aypx(self, y, beta, x):
        self.gbs.gbs_vec_aypx(self._h(y), beta, self._h(x))

    def jacobi(self, r, z):
        self.gbs.gbs_pc_apply(self.pc, self._h(r), self._h(z))

    def copy(self, x, y):
        self.gbs.gbs_vec_copy(self._h(x), self._h(y))

    def close(self):
        for h in self._handles.values():
            self.gbs.gbs_vec_destroy(h)
        self._handles.clear()
        self._keep.clear()
        if self.pc is not None:
            self.gbs.gbs_pc_destroy(self.pc)
        self.gbs.gbs_mat_destroy(self.A)


def halo_exchange(blk: LocalBlock, v, group=None):
    """Fill the ghost part of v (length ncols) from the owners: one message
    to and from each neighbour, posted together (batch_isend_irecv)."""
    import torch
    import torch.distributed as dist
    ops, fills = [], []
    for p, rows in sorted(blk.send.items()):
        idx = torch.as_tensor(rows, dtype=torch.int64, device=v.device)
        ops.append(dist.P2POp(dist.isend, v[: blk.n_own].index_select(0, idx).contiguous(), p,
                              group=group))
    for q, (off, cnt) in sorted(blk.recv.items()):
        tmp = v.new_empty(cnt)
        ops.append(dist.P2POp(dist.irecv, tmp, q, group=group))
        fills.append((off, cnt, tmp))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    for off, cnt, tmp in fills:
        v[blk.n_own + off: blk.n_own + off + cnt] = tmp


def allreduce_sum(vals, device, group=None):
    """Sum a list of host values, or a tensor of partial sums already on the
    device (summed in place), over the ranks; the totals come back to the
    host for the scalar recurrence."""
    import torch
    import torch.distributed as dist
    t = vals if isinstance(vals, torch.Tensor) else torch.tensor(vals, dtype=torch.float64,
                                                                  device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.tolist()


def sharded_pcg(blk: LocalBlock, ops, b_own, rtol: float, maxit: int, group=None):
    """Jacobi-PCG on the distributed system from x0 = 0.  Returns
    (x_own, status, iterations, ||r||, ||b||) with status 0 converged, 1
    iteration limit, -5 indefinite, -6 NaN (the library's codes).  The
    vector work runs in `ops`; the scalar recurrence (alpha, beta, the
    stopping test) runs here, on the all-reduced sums."""
    import math
    n = blk.n_own
    ops.setup(blk)
    b = ops.vec(b_own)
    x = ops.vec(np.zeros(n))
    r = ops.vec(b_own)
    z = ops.vec(np.zeros(n))
    ops.jacobi(r, z)
    p = ops.vec(np.zeros(blk.ncols))
    ops.copy(z, p[:n])
    q = ops.vec(np.zeros(n))
    rho, rr, bb = allreduce_sum(ops.dots([(r, z), (r, r), (b, b)]), ops.device, group)
    bnorm = math.sqrt(bb)
    k = 0
    status = 1
    while True:
        rn = math.sqrt(rr)
        if math.isnan(rn) or math.isnan(rho):
            status = -6
            break
        if rn <= rtol * bnorm:
            status = 0
            break
        if k >= maxit:
            break
        halo_exchange(blk, p, group)
        ops.spmv(blk, p, q)
        (pq,) = allreduce_sum(ops.dots([(p, q)]), ops.device, group)
        if math.isnan(pq):
            status = -6
            break
        if pq <= 0.0:
            status = -5
            break
        alpha = rho / pq
        ops.axpy(x, alpha, p[:n])
        ops.axpy(r, -alpha, q)
        ops.jacobi(r, z)
        rho_new, rr = allreduce_sum(ops.dots([(r, z), (r, r)]), ops.device, group)
        k += 1
        if rho_new < 0.0:
            status = -5
            break
        beta = rho_new / rho
        rho = rho_new
        ops.aypx(p[:n], beta, z)
    return x, status, k, math.sqrt(rr), bnorm
