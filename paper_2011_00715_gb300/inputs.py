"""Seeded synthetic inputs for the Jacobi-PCG solve: stencil matrices in CSR
(AIJ) layout, manufactured solutions and request streams.

This module is the only code shared by the CPU oracle's tests, the CUDA
path's tests and the benchmark.  It draws random numbers and lays out
matrix entries; it holds none of the solver's arithmetic (no SpMV, no dot
product, no Krylov step).  Right-hand sides b = A x* are therefore formed
by whichever side consumes the inputs.

Random numbers come from one counter-based generator: the SplitMix64
finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to (seed, stream, index), so any entry can
be regenerated on its own and the draw order never matters.

Matrix families (the paper's case studies use 5-point and 7-point
finite-difference stencils on structured grids, Sec. 5.3; the CSR layout is
the MATAIJ type of Sec. 4):

* ``lap2d5``  2D 5-point Laplacian, Dirichlet, diag 4, off-diagonals -1.
* ``lap3d7``  3D 7-point Laplacian, Dirichlet, diag 6, off-diagonals -1.
* ``var27``   3D 27-point variable-coefficient diffusion: one symmetric link
  weight w ~ lognormal(0, sigma) per pair of neighbouring cells, scaled by 1
  (face), 1/2 (edge), 1/4 (corner); A_ij = -c w, A_ii = sum of c w over all
  26 links, links to eliminated Dirichlet neighbours included.  Symmetric,
  weakly diagonally dominant, strictly so on boundary rows, irreducible:
  an SPD M-matrix.
* ``var5`` / ``var7``  the same construction with face links only.

Rows are numbered lexicographically (x fastest); column indices within a
row are strictly increasing.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSR", "counter_u64", "uniform01", "uniform_pm1", "normal", "lognormal",
    "lap2d5", "lap3d7", "var5", "var7", "var27", "random_csr",
    "exact_csr", "exact_vector", "c4_batch_specs", "c5_request_specs",
    "poisson_arrivals", "grid_for_n", "family_matrix", "xstar", "lap3d7_edge_triplets",
]

_U64 = np.uint64
_GOLDEN = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on an array of uint64 (wrapping arithmetic)."""
    z = z + _GOLDEN
    z = (z ^ (z >> _U64(30))) * _M1
    z = (z ^ (z >> _U64(27))) * _M2
    return z ^ (z >> _U64(31))


def counter_u64(seed: int, stream: int, index) -> np.ndarray:
    """64 random bits for each (seed, stream, index); index may be an array."""
    idx = np.asarray(index, dtype=np.int64).astype(np.uint64)
    with np.errstate(over="ignore"):
        h = _mix64(np.full(1, seed & 0xFFFFFFFFFFFFFFFF, dtype=np.uint64))
        h = _mix64(h ^ _U64(stream & 0xFFFFFFFFFFFFFFFF))
        return _mix64(h ^ idx)


def uniform01(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of the counter draw."""
    return (counter_u64(seed, stream, index) >> _U64(11)).astype(np.float64) * 2.0 ** -53


def uniform_pm1(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform in [-1, 1)."""
    return 2.0 * uniform01(seed, stream, np.arange(n)) - 1.0


def normal(seed: int, stream: int, index) -> np.ndarray:
    """Standard normals by Box-Muller from streams 2*stream and 2*stream+1."""
    u1 = uniform01(seed, 2 * stream, index)
    u2 = uniform01(seed, 2 * stream + 1, index)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def lognormal(seed: int, stream: int, index, sigma: float) -> np.ndarray:
    """exp(sigma * N(0,1))."""
    return np.exp(sigma * normal(seed, stream, index))


@dataclass
class CSR:
    """Square CSR matrix: int32 rowptr (n+1), int32 colidx (nnz), f64 vals."""
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        """Dense copy for small pins (placement only, no arithmetic)."""
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.colidx] = self.vals
        return a


def _offsets3(dims, radius_set):
    """Offsets in lexicographic (dz, dy, dx) order, which is ascending column order."""
    return sorted(radius_set, key=lambda d: (d[2], d[1], d[0]))


def _assemble(dims, offsets, value_of):
    """Lay out a stencil matrix.

    dims: (nx, ny, nz); offsets: list of (dx, dy, dz) in lexicographic
    (dz, dy, dx) order; value_of(k, valid) -> (n,) float64 entries for offset
    k (only entries where ``valid`` is true are kept).
    """
    nx, ny, nz = dims
    n = nx * ny * nz
    cell = np.arange(n, dtype=np.int64)
    x = cell % nx
    y = (cell // nx) % ny
    z = cell // (nx * ny)
    K = len(offsets)
    cols = np.empty((n, K), dtype=np.int64)
    vals = np.empty((n, K), dtype=np.float64)
    mask = np.empty((n, K), dtype=bool)
    for k, (dx, dy, dz) in enumerate(offsets):
        valid = ((x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
                 & (z + dz >= 0) & (z + dz < nz))
        mask[:, k] = valid
        cols[:, k] = cell + dx + nx * (dy + ny * dz)
        vals[:, k] = value_of(k, valid)
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 range")
    return CSR(n, rowptr.astype(np.int32), cols[mask].astype(np.int32),
               np.ascontiguousarray(vals[mask]), {"dims": tuple(dims)})


def _const_stencil(dims, offsets, diag):
    def value_of(k, valid):
        d = offsets[k]
        return np.full(valid.shape, diag if d == (0, 0, 0) else -1.0)
    return _assemble(dims, offsets, value_of)


def lap2d5(nx: int, ny: int | None = None) -> CSR:
    """2D 5-point Dirichlet Laplacian (diag 4, off-diagonals -1)."""
    ny = nx if ny is None else ny
    offs = _offsets3(None, [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)])
    m = _const_stencil((nx, ny, 1), offs, 4.0)
    m.meta.update(family="lap2d5", dims=(nx, ny))
    return m


def lap3d7_torch(nx: int, device):
    """The nx^3 3D 7-point Dirichlet Laplacian of ``lap3d7`` laid out with
    torch on ``device`` (same rows, columns in ascending order and values),
    for operators too large to lay out on the host.  Returns (rowptr,
    colidx, vals) as int32, int32, float64 tensors."""
    import torch
    n = nx ** 3
    cell = torch.arange(n, dtype=torch.int64, device=device)
    x = cell % nx
    y = (cell // nx) % nx
    z = cell // (nx * nx)
    # ascending column order: -nx^2, -nx, -1, 0, +1, +nx, +nx^2
    steps = (-nx * nx, -nx, -1, 0, 1, nx, nx * nx)
    valid = torch.stack([z > 0, y > 0, x > 0, torch.ones_like(x, dtype=torch.bool),
                         x < nx - 1, y < nx - 1, z < nx - 1], dim=1)
    del x, y, z
    counts = valid.sum(dim=1)
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=rowptr[1:])
    if int(rowptr[-1]) > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 range")
    del counts
    cols = cell[:, None] + torch.tensor(steps, dtype=torch.int64, device=device)[None, :]
    colidx = cols[valid].to(torch.int32)
    del cols
    vals = torch.where(torch.tensor([s == 0 for s in steps], device=device)[None, :].expand(n, 7),
                       6.0, -1.0)[valid].to(torch.float64)
    return rowptr.to(torch.int32), colidx, vals


def lap3d7(nx: int, ny: int | None = None, nz: int | None = None) -> CSR:
    """3D 7-point Dirichlet Laplacian (diag 6, off-diagonals -1)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    offs = _offsets3(None, [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0),
                            (1, 0, 0), (0, 1, 0), (0, 0, 1)])
    m = _const_stencil((nx, ny, nz), offs, 6.0)
    m.meta.update(family="lap3d7", dims=(nx, ny, nz))
    return m


def _link_weights(dims, seed, sigma, stream0):
    """Lognormal link weight for every cell of the grid extended by one
    Dirichlet layer and every 'positive' offset (keyed by the lower cell)."""
    nx, ny, nz = dims
    ex, ey = nx + 2, ny + 2

    def weight(k, cx, cy, cz):
        ext = (cx + 1) + ex * ((cy + 1) + ey * (cz + 1))
        return lognormal(seed, stream0 + k, ext, sigma)
    return weight


def _variable_stencil(dims, neighbour_offsets, scale_of, seed, sigma, stream0):
    nx, ny, nz = dims
    n = nx * ny * nz
    cell = np.arange(n, dtype=np.int64)
    x = cell % nx
    y = (cell // nx) % ny
    z = cell // (nx * ny)
    # 'positive' offsets: those whose linear offset in the extended grid is > 0
    ex, ey = nx + 2, ny + 2
    positive = [d for d in neighbour_offsets if d[0] + ex * (d[1] + ey * d[2]) > 0]
    pindex = {d: i for i, d in enumerate(positive)}
    weight = _link_weights(dims, seed, sigma, stream0)
    link = {}
    w_min = math.inf
    for d in neighbour_offsets:
        if d in pindex:
            w = weight(pindex[d], x, y, z)
        else:
            nd = (-d[0], -d[1], -d[2])
            w = weight(pindex[nd], x + d[0], y + d[1], z + d[2])
        if w.size:
            w_min = min(w_min, float(w.min()))
        link[d] = scale_of(d) * w
    diag = np.zeros(n)
    for d in neighbour_offsets:          # fixed order: the stencil's own order
        diag += link[d]
    offs = _offsets3(None, list(neighbour_offsets) + [(0, 0, 0)])

    def value_of(k, valid):
        d = offs[k]
        return diag if d == (0, 0, 0) else -link[d]
    m = _assemble(dims, offs, value_of)
    m.meta["w_min"] = w_min            # smallest link weight (Dirichlet links included)
    return m


def _face_offsets(ndim):
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)]
    if ndim == 3:
        offs += [(0, 0, -1), (0, 0, 1)]
    return _offsets3(None, offs)


def var5(nx: int, ny: int, seed: int, sigma: float = 0.5) -> CSR:
    """2D 5-point variable-coefficient diffusion, lognormal(0, sigma) face links."""
    m = _variable_stencil((nx, ny, 1), _face_offsets(2), lambda d: 1.0, seed, sigma, 300)
    m.meta.update(family="var5", dims=(nx, ny), seed=seed, sigma=sigma)
    return m


def var7(nx: int, ny: int, nz: int, seed: int, sigma: float = 0.5) -> CSR:
    """3D 7-point variable-coefficient diffusion, lognormal(0, sigma) face links."""
    m = _variable_stencil((nx, ny, nz), _face_offsets(3), lambda d: 1.0, seed, sigma, 300)
    m.meta.update(family="var7", dims=(nx, ny, nz), seed=seed, sigma=sigma)
    return m


_SCALE27 = {1: 1.0, 2: 0.5, 3: 0.25}


def var27(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 3,
          sigma: float = 1.0) -> CSR:
    """3D 27-point variable-coefficient diffusion (face/edge/corner links
    scaled 1, 1/2, 1/4, lognormal(0, sigma) weights)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    nb = _offsets3(None, [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                          for dx in (-1, 0, 1) if (dx, dy, dz) != (0, 0, 0)])
    m = _variable_stencil((nx, ny, nz), nb,
                          lambda d: _SCALE27[abs(d[0]) + abs(d[1]) + abs(d[2])],
                          seed, sigma, 400)
    m.meta.update(family="var27", dims=(nx, ny, nz), seed=seed, sigma=sigma)
    return m


def xstar(n: int, seed: int, column: int = 0, system: int = 0) -> np.ndarray:
    """Manufactured solution: uniform[-1, 1) keyed by (seed, system, column)."""
    return uniform_pm1(seed, 1000 + 64 * system + column, n)


def random_csr(n: int, ncols: int, per_row: int, seed: int, symmetric=False,
               diag_shift: float | None = None) -> CSR:
    """Random sparsity pattern with up to ``per_row`` draws per row, values
    uniform[-1,1).  ``symmetric`` keys each entry by its unordered (row, col)
    pair and mirrors it; ``diag_shift`` sets the diagonal to the row's
    absolute off-diagonal sum plus the shift (SPD when symmetric and the
    shift is positive)."""
    a = {}
    for i in range(n):
        idx = np.arange(per_row) + i * per_row
        c = (counter_u64(seed, 7, idx) % np.uint64(ncols)).astype(np.int64)
        v = 2.0 * uniform01(seed, 8, idx) - 1.0
        for cc, vv in zip(c.tolist(), v.tolist()):
            if symmetric:
                if cc == i:
                    continue
                a[(min(i, cc), max(i, cc))] = vv
            else:
                a[(i, cc)] = vv
    if symmetric:
        for (r_, c_) in list(a):
            a[(c_, r_)] = a[(r_, c_)]
    if diag_shift is not None:
        rowabs = np.zeros(n)
        for (r_, c_), v_ in a.items():
            if r_ != c_:
                rowabs[r_] += abs(v_)
        for i in range(n):
            a[(i, i)] = rowabs[i] + diag_shift
    return _from_dict(n, a, {"family": "random", "seed": seed}, ncols)


def exact_csr(n: int, per_row: int, seed: int, ncols: int | None = None) -> CSR:
    """Random pattern with small integer values in [-8, 8] (exactly
    representable products and sums for the exact-arithmetic pins)."""
    ncols = n if ncols is None else ncols
    a = {}
    for i in range(n):
        r = counter_u64(seed, 9, np.arange(per_row) + i * per_row)
        for j, rr in enumerate(r):
            c = int(rr % np.uint64(ncols))
            v = int((rr >> np.uint64(32)) % np.uint64(17)) - 8
            a[(i, c)] = float(v if v != 0 else 1)
    return _from_dict(n, a, {"family": "exact", "seed": seed}, ncols)


def exact_vector(n: int, seed: int, stream: int = 11) -> np.ndarray:
    """Values k / 2^20 with |k| < 2^20: products with small integers and their
    sums stay exact in binary64 for moderate lengths."""
    k = (counter_u64(seed, stream, np.arange(n)) % np.uint64(1 << 21)).astype(np.int64) - (1 << 20)
    return k.astype(np.float64) / float(1 << 20)


def _from_dict(n, a, meta, ncols=None):
    keys = sorted(a)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    for (r_, _c) in keys:
        rowptr[r_ + 1] += 1
    rowptr = np.cumsum(rowptr).astype(np.int32)
    colidx = np.array([c for (_r, c) in keys], dtype=np.int32)
    vals = np.array([a[k] for k in keys], dtype=np.float64)
    m = CSR(n, rowptr, colidx, vals, dict(meta))
    m.meta["ncols"] = n if ncols is None else ncols
    return m


def grid_for_n(family: str, n_target: float):
    """Grid dimensions for a target row count: 2D nx=floor(sqrt n),
    ny=round(n/nx); 3D nx=ny=floor(cbrt n), nz=round(n/nx^2)."""
    if family in ("var5", "lap2d5"):
        nx = max(2, int(math.isqrt(int(n_target))))
        return (nx, max(1, int(round(n_target / nx))))
    c = max(2, int(round(n_target ** (1.0 / 3.0))))
    while c ** 3 > n_target * 1.0000001 and c > 2:
        c -= 1
    return (c, c, max(1, int(round(n_target / (c * c)))))


def family_matrix(family: str, dims, seed: int, sigma: float) -> CSR:
    if family == "var5":
        return var5(dims[0], dims[1], seed, sigma)
    if family == "var7":
        return var7(dims[0], dims[1], dims[2], seed, sigma)
    if family == "var27":
        return var27(dims[0], dims[1], dims[2], seed, sigma)
    raise ValueError(family)


def c4_batch_specs(seed: int = 4, nsys: int = 512, n_lo: float = 1e3, n_hi: float = 2e5,
                   nrhs: int = 8):
    """Batch of independent systems: per system a seeded coin picks the 2D
    5-point or 3D 7-point family (lognormal(0, 0.5) face links) and the
    target row count is log-uniform in [n_lo, n_hi]."""
    s = np.arange(nsys)
    coin = uniform01(seed, 200, s)
    un = uniform01(seed, 201, s)
    specs = []
    for i in range(nsys):
        fam = "var5" if coin[i] < 0.5 else "var7"
        nt = math.exp(math.log(n_lo) + un[i] * (math.log(n_hi) - math.log(n_lo)))
        specs.append({"family": fam, "dims": grid_for_n(fam, nt), "seed": seed * 100000 + i,
                      "sigma": 0.5, "nrhs": nrhs, "system": i})
    return specs


def c5_request_specs(seed: int = 5, count: int = 2000, n_lo: float = 1e3, n_hi: float = 1e6,
                     pool: int = 0):
    """Solve requests for the serving loop: 27-point variable-coefficient
    cubes with log-uniform target size and 1..4 right-hand sides.  With
    ``pool`` > 0 the matrices repeat from a pool of that many distinct
    operators (the right-hand sides stay distinct per request)."""
    r = np.arange(count)
    un = uniform01(seed, 210, r)
    uk = uniform01(seed, 211, r)
    specs = []
    for i in range(count):
        key = i % pool if pool else i
        nt = math.exp(math.log(n_lo) + float(uniform01(seed, 210, [key])[0]) *
                      (math.log(n_hi) - math.log(n_lo))) if pool else \
            math.exp(math.log(n_lo) + un[i] * (math.log(n_hi) - math.log(n_lo)))
        c = grid_for_n("var27", nt)
        specs.append({"family": "var27", "dims": c, "seed": seed * 1000003 + key,
                      "sigma": 1.0, "nrhs": 1 + int(uk[i] * 4), "request": i,
                      "matrix_key": key})
    return specs


def poisson_arrivals(seed: int, rate: float, count: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    u = uniform01(seed, 220, np.arange(count))
    return np.cumsum(-np.log1p(-u) / rate)


def lap3d7_edge_triplets(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0):
    """Coordinate triplets (i, j, v) whose sum is the 3D 7-point Dirichlet
    Laplacian, the way a finite-element or finite-volume code produces them:
    every interior edge (p, q) of the grid adds +1 at (p, p) and (q, q) and
    -1 at (p, q) and (q, p); every edge to an eliminated Dirichlet neighbour
    adds +1 at (p, p).  The triplets come in a seeded random order (a
    permutation), so assembly has to sort and sum repeated entries."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    cell = np.arange(n, dtype=np.int64)
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    ii, jj, vv = [], [], []
    for step, coord, size in ((1, x, nx), (nx, y, ny), (nx * ny, z, nz)):
        inner = coord < size - 1
        p, q = cell[inner], cell[inner] + step
        ones = np.ones(len(p))
        ii += [p, q, p, q]
        jj += [p, q, q, p]
        vv += [ones, ones, -ones, -ones]
        # Dirichlet neighbours below and above
        for bnd in (coord == 0, coord == size - 1):
            ii.append(cell[bnd])
            jj.append(cell[bnd])
            vv.append(np.ones(int(bnd.sum())))
    i = np.concatenate(ii).astype(np.int32)
    j = np.concatenate(jj).astype(np.int32)
    v = np.concatenate(vv)
    # seeded shuffle: sort by counter-based random keys
    order = np.argsort(counter_u64(seed, 91, np.arange(len(i))), kind="stable")
    return i[order], j[order], v[order]
