"""Pins for the seeded input generators (CPU only).

The generators hold no solver arithmetic; these tests fix their structure
against closed forms: SplitMix64's published output sequence, the nnz
counts of truncated stencils, symmetry, diagonal dominance and the
closed-form eigenvalues of the Dirichlet Laplacian,
lambda = sum_d (2 - 2 cos(k_d pi / (N_d + 1))) (+ the diagonal shift).
"""
import math

import numpy as np
import pytest

from paper_2011_00715_gb300 import inputs as I


def test_splitmix64_published_sequence():
    # SplitMix64 from state 0: the first three outputs of the generator's
    # reference implementation (Steele, Lea & Flood 2014).
    z = np.zeros(3, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z[1] = I._GOLDEN
        z[2] = I._GOLDEN * np.uint64(2)
        out = I._mix64(z)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_moments():
    u = I.uniform01(7, 1, np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3
    g = I.normal(7, 2, np.arange(200000))
    assert abs(g.mean()) < 1e-2 and abs(g.var() - 1.0) < 2e-2
    # draws are keyed by index: a slice regenerates the same values
    assert np.array_equal(I.uniform01(7, 1, np.arange(100, 120)), u[100:120])


def _is_symmetric(A):
    d = A.to_dense()
    return np.array_equal(d, d.T)


@pytest.mark.parametrize("N", [2, 3, 7, 16])
def test_lap2d5_structure(N):
    A = I.lap2d5(N)
    assert A.n == N * N and A.nnz == 5 * N * N - 4 * N
    assert _is_symmetric(A)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    for i in range(A.n):
        c = A.colidx[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    # row sum = number of eliminated (Dirichlet) neighbours
    d = A.to_dense()
    x = np.arange(A.n) % N
    y = np.arange(A.n) // N
    missing = (x == 0).astype(int) + (x == N - 1) + (y == 0) + (y == N - 1)
    assert np.array_equal(d.sum(axis=1), missing.astype(float))
    assert rows.shape[0] == A.nnz


@pytest.mark.parametrize("N", [2, 3, 6])
def test_lap3d7_and_var27_nnz(N):
    assert I.lap3d7(N).nnz == 7 * N ** 3 - 6 * N ** 2
    assert I.var27(N).nnz == (3 * N - 2) ** 3


@pytest.mark.parametrize("dims", [(6, 6), (5, 7)])
def test_lap2d5_closed_form_eigenvalues(dims):
    nx, ny = dims
    lam = sorted(4 - 2 * math.cos(j * math.pi / (nx + 1)) - 2 * math.cos(k * math.pi / (ny + 1))
                 for j in range(1, nx + 1) for k in range(1, ny + 1))
    ev = np.linalg.eigvalsh(I.lap2d5(nx, ny).to_dense())
    assert np.allclose(ev, lam, atol=1e-12)


def test_lap3d7_closed_form_eigenvalues():
    nx, ny, nz = 3, 4, 5
    lam = sorted(6 - 2 * math.cos(a * math.pi / (nx + 1)) - 2 * math.cos(b * math.pi / (ny + 1))
                 - 2 * math.cos(c * math.pi / (nz + 1))
                 for a in range(1, nx + 1) for b in range(1, ny + 1) for c in range(1, nz + 1))
    ev = np.linalg.eigvalsh(I.lap3d7(nx, ny, nz).to_dense())
    assert np.allclose(ev, lam, atol=1e-12)


@pytest.mark.parametrize("maker", [
    lambda: I.var27(5, 4, 3, seed=3, sigma=1.0),
    lambda: I.var7(4, 5, 3, seed=11, sigma=0.5),
    lambda: I.var5(7, 6, seed=12, sigma=0.5),
])
def test_variable_coefficient_spd_m_matrix(maker):
    A = maker()
    d = A.to_dense()
    assert np.array_equal(d, d.T)
    off = d - np.diag(np.diag(d))
    assert np.all(off <= 0)                               # M-matrix sign pattern
    slack = np.diag(d) - np.abs(off).sum(axis=1)
    assert np.all(slack >= -1e-12)                        # weak dominance
    assert np.any(slack > 1e-3)                           # strict on boundary rows
    assert np.linalg.eigvalsh(d).min() > 0                # SPD
    # Gershgorin: the spectrum lies inside [0, 2 max diag]
    assert np.linalg.eigvalsh(d).max() <= 2 * np.diag(d).max() + 1e-12


def test_var27_link_scaling_and_interior_row_sums():
    # interior rows of the 27-point operator sum to zero (all links are
    # inside the grid), boundary rows to the eliminated links' weight
    A = I.var27(5, seed=3, sigma=1.0)
    d = A.to_dense()
    rs = d.sum(axis=1)
    c = np.arange(A.n)
    x, y, z = c % 5, (c // 5) % 5, c // 25
    interior = (x > 0) & (x < 4) & (y > 0) & (y < 4) & (z > 0) & (z < 4)
    assert np.allclose(rs[interior], 0.0, atol=1e-12)
    assert np.all(rs[~interior] > 0)
    # sigma = 0 gives unit weights: off-diagonals are exactly -1, -1/2, -1/4
    B = I.var27(4, seed=3, sigma=0.0)
    assert set(np.unique(B.vals[B.vals < 0])) == {-1.0, -0.5, -0.25}
    assert np.allclose(np.diag(B.to_dense()), 6 * 1 + 12 * 0.5 + 8 * 0.25)


def test_var27_unit_weight_closed_form_eigenvalues():
    # with unit weights the 27-point operator is 14 I minus a sum of tensor
    # products of the 1D Dirichlet shift pair T (eigenvalues 2 cos theta):
    # lambda = 14 - 2(cx+cy+cz) - 2(cx cy + cx cz + cy cz) - 2 cx cy cz
    nx, ny, nz = 3, 4, 5
    lam = []
    for a in range(1, nx + 1):
        for b in range(1, ny + 1):
            for c in range(1, nz + 1):
                cx, cy, cz = (math.cos(a * math.pi / (nx + 1)), math.cos(b * math.pi / (ny + 1)),
                              math.cos(c * math.pi / (nz + 1)))
                lam.append(14 - 2 * (cx + cy + cz) - 2 * (cx * cy + cx * cz + cy * cz)
                           - 2 * cx * cy * cz)
    A = I.var27(nx, ny, nz, seed=1, sigma=0.0)
    assert A.meta["w_min"] == 1.0
    assert np.allclose(np.linalg.eigvalsh(A.to_dense()), sorted(lam), atol=1e-12)
    # Loewner bound used by the solver tests: lambda_min(A) >= w_min lambda_min(unit)
    B = I.var27(nx, ny, nz, seed=3, sigma=1.0)
    assert np.linalg.eigvalsh(B.to_dense()).min() >= B.meta["w_min"] * min(lam) * (1 - 1e-12)


def test_random_and_exact_generators():
    A = I.random_csr(30, 30, 4, seed=5, symmetric=True, diag_shift=0.5)
    d = A.to_dense()
    assert np.array_equal(d, d.T) and np.linalg.eigvalsh(d).min() > 0
    E = I.exact_csr(40, 6, seed=9, ncols=50)
    assert E.meta["ncols"] == 50 and np.all(E.vals == np.round(E.vals))
    v = I.exact_vector(1000, seed=1)
    assert np.all(v * 2 ** 20 == np.round(v * 2 ** 20)) and np.abs(v).max() <= 1.0


def test_c4_and_c5_specs():
    s4 = I.c4_batch_specs()
    assert len(s4) == 512 and {s["family"] for s in s4} == {"var5", "var7"}
    ns = [int(np.prod(s["dims"])) for s in s4]
    assert min(ns) >= 500 and max(ns) <= 2.2e5
    assert 1.2e7 < sum(ns) < 2.6e7          # E[n] ~ 3.76e4 for log-uniform [1e3, 2e5]
    s5 = I.c5_request_specs(count=200)
    assert {s["nrhs"] for s in s5} <= {1, 2, 3, 4}
    t = I.poisson_arrivals(1, 100.0, 20000)
    assert abs(np.diff(t).mean() - 0.01) < 5e-4


@pytest.mark.parametrize("N", [1, 2, 5, 9, 16])
def test_lap3d7_torch_layout_equals_host_layout(N):
    """The torch layout of the 7-point Laplacian (used for operators too
    large for the host) is the host generator's CSR, array for array."""
    torch = pytest.importorskip("torch")
    A = I.lap3d7(N)
    rp, ci, v = I.lap3d7_torch(N, "cpu")
    assert rp.dtype == torch.int32 and ci.dtype == torch.int32 and v.dtype == torch.float64
    assert np.array_equal(A.rowptr, rp.numpy())
    assert np.array_equal(A.colidx, ci.numpy())
    assert np.array_equal(A.vals, v.numpy())
    assert int(rp[-1]) == 7 * N ** 3 - 6 * N ** 2
