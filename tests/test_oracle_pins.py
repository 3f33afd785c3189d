"""Pins that tie the CPU oracle to mathematics, not to itself (CPU only).

* SpMV: dense brute force in extended precision with Higham's componentwise
  bound |fl(a.x) - a.x| <= gamma_m |a|.|x| (Accuracy and Stability of
  Numerical Algorithms, Sec. 3.1); exact integer inputs (bitwise); row sums
  of the Dirichlet Laplacian; a non-symmetric, rectangular pattern so that a
  transposed operand cannot pass.
* Vector ops: exact inputs (bitwise), roles of alpha/beta in AXPY/AYPX.
* PCG: the k-th iterate equals the minimiser of the A-norm error over the
  Jacobi-preconditioned Krylov space (computed by dense Galerkin projection);
  finite termination after #distinct eigenvalues steps; the CG iteration
  bound from the closed-form condition number; dense solves; manufactured
  solutions; breakdown, limit and degenerate cases.
* Mixed precision: agreement with the FP64 solve and the outer-step count.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2011_00715_gb300 import inputs as I

U = 2.0 ** -53


def gamma(m):
    return m * U / (1 - m * U)


# ------------------------------------------------------------------ SpMV --

def test_spmv_dense_bruteforce_nonsymmetric_rectangular(orc):
    A = I.random_csr(150, 220, 9, seed=21)          # 150 x 220, non-symmetric
    x = I.uniform_pm1(4, 0, 220)
    d = np.zeros((150, 220), dtype=np.longdouble)
    rows = np.repeat(np.arange(150), np.diff(A.rowptr))
    d[rows, A.colidx] = A.vals
    exact = d @ x.astype(np.longdouble)
    y = orc.spmv(A, x)
    absdot = np.abs(d) @ np.abs(x).astype(np.longdouble)
    m = np.diff(A.rowptr)
    bound = np.array([gamma(int(mi)) for mi in m]) * absdot.astype(float)
    assert np.all(np.abs(y - exact.astype(float)) <= bound + 1e-300)
    # the transposed product is a different vector
    assert np.abs(y - (d.T[:150, :150] @ x[:150].astype(np.longdouble)).astype(float)).max() > 1e-3


def test_spmv_exact_inputs_bitwise(orc):
    A = I.exact_csr(300, 8, seed=3)
    x = I.exact_vector(300, seed=4)
    y = orc.spmv(A, x)
    k = np.round(x * 2 ** 20).astype(np.int64)
    for i in range(A.n):
        s = 0
        for t in range(A.rowptr[i], A.rowptr[i + 1]):
            s += int(A.vals[t]) * int(k[A.colidx[t]])
        assert y[i] == s / 2 ** 20


def test_spmv_laplacian_row_sums(orc):
    A = I.lap3d7(9)
    y = orc.spmv(A, np.ones(A.n))
    c = np.arange(A.n)
    x, yy, z = c % 9, (c // 9) % 9, c // 81
    missing = sum((v == 0).astype(int) + (v == 8) for v in (x, yy, z))
    assert np.array_equal(y, missing.astype(float))


def test_spmv_f32_matches_rounded_double(orc):
    A = I.exact_csr(200, 6, seed=8)
    x = I.exact_vector(200, seed=9)
    # exact inputs with <= 24 significant bits: the FP32 product is exact too
    x = np.round(x * 2 ** 12) / 2 ** 12
    assert np.array_equal(orc.spmv_f32(A, x).astype(np.float64), orc.spmv(A, x))


def test_csr_check(orc):
    A = I.lap2d5(4)
    assert orc.csr_check(A.n, A.n, A.rowptr, A.colidx) == 0
    bad = A.rowptr.copy(); bad[3] = bad[4] + 1
    assert orc.csr_check(A.n, A.n, bad, A.colidx) == orc.ERR_CSR
    badc = A.colidx.copy(); badc[5] = A.n
    assert orc.csr_check(A.n, A.n, A.rowptr, badc) == orc.ERR_CSR
    unsorted = A.colidx.copy(); unsorted[[0, 1]] = unsorted[[1, 0]]
    assert orc.csr_check(A.n, A.n, A.rowptr, unsorted) == orc.ERR_CSR
    bad0 = A.rowptr.copy(); bad0[0] = 1
    assert orc.csr_check(A.n, A.n, bad0, A.colidx) == orc.ERR_CSR
    dup = A.colidx.copy(); dup[1] = dup[0]                 # repeated column in row 0
    assert orc.csr_check(A.n, A.n, A.rowptr, dup) == orc.ERR_CSR
    neg = A.colidx.copy(); neg[0] = -1
    assert orc.csr_check(A.n, A.n, A.rowptr, neg) == orc.ERR_CSR


# ------------------------------------------------------------ vector ops --

def test_dot_norm_exact(orc):
    x = I.exact_vector(10000, seed=1)
    y = np.round(I.uniform_pm1(2, 0, 10000) * 8)
    kx = np.round(x * 2 ** 20).astype(np.int64)
    exact = int(np.sum(kx * y.astype(np.int64))) / 2 ** 20
    assert orc.dot(x, y) == exact
    assert orc.dot2(x, y) == exact
    assert orc.norm2(np.array([3.0, 4.0])) == 5.0
    v = np.array([1.0, 2.0, 2.0, 4.0, 10.0])             # sum of squares 125
    assert orc.norm2(v) == math.sqrt(125.0)


def test_dot2_is_twice_working_precision(orc):
    # ill-conditioned dot: huge cancellation; Dot2 error <= u|s| + gamma^2 |x|.|y|
    rng_x = I.uniform_pm1(3, 0, 2000) * np.exp(20 * I.uniform01(3, 1, np.arange(2000)))
    y = I.uniform_pm1(3, 2, 2000)
    x = np.concatenate([rng_x, -rng_x[:1000]])
    y = np.concatenate([y, y[:1000]])
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))
    s2 = orc.dot2(x, y)
    n = len(x)
    bound = U * abs(float(exact)) + gamma(n) ** 2 * float(np.abs(x) @ np.abs(y))
    assert abs(Fraction(s2) - exact) <= Fraction(bound)
    # (1 + 2^-30)^2 - (1 + 2^-29) = 2^-60 exactly; the rounded product loses
    # that term, so a plain dot returns 0 and Dot2 must return 2^-60
    a = 1.0 + 2.0 ** -30
    x = np.array([a, -(1.0 + 2.0 ** -29)])
    y = np.array([a, 1.0])
    assert orc.dot(x, y) == 0.0
    assert orc.dot2(x, y) == 2.0 ** -60


def test_axpy_aypx_roles(orc):
    x = np.array([1.0, 2.0, -3.0])
    y = np.array([10.0, 20.0, 30.0])
    assert np.array_equal(orc.axpy(2.0, x, y), [12.0, 24.0, 24.0])      # 2x + y
    assert np.array_equal(orc.aypx(2.0, x, y), [21.0, 42.0, 57.0])      # x + 2y


def test_fused_axpy_aypx_round_the_exact_value_once(orc):
    """alpha x + y computed exactly in rationals and rounded once (Python's
    float(Fraction) rounds to nearest even) equals the fused oracle entry by
    entry, including cancelling and tiny/huge operands; the separately
    rounded form differs somewhere, so the pin tells the two apart."""
    rng = np.random.default_rng(5)
    n = 400
    x = rng.standard_normal(n) * 10.0 ** rng.integers(-8, 9, n)
    y = rng.standard_normal(n) * 10.0 ** rng.integers(-8, 9, n)
    x[:50] = 1.0 + rng.random(50) * 2.0 ** -30      # alpha x close to -y: cancellation
    y[:50] = -0.37 * x[:50] + rng.standard_normal(50) * 2.0 ** -40
    for alpha in (-0.37, 1.9, 3.0 ** 0.5):
        exact = np.array([float(Fraction(alpha) * Fraction(xi) + Fraction(yi)) for xi, yi in zip(x, y)])
        assert np.array_equal(orc.axpy_fused(alpha, x, y), exact)
        exact_aypx = np.array([float(Fraction(xi) + Fraction(alpha) * Fraction(yi)) for xi, yi in zip(x, y)])
        assert np.array_equal(orc.aypx_fused(alpha, x, y), exact_aypx)
    assert not np.array_equal(orc.axpy(-0.37, x, y), orc.axpy_fused(-0.37, x, y))


def test_jacobi_dinv(orc):
    A = I.var5(5, 4, seed=2)
    st, dinv = orc.jacobi_dinv(A)
    assert st == 0 and np.array_equal(dinv, 1.0 / np.diag(A.to_dense()))
    B = I.random_csr(10, 10, 2, seed=1)                 # no guaranteed diagonal
    d = B.to_dense()
    st, _ = orc.jacobi_dinv(B)
    assert st == (0 if np.all(np.diag(d) > 0) and all(
        i in B.colidx[B.rowptr[i]:B.rowptr[i + 1]] for i in range(10)) else orc.ERR_DIAG)


# ------------------------------------------------------------------- PCG --

def krylov_minimiser(A, b, k):
    """Dense reference for the k-th PCG iterate from x0 = 0: the minimiser
    of ||x - x*||_A over span{z0, (D^-1 A) z0, ..., (D^-1 A)^(k-1) z0},
    z0 = D^-1 b, by Galerkin projection on an orthonormal basis."""
    d = A.to_dense()
    dinv = 1.0 / np.diag(d)
    v = dinv * b
    basis = []
    for _ in range(k):
        basis.append(v)
        v = dinv * (d @ v)
    Q, _ = np.linalg.qr(np.array(basis).T)
    y = np.linalg.solve(Q.T @ d @ Q, Q.T @ b)
    return Q @ y


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_pcg_iterates_are_krylov_minimisers(orc, k):
    A = I.var5(8, 7, seed=31, sigma=0.5)                # non-constant diagonal
    b = orc.spmv(A, I.xstar(A.n, 5))
    r = orc.pcg(A, b, rtol=0.0, maxit=k)
    assert r["status"] == orc.DIVERGED_ITS and r["iters"] == k
    ref = krylov_minimiser(A, b, k)
    assert np.linalg.norm(r["x"] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_pcg_energy_error_monotone_and_history(orc):
    A = I.var7(4, 4, 4, seed=5)
    d = A.to_dense()
    xs = I.xstar(A.n, 6)
    b = d @ xs
    errs = []
    for k in range(0, 25):
        r = orc.pcg(A, b, rtol=0.0, maxit=k, history=True)
        e = r["x"] - xs
        errs.append(math.sqrt(e @ d @ e))
        # recurrence residual matches the true residual on this small case
        assert abs(r["rhist"][-1] - np.linalg.norm(b - d @ r["x"])) <= 1e-10 * np.linalg.norm(b)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))
    assert errs[-1] < 1e-6 * errs[0]


def test_pcg_norms_with_constant_diagonal_scale_exactly(orc):
    """D = 4I: D^-1 v = v/4 exactly, so the preconditioned norm of every
    residual is ||r||/4 and the natural norm sqrt(r.r/4) = ||r||/2, bit for
    bit; the three tests stop at the same iteration with the same iterate."""
    A = I.lap2d5(20)
    b = orc.spmv(A, I.xstar(A.n, 3))
    runs = [orc.pcg(A, b, 1e-9, 2000, history=True, norm=m) for m in (0, 1, 2)]
    u, pr, na = runs
    assert u["status"] == pr["status"] == na["status"] == orc.CONVERGED
    assert u["iters"] == pr["iters"] == na["iters"]
    assert np.array_equal(u["x"], pr["x"]) and np.array_equal(u["x"], na["x"])
    assert np.array_equal(pr["rhist"], u["rhist"] / 4) and pr["bnorm"] == u["bnorm"] / 4
    assert np.array_equal(na["rhist"], u["rhist"] / 2) and na["bnorm"] == u["bnorm"] / 2
    assert abs(u["bnorm"] - np.linalg.norm(b)) <= gamma(A.n) * u["bnorm"]


def test_pcg_norms_follow_their_definitions(orc):
    """Variable diagonal: each run's residual history equals the chosen norm
    of the true residual of the k-step iterate (dense, numpy), and the run
    stops at the first iteration whose norm passes rtol N(b)."""
    A = I.var7(9, 8, 7, seed=12, sigma=1.0)
    dense = A.to_dense()
    dg = np.diag(dense)
    b = dense @ I.xstar(A.n, 4)
    norms = {0: lambda v: float(np.linalg.norm(v)),
             1: lambda v: float(np.linalg.norm(v / dg)),
             2: lambda v: math.sqrt(float(v @ (v / dg)))}
    rtol = 1e-6
    iterates = [orc.pcg(A, b, 0.0, k)["x"] for k in range(0, 80)]
    true_r = [b - dense @ x for x in iterates]
    stops = set()
    for m, N in norms.items():
        run = orc.pcg(A, b, rtol, 500, history=True, norm=m)
        assert run["status"] == orc.CONVERGED
        assert abs(run["bnorm"] - N(b)) <= 1e-13 * N(b)
        k = run["iters"]
        for j in range(k + 1):
            assert abs(run["rhist"][j] - N(true_r[j])) <= 1e-7 * N(true_r[j]) + 1e-12 * N(b)
        first = next(j for j in range(len(true_r)) if N(true_r[j]) <= rtol * N(b))
        assert k == first
        stops.add(k)
    assert len(stops) > 1          # the norms disagree on this system: the pin has teeth


@pytest.mark.parametrize("maker,steps", [
    (lambda: I.lap2d5(2), 3),        # eigenvalues {2, 4, 4, 6}: 3 distinct
    (lambda: I.lap3d7(2), 4),        # {3, 5, 7, 9}
    (lambda: I.lap2d5(6, 1), 6),     # 1D tridiagonal: 6 distinct
])
def test_pcg_finite_termination(orc, maker, steps):
    A = maker()
    b = orc.spmv(A, I.xstar(A.n, 1))
    r = orc.pcg(A, b, rtol=1e-12, maxit=50)
    assert r["status"] == orc.CONVERGED and r["iters"] == steps
    r1 = orc.pcg(A, b, rtol=1e-12, maxit=steps - 1)
    assert r1["status"] == orc.DIVERGED_ITS and r1["rnorm"] > 1e-6 * np.linalg.norm(b)


def cg_bound(kappa, rtol):
    """||r_k||/||b|| <= 2 sqrt(kappa) ((sqrt k - 1)/(sqrt k + 1))^k from x0 = 0."""
    s = math.sqrt(kappa)
    return math.ceil(math.log(2 * s / rtol) / math.log((s + 1) / (s - 1)))


def test_pcg_iteration_bound_2d(orc):
    N = 64
    lmin = 4 - 4 * math.cos(math.pi / (N + 1))
    lmax = 4 + 4 * math.cos(math.pi / (N + 1))
    assert abs(lmax / lmin - 1711.7) < 0.1
    bound = cg_bound(lmax / lmin, 1e-8)
    assert bound == 473
    A = I.lap2d5(N)
    xs = I.xstar(A.n, 1)
    b = orc.spmv(A, xs)
    r = orc.pcg(A, b, rtol=1e-8, maxit=2000)
    assert r["status"] == orc.CONVERGED and 50 < r["iters"] <= bound
    tr = b - orc.spmv(A, r["x"])
    assert np.linalg.norm(tr) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-3)
    assert np.linalg.norm(r["x"] - xs) <= (lmax / lmin) * 1e-8 * np.linalg.norm(xs)


def test_pcg_iteration_bound_3d(orc):
    N = 24
    c = math.cos(math.pi / (N + 1))
    kappa = (6 + 6 * c) / (6 - 6 * c)
    A = I.lap3d7(N)
    b = orc.spmv(A, I.xstar(A.n, 2))
    r = orc.pcg(A, b, rtol=1e-10, maxit=5000)
    assert r["status"] == orc.CONVERGED and r["iters"] <= cg_bound(kappa, 1e-10)


@pytest.mark.parametrize("maker", [
    lambda: I.random_csr(200, 200, 5, seed=8, symmetric=True, diag_shift=0.1),
    lambda: I.var27(6, 5, 4, seed=3, sigma=1.0),
])
def test_pcg_against_dense_solve(orc, maker):
    A = maker()
    d = A.to_dense()
    b = I.uniform_pm1(9, 0, A.n)
    r = orc.pcg(A, b, rtol=1e-12, maxit=10000)
    assert r["status"] == orc.CONVERGED
    ref = np.linalg.solve(d, b)
    kappa = np.linalg.cond(d)
    assert np.linalg.norm(r["x"] - ref) <= kappa * 1e-12 * 1.01 * np.linalg.norm(ref)
    assert np.linalg.norm(b - d @ r["x"]) <= 1e-12 * np.linalg.norm(b) * (1 + 1e-3)


def test_pcg_manufactured_solution(orc):
    A = I.var27(10, seed=3, sigma=1.0)
    xs = I.xstar(A.n, 3)
    b = orc.spmv(A, xs)
    r = orc.pcg(A, b, rtol=1e-12, maxit=10000)
    assert r["status"] == orc.CONVERGED
    assert np.linalg.norm(r["x"] - xs) <= 1e-7 * np.linalg.norm(xs)


def test_pcg_diagonal_matrix_one_step(orc):
    # Jacobi is the exact inverse of a diagonal operator: one iteration
    n = 50
    dvals = 0.5 + 10 * I.uniform01(4, 0, np.arange(n))
    A = I.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), dvals)
    b = I.uniform_pm1(4, 1, n)
    r = orc.pcg(A, b, rtol=1e-14, maxit=10)
    assert r["status"] == orc.CONVERGED and r["iters"] == 1
    assert np.allclose(r["x"], b / dvals, rtol=1e-15, atol=0)


def test_pcg_degenerate_cases(orc):
    A = I.lap2d5(5)
    # zero right-hand side: converged before any iteration, x stays 0
    r = orc.pcg(A, np.zeros(A.n), 1e-8, 100)
    assert r["status"] == orc.CONVERGED and r["iters"] == 0 and not r["x"].any()
    # initial guess equal to the solution
    xs = I.xstar(A.n, 2)
    b = orc.spmv(A, xs)
    r = orc.pcg(A, b, 1e-8, 100, x0=xs)
    assert r["status"] == orc.CONVERGED and r["iters"] == 0
    # iteration limit
    r = orc.pcg(A, b, 1e-14, 3)
    assert r["status"] == orc.DIVERGED_ITS and r["iters"] == 3
    # empty system
    E = I.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert orc.pcg(E, np.zeros(0), 1e-8, 10)["status"] == orc.CONVERGED
    # NaN in the right-hand side
    bn = b.copy(); bn[3] = np.nan
    assert orc.pcg(A, bn, 1e-8, 10)["status"] == orc.ERR_NAN
    # indefinite with a positive diagonal: [[1, 2], [2, 1]] has eigenvalue -1
    B = I.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
              np.array([1.0, 2.0, 2.0, 1.0]))
    assert orc.pcg(B, np.array([1.0, -1.0]), 1e-10, 10)["status"] == orc.ERR_INDEFINITE
    # non-positive and missing diagonals
    C = I.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, -2.0]))
    assert orc.pcg(C, np.ones(2), 1e-10, 10)["status"] == orc.ERR_DIAG
    M = I.CSR(2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    assert orc.pcg(M, np.ones(2), 1e-10, 10)["status"] == orc.ERR_DIAG


# ------------------------------------------------------- mixed precision --

def test_pcg_f32_close_to_fp64(orc):
    A = I.var7(10, 10, 10, seed=3)
    b = I.uniform_pm1(1, 0, A.n)
    r32 = orc.pcg_f32(A, b, 1e-5, 5000)
    r64 = orc.pcg(A, b, 1e-5, 5000)
    assert r32["status"] == orc.CONVERGED
    assert abs(r32["iters"] - r64["iters"]) <= 3
    ref = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(r32["x"] - ref) <= 1e-3 * np.linalg.norm(ref)


def test_mixed_refinement_reaches_fp64_accuracy(orc):
    A = I.var27(12, seed=3, sigma=1.0)
    xs = I.xstar(A.n, 3)
    b = orc.spmv(A, xs)
    ref = orc.pcg(A, b, 1e-10, 10000)
    m = orc.pcg_mixed(A, b, 1e-10, inner_rtol=1e-4)
    assert m["status"] == orc.CONVERGED
    # true FP64 residual by construction
    assert np.linalg.norm(b - orc.spmv(A, m["x"])) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(m["x"] - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    # each outer step gains about inner_rtol: ceil(log(rtol)/log(eta)) + 2
    assert m["outer"] <= math.ceil(math.log(1e-10) / math.log(1e-4)) + 2


def test_mixed_zero_rhs_and_bad_diag(orc):
    A = I.lap2d5(4)
    m = orc.pcg_mixed(A, np.zeros(A.n), 1e-10)
    assert m["status"] == orc.CONVERGED and m["outer"] == 0
    C = I.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 0.0]))
    assert orc.pcg_mixed(C, np.ones(2), 1e-10)["status"] == orc.ERR_DIAG


# ------------------------------------------------------------- Chebyshev --

def _cheb_T(k, t):
    """Chebyshev polynomial of the first kind by its three-term recurrence."""
    a, b = np.ones_like(t), t
    if k == 0:
        return a
    for _ in range(k - 1):
        a, b = b, 2 * t * b - a
    return b


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_chebyshev_error_is_the_scaled_chebyshev_polynomial(orc, k):
    """After k steps from x0, e_k = p_k(D^-1 A) e_0 with
    p_k(l) = T_k((theta - l) / delta) / T_k(theta / delta) — for any interval
    [emin, emax], here one strictly wider than the spectrum; computed from
    the eigen-decomposition of the symmetric D^-1/2 A D^-1/2."""
    A = I.var7(5, 4, 3, seed=11, sigma=0.7)
    n = A.n
    d = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    d[rows, A.colidx] = A.vals
    dg = np.diag(d).copy()
    B = d / np.sqrt(np.outer(dg, dg))
    lam, Q = np.linalg.eigh(B)
    emin, emax = 0.9 * lam[0], 1.05 * lam[-1]
    theta, delta = (emax + emin) / 2, (emax - emin) / 2
    xs = I.uniform_pm1(3, 0, n)
    b = d @ xs
    x0 = I.uniform_pm1(3, 1, n)
    r = orc.chebyshev(A, b, emin, emax, 0.0, k, x0=x0)
    assert r["iters"] == k
    p = _cheb_T(k, (theta - lam) / delta) / _cheb_T(k, np.array([theta / delta]))[0]
    S, Si = np.diag(np.sqrt(dg)), np.diag(1 / np.sqrt(dg))
    ek = Si @ Q @ np.diag(p) @ Q.T @ S @ (x0 - xs)
    assert np.linalg.norm(r["x"] - (xs + ek)) <= 1e-12 * np.linalg.norm(xs)


def test_chebyshev_rate_with_exact_bounds(orc):
    """With the exact extreme eigenvalues of D^-1 A (closed form for the 2D
    Laplacian, D = 4I), ||e_k||_A <= ||e_0||_A / T_k(sigma), and the
    iteration count meets the bound that implies (x0 = 0, as for CG)."""
    N = 24
    A = I.lap2d5(N)
    c1 = math.cos(math.pi / (N + 1))
    emin, emax = (4 - 4 * c1) / 4, (4 + 4 * c1) / 4
    sigma = (emax + emin) / (emax - emin)
    xs = I.xstar(A.n, 5)
    b = orc.spmv(A, xs)
    e0 = math.sqrt(float(xs @ orc.spmv(A, xs)))
    for k in (5, 20, 60):
        r = orc.chebyshev(A, b, emin, emax, 0.0, k)
        e = r["x"] - xs
        ek = math.sqrt(float(e @ orc.spmv(A, e)))
        assert ek <= e0 / math.cosh(k * math.acosh(sigma)) * (1 + 1e-9)
    kappa = emax / emin
    r = orc.chebyshev(A, b, emin, emax, 1e-8, 100000)
    # ||r_k|| / ||b|| <= sqrt(kappa) ||e_k||_A / ||e_0||_A <= sqrt(kappa) / T_k(sigma)
    bound = math.ceil(math.acosh(math.sqrt(kappa) / 1e-8) / math.acosh(sigma))
    assert r["status"] == 0 and r["iters"] <= bound


def test_chebyshev_single_eigenvalue_and_arguments(orc):
    """D^-1 A = I (a diagonal matrix) with emin = emax = 1: exact after one
    step; bad intervals are refused; b = 0 stops at once."""
    n = 7
    A = I.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
              np.linspace(1.0, 3.0, n))
    xs = I.uniform_pm1(2, 0, n)
    b = A.vals * xs
    r = orc.chebyshev(A, b, 1.0, 1.0, 1e-14, 10)
    assert r["status"] == 0 and r["iters"] == 1
    assert np.allclose(r["x"], xs, rtol=1e-15, atol=0)
    for lo, hi in ((0.0, 1.0), (2.0, 1.0), (-1.0, 1.0), (1.0, math.inf)):
        assert orc.chebyshev(A, b, lo, hi, 1e-8, 10)["status"] == orc.ERR_ARG
    r = orc.chebyshev(A, np.zeros(n), 0.5, 2.0, 1e-8, 10)
    assert r["status"] == 0 and r["iters"] == 0 and not r["x"].any()


# ------------------------------------------------------------- COO -> CSR --

def _random_triplets(seed, nrows, ncols, m, dup_rows=True):
    rng = np.random.default_rng(seed)
    ti = rng.integers(0, nrows, m).astype(np.int32)
    tj = rng.integers(0, ncols, m).astype(np.int32)
    if dup_rows:                      # force many duplicates
        ti[m // 2:] = ti[: m - m // 2]
        tj[m // 2:] = tj[: m - m // 2]
    return ti, tj, rng


def test_coo_assembly_equals_dense_accumulation_and_scipy(orc):
    """Integer values (exact in FP64): the assembled CSR is the dense sum of
    the triplets, with exactly the structural pattern of the triplets, rows
    in order and columns strictly increasing; scipy's coo -> csr agrees."""
    sp = pytest.importorskip("scipy.sparse")
    for seed, (nr, nc, m) in enumerate([(40, 50, 600), (7, 3, 100), (200, 200, 50)]):
        ti, tj, rng = _random_triplets(seed, nr, nc, m)
        v = rng.integers(-1000, 1000, m).astype(np.float64)
        st, rp, ci, vals = orc.coo_to_csr(nr, nc, ti, tj, v)
        assert st == 0
        assert orc.csr_check(nr, nc, rp, ci) == 0
        dense = np.zeros((nr, nc))
        np.add.at(dense, (ti, tj), v)
        got = np.zeros((nr, nc))
        rows = np.repeat(np.arange(nr), np.diff(rp))
        got[rows, ci] = vals
        assert np.array_equal(got, dense)
        assert set(zip(rows.tolist(), ci.tolist())) == set(zip(ti.tolist(), tj.tolist()))
        S = sp.coo_matrix((v, (ti, tj)), shape=(nr, nc)).tocsr()
        S.sort_indices()
        assert np.array_equal(S.indptr, rp) and np.array_equal(S.indices, ci)
        assert np.array_equal(S.data, vals)


def test_coo_duplicates_are_summed_in_triplet_order(orc):
    """Magnitudes chosen so that the order of a duplicate sum changes the
    result: the assembled value is the left-to-right sum in triplet order
    (a plain Python loop over the few triplets)."""
    ti = np.array([0, 1, 0, 0, 1, 1, 0], np.int32)
    tj = np.array([0, 2, 0, 0, 2, 2, 1], np.int32)
    v = np.array([1e16, 3.0, 1.0, -1e16, -3e16, 3e16, 7.0])
    st, rp, ci, vals = orc.coo_to_csr(2, 3, ti, tj, v)
    assert st == 0 and list(rp) == [0, 2, 3] and list(ci) == [0, 1, 2]
    expect = {}
    for a, b, x in zip(ti.tolist(), tj.tolist(), v.tolist()):
        expect[(a, b)] = expect[(a, b)] + x if (a, b) in expect else x
    assert vals[0] == expect[(0, 0)] == 0.0          # (1e16 + 1) - 1e16 rounds to 0
    assert vals[1] == 7.0 and vals[2] == expect[(1, 2)]
    rng = np.random.default_rng(9)
    ti, tj, _ = _random_triplets(9, 30, 30, 400)
    v = rng.standard_normal(400) * 10.0 ** rng.integers(-12, 13, 400)
    st, rp, ci, vals = orc.coo_to_csr(30, 30, ti, tj, v)
    expect = {}
    for a, b, x in zip(ti.tolist(), tj.tolist(), v.tolist()):
        expect[(a, b)] = expect[(a, b)] + x if (a, b) in expect else x
    rows = np.repeat(np.arange(30), np.diff(rp))
    assert all(vals[k] == expect[(int(rows[k]), int(ci[k]))] for k in range(len(ci)))


def test_coo_degenerate_and_invalid(orc):
    st, rp, ci, vals = orc.coo_to_csr(4, 4, [], [], [])
    assert st == 0 and list(rp) == [0] * 5 and len(ci) == 0
    assert orc.coo_to_csr(3, 3, [0, 3], [0, 0], [1.0, 1.0])[0] == orc.ERR_CSR
    assert orc.coo_to_csr(3, 3, [0, 1], [0, -1], [1.0, 1.0])[0] == orc.ERR_CSR
    st, rp, ci, vals = orc.coo_to_csr(0, 0, [], [], [])
    assert st == 0 and list(rp) == [0]


def test_coo_assembly_of_edge_contributions_is_the_laplacian(orc):
    """The seeded, shuffled edge contributions of the 3D grid sum to the
    7-point Dirichlet Laplacian: assembly reproduces it exactly."""
    for dims in ((6, 5, 4), (1, 1, 3), (9, 9, 9)):
        i, j, v = I.lap3d7_edge_triplets(*dims, seed=4)
        A = I.lap3d7(*dims)
        st, rp, ci, vals = orc.coo_to_csr(A.n, A.n, i, j, v)
        assert st == 0
        assert np.array_equal(rp, A.rowptr) and np.array_equal(ci, A.colidx)
        assert np.array_equal(vals, A.vals)


# -------------------------------------------------------------- block CG --

def block_rhs(orc, A, k, seed):
    return np.stack([orc.spmv(A, I.xstar(A.n, seed + 17 * j)) for j in range(k)], axis=1)


@pytest.mark.parametrize("maker", [lambda: I.lap2d5(20), lambda: I.var7(9, 8, 7, seed=3),
                                   lambda: I.var27(6, seed=5)])
def test_block_pcg_with_one_column_is_pcg_bitwise(orc, maker):
    """k = 1: every block operation reduces to the PCG operation (the 1 x 1
    LDL solve is one division), so the iterates are bitwise the PCG ones."""
    A = maker()
    b = block_rhs(orc, A, 1, 3)[:, 0]
    for rtol, maxit in ((1e-10, 5000), (0.0, 7)):
        r = orc.pcg(A, b, rtol, maxit)
        q = orc.block_pcg(A, b, rtol, maxit)
        assert q["status"] == r["status"] and q["iters"] == r["iters"]
        assert np.array_equal(q["x"][:, 0], r["x"])
        assert q["rnorm"][0] == r["rnorm"]


def block_krylov_minimiser(A, B, j):
    """Dense reference for the j-th block PCG iterate from X0 = 0: the
    minimiser of trace((X - X*)^T A (X - X*)) over X in the block Krylov
    space span{Z0, (D^-1 A) Z0, ..., (D^-1 A)^(j-1) Z0} (each column a
    combination of all jk basis vectors), Z0 = D^-1 B, by Galerkin
    projection on an orthonormal basis."""
    d = A.to_dense()
    dinv = 1.0 / np.diag(d)
    V = dinv[:, None] * B
    basis = []
    for _ in range(j):
        basis.append(V)
        V = dinv[:, None] * (d @ V)
    Q, _ = np.linalg.qr(np.concatenate(basis, axis=1))
    return Q @ np.linalg.solve(Q.T @ d @ Q, Q.T @ B)


@pytest.mark.parametrize("j", [1, 2, 3, 4])
def test_block_pcg_iterates_are_block_krylov_minimisers(orc, j):
    A = I.var5(9, 8, seed=31, sigma=0.5)                # non-constant diagonal
    B = block_rhs(orc, A, 3, 5)
    r = orc.block_pcg(A, B, rtol=0.0, maxit=j)
    assert r["status"] == orc.DIVERGED_ITS and r["iters"] == j
    ref = block_krylov_minimiser(A, B, j)
    assert np.linalg.norm(r["x"] - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("k,steps", [(1, 6), (2, 3), (3, 2), (6, 1)])
def test_block_pcg_finite_termination(orc, k, steps):
    """The 1D tridiagonal of 6 rows has 6 distinct eigenvalues (simple):
    the block Krylov space of k generic columns holds the solution after
    ceil(6 / k) block steps, and not one step earlier."""
    A = I.lap2d5(6, 1)
    B = block_rhs(orc, A, k, 2)
    r = orc.block_pcg(A, B, rtol=1e-12, maxit=50)
    assert r["status"] == orc.CONVERGED and r["iters"] == steps
    if steps > 1:
        r1 = orc.block_pcg(A, B, rtol=1e-12, maxit=steps - 1)
        assert r1["status"] == orc.DIVERGED_ITS
        assert np.max(r1["rnorm"] / r1["bnorm"]) > 1e-6


def test_block_pcg_against_dense_solve_and_fewer_steps(orc):
    A = I.var7(7, 6, 5, seed=8)
    B = block_rhs(orc, A, 4, 9)
    r = orc.block_pcg(A, B, rtol=1e-12, maxit=1000)
    X = np.linalg.solve(A.to_dense(), B)
    assert r["status"] == orc.CONVERGED
    assert np.linalg.norm(r["x"] - X) <= 1e-9 * np.linalg.norm(X)
    assert np.all(r["rnorm"] <= 1e-12 * r["bnorm"])
    # the shared block space needs fewer steps than the slowest single column
    single = max(orc.pcg(A, B[:, j], 1e-12, 1000)["iters"] for j in range(4))
    assert r["iters"] < single


def test_block_pcg_breakdown_and_degenerate(orc):
    A = I.lap2d5(5)
    b = block_rhs(orc, A, 1, 4)[:, 0]
    # two equal columns: P^T A P is singular at the first step
    r = orc.block_pcg(A, np.stack([b, b], axis=1), 1e-10, 100)
    assert r["status"] == orc.ERR_INDEFINITE
    # zero right-hand sides converge at once
    r = orc.block_pcg(A, np.zeros((A.n, 3)), 1e-10, 100)
    assert r["status"] == orc.CONVERGED and r["iters"] == 0 and not r["x"].any()
    # iteration limit
    B = block_rhs(orc, A, 2, 1)
    r = orc.block_pcg(A, B, 1e-14, 2)
    assert r["status"] == orc.DIVERGED_ITS and r["iters"] == 2


def test_mixed_last_step_stops_at_half_the_target(orc):
    """Each refinement step's inner FP32 solve stops at
    eta_j = max(eta, rtol ||b|| / (2 ||r_j||)).  With x0 = 0 and a loose
    rtol the first step alone can finish: its inner solve is then exactly
    the FP32 PCG of r0 / ||r0|| = b / ||b|| to the relative tolerance
    rtol / 2, so its iteration count is that solve's, far below what the
    fixed eta would take, and one refinement step reaches rtol."""
    A = I.var7(14, 13, 12, seed=9, sigma=1.0)
    b = orc.spmv(A, I.xstar(A.n, 9))
    rtol, eta = 1e-3, 1e-6
    m = orc.pcg_mixed(A, b, rtol, inner_rtol=eta)
    assert m["status"] == orc.CONVERGED and m["outer"] == 1
    alone = orc.pcg_f32(A, (b / orc.norm2(b)).astype(np.float32), 0.5 * rtol, 10000)
    fixed = orc.pcg_f32(A, (b / orc.norm2(b)).astype(np.float32), eta, 10000)
    assert m["inner"] == alone["iters"] < fixed["iters"]
    assert np.linalg.norm(b - orc.spmv(A, m["x"])) <= rtol * np.linalg.norm(b)
    # at a tight rtol every step but the last runs to eta: the count of
    # steps stays within the fixed-eta bound
    m2 = orc.pcg_mixed(A, b, 1e-10, inner_rtol=1e-4)
    assert m2["status"] == orc.CONVERGED
    assert m2["outer"] <= math.ceil(math.log(1e-10) / math.log(1e-4)) + 2
