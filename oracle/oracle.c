/*
 * Oracle for the Jacobi-preconditioned CG solve over a CSR (AIJ) matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential CPU
 * restatement of what the GPU path computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header or table with the
 * CUDA library.
 *
 * What it follows:
 *  - MatMult on the MATAIJ (compressed sparse row) type, Sec. 4 of the
 *    paper; the CSR traffic model of Challenge A7 (Sec. 3).
 *  - VecAXPY y <- a x + y, VecAYPX y <- x + b y, VecDot and VecNorm(NORM_2)
 *    as the paper's vector operations (Sec. 5.1, Sec. 2 stub routine).
 *  - PCJACOBI (Sec. 5.3: Jacobi-preconditioned smoothers) and KSPCG
 *    (Sec. 5.5: the CG method).  The paper names these methods but does not
 *    print them; the iteration below is the textbook preconditioned CG of
 *    Hestenes & Stiefel (1952) in the form of Saad, "Iterative Methods for
 *    Sparse Linear Systems", 2nd ed., Algorithm 9.1.
 *  - The single-precision-on-the-GPU plan of Response A7 (Sec. 4), read as
 *    classical iterative refinement (Wilkinson; Moler 1967): FP64 residual,
 *    FP32 inner PCG on the scaled residual, FP64 update.
 *
 * Readings where the paper is silent:
 *  - Stopping test: unpreconditioned ||r||_2 <= rtol * ||b||_2, taken before
 *    each iteration; the iteration count is the number of SpMVs after set-up.
 *  - Breakdown: p.Ap <= 0 or r.z < 0 is an indefinite operator or
 *    preconditioner; a NaN in any scalar is reported as such.
 *  - FP32 inner reductions accumulate in FP32 by pairwise summation.
 *
 * Threads: compiled as is (the build the tests and every check use) the
 * file is sequential.  The benchmark's CPU-baseline leg also times a second
 * build of the same source with -fopenmp, in which the loops marked
 * ORC_PAR_FOR / ORC_PAR_SUM are split across the host's cores (static
 * schedule; the sums then add in another order).  That build is only
 * timed, never used to check anything.
 *
 * Status codes (defined here independently of the CUDA library):
 *   0 converged, 1 iteration limit, -1 bad argument, -4 missing or
 *   non-positive diagonal, -5 indefinite, -6 NaN, -8 stagnation, -10 bad CSR.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#define ORC_PAR_FOR _Pragma("omp parallel for schedule(static)")
#define ORC_PAR_SUM _Pragma("omp parallel for schedule(static) reduction(+:s)")
#else
#define ORC_PAR_FOR
#define ORC_PAR_SUM
#endif

#define ORC_CONVERGED 0
#define ORC_DIVERGED_ITS 1
#define ORC_ERR_ARG (-1)
#define ORC_ERR_DIAG (-4)
#define ORC_ERR_INDEFINITE (-5)
#define ORC_ERR_NAN (-6)
#define ORC_ERR_STAGNATION (-8)
#define ORC_ERR_CSR (-10)

/* Host threads that the loops marked ORC_PAR_FOR / ORC_PAR_SUM run on:
 * 1 in the sequential build. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- CSR --- */

/* Structural check: rowptr[0] = 0, rowptr non-decreasing, every column in
 * [0, ncols) and strictly increasing within its row. */
int orc_csr_check(int64_t n, int64_t ncols, const int32_t *rowptr, const int32_t *colidx)
{
    if (n < 0 || ncols < 0) return ORC_ERR_ARG;
    if (rowptr[0] != 0) return ORC_ERR_CSR;
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return ORC_ERR_CSR;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colidx[k] < 0 || colidx[k] >= ncols) return ORC_ERR_CSR;
            if (k > rowptr[i] && colidx[k] <= colidx[k - 1]) return ORC_ERR_CSR;
        }
    }
    return 0;
}

/* MatMult: y_i = sum_k vals[k] * x[colidx[k]] over row i, in storage order. */
void orc_spmv(int64_t n, const int32_t *rowptr, const int32_t *colidx,
              const double *vals, const double *x, double *y)
{
    ORC_PAR_FOR
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s += vals[k] * x[colidx[k]];
        y[i] = s;
    }
}

/* The same product in binary32 (values, vector and sum all float). */
void orc_spmv_f32(int64_t n, const int32_t *rowptr, const int32_t *colidx,
                  const float *vals, const float *x, float *y)
{
    for (int64_t i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s += vals[k] * x[colidx[k]];
        y[i] = s;
    }
}

/* ------------------------------------------------------- vector ops --- */

/* VecDot: sum_i x_i y_i, left to right. */
double orc_dot(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    ORC_PAR_SUM
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* VecNorm(NORM_2): sqrt(x . x). */
double orc_norm2(int64_t n, const double *x)
{
    return sqrt(orc_dot(n, x, x));
}

/* Compensated dot product Dot2 (Ogita, Rump & Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26(6), 2005, Algorithm 5.3): the result is
 * as accurate as if computed in twice the working precision and then
 * rounded.  TwoProduct uses the fused multiply-add; TwoSum is Knuth's. */
double orc_dot2(int64_t n, const double *x, const double *y)
{
    double p = 0.0, s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double h = x[i] * y[i];
        double r = fma(x[i], y[i], -h);          /* exact error of the product */
        double q = p + h;                        /* TwoSum(p, h) */
        double z = q - p;
        double e = (p - (q - z)) + (h - z);
        p = q;
        s += e + r;
    }
    return p + s;
}

/* VecAXPY: y <- alpha x + y. */
void orc_axpy(int64_t n, double alpha, const double *x, double *y)
{
    ORC_PAR_FOR
    for (int64_t i = 0; i < n; ++i) y[i] = alpha * x[i] + y[i];
}

/* VecAYPX: y <- x + beta y. */
void orc_aypx(int64_t n, double beta, const double *x, double *y)
{
    ORC_PAR_FOR
    for (int64_t i = 0; i < n; ++i) y[i] = x[i] + beta * y[i];
}

/* The same two operations with one rounding per entry (the IEEE fused
 * multiply-add of C99 fma: the exact alpha x_i + y_i, rounded once), the
 * way the library's standalone VecAXPY and VecAYPX compute them. */
void orc_axpy_fused(int64_t n, double alpha, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = fma(alpha, x[i], y[i]);
}

void orc_aypx_fused(int64_t n, double beta, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = fma(beta, y[i], x[i]);
}

/* Pairwise (cascade) sum of v[0..n) in binary32: split in halves down to
 * blocks of at most 8, which are summed left to right. */
static float pairwise_f32(const float *v, int64_t n)
{
    if (n <= 8) {
        float s = 0.0f;
        for (int64_t i = 0; i < n; ++i) s += v[i];
        return s;
    }
    int64_t h = n / 2;
    return pairwise_f32(v, h) + pairwise_f32(v + h, n - h);
}

/* FP32 dot with FP32 pairwise accumulation; tmp has n floats. */
static float dot_f32(int64_t n, const float *x, const float *y, float *tmp)
{
    for (int64_t i = 0; i < n; ++i) tmp[i] = x[i] * y[i];
    return pairwise_f32(tmp, n);
}

/* ------------------------------------------------------------ Jacobi --- */

/* PCJACOBI set-up: dinv_i = 1 / a_ii.  Missing or non-positive a_ii is an
 * error (the preconditioner would not be SPD). */
int orc_jacobi_dinv(int64_t n, const int32_t *rowptr, const int32_t *colidx,
                    const double *vals, double *dinv)
{
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        int found = 0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (colidx[k] == i) { d = vals[k]; found = 1; }
        if (!found || !(d > 0.0)) return ORC_ERR_DIAG;
        dinv[i] = 1.0 / d;
    }
    return 0;
}

/* ------------------------------------------------------------ KSPCG --- */

/*
 * Norm of the stopping test.  The paper names KSPCG (Sec. 5.5) but does
 * not fix the norm its test uses; three are offered:
 *   0  unpreconditioned  N(v) = ||v||_2
 *   1  preconditioned    N(v) = ||D^-1 v||_2
 *   2  natural           N(v) = sqrt(v . D^-1 v)
 * w is scratch of n doubles.
 */
static double orc_test_norm(int norm, int64_t n, const double *v, const double *dinv, double *w)
{
    if (norm == 0) return orc_norm2(n, v);
    for (int64_t i = 0; i < n; ++i) w[i] = dinv[i] * v[i];
    return norm == 1 ? orc_norm2(n, w) : sqrt(orc_dot(n, v, w));
}

/*
 * Jacobi-preconditioned CG, FP64 (Saad, Iterative Methods for Sparse
 * Linear Systems, Alg. 9.1, the method behind KSPCG with PCJACOBI).
 *   x (in/out) initial guess -> solution; the test before each iteration
 *   is N(r) <= rtol N(b) in the chosen norm (above); maxit iterations at
 *   most; rhist (optional, maxit+1 doubles) receives N(r_k) for
 *   k = 0..iters.
 * Returns a status code; *iters = SpMVs done, *rnorm = last N(r) of the
 * recurrence, *bnorm = N(b).  The iterates do not depend on the norm.
 *
 *   r = b - A x;  z = D^-1 r;  p = z;  rho = r.z
 *   for k = 0, 1, ...:
 *       if N(r) <= rtol N(b): converged after k iterations
 *       q = A p;  pi = p.q;  (pi <= 0: indefinite)
 *       alpha = rho / pi;  x += alpha p;  r -= alpha q;  z = D^-1 r
 *       rho' = r.z;  (rho' < 0: indefinite preconditioner)
 *       beta = rho' / rho;  rho = rho';  p = z + beta p
 */
int orc_pcg_norm(int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                 const double *b, double *x, double rtol, int64_t maxit, int norm,
                 int64_t *iters, double *rnorm, double *bnorm_out, double *rhist)
{
    *iters = 0;
    *rnorm = 0.0;
    *bnorm_out = 0.0;
    if (n < 0 || maxit < 0 || !(rtol >= 0.0) || norm < 0 || norm > 2) return ORC_ERR_ARG;
    if (n == 0) return ORC_CONVERGED;
    double *dinv = malloc(sizeof(double) * n);
    double *r = malloc(sizeof(double) * n);
    double *z = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n);
    double *w = malloc(sizeof(double) * n);
    int status = orc_jacobi_dinv(n, rowptr, colidx, vals, dinv);
    if (status == 0) {
        orc_spmv(n, rowptr, colidx, vals, x, q);
        ORC_PAR_FOR
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        ORC_PAR_FOR
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        memcpy(p, z, sizeof(double) * n);
        double rho = orc_dot(n, r, z);
        const double bnorm = orc_test_norm(norm, n, b, dinv, w);
        *bnorm_out = bnorm;
        int64_t k = 0;
        status = ORC_DIVERGED_ITS;
        for (;;) {
            double rn = orc_test_norm(norm, n, r, dinv, w);
            *rnorm = rn;
            if (rhist) rhist[k] = rn;
            if (isnan(rn) || isnan(rho)) { status = ORC_ERR_NAN; break; }
            if (rn <= rtol * bnorm) { status = ORC_CONVERGED; break; }
            if (k >= maxit) break;
            orc_spmv(n, rowptr, colidx, vals, p, q);
            double pi = orc_dot(n, p, q);
            if (isnan(pi)) { status = ORC_ERR_NAN; break; }
            if (pi <= 0.0) { status = ORC_ERR_INDEFINITE; break; }
            double alpha = rho / pi;
            orc_axpy(n, alpha, p, x);
            orc_axpy(n, -alpha, q, r);
            ORC_PAR_FOR
            for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
            double rho_new = orc_dot(n, r, z);
            ++k;
            if (rho_new < 0.0) {
                *rnorm = orc_test_norm(norm, n, r, dinv, w);
                status = ORC_ERR_INDEFINITE;
                break;
            }
            double beta = rho_new / rho;
            rho = rho_new;
            orc_aypx(n, beta, z, p);
        }
        *iters = k;
    }
    free(dinv); free(r); free(z); free(p); free(q); free(w);
    return status;
}

/* orc_pcg_norm with the unpreconditioned norm. */
int orc_pcg(int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals,
            const double *b, double *x, double rtol, int64_t maxit,
            int64_t *iters, double *rnorm, double *rhist)
{
    double bnorm = 0.0;
    return orc_pcg_norm(n, rowptr, colidx, vals, b, x, rtol, maxit, 0, iters, rnorm, &bnorm,
                        rhist);
}

/*
 * The same iteration entirely in binary32 (storage, arithmetic and
 * pairwise-accumulated reductions), from x = 0.  vals32/dinv32 are the
 * rounded FP64 inputs.  rtol is relative to ||b||_2 computed in FP32.
 */
int orc_pcg_f32(int64_t n, const int32_t *rowptr, const int32_t *colidx, const float *vals32,
                const float *dinv32, const float *b, float *x, float rtol, int64_t maxit,
                int64_t *iters, float *rnorm)
{
    *iters = 0;
    *rnorm = 0.0f;
    if (n < 0 || maxit < 0 || !(rtol >= 0.0f)) return ORC_ERR_ARG;
    if (n == 0) return ORC_CONVERGED;
    float *r = malloc(sizeof(float) * n);
    float *z = malloc(sizeof(float) * n);
    float *p = malloc(sizeof(float) * n);
    float *q = malloc(sizeof(float) * n);
    float *t = malloc(sizeof(float) * n);
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0f; r[i] = b[i]; }
    for (int64_t i = 0; i < n; ++i) z[i] = dinv32[i] * r[i];
    memcpy(p, z, sizeof(float) * n);
    float rho = dot_f32(n, r, z, t);
    float bnorm = sqrtf(dot_f32(n, b, b, t));
    int64_t k = 0;
    int status = ORC_DIVERGED_ITS;
    for (;;) {
        float rn = sqrtf(dot_f32(n, r, r, t));
        *rnorm = rn;
        if (isnan(rn) || isnan(rho)) { status = ORC_ERR_NAN; break; }
        if (rn <= rtol * bnorm) { status = ORC_CONVERGED; break; }
        if (k >= maxit) break;
        orc_spmv_f32(n, rowptr, colidx, vals32, p, q);
        float pi = dot_f32(n, p, q, t);
        if (isnan(pi)) { status = ORC_ERR_NAN; break; }
        if (pi <= 0.0f) { status = ORC_ERR_INDEFINITE; break; }
        float alpha = rho / pi;
        for (int64_t i = 0; i < n; ++i) x[i] = alpha * p[i] + x[i];
        for (int64_t i = 0; i < n; ++i) r[i] = -alpha * q[i] + r[i];
        for (int64_t i = 0; i < n; ++i) z[i] = dinv32[i] * r[i];
        float rho_new = dot_f32(n, r, z, t);
        ++k;
        if (rho_new < 0.0f) { status = ORC_ERR_INDEFINITE; break; }
        float beta = rho_new / rho;
        rho = rho_new;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    *iters = k;
    free(r); free(z); free(p); free(q); free(t);
    return status;
}

/*
 * Mixed precision: FP32 inner PCG inside FP64 iterative refinement.
 *   loop: r = b - A x (FP64);  stop if ||r|| <= rtol ||b||;
 *         stagnation if ||r|| > ||r_prev|| / 2;
 *         s = ||r||;  solve A d = r / s with FP32 PCG to inner_rtol;
 *         x += s d (FP64).
 * Returns a status; *outer = refinement steps taken, *inner = FP32 PCG
 * iterations summed over them, *rnorm = last FP64 residual norm.
 */
int orc_pcg_mixed(int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                  const double *b, double *x, double rtol, double inner_rtol,
                  int64_t inner_maxit, int64_t outer_maxit,
                  int64_t *outer, int64_t *inner, double *rnorm)
{
    *outer = 0;
    *inner = 0;
    *rnorm = 0.0;
    if (n < 0 || inner_maxit < 0 || outer_maxit < 0 || !(rtol >= 0.0)) return ORC_ERR_ARG;
    if (n == 0) return ORC_CONVERGED;
    double *dinv = malloc(sizeof(double) * n);
    int status = orc_jacobi_dinv(n, rowptr, colidx, vals, dinv);
    if (status != 0) { free(dinv); return status; }
    int64_t nnz = rowptr[n];
    float *vals32 = malloc(sizeof(float) * (nnz > 0 ? nnz : 1));
    float *dinv32 = malloc(sizeof(float) * n);
    float *r32 = malloc(sizeof(float) * n);
    float *d32 = malloc(sizeof(float) * n);
    double *r = malloc(sizeof(double) * n);
    for (int64_t k = 0; k < nnz; ++k) vals32[k] = (float)vals[k];
    for (int64_t i = 0; i < n; ++i) dinv32[i] = (float)dinv[i];
    double bnorm = orc_norm2(n, b);
    double prev = INFINITY;
    status = ORC_DIVERGED_ITS;
    for (int64_t it = 0;; ++it) {
        orc_spmv(n, rowptr, colidx, vals, x, r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double rn = orc_norm2(n, r);
        *rnorm = rn;
        *outer = it;
        if (isnan(rn)) { status = ORC_ERR_NAN; break; }
        if (rn <= rtol * bnorm) { status = ORC_CONVERGED; break; }
        if (rn > 0.5 * prev) { status = ORC_ERR_STAGNATION; break; }
        if (it >= outer_maxit) break;
        prev = rn;
        for (int64_t i = 0; i < n; ++i) r32[i] = (float)(r[i] / rn);
        /* the inner solve stops at eta, or sooner where half the outer
         * target already suffices: x += rn d with ||r/rn - A d|| <= eta_j
         * leaves an outer residual of about rn eta_j */
        const double eta_j = fmax(inner_rtol, 0.5 * rtol * bnorm / rn);
        int64_t kin = 0;
        float rin = 0.0f;
        int st = orc_pcg_f32(n, rowptr, colidx, vals32, dinv32, r32, d32, (float)eta_j,
                             inner_maxit, &kin, &rin);
        *inner += kin;
        if (st < 0) { status = st; break; }
        for (int64_t i = 0; i < n; ++i) x[i] += rn * (double)d32[i];
    }
    free(dinv); free(vals32); free(dinv32); free(r32); free(d32); free(r);
    return status;
}

/*
 * Solve S Y = C for Y (k x k, column-major, k <= 8) with the symmetric
 * positive definite S (its lower triangle is used) factored as L D L^T,
 * L unit lower triangular, without square roots, so that for k = 1 the
 * solution is the single division C / S.  Returns 0, or -1 if a pivot of D
 * is not positive (S not positive definite: a breakdown of the block
 * method).
 */
static int orc_ldl_solve(int k, const double *S, const double *C, double *Y)
{
    double L[64], D[8];
    for (int j = 0; j < k; ++j) {
        double d = S[j + j * k];
        for (int m = 0; m < j; ++m) d -= L[j + m * k] * L[j + m * k] * D[m];
        if (!(d > 0.0)) return -1;
        D[j] = d;
        L[j + j * k] = 1.0;
        for (int i = j + 1; i < k; ++i) {
            double v = S[i + j * k];
            for (int m = 0; m < j; ++m) v -= L[i + m * k] * L[j + m * k] * D[m];
            L[i + j * k] = v / d;
        }
    }
    for (int c = 0; c < k; ++c) {
        double y[8];
        for (int i = 0; i < k; ++i) {          /* L y = C(:, c) */
            double v = C[i + c * k];
            for (int m = 0; m < i; ++m) v -= L[i + m * k] * y[m];
            y[i] = v;
        }
        for (int i = 0; i < k; ++i) y[i] = y[i] / D[i];
        for (int i = k - 1; i >= 0; --i) {     /* L^T Y(:, c) = y */
            double v = y[i];
            for (int m = i + 1; m < k; ++m) v -= L[m + i * k] * Y[m + c * k];
            Y[i + c * k] = v;
        }
    }
    return 0;
}

/* G = U^T V for n x k blocks (column-major), entry (a, b) = sum_i U_ia V_ib
 * left to right. */
static void orc_gram(int64_t n, int k, const double *U, const double *V, double *G)
{
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) G[a + b * k] = orc_dot(n, U + a * n, V + b * n);
}

/*
 * Block Jacobi-preconditioned CG for k right-hand sides at once (O'Leary,
 * "The block conjugate gradient algorithm and related methods", Linear
 * Algebra Appl. 29, 1980), FP64; the paper's Challenge F2 / KSPHPDDM point
 * that methods for several right-hand sides raise arithmetic intensity.
 * B, X: n x k column-major (column j at B + j n), X the initial guess in
 * and the solution out; 1 <= k <= 8.
 *
 *   R = B - A X;  Z = D^-1 R;  P = Z;  rho = Z^T R                (k x k)
 *   for it = 0, 1, ...:
 *       if ||R_j|| <= rtol ||B_j|| for every column j: converged
 *       Q = A P;  pi = P^T Q;  alpha = pi^-1 rho
 *       X += P alpha;  R -= Q alpha;  Z = D^-1 R
 *       rho' = Z^T R;  beta = rho^-1 rho';  P = Z + P beta;  rho = rho'
 *
 * The k x k systems are solved by orc_ldl_solve (pi or rho not positive
 * definite: ORC_ERR_INDEFINITE).  The products X + P alpha etc. add the k
 * terms left to right onto the first operand, so for k = 1 every operation
 * is the one orc_pcg does.  *iters = block iterations (SpMV passes over
 * the block); rnorm[j] = ||R_j|| at the end, bnorm[j] = ||B_j||.
 */
int orc_block_pcg(int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                  int k, const double *B, double *X, double rtol, int64_t maxit,
                  int64_t *iters, double *rnorm, double *bnorm)
{
    *iters = 0;
    if (n < 0 || k < 1 || k > 8 || maxit < 0 || !(rtol >= 0.0)) return ORC_ERR_ARG;
    for (int j = 0; j < k; ++j) rnorm[j] = bnorm[j] = 0.0;
    if (n == 0) return ORC_CONVERGED;
    const size_t nk = (size_t)n * k;
    double *dinv = malloc(sizeof(double) * n);
    double *R = malloc(sizeof(double) * nk);
    double *Z = malloc(sizeof(double) * nk);
    double *P = malloc(sizeof(double) * nk);
    double *Q = malloc(sizeof(double) * nk);
    double rho[64], pi[64], alpha[64], rho2[64], beta[64], t[8];
    int status = orc_jacobi_dinv(n, rowptr, colidx, vals, dinv);
    if (status == 0) {
        for (int j = 0; j < k; ++j) {
            orc_spmv(n, rowptr, colidx, vals, X + j * n, Q + j * n);
            for (int64_t i = 0; i < n; ++i) R[i + j * n] = B[i + j * n] - Q[i + j * n];
            for (int64_t i = 0; i < n; ++i) Z[i + j * n] = dinv[i] * R[i + j * n];
            bnorm[j] = orc_norm2(n, B + j * n);
        }
        memcpy(P, Z, sizeof(double) * nk);
        orc_gram(n, k, Z, R, rho);
        int64_t it = 0;
        status = ORC_DIVERGED_ITS;
        for (;;) {
            int done = 1, bad = 0;
            for (int j = 0; j < k; ++j) {
                rnorm[j] = orc_norm2(n, R + j * n);
                if (isnan(rnorm[j])) bad = 1;
                if (!(rnorm[j] <= rtol * bnorm[j])) done = 0;
            }
            if (bad) { status = ORC_ERR_NAN; break; }
            if (done) { status = ORC_CONVERGED; break; }
            if (it >= maxit) break;
            for (int j = 0; j < k; ++j) orc_spmv(n, rowptr, colidx, vals, P + j * n, Q + j * n);
            orc_gram(n, k, P, Q, pi);
            if (orc_ldl_solve(k, pi, rho, alpha)) { status = ORC_ERR_INDEFINITE; break; }
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < k; ++j) {
                    double x = X[i + j * n], r = R[i + j * n];
                    for (int m = 0; m < k; ++m) {
                        x = x + P[i + m * n] * alpha[m + j * k];
                        r = r - Q[i + m * n] * alpha[m + j * k];
                    }
                    X[i + j * n] = x;
                    R[i + j * n] = r;
                }
            for (size_t e = 0; e < nk; ++e) Z[e] = dinv[e % (size_t)n] * R[e];
            orc_gram(n, k, Z, R, rho2);
            ++it;
            if (orc_ldl_solve(k, rho, rho2, beta)) { status = ORC_ERR_INDEFINITE; break; }
            for (int64_t i = 0; i < n; ++i) {
                for (int j = 0; j < k; ++j) {
                    double p = Z[i + j * n];
                    for (int m = 0; m < k; ++m) p = p + P[i + m * n] * beta[m + j * k];
                    t[j] = p;
                }
                for (int j = 0; j < k; ++j) P[i + j * n] = t[j];
            }
            memcpy(rho, rho2, sizeof(rho));
        }
        if (status == ORC_ERR_INDEFINITE)
            for (int j = 0; j < k; ++j) rnorm[j] = orc_norm2(n, R + j * n);
        *iters = it;
    }
    free(dinv); free(R); free(Z); free(P); free(Q);
    return status;
}

/*
 * Jacobi-preconditioned Chebyshev iteration (KSPCHEBYSHEV with PCJACOBI,
 * the paper's multigrid smoother of Sec. 5.3): Chebyshev acceleration of
 * the preconditioned Richardson iteration for a spectrum of D^-1 A inside
 * [emin, emax] (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
 * Algorithm 12.1, Chebyshev acceleration, with the preconditioned residual
 * z = D^-1 r in place of r where the direction is formed).
 *
 *   theta = (emax + emin) / 2,  delta = (emax - emin) / 2,  sigma = theta / delta
 *   r = b - A x,  d = z / theta,  rho = 1 / sigma
 *   repeat:  x += d;  r -= A d;  rho' = 1 / (2 sigma - rho);
 *            d = rho' rho d + (2 rho' / delta) z;  rho = rho'
 *
 * The recurrence is carried as rho = delta / (2 theta - rho delta), so
 * that d = (rho delta / c) d + (2 / c) z with c = 2 theta - rho delta:
 * algebraically the same, and delta = 0 (a single eigenvalue) needs no
 * division by zero.  Stopping test as in orc_pcg, before each iteration.
 * There are no inner products in the iteration itself.
 */
int orc_chebyshev(int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                  const double *b, double *x, double emin, double emax, double rtol,
                  int64_t maxit, int64_t *iters, double *rnorm, double *rhist)
{
    *iters = 0;
    *rnorm = 0.0;
    if (n < 0 || maxit < 0 || !(rtol >= 0.0) || !(emin > 0.0) || !(emax >= emin) ||
        isinf(emax))
        return ORC_ERR_ARG;
    if (n == 0) return ORC_CONVERGED;
    double *dinv = malloc(sizeof(double) * n);
    double *r = malloc(sizeof(double) * n);
    double *d = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n);
    int status = orc_jacobi_dinv(n, rowptr, colidx, vals, dinv);
    if (status == 0) {
        const double theta = 0.5 * (emax + emin), delta = 0.5 * (emax - emin);
        orc_spmv(n, rowptr, colidx, vals, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        for (int64_t i = 0; i < n; ++i) d[i] = (dinv[i] * r[i]) / theta;
        double rho = delta / theta;
        const double bnorm = orc_norm2(n, b);
        int64_t k = 0;
        status = ORC_DIVERGED_ITS;
        for (;;) {
            const double rn = orc_norm2(n, r);
            *rnorm = rn;
            if (rhist) rhist[k] = rn;
            if (isnan(rn)) { status = ORC_ERR_NAN; break; }
            if (rn <= rtol * bnorm) { status = ORC_CONVERGED; break; }
            if (k >= maxit) break;
            orc_spmv(n, rowptr, colidx, vals, d, q);
            for (int64_t i = 0; i < n; ++i) x[i] = x[i] + d[i];
            for (int64_t i = 0; i < n; ++i) r[i] = r[i] - q[i];
            const double c = 2.0 * theta - rho * delta;
            const double a1 = (rho * delta) / c, a2 = 2.0 / c;
            for (int64_t i = 0; i < n; ++i) d[i] = a1 * d[i] + a2 * (dinv[i] * r[i]);
            rho = delta / c;
            ++k;
        }
        *iters = k;
    }
    free(dinv); free(r); free(d); free(q);
    return status;
}

/*
 * Assembly from coordinate triplets (MatSetPreallocationCOO followed by
 * MatSetValuesCOO, Sec. 4): triplet k adds v[k] at (ti[k], tj[k]).  The
 * result is CSR with rows in order and columns strictly increasing;
 * duplicates of one (row, column) are summed in the order the triplets
 * come (k increasing), left to right.  rowptr has nrows + 1 entries; colidx
 * and vals hold at most nnz_in entries; *nnz_out gets the count.  An index
 * out of range gives ORC_ERR_CSR.  Plain counting sort by row (stable),
 * then insertion sort by column within each row (stable), then a merge.
 */
int orc_coo_to_csr(int64_t nrows, int64_t ncols, int64_t nnz_in, const int32_t *ti,
                   const int32_t *tj, const double *v, int32_t *rowptr, int32_t *colidx,
                   double *vals, int64_t *nnz_out)
{
    *nnz_out = 0;
    if (nrows < 0 || ncols < 0 || nnz_in < 0) return ORC_ERR_ARG;
    for (int64_t k = 0; k < nnz_in; ++k)
        if (ti[k] < 0 || ti[k] >= nrows || tj[k] < 0 || tj[k] >= ncols) return ORC_ERR_CSR;
    int64_t *start = calloc((size_t)nrows + 1, sizeof(int64_t));
    int64_t *order = malloc(sizeof(int64_t) * (size_t)(nnz_in > 0 ? nnz_in : 1));
    for (int64_t k = 0; k < nnz_in; ++k) start[ti[k] + 1] += 1;
    for (int64_t r = 0; r < nrows; ++r) start[r + 1] += start[r];
    int64_t *fill = calloc((size_t)nrows + 1, sizeof(int64_t));
    for (int64_t k = 0; k < nnz_in; ++k) order[start[ti[k]] + fill[ti[k]]++] = k;
    int64_t out = 0;
    rowptr[0] = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t a = start[r], b = start[r + 1];
        for (int64_t p = a + 1; p < b; ++p) {        /* stable insertion sort by column */
            const int64_t key = order[p];
            int64_t q = p - 1;
            while (q >= a && tj[order[q]] > tj[key]) {
                order[q + 1] = order[q];
                --q;
            }
            order[q + 1] = key;
        }
        for (int64_t p = a; p < b;) {
            const int32_t c = tj[order[p]];
            double s = v[order[p]];
            ++p;
            while (p < b && tj[order[p]] == c) {
                s = s + v[order[p]];
                ++p;
            }
            colidx[out] = c;
            vals[out] = s;
            ++out;
        }
        rowptr[r + 1] = (int32_t)out;
    }
    *nnz_out = out;
    free(start);
    free(order);
    free(fill);
    return ORC_CONVERGED;
}

