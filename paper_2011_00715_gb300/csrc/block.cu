// Block Jacobi-preconditioned CG for k <= 8 right-hand sides of one matrix
// (O'Leary's block CG; the paper's Challenge F2 / Sec. 4: methods for
// several right-hand sides raise the arithmetic intensity of the solve and
// cut the number of sequentially launched kernels), FP64, one cooperative
// persistent launch per solve.
//
// The k columns are interleaved with a padded stride kp (entry (row, c) at
// row * kp + c, kp = k rounded up to 1, 2, 4 or 8; padding holds zeros), so
// the kp operands one nonzero gathers are one aligned vector load.  Per
// iteration, as in the single-vector kernel, three phases end at grid
// barriers:
//   S  Q = A P (the CTA's warp tiles staged in shared memory, one row per
//      lane, all kp columns per gather), then the CTA's part of the Gram
//      matrix P^T Q (lower triangle)
//   U  alpha = (P^T Q)^-1 rho; X += P alpha; R -= Q alpha; Z = D^-1 R; the
//      CTA's part of Z^T R (lower triangle) and of the column norms ||R_j||^2
//   P  beta = rho^-1 (Z^T R); P = Z + P beta
// Every CTA sums the per-CTA parts in the same fixed order and solves the
// k x k systems the same way (LDL^T without square roots, one lane per
// right-hand-side column), so all CTAs hold bitwise-identical alpha, beta
// and decisions.  The stopping test (every column ||R_j|| <= rtol ||B_j||)
// is taken before each iteration.

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "gbs_impl.cuh"

namespace {

constexpr int kBT = GBS_PBLOCK;       // threads per CTA
constexpr int kBW = kBT / 32;         // warps per CTA
constexpr int kKmax = 8;
constexpr int kNPair = kKmax * (kKmax + 1) / 2;   // lower-triangle entries
constexpr int kSlotsB = 2 * kNPair + kKmax;       // P^T Q | Z^T R | ||R_j||^2

struct BcgResult {
    int status, iters, pad[2];
    double rnorm[kKmax], bnorm[kKmax];
};

struct BcgArgs {
    int64_t n, ntiles;
    const int32_t *tdesc, *rowptr, *colidx;
    const double *vals, *dinv;
    const double *b;            // n x kp interleaved
    double *x, *r, *z, *p, *q;  // n x kp interleaved
    double *part;               // kSlotsB * G
    gbs_grid_barrier *bar;
    BcgResult *res;
    double rtol;
    int k, maxit;
    unsigned long long timeout_ns;
};

// Shared state of a CTA.
struct BcgShared {
    double tot[kSlotsB];          // grid totals of the last reduction
    double rho[kKmax * kKmax];    // Z^T R (column-major, full)
    double mat[kKmax * kKmax];    // alpha or beta (column-major)
    double fac[kKmax * kKmax + kKmax];   // L and 1 / D of the last LDL^T
    double bn[kKmax];
    int go, status, it, pad;
};

// Lower-triangle entry index of (a, b), a >= b.
__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }

// Solve S Y = C (k x k, column-major, S symmetric positive definite) with
// S = L D L^T, L unit lower triangular, no square roots.  Warp 0 only.
// Factorisation: lane i holds row i of L; at step j every lane forms the
// pivot d_j from row j (shuffled from lane j), then lanes i > j form
// L_ij; one reciprocal per pivot.  The factors go to shared memory (fl,
// 64 + 8 entries), then lane c < k solves for column c by forward and back
// substitution.  Returns false in every lane if a pivot is not positive.
__device__ __noinline__ bool ldl_solve_warp(int k, const double *S, const double *C, double *Y,
                                            double *fl)
{
    const int lane = threadIdx.x & 31;
    double Lrow[kKmax];   // this lane's row of L (lane < k), columns < lane
    double D[kKmax], Di[kKmax];
#pragma unroll
    for (int m = 0; m < kKmax; ++m) Lrow[m] = 0.0;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < kKmax; ++j) {
        if (j >= k) break;
        // row j of L from lane j, and the pivot
        double lj[kKmax];
#pragma unroll
        for (int m = 0; m < kKmax; ++m) lj[m] = __shfl_sync(0xffffffffu, Lrow[m], j);
        double d = S[j + j * k];
#pragma unroll
        for (int m = 0; m < kKmax; ++m)
            if (m < j) d -= lj[m] * lj[m] * D[m];
        if (!(d > 0.0)) ok = false;
        D[j] = d;
        Di[j] = 1.0 / d;
        if (lane > j && lane < k) {
            double v = S[lane + j * k];
#pragma unroll
            for (int m = 0; m < kKmax; ++m)
                if (m < j) v -= Lrow[m] * lj[m] * D[m];
            Lrow[j] = v * Di[j];
        }
    }
    if (lane < k)
#pragma unroll
        for (int m = 0; m < kKmax; ++m)
            if (m < lane) fl[lane + m * k] = Lrow[m];
    if (lane < k) fl[64 + lane] = Di[lane];
    __syncwarp();
    if (ok && lane < k) {
        const int c = lane;
        double y[kKmax];
#pragma unroll
        for (int i = 0; i < kKmax; ++i) {
            if (i >= k) break;
            double v = C[i + c * k];
#pragma unroll
            for (int m = 0; m < kKmax; ++m)
                if (m < i) v -= fl[i + m * k] * y[m];
            y[i] = v;
        }
#pragma unroll
        for (int i = 0; i < kKmax; ++i)
            if (i < k) y[i] = y[i] * fl[64 + i];
#pragma unroll
        for (int i = kKmax - 1; i >= 0; --i) {
            if (i >= k) continue;
            double v = y[i];
#pragma unroll
            for (int m = 0; m < kKmax; ++m)
                if (m > i && m < k) v -= fl[m + i * k] * y[m];
            y[i] = v;
        }
#pragma unroll
        for (int i = 0; i < kKmax; ++i)
            if (i < k) Y[i + c * k] = y[i];
    }
    __syncwarp();
    return ok;
}

// The kp operands of row c of an interleaved multi-vector.
template <int KP>
__device__ __forceinline__ void ld_row(const double *v, int64_t c, double (&o)[KP])
{
    if (KP == 1) {
        o[0] = __ldcg(v + c);
    } else {
#pragma unroll
        for (int j = 0; j < KP; j += 2) {
            const double2 t = __ldcg(reinterpret_cast<const double2 *>(v + c * KP + j));
            o[j] = t.x;
            o[j + 1] = t.y;
        }
    }
}

template <int KP>
__device__ __forceinline__ void st_row(double *v, int64_t c, const double (&o)[KP])
{
    if (KP == 1) {
        __stcg(v + c, o[0]);
    } else {
#pragma unroll
        for (int j = 0; j < KP; j += 2)
            __stcg(reinterpret_cast<double2 *>(v + c * KP + j), make_double2(o[j], o[j + 1]));
    }
}

// Y = A V over the CTA's warp tiles [t0, t1): each warp stages a tile's
// column indices and values in shared memory with coalesced loads, then
// lane l accumulates row r0 + l over all kp columns (left to right in
// storage order); a row longer than a tile is summed by the whole warp
// with a fixed shuffle tree.
template <int KP>
__device__ void block_spmv(const BcgArgs &a, int64_t t0, int64_t t1, const double *V, double *Y,
                           GbsWarpTile<double> &wt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t = t0 + warp; t < t1; t += kBW) {
        const int r0 = __ldg(a.tdesc + 2 * t), r1 = __ldg(a.tdesc + 2 * t + 2);
        const int k0 = __ldg(a.tdesc + 2 * t + 1), k1 = __ldg(a.tdesc + 2 * t + 3);
        double s[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) s[j] = 0.0;
        if (k1 - k0 > GBS_WT_NNZ) {   // one long row
            for (int e = k0 + lane; e < k1; e += 32) {
                double o[KP];
                ld_row<KP>(V, __ldg(a.colidx + e), o);
                const double av = __ldg(a.vals + e);
#pragma unroll
                for (int j = 0; j < KP; ++j) s[j] = fma(av, o[j], s[j]);
            }
#pragma unroll
            for (int j = 0; j < KP; ++j)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], off);
            if (lane == 0) st_row<KP>(Y, r0, s);
            continue;
        }
        for (int e = k0 + lane; e < k1; e += 32) {
            wt.col[e - k0] = __ldg(a.colidx + e);
            wt.val[e - k0] = __ldg(a.vals + e);
        }
        __syncwarp();
        if (r0 + lane < r1) {
            const int row = r0 + lane;
            const int beg = __ldg(a.rowptr + row) - k0, end = __ldg(a.rowptr + row + 1) - k0;
            for (int e = beg; e < end; ++e) {
                double o[KP];
                ld_row<KP>(V, wt.col[e], o);
                const double av = wt.val[e];
#pragma unroll
                for (int j = 0; j < KP; ++j) s[j] = fma(av, o[j], s[j]);
            }
            st_row<KP>(Y, row, s);
        }
        __syncwarp();
    }
}

// The CTA's part over its rows [rb, re) of: (MODE 0) the lower triangle of
// U^T V, (MODE 1) that and the column norms ||V_j||^2 in the k slots after
// it, (MODE 2) the column norms ||V_j||^2 alone; into part[slot0 + e][c].
// Thread t takes entry e = t mod ne on rows t / ne, t / ne + ng, ...; the
// ng row groups are added in order.
template <int KP, int MODE>
__device__ void block_gram(const BcgArgs &a, int k, int64_t rb, int64_t re, const double *U,
                           const double *V, int slot0, double *s_red)
{
    const int np = MODE == 2 ? 0 : k * (k + 1) / 2, ne = MODE == 0 ? np : np + k;
    const int ng = kBT / ne, t = threadIdx.x;
    const int e = t % ne, g = t / ne;
    if (g < ng) {
        int ea, eb;
        if (e < np) {
            ea = 0;
            while (tri(ea + 1, 0) <= e) ++ea;
            eb = e - tri(ea, 0);
        } else {
            ea = eb = e - np;
        }
        const double *uu = e < np ? U : V;
        double acc = 0.0;
        for (int64_t i = rb + g; i < re; i += ng)
            acc = fma(__ldcg(uu + i * KP + ea), __ldcg(V + i * KP + eb), acc);
        s_red[g * ne + e] = acc;
    }
    __syncthreads();
    if (t < ne) {
        double s = 0.0;
        for (int h = 0; h < ng; ++h) s += s_red[h * ne + t];
        a.part[(size_t)(slot0 + t) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
}

// Grid totals of slots [slot0, slot0 + ne) into sh.tot (every CTA, same
// order: lane l adds CTAs l, l + 32, ... left to right, then a fixed
// shuffle tree; warps take the slots in turn).
__device__ void block_grid_sum(const BcgArgs &a, int slot0, int ne, BcgShared &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
    for (int e = warp; e < ne; e += kBW) {
        const double *src = a.part + (size_t)(slot0 + e) * G;
        double s = 0.0;
        for (int c = lane; c < G; c += 32) s += __ldcg(src + c);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) sh.tot[slot0 + e] = s;
    }
    __syncthreads();
}

template <int KP>
__global__ void __launch_bounds__(kBT, 1) k_block_cg(BcgArgs a)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];   // kBW warp tiles
    __shared__ double s_red[kBT];
    __shared__ BcgShared sh;
    __shared__ int s_flag;
    const int k = a.k, G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = k * (k + 1) / 2;
    const int64_t t0 = a.ntiles * blockIdx.x / G, t1 = a.ntiles * (blockIdx.x + 1) / G;
    const int64_t rb = t0 < t1 ? __ldg(a.tdesc + 2 * t0) : 0;
    const int64_t re = t0 < t1 ? __ldg(a.tdesc + 2 * t1) : 0;
    int bno = 0;
    GbsWarpTile<double> &wt = reinterpret_cast<GbsWarpTile<double> *>(s_dyn)[warp];
    if (threadIdx.x == 0) {
        sh.status = GBS_DIVERGED_ITS;
        sh.it = 0;
    }

    // ---- set-up: R = B - A X, Z = D^-1 R, P = Z; Z^T R, ||R_j||^2, ||B_j||^2
    block_spmv<KP>(a, t0, t1, a.x, a.q, wt);
    __syncthreads();
    for (int64_t i = rb + threadIdx.x; i < re; i += kBT) {
        double bv[KP], av[KP], rv[KP], zv[KP];
        ld_row<KP>(a.b, i, bv);
        ld_row<KP>(a.q, i, av);
        const double di = __ldg(a.dinv + i);
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            rv[j] = bv[j] - av[j];
            zv[j] = di * rv[j];
        }
        st_row<KP>(a.r, i, rv);
        st_row<KP>(a.z, i, zv);
        st_row<KP>(a.p, i, zv);
    }
    __syncthreads();
    block_gram<KP, 1>(a, k, rb, re, a.z, a.r, np, s_red);   // Z^T R, ||R_j||^2: slots np ..
    block_gram<KP, 2>(a, k, rb, re, a.b, a.b, 0, s_red);    // ||B_j||^2: slots 0 .. k - 1
    if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) goto out;
    block_grid_sum(a, 0, 2 * np + k, sh);
    if (threadIdx.x == 0) {
        for (int c = 0; c < k; ++c) sh.bn[c] = sqrt(sh.tot[c]);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j <= i; ++j)
                sh.rho[i + j * k] = sh.rho[j + i * k] = sh.tot[np + tri(i, j)];
        sh.go = 1;
        bool done = true, nan_ = false;
        for (int c = 0; c < k; ++c) {
            const double rn = sqrt(sh.tot[2 * np + c]);
            a.res->rnorm[c] = rn;
            if (isnan(rn)) nan_ = true;
            if (!(rn <= a.rtol * sh.bn[c])) done = false;
        }
        if (nan_) { sh.status = GBS_ERR_NAN; sh.go = 0; }
        else if (done) { sh.status = GBS_OK; sh.go = 0; }
        else if (a.maxit <= 0) sh.go = 0;
    }
    __syncthreads();

    for (int it = 0; sh.go && it <= a.maxit; ++it) {
        // ---- S: Q = A P, P^T Q
        block_spmv<KP>(a, t0, t1, a.p, a.q, wt);
        __syncthreads();
        block_gram<KP, 0>(a, k, rb, re, a.p, a.q, 0, s_red);
        if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) goto out;
        block_grid_sum(a, 0, np, sh);
        if (warp == 0) {
            double pi[kKmax * kKmax];
            for (int i = 0; i < k; ++i)
                for (int j = 0; j <= i; ++j) pi[i + j * k] = pi[j + i * k] = sh.tot[tri(i, j)];
            const bool ok = ldl_solve_warp(k, pi, sh.rho, sh.mat, sh.fac);   // alpha
            if (lane == 0 && !ok) {
                sh.status = GBS_ERR_INDEFINITE;
                sh.go = 0;
            }
        }
        __syncthreads();
        if (!sh.go) break;

        // ---- U: X += P alpha, R -= Q alpha, Z = D^-1 R; Z^T R, ||R_j||^2
        for (int64_t i = rb + threadIdx.x; i < re; i += kBT) {
            double pv[KP], qv[KP], xv[KP], rv[KP], zv[KP];
            ld_row<KP>(a.p, i, pv);
            ld_row<KP>(a.q, i, qv);
            ld_row<KP>(a.x, i, xv);
            ld_row<KP>(a.r, i, rv);
            const double di = __ldg(a.dinv + i);
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                double xn = xv[j], rn = rv[j];
                if (j < k) {
#pragma unroll
                    for (int m = 0; m < KP; ++m)
                        if (m < k) {
                            const double al = sh.mat[m + j * k];
                            xn = fma(pv[m], al, xn);
                            rn = fma(-qv[m], al, rn);
                        }
                }
                xv[j] = xn;
                rv[j] = rn;
                zv[j] = di * rn;
            }
            st_row<KP>(a.x, i, xv);
            st_row<KP>(a.r, i, rv);
            st_row<KP>(a.z, i, zv);
        }
        __syncthreads();
        block_gram<KP, 1>(a, k, rb, re, a.z, a.r, np, s_red);
        if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) goto out;
        block_grid_sum(a, np, np + k, sh);
        if (warp == 0) {
            double rho2[kKmax * kKmax];
            for (int i = 0; i < k; ++i)
                for (int j = 0; j <= i; ++j) rho2[i + j * k] = rho2[j + i * k] = sh.tot[np + tri(i, j)];
            const bool ok = ldl_solve_warp(k, sh.rho, rho2, sh.mat, sh.fac);   // beta
            __syncwarp();
            if (lane == 0) {
                sh.it = it + 1;
                bool done = true, nan_ = false;
                for (int c = 0; c < k; ++c) {
                    const double rn = sqrt(sh.tot[2 * np + c]);
                    a.res->rnorm[c] = rn;
                    if (isnan(rn)) nan_ = true;
                    if (!(rn <= a.rtol * sh.bn[c])) done = false;
                }
                // the order of the tests: a breakdown of beta first, then
                // the stopping test of the new residual, then the limit
                if (!ok) { sh.status = GBS_ERR_INDEFINITE; sh.go = 0; }
                else if (nan_) { sh.status = GBS_ERR_NAN; sh.go = 0; }
                else if (done) { sh.status = GBS_OK; sh.go = 0; }
                else if (it + 1 >= a.maxit) { sh.status = GBS_DIVERGED_ITS; sh.go = 0; }
                for (int e = 0; e < k * k; ++e) sh.rho[e] = rho2[e];
            }
        }
        __syncthreads();
        if (!sh.go) break;

        // ---- P: P = Z + P beta
        for (int64_t i = rb + threadIdx.x; i < re; i += kBT) {
            double pv[KP], zv[KP], pn[KP];
            ld_row<KP>(a.p, i, pv);
            ld_row<KP>(a.z, i, zv);
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                double v = zv[j];
                if (j < k) {
#pragma unroll
                    for (int m = 0; m < KP; ++m)
                        if (m < k) v = fma(pv[m], sh.mat[m + j * k], v);
                }
                pn[j] = v;
            }
            st_row<KP>(a.p, i, pn);
        }
        if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) goto out;
    }
out:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const bool timed_out = a.bar->error != 0;
        a.res->status = timed_out ? GBS_ERR_TIMEOUT : sh.status;
        a.res->iters = sh.it;
        for (int c = 0; c < k; ++c) a.res->bnorm[c] = sh.bn[c];
    }
}

// Column-major (c * n + i) <-> interleaved (i * kp + c); padding zero.
__global__ void k_block_interleave(int64_t n, int k, int kp, const double *src, double *dst, int dir)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * kp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kp, c = e % kp;
        if (dir == 0) dst[e] = c < k ? src[c * n + i] : 0.0;
        else if (c < k) dst[c * n + i] = src[e];
    }
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int gbs_ksp_solve_cg_block(gbs_mat A, int k, gbs_vec B, gbs_vec X, double rtol, int maxit,
                                      gbs_solve_info *info, double *rnorm)
{
    if (!A || !B || !X || k < 1 || k > kKmax || !(rtol >= 0.0) || maxit < 0) return GBS_ERR_ARG;
    gbs_ctx c = A->ctx;
    if (B->ctx != c || X->ctx != c || A->n != A->ncols) return GBS_ERR_ARG;
    if (B->n != A->n * k || X->n != A->n * k || B->dtype != GBS_F64 || X->dtype != GBS_F64)
        return GBS_ERR_ARG;
    if (B->data == X->data && A->n > 0) return GBS_ERR_ARG;
    gbs_solve_info tmp;
    memset(&tmp, 0, sizeof(tmp));
    int st = GBS_OK;
    if (rnorm)
        for (int j = 0; j < k; ++j) rnorm[j] = 0.0;
    if (A->n == 0) {
        tmp.status = GBS_OK;
    } else if (!A->diag_ok) {
        st = tmp.status = GBS_ERR_DIAG;
    } else {
        GBS_CUDA_TRY(cudaSetDevice(c->device));
        if (!c->coop_supported) return GBS_ERR_UNSUPPORTED;
        const int kp = k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : 8;
        const void *fn = kp == 1 ? (const void *)k_block_cg<1>
                       : kp == 2 ? (const void *)k_block_cg<2>
                       : kp == 4 ? (const void *)k_block_cg<4> : (const void *)k_block_cg<8>;
        const size_t smem = sizeof(GbsWarpTile<double>) * kBW;
        GBS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBT, smem));
        if (per_sm < 1) return GBS_ERR_CUDA;
        // one CTA per 4 warp tiles at most: a block iteration's vector work
        // (about 3 k^2 + k^2 FP64 operations per row) is bound by the FP64
        // rate, so it wants every SM well before the SpMV does
        int64_t g = (int64_t)per_sm * c->num_sms;
        const int64_t need = (A->ntiles + 3) / 4;
        if (g > need) g = need;
        if (c->opts.persistent_ctas > 0 && c->opts.persistent_ctas < g) g = c->opts.persistent_ctas;
        const int G = g < 1 ? 1 : (int)g;
        const size_t n = (size_t)A->n, vec = al256(sizeof(double) * n * kp);
        const size_t head = 512, part = al256(sizeof(double) * kSlotsB * (size_t)G);
        const size_t total = head + al256(sizeof(BcgResult)) + part + 6 * vec;
        void *scr = nullptr;
        st = gbs_ctx_reserve(c, total, &scr);
        if (st) return st;
        char *base = (char *)scr;
        BcgArgs a;
        memset(&a, 0, sizeof(a));
        a.bar = (gbs_grid_barrier *)base;
        a.res = (BcgResult *)(base + head);
        a.part = (double *)(base + head + al256(sizeof(BcgResult)));
        char *v = base + head + al256(sizeof(BcgResult)) + part;
        double *bI = (double *)v; v += vec;
        a.x = (double *)v; v += vec;
        a.r = (double *)v; v += vec;
        a.z = (double *)v; v += vec;
        a.p = (double *)v; v += vec;
        a.q = (double *)v; v += vec;
        a.b = bI;
        a.n = A->n;
        a.ntiles = A->ntiles;
        a.tdesc = A->tdesc;
        a.rowptr = A->rowptr;
        a.colidx = A->colidx;
        a.vals = A->vals;
        a.dinv = A->dinv;
        a.rtol = rtol;
        a.k = k;
        a.maxit = maxit;
        a.timeout_ns = (unsigned long long)c->opts.barrier_timeout_ms * 1000000ull;
        const int gi = (int)std::min<int64_t>((int64_t)(n * kp + 255) / 256, (int64_t)c->num_sms * 8);
        GBS_CUDA_TRY(cudaMemsetAsync(base, 0, head + al256(sizeof(BcgResult)), c->stream));
        k_block_interleave<<<gi, 256, 0, c->stream>>>(A->n, k, kp, (const double *)B->data, bI, 0);
        k_block_interleave<<<gi, 256, 0, c->stream>>>(A->n, k, kp, (const double *)X->data, a.x, 0);
        gbs_count_launch(c, 2);
        GBS_CUDA_TRY(cudaGetLastError());
        GBS_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        void *args[] = {&a};
        GBS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBT), args, smem, c->stream));
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
        k_block_interleave<<<gi, 256, 0, c->stream>>>(A->n, k, kp, a.x, (double *)X->data, 1);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
        GBS_CUDA_TRY(cudaMemcpyAsync(c->pinned, a.res, sizeof(BcgResult), cudaMemcpyDeviceToHost,
                                     c->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        BcgResult r;
        memcpy(&r, c->pinned, sizeof(r));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        tmp.status = r.status;
        tmp.iters = r.iters;
        double mx = 0.0, bmx = 0.0;
        for (int j = 0; j < k; ++j) {
            if (rnorm) rnorm[j] = r.rnorm[j];
            if (r.rnorm[j] > mx) mx = r.rnorm[j];
            if (r.bnorm[j] > bmx) bmx = r.bnorm[j];
        }
        tmp.rnorm = mx;
        tmp.bnorm = bmx;
        tmp.device_ms = ms;
        // algorithmic bytes per iteration: matrix 12 nnz + row pointers 4n
        // and the P gather + Q write (16 n kp) in S, the P^T Q pass (16 n kp),
        // U (P, Q, X, R read, X, R, Z written: 56 n kp, D^-1 8n), the Z^T R
        // pass (16 n kp), P (P, Z read, P written: 24 n kp)
        const double nn = (double)A->n, nnz = (double)A->nnz;
        tmp.model_bytes = (double)r.iters * (12.0 * nnz + 12.0 * nn + 128.0 * nn * kp);
        st = r.status;
    }
    c->last = tmp;
    if (info) *info = tmp;
    return st;
}
