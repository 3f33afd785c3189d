// Jacobi-preconditioned Chebyshev iteration in one persistent cooperative
// kernel (KSPCHEBYSHEV with PCJACOBI: the paper's multigrid smoother,
// Sec. 5.3).  Chebyshev acceleration of the preconditioned Richardson
// iteration for a spectrum of D^-1 A inside [emin, emax] (Saad, Iterative
// Methods for Sparse Linear Systems, Algorithm 12.1, with z = D^-1 r where
// the direction is formed):
//
//   theta = (emax + emin) / 2, delta = (emax - emin) / 2
//   r = b - A x, d = z / theta, rho = delta / theta
//   repeat: c = 2 theta - rho delta
//           x += d;  r -= A d;  d = (rho delta / c) d + (2 / c) D^-1 r;  rho = delta / c
//
// The iteration has no inner product, so one grid barrier per iteration
// suffices: the SpMV's epilogue updates x, r and writes the next direction
// into the other half of a double buffer (neighbouring rows still gather
// the current one), and accumulates ||r||^2 for the stopping test, which
// every CTA evaluates from the same partials in the same order after the
// barrier.  The scalar recurrence does not depend on the data, so every
// thread carries it itself.

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "gbs_impl.cuh"

namespace {

constexpr size_t kChebSmem = (size_t)GBS_WARP_STAGE_BYTES * GBS_PWARPS;

struct ChebArgs {
    int64_t n, ntiles;
    const int32_t *tiles, *tdesc, *rowptr, *colidx;
    const int16_t *colrel16;   // col - row, streamed instead of colidx when set
    const double *vals, *dinv, *b;
    double *x, *r, *d0, *d1;
    double *part;   // [parity][r.r, b.b][G]
    GbsPipeCfg pipe;
    double theta, delta, rtol;
    int maxit;
    gbs_grid_barrier *bar;
    gbs_result_dev *res;
    unsigned long long timeout_ns;
};

// A row's own entries the iteration's epilogue needs.
struct RowVals {
    double x, r, dinv;
};

template <int NT>
struct ChebShared {
    double buf[2 * NT];
    double out[8];   // totals and part sums
    double rn, bn;
    int status;   // -100 while the iteration goes on
};

// Stopping test before iteration k (the oracle's order): NaN, converged,
// iteration limit, else go on (-100).
__device__ __forceinline__ int cheb_check(double rn, double tol, int k, int maxit)
{
    if (isnan(rn)) return GBS_ERR_NAN;
    if (rn <= tol) return GBS_OK;
    if (k >= maxit) return GBS_DIVERGED_ITS;
    return -100;
}

// NT threads per CTA (one CTA per SM), WB bytes of copy ring per warp: 32
// warps with 6.4 KB rings for large systems (more gathers in flight), else
// 16 warps with 12.8 KB rings.
// IX: the column indices the SpMV streams (int32, or 16-bit col - row).
template <int NT, int WB, typename IX>
__global__ void __launch_bounds__(NT, 1) k_chebyshev(ChebArgs a)
{
    const IX *cols = sizeof(IX) == 2 ? (const IX *)(const void *)a.colrel16
                                     : (const IX *)(const void *)a.colidx;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ChebShared<NT> sh;
    __shared__ GbsWarpQ s_q[NT / 32];
    __shared__ int s_next;
    __shared__ int s_flag;
    const int warp = threadIdx.x >> 5, G = gridDim.x, cta = blockIdx.x;
    gbs_warpq_init(s_q[warp]);
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const uint64_t ps = gbs_policy_stream(), pk = gbs_policy_keep();
    uint32_t parity = 0;
    unsigned char *wsm = smem + (size_t)warp * WB;
    const int64_t t0 = a.ntiles * cta / G, t1 = a.ntiles * (cta + 1) / G;
    const double theta = a.theta, delta = a.delta;
    int bno = 0, k = 0, status = GBS_ERR_TIMEOUT;

    // after each pass: CTA partials, grid barrier, every CTA's stopping test
    auto finish_pass = [&](double (&acc)[2], int par, int kk) -> bool {
        gbs_block_sum_staged<double, 2, NT>(acc, sh.buf, sh.out);
        if (threadIdx.x == 0) {
            s_next = 0;
            a.part[(2 * par + 0) * G + cta] = sh.out[0];
            a.part[(2 * par + 1) * G + cta] = sh.out[1];
        }
        if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) return false;
        if (warp == 0) {
            double t[2];
            gbs_warp_grid_sum<double, 2>(a.part + 2 * par * G, G, G, t);
            if (threadIdx.x == 0) {
                if (kk == 0) sh.bn = sqrt(t[1]);
                sh.rn = sqrt(t[0]);
                sh.status = cheb_check(sh.rn, a.rtol * sh.bn, kk, a.maxit);
            }
        }
        __syncthreads();
        return true;
    };

    // ---- set-up: r = b - A x, d = D^-1 r / theta; partials r.r, b.b
    {
        double acc[2] = {0.0, 0.0};
        auto epi = [&](int64_t i, double s, double) {
            const double bi = gbs_ld(a.b + i, pk);
            const double ri = bi - s;
            gbs_st(a.r + i, ri, pk);
            gbs_st(a.d0 + i, (gbs_ld(a.dinv + i, pk) * ri) / theta, pk);
            acc[0] += ri * ri;
            acc[1] += bi * bi;
        };
        if (!gbs_spmv_pipe<double, IX>(a.tdesc, t0, t1, &s_next, a.rowptr, cols, a.vals, a.x, wsm,
                                   s_q[warp], parity, a.pipe, ps, pk, a.timeout_ns, epi) &&
            (threadIdx.x & 31) == 0)
            atomicCAS(&a.bar->error, 0, GBS_ERR_TIMEOUT);
        if (!finish_pass(acc, 0, 0)) goto out;
    }
    status = sh.status;
    {
        double rho = delta / theta;
        // every thread also bounds its own loop, whatever the shared record says
        for (int it = 0; status == -100 && it <= a.maxit; ++it) {
            const double cc = 2.0 * theta - rho * delta;
            const double a1 = (rho * delta) / cc, a2 = 2.0 / cc;
            const double *dc = (k & 1) ? a.d1 : a.d0;
            double *dn = (k & 1) ? a.d0 : a.d1;
            double acc[2] = {0.0, 0.0};
            // ---- q = A d; x += d; r -= q; next d; partial r.r (d_i is the
            // operand the row's diagonal entry gathered; x_i, r_i and D^-1_i
            // are loaded before the row's gathers, so they arrive with them)
            auto pre = [&](int64_t i) {
                RowVals v;
                v.x = gbs_ld(a.x + i, pk);
                v.r = gbs_ld(a.r + i, pk);
                v.dinv = gbs_ld(a.dinv + i, pk);
                return v;
            };
            auto epi = [&](int64_t i, double s, double di, const RowVals &v) {
                gbs_st(a.x + i, v.x + di, pk);
                const double ri = v.r - s;
                gbs_st(a.r + i, ri, pk);
                gbs_st(dn + i, fma(a1, di, a2 * (v.dinv * ri)), pk);
                acc[0] += ri * ri;
            };
            if (!gbs_spmv_pipe_pre<double, IX>(a.tdesc, t0, t1, &s_next, a.rowptr, cols, a.vals, dc,
                                           wsm, s_q[warp], parity, a.pipe, ps, pk, a.timeout_ns, pre,
                                           epi) &&
                (threadIdx.x & 31) == 0)
                atomicCAS(&a.bar->error, 0, GBS_ERR_TIMEOUT);
            rho = delta / cc;
            ++k;
            if (!finish_pass(acc, k & 1, k)) {
                status = GBS_ERR_TIMEOUT;
                break;
            }
            status = sh.status;
        }
        if (status == -100) status = GBS_DIVERGED_ITS;
    }
out:
    if (cta == 0 && threadIdx.x == 0) {
        a.res->status = status;
        a.res->iters = k;
        a.res->outer = 0;
        a.res->rnorm = sh.rn;
        a.res->bnorm = sh.bn;
        a.res->timeout_where = status == GBS_ERR_TIMEOUT ? a.bar->where : -1;
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int gbs_ksp_solve_chebyshev(gbs_mat A, gbs_vec b, gbs_vec x, double emin, double emax,
                                       double rtol, int maxit, gbs_solve_info *info)
{
    if (!A || !b || !x) return GBS_ERR_ARG;
    gbs_ctx c = A->ctx;
    if (b->ctx != c || x->ctx != c) return GBS_ERR_ARG;
    if (A->n != A->ncols || b->n != A->n || x->n != A->n) return GBS_ERR_ARG;
    if (b->dtype != GBS_F64 || x->dtype != GBS_F64) return GBS_ERR_ARG;
    if (b->data == x->data && A->n > 0) return GBS_ERR_ARG;
    if (!(rtol >= 0.0) || maxit < 0) return GBS_ERR_ARG;
    if (!(emin > 0.0) || !(emax >= emin) || isinf(emax)) return GBS_ERR_ARG;
    gbs_solve_info tmp;
    memset(&tmp, 0, sizeof(tmp));
    int st = GBS_OK;
    if (A->n == 0) {
        tmp.status = GBS_OK;
    } else if (!A->diag_ok) {
        st = tmp.status = GBS_ERR_DIAG;
    } else {
        GBS_CUDA_TRY(cudaSetDevice(c->device));
        if (!c->coop_supported) return GBS_ERR_UNSUPPORTED;
        // launch shape: 32 warps with 6.4 KB rings when two stages of the largest
        // tile fit and there are at least 32 tiles per SM
        constexpr int kWide = 2 * GBS_PBLOCK, kRing = GBS_WARP_STAGE_BYTES / 2;
        if (!c->opts.no_rel16) {
            st = gbs_mat_ensure_rel16(A);
            if (st) return st;
        }
        const bool rel = A->colrel16 && !c->opts.no_rel16;
        GbsPipeCfg cfg = rel ? A->pipe64r : A->pipe64;
        const int st6 = kRing / cfg.sbytes;
        const bool wide = st6 >= 2 && A->ntiles >= (int64_t)c->num_sms * (kWide / 32);
        const void *fn =
            rel ? (wide ? (const void *)k_chebyshev<kWide, kRing, int16_t>
                        : (const void *)k_chebyshev<GBS_PBLOCK, GBS_WARP_STAGE_BYTES, int16_t>)
                : (wide ? (const void *)k_chebyshev<kWide, kRing, int32_t>
                        : (const void *)k_chebyshev<GBS_PBLOCK, GBS_WARP_STAGE_BYTES, int32_t>);
        const int nt = wide ? kWide : GBS_PBLOCK;
        const size_t smem = wide ? (size_t)kRing * (kWide / 32) : kChebSmem;
        if (wide) cfg.stages = st6 < GBS_MAX_STAGES ? st6 : GBS_MAX_STAGES;
        GBS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        int per_sm = 0;
        GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
        if (per_sm < 1) return GBS_ERR_CUDA;
        int64_t g = (int64_t)per_sm * c->num_sms;
        const int64_t need = (A->ntiles + nt / 32 - 1) / (nt / 32);
        if (g > need) g = need;
        const int G = g < 1 ? 1 : (int)g;
        const size_t head = 512;   // barrier + result record
        const size_t part = align256(sizeof(double) * 4 * (size_t)G);
        const size_t vec = align256(sizeof(double) * (size_t)A->n);
        void *scr = nullptr;
        st = gbs_ctx_reserve(c, head + part + 3 * vec, &scr);
        if (st) return st;
        char *base = (char *)scr;
        ChebArgs a;
        memset(&a, 0, sizeof(a));
        a.bar = (gbs_grid_barrier *)base;
        a.res = (gbs_result_dev *)(base + 256);
        a.part = (double *)(base + head);
        a.r = (double *)(base + head + part);
        a.d0 = (double *)(base + head + part + vec);
        a.d1 = (double *)(base + head + part + 2 * vec);
        a.n = A->n;
        a.ntiles = A->ntiles;
        a.tiles = A->tiles;
        a.tdesc = A->tdesc;
        a.rowptr = A->rowptr;
        a.colidx = A->colidx;
        a.colrel16 = rel ? A->colrel16 : nullptr;
        a.vals = A->vals;
        a.dinv = A->dinv;
        a.pipe = cfg;
        a.b = (const double *)b->data;
        a.x = (double *)x->data;
        a.theta = 0.5 * (emax + emin);
        a.delta = 0.5 * (emax - emin);
        a.rtol = rtol;
        a.maxit = maxit;
        a.timeout_ns = (unsigned long long)c->opts.barrier_timeout_ms * 1000000ull;
        GBS_CUDA_TRY(cudaMemsetAsync(base, 0, head, c->stream));
        GBS_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        void *args[] = {&a};
        GBS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(nt), args, smem, c->stream));
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
        GBS_CUDA_TRY(cudaMemcpyAsync(c->pinned, a.res, sizeof(gbs_result_dev),
                                     cudaMemcpyDeviceToHost, c->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        gbs_result_dev r;
        memcpy(&r, c->pinned, sizeof(r));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        tmp.status = r.status;
        tmp.iters = r.iters;
        tmp.rnorm = r.rnorm;
        tmp.bnorm = r.bnorm;
        tmp.device_ms = ms;
        // algorithmic bytes: the set-up pass (matrix, rowptr, x gather, b and
        // D^-1 read, r and d written), then per iteration the matrix, rowptr,
        // the d gather, x and r read and written, D^-1 read, d written; a
        // nonzero is 8 bytes of value and 4 or 2 of column index
        const double n = (double)A->n, nnz = (double)A->nnz, bnz = rel ? 10.0 : 12.0;
        tmp.model_bytes = (bnz * nnz + 4 * (n + 1) + 40 * n) + r.iters * (bnz * nnz + 4 * (n + 1) + 56 * n);
        st = r.status;
    }
    c->last = tmp;
    if (info) *info = tmp;
    return st;
}
