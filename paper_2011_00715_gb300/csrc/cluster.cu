// FP64 Jacobi-PCG for small systems in one thread-block cluster
// (Challenge A1: below a few tens of thousands of rows a solve is bound by
// synchronisation latency, not by bandwidth).
//
// The grid-wide persistent kernel pays three software grid barriers per
// iteration across all 152 SMs.  A small system instead runs in one cluster
// of up to 16 CTAs: CTA k owns the rows [k R, (k+1) R), R = ceil(n / CTAs),
// and keeps x, r, p, A p and D^-1 of those rows in its shared memory.  The
// SpMV reads the direction vector p of other CTAs' rows through distributed
// shared memory, and the CTAs synchronise with the hardware cluster
// barrier.  One SM alone would not do: GB300 issues about two FP64 FMAs per
// clock per SM, so the iteration's FP64 work is spread over the cluster.
//
// Same iteration, stopping test and statuses as the persistent kernel
// (textbook PCG, Saad Alg. 9.1; ||r|| <= rtol ||b|| before each iteration).
// z = D^-1 r is not stored: it is recomputed as one rounded product where
// it is needed.
//
// Reductions are deterministic: each thread sums its rows in order, a fixed
// staged tree over the threads' values gives the CTA's partial,
// which every CTA writes into its slot of every CTA's shared memory; after
// the cluster barrier every CTA adds the slots by the same fixed tree, so
// all CTAs hold bitwise the same scalars and take the same branches (every
// CTA meets every cluster barrier).  No wait in this kernel spins on memory: the only
// waits are the CTA and cluster barriers, which all CTAs reach on the same
// control path.

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <atomic>

#include "gbs_impl.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kCT = 512;                 // threads per CTA (256 when a CTA owns at most 256 rows)
constexpr int kCTSmall = 256;
constexpr int kMaxCluster = 16;          // the opt-in (non-portable) cluster size
constexpr int kPortableCluster = 8;
constexpr int kMinRows = 128;            // rows per CTA at least
constexpr int kMaxRowsPerCta = GBS_CLUSTER_MAX_ROWS / kPortableCluster;
constexpr size_t kMaxSmem = (size_t)5 * kMaxRowsPerCta * sizeof(double);
static_assert(kMaxSmem <= 200 * 1024, "five FP64 vectors of R rows fit in shared memory");
static_assert((uint64_t)GBS_CLUSTER_MAX_ROWS * kMaxRowsPerCta < (1ull << 32),
              "column / R by a multiply-high is exact");

struct ClArgs {
    int n;
    int rows;                // rows per CTA (R)
    unsigned int rmagic;     // floor(2^32 / R) + 1: c / R = umulhi(c, rmagic) for c < n
    const int32_t *rowptr, *colidx;
    const double *vals, *dinv, *b;
    double *x;               // initial guess in, solution out (global)
    double rtol;
    int maxit;
    int norm;                // GBS_NORM_* of the stopping test
    gbs_result_dev *res;
};

template <int CT>
struct ClShared {
    double *pseg[kMaxCluster];           // each rank's p segment, as this CTA addresses it
    double init[3 * kMaxCluster];        // set-up partials r.z, r.r, b.b; slot = writing rank
    double pq[kMaxCluster];              // p.Ap partials
    double u[2 * kMaxCluster];           // r.z, r.r partials after the update
    double stage[3][CT];                 // per-thread values of a CTA sum
    double part[3][4];                   // per-warp sums of a CTA sum
    double alpha, beta;
    double rn;                           // square root of the stopping test (warp 1)
    int go, status;
};

__device__ __forceinline__ int cl_check(double rn, double rho, double tol, int k, int maxit)
{
    if (isnan(rn) || isnan(rho)) return GBS_ERR_NAN;
    if (rn <= tol) return GBS_OK;
    if (k >= maxit) return GBS_DIVERGED_ITS;
    return -100;
}

// The CTA's sum of v, written into slot `rank` of dst[k * kMaxCluster] in
// the shared memory of every CTA of the cluster; the caller's next cluster
// barrier publishes the writes.  Staged so as to spend few FP64
// instructions: an SM partition retires about one FP64 warp instruction
// per 76 cycles, whether or not its lanes are all useful, so a shuffle
// tree in every warp is costly.  Every thread stages its K values; W = 4/K
// warps per value (one per SM partition where possible) each add their
// share of the entries per lane and finish with a shuffle tree; one lane
// per value adds the W part sums.  A fixed order throughout.
template <int K, int CT>
__device__ __forceinline__ void cta_publish(const double (&v)[K], double *dst, ClShared<CT> &s,
                                            cg::cluster_group &cl, int rank, int cs)
{
    constexpr int W = K >= 3 ? 1 : 4 / K;   // warps per value
    constexpr int PER = CT / 32 / W;        // entries per lane
    static_assert(W * K <= CT / 32 && W <= 4, "warps per value");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) s.stage[k][threadIdx.x] = v[k];
    __syncthreads();
    if (warp < W * K) {
        const int k = warp / W, j = warp % W;
        const double *src = s.stage[k] + j * (CT / W) + lane;
        double t = src[0];
#pragma unroll
        for (int m = 1; m < PER; ++m) t += src[32 * m];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) s.part[k][j] = t;
    }
    __syncthreads();
    if (warp == 0) {
        double t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (W == 4) t[k] = (s.part[k][0] + s.part[k][1]) + (s.part[k][2] + s.part[k][3]);
            else if (W == 2) t[k] = s.part[k][0] + s.part[k][1];
            else t[k] = s.part[k][0];
        }
        if (lane < cs) {
#pragma unroll
            for (int k = 0; k < K; ++k) cl.map_shared_rank(dst + k * kMaxCluster, lane)[rank] = t[k];
        }
    }
}

// Sum of the cs published partials by a fixed tree over the slots (the
// same in every CTA); called by a whole warp, the total is in its lane 0.  A
// tree rather than a running sum: each dependent FP64 step costs a full
// pass of the warp through the narrow FP64 pipe.
__device__ __forceinline__ double cluster_total(const double *slots, int cs)
{
    const int lane = threadIdx.x & 31;
    double t = lane < cs ? slots[lane] : 0.0;
#pragma unroll
    for (int off = kMaxCluster / 2; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    return t;
}

template <int CT>
__global__ void __launch_bounds__(CT, 1) k_pcg_cluster(ClArgs a)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ ClShared<CT> s;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), cs = (int)cl.num_blocks();
    const int R = a.rows, lo = rank * R;
    const int nl = max(0, min(a.n - lo, R));   // rows this CTA owns
    double *x = sm, *r = sm + R, *p = sm + 2 * R, *q = sm + 3 * R, *dinv = sm + 4 * R;
    if (threadIdx.x < cs) s.pseg[threadIdx.x] = cl.map_shared_rank(p, (int)threadIdx.x);

    // ---- set-up: r = b - A x0 (x0 read from global memory), p = z = D^-1 r
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nl; i += CT) {
        const int gi = lo + i;
        double sum = 0.0;
        const int e1 = __ldg(a.rowptr + gi + 1);
        for (int e = __ldg(a.rowptr + gi); e < e1; ++e)
            sum = fma(__ldg(a.vals + e), __ldg(a.x + __ldg(a.colidx + e)), sum);
        const double bi = __ldg(a.b + gi), di = __ldg(a.dinv + gi);
        const double ri = bi - sum, zi = __dmul_rn(di, ri);
        x[i] = __ldg(a.x + gi);
        dinv[i] = di;
        r[i] = ri;
        p[i] = zi;
        acc[0] = fma(ri, zi, acc[0]);
        const double w = a.norm == GBS_NORM_PRECONDITIONED ? zi : ri;
        acc[1] = fma(w, w, acc[1]);
        if (a.norm == GBS_NORM_UNPRECONDITIONED) {
            acc[2] = fma(bi, bi, acc[2]);
        } else {
            const double db = __dmul_rn(di, bi);
            acc[2] = a.norm == GBS_NORM_PRECONDITIONED ? fma(db, db, acc[2]) : fma(bi, db, acc[2]);
        }
    }
    // every CTA of the cluster is running before the first remote access
    cl.sync();
    cta_publish<3, CT>(acc, s.init, s, cl, rank, cs);
    cl.sync();
    // scalar state, meaningful in thread 0 only; rr holds N(r)^2 of the
    // stopping-test norm N (r.r, z.z, or r.z for the natural norm)
    const bool natural = a.norm == GBS_NORM_NATURAL;
    double rho = 0.0, rr = 0.0, bnorm = 0.0;
    int k = 0, status = GBS_DIVERGED_ITS;
    if (threadIdx.x < 32) {
        rho = cluster_total(s.init, cs);
        rr = natural ? rho : cluster_total(s.init + kMaxCluster, cs);
        bnorm = cluster_total(s.init + 2 * kMaxCluster, cs);
    }
    if (threadIdx.x == 0) {
        bnorm = sqrt(bnorm);
        const int st = cl_check(sqrt(rr), rho, a.rtol * bnorm, 0, a.maxit);
        s.go = st == -100;
        if (!s.go) status = st;
    }
    __syncthreads();

    const unsigned int rm = a.rmagic;
    for (int kk = 0; s.go && kk <= a.maxit; ++kk) {
        // ---- S: q = A p (p of other CTAs' rows through distributed shared
        // memory), partial p.q
        double pq[1] = {0.0};
        for (int i = threadIdx.x; i < nl; i += CT) {
            const int gi = lo + i;
            double sum = 0.0;
            const int e1 = __ldg(a.rowptr + gi + 1);
            for (int e = __ldg(a.rowptr + gi); e < e1; ++e) {
                const int c = __ldg(a.colidx + e);
                const int owner = (int)__umulhi((unsigned int)c, rm), off = c - owner * R;
                const double pc = owner == rank ? p[off] : s.pseg[owner][off];
                sum = fma(__ldg(a.vals + e), pc, sum);
            }
            q[i] = sum;
            pq[0] = fma(p[i], sum, pq[0]);
        }
        cta_publish<1, CT>(pq, s.pq, s, cl, rank, cs);
        cl.sync();
        double pi = 0.0;
        if (threadIdx.x < 32) pi = cluster_total(s.pq, cs);
        if (threadIdx.x == 0) {
            if (isnan(pi)) status = GBS_ERR_NAN;
            else if (pi <= 0.0) status = GBS_ERR_INDEFINITE;
            s.go = !(isnan(pi) || pi <= 0.0);
            s.alpha = rho / pi;
        }
        __syncthreads();
        if (!s.go) break;
        const double alpha = s.alpha;

        // ---- U: x += alpha p; r -= alpha q; partials r.z, r.r
        double u[2] = {0.0, 0.0};
        for (int i = threadIdx.x; i < nl; i += CT) {
            x[i] = fma(alpha, p[i], x[i]);
            const double ri = fma(-alpha, q[i], r[i]);
            r[i] = ri;
            const double zi = __dmul_rn(dinv[i], ri);
            u[0] = fma(ri, zi, u[0]);
            const double w = a.norm == GBS_NORM_PRECONDITIONED ? zi : ri;
            u[1] = fma(w, w, u[1]);
        }
        cta_publish<2, CT>(u, s.u, s, cl, rank, cs);
        cl.sync();
        // warps 0 and 1 form the same totals; warp 0 divides for beta while
        // warp 1 takes the stopping test's square root, side by side
        double rho_new = 0.0, rr_new = 0.0;
        if (threadIdx.x < 64) {
            rho_new = cluster_total(s.u, cs);
            rr_new = cluster_total(s.u + kMaxCluster, cs);
            if (threadIdx.x == 32) s.rn = sqrt(natural ? rho_new : rr_new);
            if (threadIdx.x == 0) s.beta = rho_new / rho;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ++k;
            rr = natural ? rho_new : rr_new;
            if (rho_new < 0.0) {
                status = GBS_ERR_INDEFINITE;
                s.go = 0;
            } else {
                rho = rho_new;
                const int st = cl_check(s.rn, rho, a.rtol * bnorm, k, a.maxit);
                s.go = st == -100;
                if (!s.go) status = st;
            }
        }
        __syncthreads();
        if (!s.go) break;
        const double beta = s.beta;

        // ---- P: p = z + beta p on this CTA's rows; the barrier publishes
        // them to the next SpMV of every CTA
        for (int i = threadIdx.x; i < nl; i += CT) p[i] = fma(beta, p[i], __dmul_rn(dinv[i], r[i]));
        cl.sync();
    }
    for (int i = threadIdx.x; i < nl; i += CT) a.x[lo + i] = x[i];
    if (rank == 0 && threadIdx.x == 0) {
        a.res->status = status;
        a.res->iters = k;
        a.res->outer = 0;
        a.res->rnorm = sqrt(rr);
        a.res->bnorm = bnorm;
        a.res->timeout_where = -1;
    }
    // no CTA leaves while another may still address its shared memory
    cl.sync();
}

// Largest cluster a launch of k_pcg_cluster with the largest shared-memory
// size can keep resident on the device: 16 where the opt-in size fits, 8
// (portable) otherwise, 0 if not even that.  Cached per device.
std::atomic<int> g_cluster_max[64];

int cluster_max(int device)
{
    if (device < 0 || device >= 64) return 0;
    int v = g_cluster_max[device].load();
    if (v) return v > 0 ? v : 0;
    const void *fn = (const void *)k_pcg_cluster<kCT>;
    const void *fn_small = (const void *)k_pcg_cluster<kCTSmall>;
    int found = -1;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem) ==
            cudaSuccess &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(fn_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMaxSmem) == cudaSuccess &&
        cudaFuncSetAttribute(fn_small, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
        for (int cs : {kMaxCluster, kPortableCluster}) {
            cudaLaunchConfig_t cfg;
            memset(&cfg, 0, sizeof(cfg));
            cfg.gridDim = dim3(cs);
            cfg.blockDim = dim3(kCT);
            cfg.dynamicSmemBytes = kMaxSmem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cs;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc > 0) {
                found = cs;
                break;
            }
        }
    }
    cudaGetLastError();   // a refused query leaves no sticky error behind
    g_cluster_max[device].store(found);
    return found > 0 ? found : 0;
}

}  // namespace

int gbs_solve_cluster(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit, int norm,
                      gbs_solve_info *info)
{
    gbs_ctx c = A->ctx;
    const int64_t n = A->n;
    if (n <= 0 || n > GBS_CLUSTER_MAX_ROWS) return GBS_ERR_UNSUPPORTED;
    const int csmax = cluster_max(c->device);
    if (csmax == 0) return GBS_ERR_UNSUPPORTED;
    // as many CTAs as the cluster allows while each keeps kMinRows rows
    int64_t want = (n + kMinRows - 1) / kMinRows;
    const int cs = (int)(want < csmax ? want : csmax);
    const int rows = (int)((n + cs - 1) / cs);
    if (rows > kMaxRowsPerCta) return GBS_ERR_UNSUPPORTED;
    void *scr = nullptr;
    const int st = gbs_ctx_reserve(c, 256, &scr);
    if (st) return st;
    ClArgs a;
    memset(&a, 0, sizeof(a));
    a.n = (int)n;
    a.rows = rows;
    // one CTA: every column is its own (umulhi(c, 0) = 0); else rows >= 64,
    // so the multiplier fits in 32 bits
    a.rmagic = cs == 1 ? 0u : (unsigned int)((1ull << 32) / (uint64_t)rows) + 1u;
    a.rowptr = A->rowptr;
    a.colidx = A->colidx;
    a.vals = A->vals;
    a.dinv = A->dinv;
    a.b = (const double *)b->data;
    a.x = (double *)x->data;
    a.rtol = rtol;
    a.maxit = maxit;
    a.norm = norm;
    a.res = (gbs_result_dev *)scr;
    // one row per thread where the CTA owns at most 256 rows: fewer warps
    // make the CTA-wide sums and barriers cheaper
    const bool small = rows <= kCTSmall;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(small ? kCTSmall : kCT);
    cfg.dynamicSmemBytes = (size_t)5 * rows * sizeof(double);
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GBS_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    if (small)
        GBS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_pcg_cluster<kCTSmall>, a));
    else
        GBS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_pcg_cluster<kCT>, a));
    gbs_count_launch(c);
    GBS_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    GBS_CUDA_TRY(cudaMemcpyAsync(c->pinned, a.res, sizeof(gbs_result_dev), cudaMemcpyDeviceToHost,
                                 c->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    gbs_result_dev r;
    memcpy(&r, c->pinned, sizeof(r));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->status = r.status;
    info->iters = r.iters;
    info->outer_iters = 0;
    info->rnorm = r.rnorm;
    info->bnorm = r.bnorm;
    info->device_ms = ms;
    return r.status;
}
