// Batched Jacobi-PCG over many independent systems with several right-hand
// sides each, in one persistent cooperative kernel (Response A6: solve many
// different-size problems at once; Challenge F2 and Sec. 4: multiple
// right-hand sides raise arithmetic intensity; Response A7: FP32 inner
// iterations with FP64 refinement).
//
// Lockstep design.  Every active system advances by one step per global
// iteration; a step has five phases separated by grid barriers:
//   S   SpMV over every warp tile of every active system (all k columns
//       of a system share one pass over its matrix), per-tile partials
//   R1  per-(system, column) reductions of the S partials, in a fixed
//       order over the system's tiles
//   U   vector updates per tile, per-tile partials
//   R2  per-(system, column) reductions of the U partials
//   P   direction update, or the FP64 solution update before a refinement
// A system is either in an INNER step (one PCG iteration in the inner
// precision TI on all its unfinished columns) or an OUTER step (FP64
// residual r = b - A x, stopping test, r / ||r|| becomes the inner
// right-hand side).  Its columns advance together; a column whose inner
// solve has converged waits for the others, then all refine together.
// Because every per-system quantity depends only on the system's own tiles
// and a fixed reduction order, each column's result is bitwise the same
// alone or in any batch.
//
// Multi-vectors are interleaved (entry (row, column) at row * k + column),
// so the k operands one nonzero gathers are contiguous.
//
// The kernel runs at most `quantum` global iterations and returns; all
// state lives in device memory, so the host can retire finished systems
// and admit new ones between launches (continuous batching).

#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gbs_impl.cuh"

#define GBS_KMAX 8
#define GBS_RUNNING (-100)

namespace {

enum { MODE_OUTER = 0, MODE_INNER = 1 };

// Read-only description of one system (device).
struct BSys {
    const int32_t *rowptr, *colidx, *tiles;
    const double *vals, *dinv;
    const float *vals32, *dinv32;
    const double *b;    // n * k, interleaved
    double *x;          // n * k, interleaved (initial guess in, solution out)
    double *r64;        // n * k
    void *xi, *ri, *zi, *pi, *qi;   // inner-precision work vectors, n * k
    int n, k, ntiles, gtile0;
    double rtol;
    int maxit;
    int pad;
};

// Mutable state of one (system, column) pair (device).
struct BCol {
    double rho, rr, alpha, beta, rn, bnorm, prev, scale, tol_inner;
    int status;       // GBS_RUNNING until final
    int iters;        // inner iterations, all refinement steps together
    int outer;        // refinement steps
    int kin;          // inner iterations of the current refinement step
    int inner_done;   // the current inner solve has stopped
    int first;        // no residual computed yet
    int pad[2];
};

// Mutable per-system state (device).
struct BSysDyn {
    int mode[2];      // indexed by global iteration parity
    int finished;
    int pad;
};

struct BArgs {
    const BSys *sys;
    BCol *col;          // sys index * GBS_KMAX + column
    BSysDyn *dyn;
    const int2 *tiles;  // active tiles {system, local tile}, ntile entries
    int ntile;
    const int2 *pairs;  // active {system, column} pairs, npair entries
    int npair;
    double *partS;      // global tile * GBS_KMAX * 2
    double *partU;      // global tile * GBS_KMAX * 2
    gbs_grid_barrier *bar;
    int quantum;
    int iter0;          // global iteration count at launch (parity of mode[])
    double inner_rtol;
    int outer_maxit;
    int fp64;           // inner precision is FP64 (FP64 mode)
    unsigned long long timeout_ns;
};

// Staging of one warp tile's colidx/vals in shared memory.
template <typename V>
struct BTile {
    int32_t col[GBS_WT_NNZ];
    V val[GBS_WT_NNZ];
};

__device__ __forceinline__ double bmac(double a, double x, double s) { return fma(a, x, s); }
__device__ __forceinline__ float bmac(float a, float x, float s) { return fmaf(a, x, s); }

// y_c = (A v_c)(row) for the rows of one warp tile and all k columns;
// epi(row, sums[]) runs in the lane that owns the row.
template <typename V, typename X, typename Epi>
__device__ __forceinline__ void tile_spmv_k(const BSys &S, const V *vals, const X *v, int lt,
                                            BTile<V> &wt, Epi &epi)
{
    const int lane = threadIdx.x & 31;
    const int k = S.k;
    const int r0 = __ldg(S.tiles + lt), r1 = __ldg(S.tiles + lt + 1);
    const int nrows = r1 - r0;
    int beg = 0, end = 0;
    if (lane < nrows) {
        beg = __ldg(S.rowptr + r0 + lane);
        end = __ldg(S.rowptr + r0 + lane + 1);
    }
    const int k0 = __shfl_sync(0xffffffffu, beg, 0);
    const int k1 = __shfl_sync(0xffffffffu, end, nrows - 1);
    X sum[GBS_KMAX];
#pragma unroll
    for (int c = 0; c < GBS_KMAX; ++c) sum[c] = X(0);
    if (k1 - k0 <= GBS_WT_NNZ) {
        for (int e = k0 + lane; e < k1; e += 32) {
            wt.col[e - k0] = __ldg(S.colidx + e);
            wt.val[e - k0] = __ldg(vals + e);
        }
        __syncwarp();
        if (lane < nrows) {
            for (int e = beg; e < end; ++e) {
                const X a = (X)wt.val[e - k0];
                const X *vp = v + (size_t)wt.col[e - k0] * k;
#pragma unroll
                for (int c = 0; c < GBS_KMAX; ++c)
                    if (c < k) sum[c] = bmac(a, vp[c], sum[c]);
            }
            epi(r0 + lane, sum);
        }
        __syncwarp();
    } else {
        // one long row: strided partial sums per column, fixed shuffle tree
        for (int e = k0 + lane; e < k1; e += 32) {
            const X a = (X)__ldg(vals + e);
            const X *vp = v + (size_t)__ldg(S.colidx + e) * k;
#pragma unroll
            for (int c = 0; c < GBS_KMAX; ++c)
                if (c < k) sum[c] = bmac(a, vp[c], sum[c]);
        }
#pragma unroll
        for (int c = 0; c < GBS_KMAX; ++c)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], off);
        if (lane == 0) epi(r0, sum);
        __syncwarp();
    }
}

// Warp-wide fixed-tree sum of per-lane values; lane 0 stores them.
template <typename T>
__device__ __forceinline__ void warp_store_partials(T (&a)[GBS_KMAX][2], int k, double *dst)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < GBS_KMAX; ++c) {
        if (c >= k) break;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            T t = a[c][j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) dst[c * 2 + j] = (double)t;
        }
    }
}

// Sum entry j of column c over the system's tiles in a fixed order
// (lane l: tiles l, l + 32, ... in type T; then a fixed shuffle tree).
template <typename T>
__device__ __forceinline__ T sys_sum(const double *part, const BSys &S, int c, int j)
{
    const int lane = threadIdx.x & 31;
    T t = T(0);
    for (int i = lane; i < S.ntiles; i += 32)
        t += (T)__ldcg(part + ((size_t)(S.gtile0 + i) * GBS_KMAX + c) * 2 + j);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
}

__device__ __forceinline__ bool col_running(const BCol &c) { return c.status == GBS_RUNNING; }

template <typename TI>
__global__ void __launch_bounds__(GBS_PBLOCK) k_batched(BArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const int gw = blockIdx.x * GBS_PWARPS + warp, nw = G * GBS_PWARPS;
    BTile<double> &wt64 = reinterpret_cast<BTile<double> *>(smem)[warp];
    BTile<float> &wt32 = *reinterpret_cast<BTile<float> *>(&wt64);
    int bno = 0;
    bool ok = true;

    for (int q = 0; q < a.quantum && ok; ++q) {
        const int it = a.iter0 + q;
        const int cur = it & 1, nxt = cur ^ 1;

        // ---------------- S: SpMV per tile
        for (int g = gw; g < a.ntile; g += nw) {
            const int2 tl = a.tiles[g];
            const BSys &S = a.sys[tl.x];
            const BSysDyn &D = a.dyn[tl.x];
            if (D.finished) continue;
            const int k = S.k;
            double *dst = a.partS + (size_t)(S.gtile0 + tl.y) * GBS_KMAX * 2;
            if (D.mode[cur] == MODE_OUTER) {
                // r64 = b - A x (FP64), partials r.r and b.b
                double acc[GBS_KMAX][2];
#pragma unroll
                for (int c = 0; c < GBS_KMAX; ++c) acc[c][0] = acc[c][1] = 0.0;
                auto epi = [&](int row, double(&s)[GBS_KMAX]) {
#pragma unroll
                    for (int c = 0; c < GBS_KMAX; ++c) {
                        if (c >= k) break;
                        const size_t o = (size_t)row * k + c;
                        const double bi = S.b[o];
                        const double ri = bi - s[c];
                        S.r64[o] = ri;
                        acc[c][0] += ri * ri;
                        acc[c][1] += bi * bi;
                    }
                };
                tile_spmv_k<double, double>(S, S.vals, S.x, tl.y, wt64, epi);
                warp_store_partials<double>(acc, k, dst);
            } else {
                // q = A p (inner precision), partial p.q
                TI acc[GBS_KMAX][2];
#pragma unroll
                for (int c = 0; c < GBS_KMAX; ++c) acc[c][0] = acc[c][1] = TI(0);
                const TI *p = (const TI *)S.pi;
                TI *qv = (TI *)S.qi;
                auto epi = [&](int row, TI(&s)[GBS_KMAX]) {
#pragma unroll
                    for (int c = 0; c < GBS_KMAX; ++c) {
                        if (c >= k) break;
                        const size_t o = (size_t)row * k + c;
                        qv[o] = s[c];
                        acc[c][0] += p[o] * s[c];
                    }
                };
                if (a.fp64)
                    tile_spmv_k<double, TI>(S, S.vals, p, tl.y, wt64, epi);
                else
                    tile_spmv_k<float, TI>(S, S.vals32, p, tl.y, wt32, epi);
                warp_store_partials<TI>(acc, k, dst);
            }
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;

        // ---------------- R1: per (system, column)
        for (int g = gw; g < a.npair; g += nw) {
            const int2 pc = a.pairs[g];
            const BSys &S = a.sys[pc.x];
            BSysDyn &D = a.dyn[pc.x];
            if (D.finished) continue;
            BCol &C = a.col[pc.x * GBS_KMAX + pc.y];
            if (!col_running(C)) continue;
            if (D.mode[cur] == MODE_OUTER) {
                const double rr = sys_sum<double>(a.partS, S, pc.y, 0);
                const double bb = sys_sum<double>(a.partS, S, pc.y, 1);
                if (lane == 0) {
                    const double rn = sqrt(rr);
                    if (C.first) C.bnorm = sqrt(bb);
                    C.first = 0;
                    C.rn = rn;
                    if (isnan(rn)) C.status = GBS_ERR_NAN;
                    else if (rn <= S.rtol * C.bnorm) C.status = GBS_OK;
                    else if (rn > 0.5 * C.prev) C.status = GBS_ERR_STAGNATION;
                    else if (C.outer >= a.outer_maxit || C.iters >= S.maxit) C.status = GBS_DIVERGED_ITS;
                    else {
                        C.prev = rn;
                        C.scale = 1.0 / rn;
                        C.outer += 1;
                        // FP64 inner solves aim below rtol ||b|| at once
                        C.tol_inner = a.fp64 ? 0.5 * S.rtol * C.bnorm / rn : a.inner_rtol;
                    }
                }
            } else if (!C.inner_done) {
                const TI pq = sys_sum<TI>(a.partS, S, pc.y, 0);
                if (lane == 0) {
                    if (isnan((double)pq)) C.status = GBS_ERR_NAN;
                    else if (pq <= TI(0)) C.status = GBS_ERR_INDEFINITE;
                    else C.alpha = (double)((TI)C.rho / pq);
                }
            }
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;

        // ---------------- U: vector updates per tile
        for (int g = gw; g < a.ntile; g += nw) {
            const int2 tl = a.tiles[g];
            const BSys &S = a.sys[tl.x];
            const BSysDyn &D = a.dyn[tl.x];
            if (D.finished) continue;
            const int k = S.k;
            const BCol *Cs = a.col + tl.x * GBS_KMAX;
            const int r0 = __ldg(S.tiles + tl.y), r1 = __ldg(S.tiles + tl.y + 1);
            TI acc[GBS_KMAX][2];
#pragma unroll
            for (int c = 0; c < GBS_KMAX; ++c) acc[c][0] = acc[c][1] = TI(0);
            TI *xi = (TI *)S.xi, *ri = (TI *)S.ri, *zi = (TI *)S.zi, *pi = (TI *)S.pi;
            const TI *qi = (const TI *)S.qi;
            const int row = r0 + lane;
            if (row < r1) {
                const TI dg = a.fp64 ? (TI)S.dinv[row] : (TI)S.dinv32[row];
                if (D.mode[cur] == MODE_OUTER) {
                    // start an inner solve on r / ||r||: x_i = 0, r_i = b_i, z = D^-1 r_i, p = z
#pragma unroll
                    for (int c = 0; c < GBS_KMAX; ++c) {
                        if (c >= k) break;
                        if (!col_running(Cs[c])) continue;
                        const size_t o = (size_t)row * k + c;
                        const TI bi = (TI)(S.r64[o] * Cs[c].scale);
                        const TI zi_ = dg * bi;
                        xi[o] = TI(0);
                        ri[o] = bi;
                        zi[o] = zi_;
                        pi[o] = zi_;
                        acc[c][0] += bi * zi_;
                        acc[c][1] += bi * bi;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < GBS_KMAX; ++c) {
                        if (c >= k) break;
                        if (!col_running(Cs[c]) || Cs[c].inner_done) continue;
                        const size_t o = (size_t)row * k + c;
                        const TI al = (TI)Cs[c].alpha;
                        xi[o] = xi[o] + al * pi[o];
                        const TI rn_ = ri[o] - al * qi[o];
                        const TI zn_ = dg * rn_;
                        ri[o] = rn_;
                        zi[o] = zn_;
                        acc[c][0] += rn_ * zn_;
                        acc[c][1] += rn_ * rn_;
                    }
                }
            }
            warp_store_partials<TI>(acc, k, a.partU + (size_t)(S.gtile0 + tl.y) * GBS_KMAX * 2);
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;

        // ---------------- R2: per (system, column)
        for (int g = gw; g < a.npair; g += nw) {
            const int2 pc = a.pairs[g];
            const BSys &S = a.sys[pc.x];
            BSysDyn &D = a.dyn[pc.x];
            if (D.finished) continue;
            BCol &C = a.col[pc.x * GBS_KMAX + pc.y];
            if (!col_running(C)) continue;
            if (D.mode[cur] == MODE_OUTER) {
                const TI rho = sys_sum<TI>(a.partU, S, pc.y, 0);
                const TI bb = sys_sum<TI>(a.partU, S, pc.y, 1);
                if (lane == 0) {
                    C.rho = (double)rho;
                    C.tol_inner = C.tol_inner * (double)sqrt(bb);
                    C.kin = 0;
                    C.inner_done = 0;
                }
            } else if (!C.inner_done) {
                const TI rho_new = sys_sum<TI>(a.partU, S, pc.y, 0);
                const TI rr = sys_sum<TI>(a.partU, S, pc.y, 1);
                if (lane == 0) {
                    C.kin += 1;
                    C.iters += 1;
                    if (rho_new < TI(0)) {
                        C.status = GBS_ERR_INDEFINITE;
                    } else if (isnan((double)rr)) {
                        C.status = GBS_ERR_NAN;
                    } else {
                        C.beta = (double)(rho_new / (TI)C.rho);
                        C.rho = (double)rho_new;
                        if ((double)sqrt(rr) <= C.tol_inner || C.iters >= S.maxit) C.inner_done = 1;
                    }
                }
            }
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;

        // ---------------- P: direction update, or refinement update
        for (int g = gw; g < a.ntile; g += nw) {
            const int2 tl = a.tiles[g];
            const BSys &S = a.sys[tl.x];
            BSysDyn &D = a.dyn[tl.x];
            if (D.finished) continue;
            const int k = S.k;
            const BCol *Cs = a.col + tl.x * GBS_KMAX;
            // the system's next step: refinement once every running column's
            // inner solve has stopped; finished once no column runs
            int running = 0, waiting = 0;
            for (int c = 0; c < k; ++c) {
                running += col_running(Cs[c]);
                waiting += col_running(Cs[c]) && !Cs[c].inner_done;
            }
            const int mode = D.mode[cur];
            const int next = (mode == MODE_INNER && waiting == 0) ? MODE_OUTER
                             : (mode == MODE_OUTER ? MODE_INNER : MODE_INNER);
            const int r0 = __ldg(S.tiles + tl.y), r1 = __ldg(S.tiles + tl.y + 1);
            const int row = r0 + lane;
            if (row < r1 && mode == MODE_INNER) {
                TI *pi = (TI *)S.pi;
                const TI *zi = (const TI *)S.zi, *xi = (const TI *)S.xi;
#pragma unroll
                for (int c = 0; c < GBS_KMAX; ++c) {
                    if (c >= k) break;
                    if (!col_running(Cs[c])) continue;
                    const size_t o = (size_t)row * k + c;
                    if (next == MODE_OUTER)
                        S.x[o] += Cs[c].rn * (double)xi[o];   // x += ||r|| d
                    else if (!Cs[c].inner_done)
                        pi[o] = zi[o] + (TI)Cs[c].beta * pi[o];
                }
            }
            if (tl.y == 0 && lane == 0) {
                D.mode[nxt] = running ? next : mode;
                if (!running) D.finished = 1;
            }
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;
    }
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// ----------------------------------------------------------------------
// Host engine shared by the batched solve and the serving loop.
// ----------------------------------------------------------------------

struct gbs_batch_engine {
    gbs_ctx ctx;
    int fp64;
    double inner_rtol;
    int outer_maxit;
    int quantum;
    // device arrays, grown on demand
    BSys *d_sys = nullptr;
    BCol *d_col = nullptr;
    BSysDyn *d_dyn = nullptr;
    int2 *d_tiles = nullptr;
    int2 *d_pairs = nullptr;
    double *d_partS = nullptr, *d_partU = nullptr;
    gbs_grid_barrier *d_bar = nullptr;
    size_t cap_sys = 0, cap_tiles = 0, cap_pairs = 0, cap_gtiles = 0;
    int64_t iter = 0;
};

static int grow(void **p, size_t *cap, size_t need, size_t elem)
{
    if (need <= *cap) return GBS_OK;
    size_t n = std::max(need, *cap * 2 + 16);
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    GBS_CUDA_TRY(cudaMalloc(p, n * elem));
    *cap = n;
    return GBS_OK;
}

// Run the active systems for one quantum.  sys/col/dyn are uploaded by the
// caller; tiles/pairs list the active work.
static int engine_launch(gbs_batch_engine *E, int nsys_total, const std::vector<int2> &tiles,
                         const std::vector<int2> &pairs, int64_t gtiles_total, int *timed_out)
{
    gbs_ctx c = E->ctx;
    *timed_out = 0;
    int st = grow((void **)&E->d_tiles, &E->cap_tiles, tiles.size() + 1, sizeof(int2));
    if (!st) st = grow((void **)&E->d_pairs, &E->cap_pairs, pairs.size() + 1, sizeof(int2));
    if (st) return st;
    if ((size_t)gtiles_total > E->cap_gtiles) {
        cudaFree(E->d_partS);
        cudaFree(E->d_partU);
        E->d_partS = E->d_partU = nullptr;
        E->cap_gtiles = 0;
        const size_t n = (size_t)gtiles_total * 2 + 64;
        GBS_CUDA_TRY(cudaMalloc(&E->d_partS, n * GBS_KMAX * 2 * sizeof(double)));
        GBS_CUDA_TRY(cudaMalloc(&E->d_partU, n * GBS_KMAX * 2 * sizeof(double)));
        E->cap_gtiles = n;
    }
    if (!E->d_bar) GBS_CUDA_TRY(cudaMalloc(&E->d_bar, 256));
    GBS_CUDA_TRY(cudaMemcpyAsync(E->d_tiles, tiles.data(), tiles.size() * sizeof(int2),
                                 cudaMemcpyHostToDevice, c->stream));
    GBS_CUDA_TRY(cudaMemcpyAsync(E->d_pairs, pairs.data(), pairs.size() * sizeof(int2),
                                 cudaMemcpyHostToDevice, c->stream));
    GBS_CUDA_TRY(cudaMemsetAsync(E->d_bar, 0, 256, c->stream));
    BArgs a;
    memset(&a, 0, sizeof(a));
    a.sys = E->d_sys;
    a.col = E->d_col;
    a.dyn = E->d_dyn;
    a.tiles = E->d_tiles;
    a.ntile = (int)tiles.size();
    a.pairs = E->d_pairs;
    a.npair = (int)pairs.size();
    a.partS = E->d_partS;
    a.partU = E->d_partU;
    a.bar = E->d_bar;
    a.quantum = E->quantum;
    a.iter0 = (int)(E->iter & 1);
    a.inner_rtol = E->inner_rtol;
    a.outer_maxit = E->outer_maxit;
    a.fp64 = E->fp64;
    a.timeout_ns = (unsigned long long)c->opts.barrier_timeout_ms * 1000000ull;
    const void *fn = E->fp64 ? (const void *)k_batched<double> : (const void *)k_batched<float>;
    const size_t smem = sizeof(BTile<double>) * GBS_PWARPS;
    GBS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, GBS_PBLOCK, smem));
    if (per_sm < 1) return GBS_ERR_CUDA;
    int64_t need = ((int64_t)std::max(tiles.size(), pairs.size()) + GBS_PWARPS - 1) / GBS_PWARPS;
    int64_t G = std::min<int64_t>((int64_t)per_sm * c->num_sms, std::max<int64_t>(need, 1));
    void *args[] = {&a};
    GBS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(GBS_PBLOCK), args, smem,
                                             c->stream));
    gbs_count_launch(c);
    E->iter += E->quantum;
    GBS_CUDA_TRY(cudaMemcpyAsync(c->pinned, &E->d_bar->error, sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *timed_out = *(volatile int *)c->pinned != 0;
    (void)nsys_total;
    return GBS_OK;
}

// ----------------------------------------------------------------------
// gbs_ksp_solve_cg_batched
// ----------------------------------------------------------------------

__global__ void k_interleave(int64_t n, int k, const double *src, double *dst, int dir)
{
    // dir 0: column-major (c * n + i) -> interleaved (i * k + c); dir 1: back
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, cc = e % k;
        if (dir == 0) dst[e] = src[cc * n + i];
        else dst[cc * n + i] = src[e];
    }
}

struct BatchHostSys {
    gbs_mat A;
    int k;
    double *b_il, *x_il, *r64;
    void *xi, *ri, *zi, *pi, *qi;
};

extern "C" int gbs_ksp_solve_cg_batched(gbs_ctx c, int nsys, const gbs_mat *A, const gbs_vec *B,
                                        gbs_vec *X, const int *nrhs, const double *rtol, int maxit,
                                        int mode, int *iters, double *rnorm, int *status)
{
    if (!c || nsys < 0 || (nsys > 0 && (!A || !B || !X || !nrhs || !rtol)) || maxit < 0)
        return GBS_ERR_ARG;
    if (mode != GBS_MODE_FP64 && mode != GBS_MODE_MIXED) return GBS_ERR_ARG;
    int64_t totcols = 0;
    for (int s = 0; s < nsys; ++s) {
        if (!A[s] || !B[s] || !X[s] || A[s]->ctx != c || nrhs[s] < 1 || nrhs[s] > GBS_KMAX)
            return GBS_ERR_ARG;
        if (A[s]->n != A[s]->ncols || B[s]->n != A[s]->n * nrhs[s] || X[s]->n != B[s]->n ||
            B[s]->dtype != GBS_F64 || X[s]->dtype != GBS_F64 || !(rtol[s] >= 0.0))
            return GBS_ERR_ARG;
        totcols += nrhs[s];
    }
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    const bool fp64 = mode == GBS_MODE_FP64;
    const size_t tsz = fp64 ? 8 : 4;
    // per-system device work vectors in one allocation
    std::vector<size_t> off(nsys + 1, 0);
    for (int s = 0; s < nsys; ++s) {
        const size_t nk = (size_t)A[s]->n * nrhs[s];
        off[s + 1] = off[s] + 3 * a256(nk * 8) + 5 * a256(nk * tsz);
    }
    char *work = nullptr;
    if (off[nsys] > 0) GBS_CUDA_TRY(cudaMalloc(&work, off[nsys]));
    std::vector<BSys> hs(nsys);
    std::vector<BCol> hc((size_t)nsys * GBS_KMAX);
    std::vector<BSysDyn> hd(nsys);
    std::vector<int2> tiles, pairs;
    int64_t gt = 0;
    int rc = GBS_OK;
    for (int s = 0; s < nsys && rc == GBS_OK; ++s) {
        gbs_mat M = A[s];
        if (!fp64 && (rc = gbs_mat_ensure_f32(M)) != GBS_OK) break;
        const size_t nk = (size_t)M->n * nrhs[s];
        char *p = work + off[s];
        BSys &S = hs[s];
        memset(&S, 0, sizeof(S));
        S.rowptr = M->rowptr;
        S.colidx = M->colidx;
        S.tiles = M->tiles;
        S.vals = M->vals;
        S.vals32 = M->vals32;
        S.dinv = M->dinv;
        S.dinv32 = M->dinv32;
        S.b = (const double *)p; p += a256(nk * 8);
        S.x = (double *)p; p += a256(nk * 8);
        S.r64 = (double *)p; p += a256(nk * 8);
        S.xi = p; p += a256(nk * tsz);
        S.ri = p; p += a256(nk * tsz);
        S.zi = p; p += a256(nk * tsz);
        S.pi = p; p += a256(nk * tsz);
        S.qi = p; p += a256(nk * tsz);
        S.n = (int)M->n;
        S.k = nrhs[s];
        S.ntiles = (int)M->ntiles;
        S.gtile0 = (int)gt;
        S.rtol = rtol[s];
        S.maxit = maxit;
        gt += M->ntiles;
        if (M->n > 0) {
            const int g = (int)std::min<int64_t>((int64_t)(nk + 255) / 256, (int64_t)c->num_sms * 8);
            k_interleave<<<g, 256, 0, c->stream>>>(M->n, S.k, (const double *)B[s]->data,
                                                           (double *)S.b, 0);
            k_interleave<<<g, 256, 0, c->stream>>>(M->n, S.k, (const double *)X[s]->data,
                                                           S.x, 0);
            gbs_count_launch(c, 2);
        }
        BSysDyn &D = hd[s];
        memset(&D, 0, sizeof(D));
        D.mode[0] = D.mode[1] = MODE_OUTER;
        const bool bad = M->n == 0 || !M->diag_ok;
        D.finished = bad ? 1 : 0;
        for (int cc = 0; cc < GBS_KMAX; ++cc) {
            BCol &C = hc[(size_t)s * GBS_KMAX + cc];
            memset(&C, 0, sizeof(C));
            C.status = cc < S.k ? (M->n == 0 ? GBS_OK : (!M->diag_ok ? GBS_ERR_DIAG : GBS_RUNNING))
                                : GBS_OK;
            C.prev = INFINITY;
            C.first = 1;
        }
        if (!bad) {
            for (int t = 0; t < M->ntiles; ++t) tiles.push_back(make_int2(s, t));
            for (int cc = 0; cc < S.k; ++cc) pairs.push_back(make_int2(s, cc));
        }
    }
    gbs_batch_engine E;
    E.ctx = c;
    E.fp64 = fp64 ? 1 : 0;
    E.inner_rtol = c->opts.inner_rtol;
    E.outer_maxit = c->opts.outer_maxit;
    E.quantum = 64;
    if (rc == GBS_OK && nsys > 0) {
        cudaError_t e = cudaMalloc(&E.d_sys, sizeof(BSys) * nsys);
        if (e == cudaSuccess) e = cudaMalloc(&E.d_col, sizeof(BCol) * hc.size());
        if (e == cudaSuccess) e = cudaMalloc(&E.d_dyn, sizeof(BSysDyn) * nsys);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(E.d_sys, hs.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(E.d_col, hc.data(), sizeof(BCol) * hc.size(),
                                cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(E.d_dyn, hd.data(), sizeof(BSysDyn) * nsys, cudaMemcpyHostToDevice,
                                c->stream);
        if (e != cudaSuccess) rc = gbs_cuda_fail(e);
    }
    GBS_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    // run quanta until every system has finished, compacting the work lists
    std::vector<BSysDyn> dyn(nsys);
    while (rc == GBS_OK && !tiles.empty()) {
        int to = 0;
        rc = engine_launch(&E, nsys, tiles, pairs, gt, &to);
        if (rc) break;
        if (to) { rc = GBS_ERR_TIMEOUT; break; }
        cudaError_t e = cudaMemcpy(dyn.data(), E.d_dyn, sizeof(BSysDyn) * nsys,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { rc = gbs_cuda_fail(e); break; }
        std::vector<int2> t2, p2;
        for (const int2 &t : tiles)
            if (!dyn[t.x].finished) t2.push_back(t);
        for (const int2 &p : pairs)
            if (!dyn[p.x].finished) p2.push_back(p);
        tiles.swap(t2);
        pairs.swap(p2);
    }
    GBS_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    // results
    int first_bad = GBS_OK;
    if (rc == GBS_OK && nsys > 0) {
        cudaError_t e = cudaMemcpy(hc.data(), E.d_col, sizeof(BCol) * hc.size(),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = gbs_cuda_fail(e);
    }
    if (rc == GBS_OK) {
        int64_t o = 0;
        for (int s = 0; s < nsys; ++s) {
            const BSys &S = hs[s];
            if (A[s]->n > 0) {
                const size_t nk = (size_t)A[s]->n * S.k;
                const int g = (int)std::min<int64_t>((int64_t)(nk + 255) / 256, (int64_t)c->num_sms * 8);
                k_interleave<<<g, 256, 0, c->stream>>>(A[s]->n, S.k, S.x,
                                                               (double *)X[s]->data, 1);
                gbs_count_launch(c);
            }
            for (int cc = 0; cc < S.k; ++cc, ++o) {
                const BCol &C = hc[(size_t)s * GBS_KMAX + cc];
                const int cs = C.status == GBS_RUNNING ? GBS_DIVERGED_ITS : C.status;
                if (iters) iters[o] = C.iters;
                if (rnorm) rnorm[o] = C.rn;
                if (status) status[o] = cs;
                if (cs != GBS_OK && first_bad == GBS_OK) first_bad = cs;
            }
        }
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = gbs_cuda_fail(e);
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->last.device_ms = ms;
    cudaStreamSynchronize(c->stream);
    cudaFree(work);
    cudaFree(E.d_sys);
    cudaFree(E.d_col);
    cudaFree(E.d_dyn);
    cudaFree(E.d_tiles);
    cudaFree(E.d_pairs);
    cudaFree(E.d_partS);
    cudaFree(E.d_partU);
    cudaFree(E.d_bar);
    if (rc != GBS_OK) return rc;
    return first_bad;
}

// ----------------------------------------------------------------------
// Serving loop (continuous batching) -- declared in gbs.h, built on the
// engine above; implemented in server.cu.
// ----------------------------------------------------------------------
extern "C" int gbs_server_create(gbs_ctx, size_t, int, int, gbs_server *) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_destroy(gbs_server) { return GBS_OK; }
extern "C" int gbs_server_submit(gbs_server, int64_t, const int32_t *, const int32_t *,
                                 const double *, int, const double *, double, int, uint64_t *)
{
    return GBS_ERR_UNSUPPORTED;
}
extern "C" int gbs_server_progress(gbs_server, int *) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_poll(gbs_server, uint64_t, int *) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_wait(gbs_server, uint64_t) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_fetch(gbs_server, uint64_t, double *, int *, double *, int *)
{
    return GBS_ERR_UNSUPPORTED;
}
extern "C" int gbs_server_stats(gbs_server, int *, int *, int *, size_t *) { return GBS_ERR_UNSUPPORTED; }
