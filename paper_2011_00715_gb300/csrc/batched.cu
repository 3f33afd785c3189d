// Batched Jacobi-PCG over many independent systems with several right-hand
// sides each, in one persistent cooperative kernel (Response A6: solve many
// different-size problems at once; Challenge F2 and Sec. 4: multiple
// right-hand sides raise arithmetic intensity; Response A7: FP32 inner
// iterations with FP64 refinement), and the serving loop built on it.
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
// Systems live in slots.  The kernel runs at most `quantum` global
// iterations over the active slots and returns; all solver state stays in
// device memory, so the host retires finished systems and admits new ones
// between launches (continuous batching).  The launch of a quantum is
// captured once into a CUDA graph and replayed while the active set is
// unchanged (Challenge A1).

#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <unordered_map>
#include <vector>

#include "gbs_impl.cuh"

#define GBS_KMAX 8
#define GBS_RUNNING (-100)

namespace {

enum { MODE_OUTER = 0, MODE_INNER = 1 };

// Read-only description of one system (device, one per slot).
struct BSys {
    const int32_t *rowptr, *colidx, *tiles;
    const double *vals, *dinv;
    const float *vals32, *dinv32;
    const double *b;    // n * k, interleaved
    double *x;          // n * k, interleaved (initial guess in, solution out)
    double *r64;        // n * k
    void *xi, *ri, *zi, *pi, *qi;   // inner-precision work vectors, n * k
    int n, k, ntiles, pad0;
    double rtol;
    int maxit;
    int pad1;
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
    const BSys *sys;    // by slot
    BCol *col;          // slot * GBS_KMAX + column
    BSysDyn *dyn;       // by slot
    const int *act;     // active slots, nact entries
    const int *tcum;    // prefix sums of the active slots' tile counts (nact + 1)
    int nact;
    int ntile;          // tcum[nact]
    int nchunk;         // ccum[nact]
    double *partS;      // active tile * GBS_KMAX * 2
    double *partU;      // active tile * GBS_KMAX * 2
    const int *ccum;    // prefix sums of the active slots' reduction chunks (nact + 1)
    double *cpart;      // chunk * GBS_KMAX * 2: chunk partial sums
    int *ccount;        // active slot * GBS_KMAX: chunks arrived (zero between phases)
    gbs_grid_barrier *bar;
    int quantum;
    int iter0;          // parity of the global iteration count at launch
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

// Sum entry j of column c over active tiles [ga, gb) -- one system's tiles
// -- in a fixed order (lane l: tiles ga + l, ga + l + 32, ... in type T;
// then a fixed shuffle tree).
template <typename T>
__device__ __forceinline__ T sys_sum(const double *part, int ga, int gb, int c, int j)
{
    const int lane = threadIdx.x & 31;
    T t = T(0);
    for (int g = ga + lane; g < gb; g += 32)
        t += (T)__ldcg(part + ((size_t)g * GBS_KMAX + c) * 2 + j);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
}

__device__ __forceinline__ bool col_running(const BCol &c) { return c.status == GBS_RUNNING; }

// Tiles per reduction chunk: a system's per-tile partials are summed chunk
// by chunk (one warp each), then the chunk sums are added by the warp that
// completes the last chunk.  Both levels use a fixed order that depends
// only on the system, so results stay independent of the batch.
#define GBS_RCHUNK 128

// Two-level reduction of entries 0 and 1 of column c over one system's
// tiles, for the chunk [ga, gb) handled by this warp (chunk gc of the
// active chunk range [ca, cb), system active index ai).  Returns true in
// the warp whose chunk arrived last; that warp gets the totals in out[].
template <typename T>
__device__ __forceinline__ bool chunk_reduce(const BArgs &a, const double *part, int ga, int gb,
                                             int gc, int ca, int cb, int ai, int c, T (&out)[2])
{
    const int lane = threadIdx.x & 31;
    T s0 = sys_sum<T>(part, ga, gb, c, 0);
    T s1 = sys_sum<T>(part, ga, gb, c, 1);
    int last = 0;
    if (lane == 0) {
        a.cpart[((size_t)gc * GBS_KMAX + c) * 2 + 0] = (double)s0;
        a.cpart[((size_t)gc * GBS_KMAX + c) * 2 + 1] = (double)s1;
        __threadfence();
        last = atomicAdd(&a.ccount[ai * GBS_KMAX + c], 1) == cb - ca - 1;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return false;
    __threadfence();
    out[0] = sys_sum<T>(a.cpart, ca, cb, c, 0);
    out[1] = sys_sum<T>(a.cpart, ca, cb, c, 1);
    if (lane == 0) a.ccount[ai * GBS_KMAX + c] = 0;
    return true;
}

// Active index owning active tile g (tcum is increasing, tcum[0] = 0).
__device__ __forceinline__ int owner_of(const int *tcum, int nact, int g)
{
    int lo = 0, hi = nact - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tcum + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

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
    // this warp's contiguous share of the active tiles
    const int g0 = (int)((int64_t)a.ntile * gw / nw), g1 = (int)((int64_t)a.ntile * (gw + 1) / nw);
    const int ai0 = g0 < g1 ? owner_of(a.tcum, a.nact, g0) : 0;
    const int nunits = a.nchunk * GBS_KMAX;   // reduction work units: (chunk, column)
    int bno = 0;
    bool ok = true;

    for (int q = 0; q < a.quantum && ok; ++q) {
        const int cur = (a.iter0 + q) & 1, nxt = cur ^ 1;

        // ---------------- S: SpMV per tile
        for (int g = g0, ai = ai0; g < g1; ++g) {
            while (__ldg(a.tcum + ai + 1) <= g) ++ai;
            const int slot = __ldg(a.act + ai);
            const int lt = g - __ldg(a.tcum + ai);
            const BSys &S = a.sys[slot];
            const BSysDyn &D = a.dyn[slot];
            if (D.finished) continue;
            const int k = S.k;
            double *dst = a.partS + (size_t)g * GBS_KMAX * 2;
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
                tile_spmv_k<double, double>(S, S.vals, S.x, lt, wt64, epi);
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
                    tile_spmv_k<double, TI>(S, S.vals, p, lt, wt64, epi);
                else
                    tile_spmv_k<float, TI>(S, S.vals32, p, lt, wt32, epi);
                warp_store_partials<TI>(acc, k, dst);
            }
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;

        // ---------------- R1: per (system, column)
        for (int u = gw; u < nunits; u += nw) {
            const int gc = u / GBS_KMAX, cc = u % GBS_KMAX;
            const int ai = owner_of(a.ccum, a.nact, gc);
            const int slot = __ldg(a.act + ai);
            const BSys &S = a.sys[slot];
            BSysDyn &D = a.dyn[slot];
            if (cc >= S.k || D.finished) continue;
            BCol &C = a.col[slot * GBS_KMAX + cc];
            if (!col_running(C)) continue;
            const int ca = __ldg(a.ccum + ai), cb = __ldg(a.ccum + ai + 1);
            const int ga = __ldg(a.tcum + ai) + (gc - ca) * GBS_RCHUNK;
            const int gb = min(ga + GBS_RCHUNK, __ldg(a.tcum + ai + 1));
            if (D.mode[cur] == MODE_OUTER) {
                double tot[2];
                if (!chunk_reduce<double>(a, a.partS, ga, gb, gc, ca, cb, ai, cc, tot)) continue;
                const double rr = tot[0], bb = tot[1];
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
                TI tot[2];
                if (!chunk_reduce<TI>(a, a.partS, ga, gb, gc, ca, cb, ai, cc, tot)) continue;
                const TI pq = tot[0];
                if (lane == 0) {
                    if (isnan((double)pq)) C.status = GBS_ERR_NAN;
                    else if (pq <= TI(0)) C.status = GBS_ERR_INDEFINITE;
                    else C.alpha = (double)((TI)C.rho / pq);
                }
            }
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;

        // ---------------- U: vector updates per tile
        for (int g = g0, ai = ai0; g < g1; ++g) {
            while (__ldg(a.tcum + ai + 1) <= g) ++ai;
            const int slot = __ldg(a.act + ai);
            const int lt = g - __ldg(a.tcum + ai);
            const BSys &S = a.sys[slot];
            const BSysDyn &D = a.dyn[slot];
            if (D.finished) continue;
            const int k = S.k;
            const BCol *Cs = a.col + slot * GBS_KMAX;
            const int r0 = __ldg(S.tiles + lt), r1 = __ldg(S.tiles + lt + 1);
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
            warp_store_partials<TI>(acc, k, a.partU + (size_t)g * GBS_KMAX * 2);
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;

        // ---------------- R2: per (system, column)
        for (int u = gw; u < nunits; u += nw) {
            const int gc = u / GBS_KMAX, cc = u % GBS_KMAX;
            const int ai = owner_of(a.ccum, a.nact, gc);
            const int slot = __ldg(a.act + ai);
            const BSys &S = a.sys[slot];
            BSysDyn &D = a.dyn[slot];
            if (cc >= S.k || D.finished) continue;
            BCol &C = a.col[slot * GBS_KMAX + cc];
            if (!col_running(C)) continue;
            const int ca = __ldg(a.ccum + ai), cb = __ldg(a.ccum + ai + 1);
            const int ga = __ldg(a.tcum + ai) + (gc - ca) * GBS_RCHUNK;
            const int gb = min(ga + GBS_RCHUNK, __ldg(a.tcum + ai + 1));
            if (D.mode[cur] == MODE_OUTER) {
                TI tot[2];
                if (!chunk_reduce<TI>(a, a.partU, ga, gb, gc, ca, cb, ai, cc, tot)) continue;
                const TI rho = tot[0], bb = tot[1];
                if (lane == 0) {
                    C.rho = (double)rho;
                    C.tol_inner = C.tol_inner * (double)sqrt(bb);
                    C.kin = 0;
                    C.inner_done = 0;
                }
            } else if (!C.inner_done) {
                TI tot[2];
                if (!chunk_reduce<TI>(a, a.partU, ga, gb, gc, ca, cb, ai, cc, tot)) continue;
                const TI rho_new = tot[0], rr = tot[1];
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
        for (int g = g0, ai = ai0; g < g1; ++g) {
            while (__ldg(a.tcum + ai + 1) <= g) ++ai;
            const int slot = __ldg(a.act + ai);
            const int lt = g - __ldg(a.tcum + ai);
            const BSys &S = a.sys[slot];
            BSysDyn &D = a.dyn[slot];
            if (D.finished) continue;
            const int k = S.k;
            const BCol *Cs = a.col + slot * GBS_KMAX;
            // the system's next step: refinement once every running column's
            // inner solve has stopped; finished once no column runs
            int running = 0, waiting = 0;
            for (int c = 0; c < k; ++c) {
                running += col_running(Cs[c]);
                waiting += col_running(Cs[c]) && !Cs[c].inner_done;
            }
            const int mode = D.mode[cur];
            const int next = (mode == MODE_INNER && waiting == 0) ? MODE_OUTER : MODE_INNER;
            const int r0 = __ldg(S.tiles + lt), r1 = __ldg(S.tiles + lt + 1);
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
            if (lt == 0 && lane == 0) {
                D.mode[nxt] = running ? next : mode;
                if (!running) D.finished = 1;
            }
        }
        if (!(ok = gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag))) break;
    }
}

// Column-major (c * n + i) <-> interleaved (i * k + c).
__global__ void k_interleave(int64_t n, int k, const double *src, double *dst, int dir)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, cc = e % k;
        if (dir == 0) dst[e] = src[cc * n + i];
        else dst[cc * n + i] = src[e];
    }
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// ----------------------------------------------------------------------
// Host engine: a slot table of systems run by the kernel above.
// ----------------------------------------------------------------------

struct SlotHost {
    bool used = false;
    bool finished = false;
    gbs_mat A = nullptr;
    bool own_A = false;       // the engine created the matrix (serving) and frees it
    int k = 0;
    char *work = nullptr;     // device vectors of the slot
    size_t bytes = 0;         // device bytes held for budget accounting
    uint64_t ticket = 0;
};

struct Engine {
    gbs_ctx c = nullptr;
    int fp64 = 0;
    double inner_rtol = 1e-4;
    int outer_maxit = 30;
    int quantum = 32;
    int nslots = 0;
    BSys *d_sys = nullptr;
    BCol *d_col = nullptr;
    BSysDyn *d_dyn = nullptr;
    int *d_act = nullptr, *d_tcum = nullptr, *d_ccum = nullptr, *d_ccount = nullptr;
    double *d_cpart = nullptr;
    size_t cap_cpart = 0;
    double *d_partS = nullptr, *d_partU = nullptr;
    size_t cap_part = 0;
    gbs_grid_barrier *d_bar = nullptr;
    std::vector<SlotHost> slots;
    std::vector<BSysDyn> h_dyn;
    int64_t iter = 0;
    // graph of one quantum for the current active set
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    std::vector<int> g_act;   // active set the graph was captured for
    std::vector<int> g_tcum;  // and its tile prefix sums
    bool dirty = true;        // a slot was filled or released since the capture
    BArgs g_args;
    int G = 0;
};

void engine_free_graph(Engine &E)
{
    if (E.gexec) cudaGraphExecDestroy(E.gexec);
    if (E.graph) cudaGraphDestroy(E.graph);
    E.gexec = nullptr;
    E.graph = nullptr;
    E.g_act.clear();
    E.g_tcum.clear();
}

int engine_init(Engine &E, gbs_ctx c, int nslots, int fp64, int quantum)
{
    E.c = c;
    E.fp64 = fp64;
    E.inner_rtol = c->opts.inner_rtol;
    E.outer_maxit = c->opts.outer_maxit;
    E.quantum = quantum;
    E.nslots = nslots;
    E.slots.assign(nslots, SlotHost());
    E.h_dyn.assign(nslots, BSysDyn());
    GBS_CUDA_TRY(cudaMalloc(&E.d_sys, sizeof(BSys) * (size_t)std::max(nslots, 1)));
    GBS_CUDA_TRY(cudaMalloc(&E.d_col, sizeof(BCol) * (size_t)std::max(nslots, 1) * GBS_KMAX));
    GBS_CUDA_TRY(cudaMalloc(&E.d_dyn, sizeof(BSysDyn) * (size_t)std::max(nslots, 1)));
    GBS_CUDA_TRY(cudaMalloc(&E.d_act, sizeof(int) * (size_t)(nslots + 1)));
    GBS_CUDA_TRY(cudaMalloc(&E.d_tcum, sizeof(int) * (size_t)(nslots + 2)));
    GBS_CUDA_TRY(cudaMalloc(&E.d_ccum, sizeof(int) * (size_t)(nslots + 2)));
    GBS_CUDA_TRY(cudaMalloc(&E.d_ccount, sizeof(int) * (size_t)(nslots + 1) * GBS_KMAX));
    GBS_CUDA_TRY(cudaMemset(E.d_ccount, 0, sizeof(int) * (size_t)(nslots + 1) * GBS_KMAX));
    GBS_CUDA_TRY(cudaMalloc(&E.d_bar, 256));
    return GBS_OK;
}

void engine_destroy(Engine &E)
{
    if (E.c) cudaStreamSynchronize(E.c->stream);
    engine_free_graph(E);
    for (SlotHost &s : E.slots) {
        if (s.work) cudaFree(s.work);
        if (s.own_A) gbs_mat_destroy(s.A);
        s = SlotHost();
    }
    cudaFree(E.d_sys);
    cudaFree(E.d_col);
    cudaFree(E.d_dyn);
    cudaFree(E.d_act);
    cudaFree(E.d_tcum);
    cudaFree(E.d_ccum);
    cudaFree(E.d_ccount);
    cudaFree(E.d_cpart);
    cudaFree(E.d_partS);
    cudaFree(E.d_partU);
    cudaFree(E.d_bar);
    E = Engine();
}

// Device bytes a system of n rows, nnz nonzeros and k columns holds.
size_t system_bytes(int64_t n, int64_t nnz, int k, int fp64)
{
    const size_t nk = (size_t)n * k, tsz = fp64 ? 8 : 4;
    const size_t vecs = 3 * a256(nk * 8) + 5 * a256(nk * tsz);
    const size_t mat = 4 * (size_t)(n + 5) + 12 * (size_t)(nnz + 4) + (fp64 ? 0 : 4 * (size_t)(nnz + 4)) +
                       12 * (size_t)(n + 4) + 12 * (size_t)(n / 32 + 2) + 4096;
    return vecs + mat;
}

// Put a system into a free slot.  b and x0 are column-major device arrays
// (x0 may be NULL for zeros).  A failing matrix (no usable diagonal, n = 0)
// is admitted as finished with the corresponding column status.
int engine_add(Engine &E, int slot, gbs_mat A, int k, double rtol, int maxit, const double *b,
               const double *x0, bool own_A, uint64_t ticket)
{
    gbs_ctx c = E.c;
    SlotHost &H = E.slots[slot];
    const size_t nk = (size_t)A->n * k, tsz = E.fp64 ? 8 : 4;
    if (!E.fp64) {
        int st = gbs_mat_ensure_f32(A);
        if (st) return st;
    }
    const size_t bytes = 3 * a256(nk * 8) + 5 * a256(nk * tsz);
    char *p = nullptr;
    if (bytes) GBS_CUDA_TRY(cudaMalloc(&p, bytes));
    // a reused slot may hold a system of another size: the active lists and
    // the captured launch must be rebuilt before the next quantum
    E.dirty = true;
    H.used = true;
    H.finished = false;
    H.A = A;
    H.own_A = own_A;
    H.k = k;
    H.work = p;
    H.bytes = bytes;
    H.ticket = ticket;
    BSys S;
    memset(&S, 0, sizeof(S));
    S.rowptr = A->rowptr;
    S.colidx = A->colidx;
    S.tiles = A->tiles;
    S.vals = A->vals;
    S.vals32 = A->vals32;
    S.dinv = A->dinv;
    S.dinv32 = A->dinv32;
    if (p) {
        S.b = (const double *)p; p += a256(nk * 8);
        S.x = (double *)p; p += a256(nk * 8);
        S.r64 = (double *)p; p += a256(nk * 8);
        S.xi = p; p += a256(nk * tsz);
        S.ri = p; p += a256(nk * tsz);
        S.zi = p; p += a256(nk * tsz);
        S.pi = p; p += a256(nk * tsz);
        S.qi = p; p += a256(nk * tsz);
    }
    S.n = (int)A->n;
    S.k = k;
    S.ntiles = (int)A->ntiles;
    S.rtol = rtol;
    S.maxit = maxit;
    if (nk) {
        const int g = (int)std::min<int64_t>((int64_t)(nk + 255) / 256, (int64_t)c->num_sms * 8);
        k_interleave<<<g, 256, 0, c->stream>>>(A->n, k, b, (double *)S.b, 0);
        if (x0)
            k_interleave<<<g, 256, 0, c->stream>>>(A->n, k, x0, S.x, 0);
        else
            GBS_CUDA_TRY(cudaMemsetAsync(S.x, 0, nk * 8, c->stream));
        gbs_count_launch(c, x0 ? 2 : 1);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    BSysDyn D;
    memset(&D, 0, sizeof(D));
    D.mode[0] = D.mode[1] = MODE_OUTER;
    const bool bad = A->n == 0 || !A->diag_ok;
    D.finished = bad ? 1 : 0;
    BCol C[GBS_KMAX];
    for (int cc = 0; cc < GBS_KMAX; ++cc) {
        memset(&C[cc], 0, sizeof(BCol));
        C[cc].status = cc < k ? (A->n == 0 ? GBS_OK : (!A->diag_ok ? GBS_ERR_DIAG : GBS_RUNNING))
                              : GBS_OK;
        C[cc].prev = INFINITY;
        C[cc].first = 1;
    }
    H.finished = bad;
    E.h_dyn[slot] = D;
    GBS_CUDA_TRY(cudaMemcpyAsync(E.d_sys + slot, &S, sizeof(S), cudaMemcpyHostToDevice, c->stream));
    GBS_CUDA_TRY(cudaMemcpyAsync(E.d_col + (size_t)slot * GBS_KMAX, C, sizeof(C),
                                 cudaMemcpyHostToDevice, c->stream));
    GBS_CUDA_TRY(cudaMemcpyAsync(E.d_dyn + slot, &D, sizeof(D), cudaMemcpyHostToDevice, c->stream));
    // the host arrays above are copied from pageable memory: make sure they
    // are consumed before they go out of scope
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GBS_OK;
}

// Copy a slot's results out (x column-major into x_out, device or host per
// memspace) and release the slot.
int engine_collect(Engine &E, int slot, double *x_out, int memspace, int *iters, double *rnorm,
                   int *status)
{
    gbs_ctx c = E.c;
    SlotHost &H = E.slots[slot];
    BCol C[GBS_KMAX];
    GBS_CUDA_TRY(cudaMemcpyAsync(C, E.d_col + (size_t)slot * GBS_KMAX, sizeof(C),
                                 cudaMemcpyDeviceToHost, c->stream));
    const int64_t n = H.A->n;
    const size_t nk = (size_t)n * H.k;
    if (nk && x_out) {
        const double *xil = (const double *)(H.work + a256(nk * 8));
        const int g = (int)std::min<int64_t>((int64_t)(nk + 255) / 256, (int64_t)c->num_sms * 8);
        if (memspace == GBS_MEM_DEVICE) {
            k_interleave<<<g, 256, 0, c->stream>>>(n, H.k, xil, x_out, 1);
            gbs_count_launch(c);
            GBS_CUDA_TRY(cudaGetLastError());
        } else {
            std::vector<double> tmp(nk);
            GBS_CUDA_TRY(cudaMemcpyAsync(tmp.data(), xil, nk * 8, cudaMemcpyDeviceToHost, c->stream));
            GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
            for (size_t e = 0; e < nk; ++e) x_out[(e % H.k) * n + e / H.k] = tmp[e];
        }
    }
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int cc = 0; cc < H.k; ++cc) {
        const int cs = C[cc].status == GBS_RUNNING ? GBS_DIVERGED_ITS : C[cc].status;
        if (iters) iters[cc] = C[cc].iters;
        if (rnorm) rnorm[cc] = C[cc].rn;
        if (status) status[cc] = cs;
    }
    return GBS_OK;
}

void engine_release(Engine &E, int slot)
{
    E.dirty = true;
    SlotHost &H = E.slots[slot];
    if (H.work) cudaFree(H.work);
    if (H.own_A) gbs_mat_destroy(H.A);
    H = SlotHost();
}

// Run one quantum over the active slots; refresh the finished flags.
int engine_step(Engine &E, int *ran)
{
    gbs_ctx c = E.c;
    *ran = 0;
    std::vector<int> act, tcum(1, 0), ccum(1, 0);
    for (int s = 0; s < E.nslots; ++s) {
        const SlotHost &H = E.slots[s];
        if (H.used && !H.finished && H.A->ntiles > 0) {
            act.push_back(s);
            tcum.push_back(tcum.back() + (int)H.A->ntiles);
            ccum.push_back(ccum.back() + (int)((H.A->ntiles + GBS_RCHUNK - 1) / GBS_RCHUNK));
        }
    }
    if (act.empty()) return GBS_OK;
    const int nact = (int)act.size(), ntile = tcum.back(), nchunk = ccum.back();
    const void *fn = E.fp64 ? (const void *)k_batched<double> : (const void *)k_batched<float>;
    const size_t smem = sizeof(BTile<double>) * GBS_PWARPS;
    if (E.dirty || act != E.g_act || tcum != E.g_tcum) {
        engine_free_graph(E);
        E.dirty = false;
        if ((size_t)ntile > E.cap_part) {
            cudaFree(E.d_partS);
            cudaFree(E.d_partU);
            E.d_partS = E.d_partU = nullptr;
            E.cap_part = 0;
            const size_t cap = (size_t)ntile + ntile / 2 + 64;
            GBS_CUDA_TRY(cudaMalloc(&E.d_partS, cap * GBS_KMAX * 2 * sizeof(double)));
            GBS_CUDA_TRY(cudaMalloc(&E.d_partU, cap * GBS_KMAX * 2 * sizeof(double)));
            E.cap_part = cap;
        }
        if ((size_t)nchunk > E.cap_cpart) {
            cudaFree(E.d_cpart);
            E.d_cpart = nullptr;
            E.cap_cpart = 0;
            const size_t cap = (size_t)nchunk + nchunk / 2 + 64;
            GBS_CUDA_TRY(cudaMalloc(&E.d_cpart, cap * GBS_KMAX * 2 * sizeof(double)));
            E.cap_cpart = cap;
        }
        GBS_CUDA_TRY(cudaMemcpyAsync(E.d_ccum, ccum.data(), sizeof(int) * (nact + 1),
                                     cudaMemcpyHostToDevice, c->stream));
        GBS_CUDA_TRY(cudaMemcpyAsync(E.d_act, act.data(), sizeof(int) * nact, cudaMemcpyHostToDevice,
                                     c->stream));
        GBS_CUDA_TRY(cudaMemcpyAsync(E.d_tcum, tcum.data(), sizeof(int) * (nact + 1),
                                     cudaMemcpyHostToDevice, c->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));   // act/tcum are stack vectors
        GBS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, GBS_PBLOCK, smem));
        if (per_sm < 1) return GBS_ERR_CUDA;
        const int64_t need = ((int64_t)std::max(ntile, nchunk * GBS_KMAX) + GBS_PWARPS - 1) / GBS_PWARPS;
        E.G = (int)std::min<int64_t>((int64_t)per_sm * c->num_sms, std::max<int64_t>(need, 1));
        BArgs &a = E.g_args;
        memset(&a, 0, sizeof(a));
        a.sys = E.d_sys;
        a.col = E.d_col;
        a.dyn = E.d_dyn;
        a.act = E.d_act;
        a.tcum = E.d_tcum;
        a.nact = nact;
        a.ntile = ntile;
        a.nchunk = nchunk;
        a.ccum = E.d_ccum;
        a.cpart = E.d_cpart;
        a.ccount = E.d_ccount;
        a.partS = E.d_partS;
        a.partU = E.d_partU;
        a.bar = E.d_bar;
        a.quantum = E.quantum;   // even: the parity of the global iteration is unchanged
        a.iter0 = 0;
        a.inner_rtol = E.inner_rtol;
        a.outer_maxit = E.outer_maxit;
        a.fp64 = E.fp64;
        a.timeout_ns = (unsigned long long)c->opts.barrier_timeout_ms * 1000000ull;
        // capture barrier reset + cooperative launch once for this active set
        cudaStream_t cap = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(E.d_bar, 0, 256, cap);
            void *args[] = {&E.g_args};
            cudaLaunchCooperativeKernel(fn, dim3((unsigned)E.G), dim3(GBS_PBLOCK), args, smem, cap);
            e = cudaStreamEndCapture(cap, &E.graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&E.gexec, E.graph, 0);
        if (cap) cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            engine_free_graph(E);   // launch directly below
        } else {
            E.g_act = act;
            E.g_tcum = tcum;
        }
    }
    if (E.gexec) {
        GBS_CUDA_TRY(cudaGraphLaunch(E.gexec, c->stream));
    } else {
        GBS_CUDA_TRY(cudaMemsetAsync(E.d_bar, 0, 256, c->stream));
        void *args[] = {&E.g_args};
        GBS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3((unsigned)E.G), dim3(GBS_PBLOCK), args,
                                                 smem, c->stream));
    }
    gbs_count_launch(c);
    E.iter += E.quantum;
    *ran = 1;
    // barrier error word and the finished flags of every slot
    GBS_CUDA_TRY(cudaMemcpyAsync(c->pinned, &E.d_bar->error, sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream));
    GBS_CUDA_TRY(cudaMemcpyAsync(E.h_dyn.data(), E.d_dyn, sizeof(BSysDyn) * E.nslots,
                                 cudaMemcpyDeviceToHost, c->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (*(volatile int *)c->pinned) return GBS_ERR_TIMEOUT;
    for (int s = 0; s < E.nslots; ++s)
        if (E.slots[s].used) E.slots[s].finished = E.h_dyn[s].finished != 0;
    return GBS_OK;
}

}  // namespace

// ----------------------------------------------------------------------
// gbs_ksp_solve_cg_batched
// ----------------------------------------------------------------------

extern "C" int gbs_ksp_solve_cg_batched(gbs_ctx c, int nsys, const gbs_mat *A, const gbs_vec *B,
                                        gbs_vec *X, const int *nrhs, const double *rtol, int maxit,
                                        int mode, int *iters, double *rnorm, int *status)
{
    if (!c || nsys < 0 || (nsys > 0 && (!A || !B || !X || !nrhs || !rtol)) || maxit < 0)
        return GBS_ERR_ARG;
    if (mode != GBS_MODE_FP64 && mode != GBS_MODE_MIXED) return GBS_ERR_ARG;
    for (int s = 0; s < nsys; ++s) {
        if (!A[s] || !B[s] || !X[s] || A[s]->ctx != c || nrhs[s] < 1 || nrhs[s] > GBS_KMAX)
            return GBS_ERR_ARG;
        if (A[s]->n != A[s]->ncols || B[s]->n != A[s]->n * nrhs[s] || X[s]->n != B[s]->n ||
            B[s]->dtype != GBS_F64 || X[s]->dtype != GBS_F64 || !(rtol[s] >= 0.0))
            return GBS_ERR_ARG;
    }
    if (nsys == 0) return GBS_OK;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    Engine E;
    int rc = engine_init(E, c, nsys, mode == GBS_MODE_FP64, 64);
    for (int s = 0; s < nsys && rc == GBS_OK; ++s)
        rc = engine_add(E, s, A[s], nrhs[s], rtol[s], maxit, (const double *)B[s]->data,
                        (const double *)X[s]->data, false, 0);
    if (rc == GBS_OK) {
        cudaEventRecord(c->ev0, c->stream);
        for (int ran = 1; rc == GBS_OK && ran;) rc = engine_step(E, &ran);
        cudaEventRecord(c->ev1, c->stream);
    }
    int first_bad = GBS_OK;
    int64_t o = 0;
    for (int s = 0; s < nsys && rc == GBS_OK; ++s) {
        int it[GBS_KMAX], stc[GBS_KMAX];
        double rn[GBS_KMAX];
        rc = engine_collect(E, s, (double *)X[s]->data, GBS_MEM_DEVICE, it, rn, stc);
        for (int cc = 0; cc < nrhs[s] && rc == GBS_OK; ++cc, ++o) {
            if (iters) iters[o] = it[cc];
            if (rnorm) rnorm[o] = rn[cc];
            if (status) status[o] = stc[cc];
            if (stc[cc] != GBS_OK && first_bad == GBS_OK) first_bad = stc[cc];
        }
    }
    if (rc == GBS_OK) {
        cudaStreamSynchronize(c->stream);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->last.device_ms = ms;
    }
    engine_destroy(E);
    return rc != GBS_OK ? rc : first_bad;
}

// ----------------------------------------------------------------------
// Serving loop: continuous batching of solve requests under a memory budget
// ----------------------------------------------------------------------

namespace {

struct Request {
    uint64_t ticket;
    int64_t n;
    int k;
    double rtol;
    int maxit;
    std::vector<int32_t> rowptr, colidx;
    std::vector<double> vals, b;
    size_t bytes;
    int slot = -1;
    bool done = false;
    std::vector<double> x;
    std::vector<int> iters, status;
    std::vector<double> rnorm;
};

}  // namespace

struct gbs_server_s {
    gbs_ctx c;
    Engine E;
    size_t budget;
    size_t used = 0;
    int mode;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;                       // waiting for admission, FIFO
    std::unordered_map<uint64_t, Request> reqs;       // queued, running or done
    int running = 0, finished = 0;
};

extern "C" int gbs_server_create(gbs_ctx c, size_t budget, int max_slots, int mode, gbs_server *out)
{
    if (!c || !out || budget == 0 || max_slots < 0) return GBS_ERR_ARG;
    if (mode != GBS_MODE_FP64 && mode != GBS_MODE_MIXED) return GBS_ERR_ARG;
    *out = nullptr;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    gbs_server srv = new (std::nothrow) gbs_server_s();
    if (!srv) return GBS_ERR_OOM;
    srv->c = c;
    srv->budget = budget;
    srv->mode = mode;
    const int st = engine_init(srv->E, c, max_slots ? max_slots : 256, mode == GBS_MODE_FP64, 32);
    if (st) {
        engine_destroy(srv->E);
        delete srv;
        return st;
    }
    *out = srv;
    return GBS_OK;
}

extern "C" int gbs_server_destroy(gbs_server srv)
{
    if (!srv) return GBS_OK;
    cudaSetDevice(srv->c->device);
    engine_destroy(srv->E);
    delete srv;
    return GBS_OK;
}

extern "C" int gbs_server_submit(gbs_server srv, int64_t nrows, const int32_t *rowptr,
                                 const int32_t *colidx, const double *vals, int k, const double *b,
                                 double rtol, int maxit, uint64_t *ticket)
{
    if (!srv || !ticket || nrows < 0 || nrows >= INT32_MAX || !rowptr || k < 1 || k > GBS_KMAX ||
        !(rtol >= 0.0) || maxit < 0 || (nrows > 0 && !b))
        return GBS_ERR_ARG;
    const int64_t nnz = rowptr[nrows];
    if (nnz < 0 || (nnz > 0 && (!colidx || !vals))) return GBS_ERR_ARG;
    const size_t bytes = system_bytes(nrows, nnz, k, srv->mode == GBS_MODE_FP64);
    if (bytes > srv->budget) return GBS_ERR_BUDGET;
    Request r;
    r.ticket = srv->next_ticket++;
    r.n = nrows;
    r.k = k;
    r.rtol = rtol;
    r.maxit = maxit;
    r.rowptr.assign(rowptr, rowptr + nrows + 1);
    r.colidx.assign(colidx, colidx + nnz);
    r.vals.assign(vals, vals + nnz);
    r.b.assign(b, b + nrows * k);
    r.bytes = bytes;
    *ticket = r.ticket;
    srv->queue.push_back(r.ticket);
    srv->reqs.emplace(r.ticket, std::move(r));
    return GBS_OK;
}

// Admit queued requests (FIFO) while a slot and budget are free.
static int server_admit(gbs_server srv)
{
    Engine &E = srv->E;
    while (!srv->queue.empty()) {
        Request &r = srv->reqs.at(srv->queue.front());
        int slot = -1;
        for (int s = 0; s < E.nslots; ++s)
            if (!E.slots[s].used) { slot = s; break; }
        if (slot < 0 || srv->used + r.bytes > srv->budget) break;
        srv->queue.pop_front();
        gbs_mat A = nullptr;
        int st = gbs_mat_create_aij(srv->c, r.n, r.n, r.rowptr.data(), r.colidx.data(),
                                    r.vals.data(), GBS_MEM_HOST, &A);
        if (st != GBS_OK) {
            // a malformed request finishes at once with that status
            r.done = true;
            r.x.assign((size_t)r.n * r.k, 0.0);
            r.iters.assign(r.k, 0);
            r.rnorm.assign(r.k, 0.0);
            r.status.assign(r.k, st);
            ++srv->finished;
            continue;
        }
        double *db = nullptr;
        const size_t nb = (size_t)r.n * r.k * sizeof(double);
        if (nb) {
            cudaError_t e = cudaMalloc(&db, nb);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(db, r.b.data(), nb, cudaMemcpyHostToDevice, srv->c->stream);
            if (e != cudaSuccess) {
                cudaFree(db);
                gbs_mat_destroy(A);
                return gbs_cuda_fail(e);
            }
        }
        st = engine_add(E, slot, A, r.k, r.rtol, r.maxit, db, nullptr, true, r.ticket);
        cudaFree(db);   // engine_add synchronised the stream after interleaving b
        if (st) {
            gbs_mat_destroy(A);
            return st;
        }
        r.slot = slot;
        srv->used += r.bytes;
        ++srv->running;
        std::vector<double>().swap(r.b);
        std::vector<int32_t>().swap(r.colidx);
        std::vector<double>().swap(r.vals);
    }
    return GBS_OK;
}

// Retire finished slots: results to the host, memory and slot released.
static int server_retire(gbs_server srv, int *retired)
{
    Engine &E = srv->E;
    for (int s = 0; s < E.nslots; ++s) {
        SlotHost &H = E.slots[s];
        if (!H.used || !H.finished) continue;
        Request &r = srv->reqs.at(H.ticket);
        r.x.assign((size_t)r.n * r.k, 0.0);
        r.iters.assign(r.k, 0);
        r.rnorm.assign(r.k, 0.0);
        r.status.assign(r.k, 0);
        const int st = engine_collect(E, s, r.x.data(), GBS_MEM_HOST, r.iters.data(), r.rnorm.data(),
                                      r.status.data());
        if (st) return st;
        engine_release(E, s);
        srv->used -= r.bytes;
        r.done = true;
        r.slot = -1;
        --srv->running;
        ++srv->finished;
        ++*retired;
    }
    return GBS_OK;
}

extern "C" int gbs_server_progress(gbs_server srv, int *retired)
{
    if (!srv) return GBS_ERR_ARG;
    int n = 0;
    GBS_CUDA_TRY(cudaSetDevice(srv->c->device));
    int st = server_retire(srv, &n);   // systems that finished at admission
    if (!st) st = server_admit(srv);
    int ran = 0;
    if (!st) st = engine_step(srv->E, &ran);
    if (!st) st = server_retire(srv, &n);
    if (retired) *retired = n;
    return st;
}

extern "C" int gbs_server_poll(gbs_server srv, uint64_t ticket, int *done)
{
    if (!srv || !done) return GBS_ERR_ARG;
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return GBS_ERR_NOT_FOUND;
    *done = it->second.done ? 1 : 0;
    return GBS_OK;
}

extern "C" int gbs_server_wait(gbs_server srv, uint64_t ticket)
{
    if (!srv) return GBS_ERR_ARG;
    for (;;) {
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return GBS_ERR_NOT_FOUND;
        if (it->second.done) return GBS_OK;
        const int st = gbs_server_progress(srv, nullptr);
        if (st) return st;
    }
}

extern "C" int gbs_server_fetch(gbs_server srv, uint64_t ticket, double *x, int *iters,
                                double *rnorm, int *status)
{
    if (!srv) return GBS_ERR_ARG;
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end() || !it->second.done) return GBS_ERR_NOT_FOUND;
    Request &r = it->second;
    if (x && !r.x.empty()) memcpy(x, r.x.data(), r.x.size() * sizeof(double));
    for (int cc = 0; cc < r.k; ++cc) {
        if (iters) iters[cc] = r.iters[cc];
        if (rnorm) rnorm[cc] = r.rnorm[cc];
        if (status) status[cc] = r.status[cc];
    }
    srv->reqs.erase(it);
    return GBS_OK;
}

extern "C" int gbs_server_stats(gbs_server srv, int *queued, int *running, int *finished,
                                size_t *bytes_in_use)
{
    if (!srv) return GBS_ERR_ARG;
    if (queued) *queued = (int)srv->queue.size();
    if (running) *running = srv->running;
    if (finished) *finished = srv->finished;
    if (bytes_in_use) *bytes_in_use = srv->used;
    return GBS_OK;
}
