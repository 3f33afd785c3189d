// Batched Jacobi-PCG over many independent systems with several right-hand
// sides each, in one persistent cooperative kernel (Response A6: solve many
// different-size problems at once; Challenge F2 and Sec. 4: multiple
// right-hand sides raise arithmetic intensity; Response A7: FP32 inner
// iterations with FP64 refinement), and the serving loop built on it.
//
// Lockstep design.  Every active system advances by one step per global
// iteration; a step has three phases separated by grid barriers:
//   S   SpMV over every warp tile of every active system (all k columns
//       of a system share one pass over its matrix; INNER tiles are staged
//       through a per-warp TMA ring), per-unit partials of p.q (or of
//       r.r and b.b for the refinement residual)
//   U   vector updates, per-unit partials of r.z and r.r
//   P   direction update, or the FP64 solution update before a refinement
// The reductions need no phase of their own: each unit of work stores its
// partial sums and counts itself in; the warp that completes a chunk of
// units adds the chunk up, and the warp that completes a system's last
// chunk adds the chunks up and computes the system's scalars for the next
// phase.  Both orders are fixed by the system alone.
// A system is either in an INNER step (one PCG iteration in the inner
// precision TI on all its unfinished columns) or an OUTER step (FP64
// residual r = b - A x, stopping test, r / ||r|| becomes the inner
// right-hand side).  Its columns advance together; a column whose inner
// solve has converged waits for the others, then all refine together.
// Because every per-system quantity depends only on the system's own data
// and a fixed reduction order, each column's result is bitwise the same
// alone or in any batch.
//
// Multi-vectors are interleaved with the column count padded to a power of
// two, so the operands of one nonzero are one aligned vector load and the
// update phases stream contiguous, coalesced entries.

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
#include <type_traits>
#include <chrono>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

#include "gbs_impl.cuh"

#define GBS_KMAX 8
#define GBS_RUNNING (-100)
#define GBS_RCHUNK 128          // reduction units per chunk
#define GBS_SUB 256             // vector entries per update sub-block (8 per lane)
#define GBS_BWARP_BYTES 13312   // bytes of one warp's stage ring

namespace {

enum { MODE_OUTER = 0, MODE_INNER = 1 };

// Read-only description of one system (device, one per slot).  Its
// multi-vectors are interleaved with a padded stride kp (entry (row, c) at
// row * kp + c, kp = k rounded up to 1, 2, 4 or 8; the padding columns
// hold zeros), so the kp operands one nonzero gathers are one aligned
// vector load.
struct BSys {
    const int32_t *rowptr, *colidx, *tdesc;   // tdesc: {row start, nonzero start} per warp tile
    const int16_t *colrel16;                  // col - row, for INNER tiles (may be NULL)
    const double *vals, *dinv;
    const float *vals32, *dinv32;
    const double *b;    // n x kp
    double *x;          // n x kp (initial guess in, solution out)
    double *r64;        // n x kp
    void *xi, *ri, *pi, *qi;   // inner-precision work vectors, n x kp
    int n, k, kp, ntiles;
    int tg;             // warp tiles per S-phase reduction unit
    int usub;           // update sub-blocks per U/P-phase unit
    int maxit;
    int lanes_log;      // log2 of the lanes sharing a row in the INNER SpMV
    double rtol;
};

// Mutable state of one (system, column) pair, touched only by the warp that
// completes the system's reduction of a phase (device).
struct BCol {
    double rho, alpha, beta, rn, bnorm, prev, scale, tol_inner;
    int status;       // GBS_RUNNING until final
    int iters;        // inner iterations, all refinement steps together
    int outer;        // refinement steps
    int kin;          // inner iterations of the current refinement step
    int inner_done;   // the current inner solve has stopped
    int first;        // no residual computed yet
    int pad[2];
};

// Per-system scalars a phase hands to the next (device; written by the
// warp that completes a reduction, read by every unit of the next phase).
struct BPh {
    double alpha64[GBS_KMAX], beta64[GBS_KMAX];   // inner step scalars (FP64 inner)
    double scale[GBS_KMAX];                       // 1 / ||r|| of the refinement residual
    double rn[GBS_KMAX];                          // ||r|| (the solution update x += ||r|| d)
    float alpha32[GBS_KMAX], beta32[GBS_KMAX];    // inner step scalars (FP32 inner)
    unsigned run;   // columns still running
    unsigned upd;   // columns whose inner solve advances
    int pad[14];
};

// Mutable per-system state (device).
struct BSysDyn {
    int mode[2];      // indexed by global iteration parity
    int finished;
    int isteps;       // INNER steps taken
    int osteps;       // OUTER steps taken
    int pad[3];
};

struct BArgs {
    const BSys *sys;    // by slot
    BCol *col;          // slot * GBS_KMAX + column
    BPh *ph;            // by slot
    BSysDyn *dyn;       // by slot
    const int *act;     // active slots, nact entries
    const int *scum;    // prefix sums of the active systems' S units (nact + 1)
    const int *ucum;    // prefix sums of the active systems' U/P units (nact + 1)
    const int *ccs;     // prefix sums of their S reduction chunks (nact + 1)
    const int *ccu;     // prefix sums of their U reduction chunks (nact + 1)
    int nact, nsu, nuu; // active systems; S units; U/P units
    double *partS, *partU;     // unit * 16: per-unit partial sums
    double *cpartS, *cpartU;   // chunk * 16: per-chunk sums
    int *cntS, *cntU;          // per chunk: units arrived (zero between phases)
    int *sysS, *sysU;          // per active system: chunks arrived
    int *claim;                // next unclaimed unit of S, U, P: 4 rotating sets of 3
    int *nfin;                 // active systems finished during the launch
    gbs_grid_barrier *bar;
    GbsPipeCfg cfg;     // stage geometry covering every active system's tiles
    int ring;           // bytes of one warp's stage ring (cfg.stages stages, 128-aligned)
    int quantum;        // global iterations at most (even)
    int iter0;          // parity of the global iteration count at launch
    double inner_rtol;
    int outer_maxit;
    int fp64;           // inner precision is FP64 (FP64 mode)
    unsigned long long timeout_ns;
};

// Per-warp ring bookkeeping in shared memory.
struct BWarpQ {
    uint64_t bar[GBS_MAX_STAGES];
    int4 desc[GBS_MAX_STAGES];    // {r0, k0, r1, k1}
    int unit[GBS_MAX_STAGES];     // S unit of the tile in the stage (-1: none)
    int ai[GBS_MAX_STAGES];       // its system's active index
    int flags[GBS_MAX_STAGES];    // 1: copied into the stage; 2: first tile of the unit;
                                  // 4: last tile of the unit; 8: INNER step;
                                  // 16: 16-bit relative column indices
};

template <typename TI> __device__ __forceinline__ const TI *bvals(const BSys &S);
template <> __device__ __forceinline__ const float *bvals<float>(const BSys &S) { return S.vals32; }
template <> __device__ __forceinline__ const double *bvals<double>(const BSys &S) { return S.vals; }
template <typename TI> __device__ __forceinline__ const TI *bdinv(const BSys &S);
template <> __device__ __forceinline__ const float *bdinv<float>(const BSys &S) { return S.dinv32; }
template <> __device__ __forceinline__ const double *bdinv<double>(const BSys &S) { return S.dinv; }

__device__ __forceinline__ float ph_alpha(const BPh &P, int c, float) { return P.alpha32[c]; }
__device__ __forceinline__ double ph_alpha(const BPh &P, int c, double) { return P.alpha64[c]; }
__device__ __forceinline__ float ph_beta(const BPh &P, int c, float) { return P.beta32[c]; }
__device__ __forceinline__ double ph_beta(const BPh &P, int c, double) { return P.beta64[c]; }
__device__ __forceinline__ void ph_set(BPh &P, int c, float al, float be, bool a)
{
    if (a) P.alpha32[c] = al;
    else P.beta32[c] = be;
}
__device__ __forceinline__ void ph_set(BPh &P, int c, double al, double be, bool a)
{
    if (a) P.alpha64[c] = al;
    else P.beta64[c] = be;
}

// Rounded product (kept out of any fused multiply-add).
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

// KP consecutive entries of type T at p, KP * sizeof(T) aligned.
template <typename T, int KP>
__device__ __forceinline__ void vload(const T *p, T (&v)[KP])
{
    constexpr int B = KP * (int)sizeof(T);
    if constexpr (B >= 16) {
        constexpr int W = 16 / (int)sizeof(T);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            const float4 w = reinterpret_cast<const float4 *>(p)[i];
            T t[W];
            memcpy(t, &w, 16);
#pragma unroll
            for (int l = 0; l < W; ++l) v[i * W + l] = t[l];
        }
    } else if constexpr (B == 8) {
        const float2 w = *reinterpret_cast<const float2 *>(p);
        memcpy(v, &w, 8);
    } else {
        v[0] = *p;
    }
}

template <typename T, int KP>
__device__ __forceinline__ void vstore(T *p, const T (&v)[KP])
{
    constexpr int B = KP * (int)sizeof(T);
    if constexpr (B >= 16) {
        constexpr int W = 16 / (int)sizeof(T);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            T t[W];
#pragma unroll
            for (int l = 0; l < W; ++l) t[l] = v[i * W + l];
            float4 w;
            memcpy(&w, t, 16);
            reinterpret_cast<float4 *>(p)[i] = w;
        }
    } else if constexpr (B == 8) {
        float2 w;
        memcpy(&w, v, 8);
        *reinterpret_cast<float2 *>(p) = w;
    } else {
        *p = v[0];
    }
}

// ---------------------------------------------------------------------
// S phase: one warp tile
// ---------------------------------------------------------------------

// INNER step, tile staged in shared memory: q = A p on its rows.  L = 2^li
// lanes share a row: lane l takes row r0 + l / L and every L-th nonzero of
// it from l mod L on (all KP columns at once); the L partial sums are added
// by a fixed shuffle tree.  acc[c][0] += p_row,c q_row,c (p_row loaded once
// per row: every row of an admitted system has its diagonal entry, so this
// is the operand the diagonal's gather reads; picking it out of the
// gathers instead cost KP selects per nonzero).
template <typename TI, int KP, bool REL>
__device__ __forceinline__ void s_tile_inner(const BSys &S, const unsigned char *st,
                                             const GbsPipeCfg &cfg, int4 d, TI (&acc)[KP][2])
{
    using IX = typename std::conditional<REL, int16_t, int32_t>::type;
    constexpr int E = 16 / (int)sizeof(TI), CE = 16 / (int)sizeof(IX);
    const int lane = threadIdx.x & 31;
    const int li = S.lanes_log, L = 1 << li;
    const int r0 = d.x, k0 = d.y, r1 = d.z;
    const int rl = lane >> li, h = lane & (L - 1);
    const bool act = rl < r1 - r0;
    const int row = r0 + rl;
    TI sum[KP];
#pragma unroll
    for (int i = 0; i < KP; ++i) sum[i] = TI(0);
    if (act) {
        const TI *sval = reinterpret_cast<const TI *>(st);
        const IX *scol = reinterpret_cast<const IX *>(st + cfg.coloff);
        const int32_t *srp = reinterpret_cast<const int32_t *>(st + cfg.rpoff);
        const int vb = k0 & ~(E - 1), cb = k0 & ~(CE - 1), rb = r0 & ~3;
        const int beg = srp[row - rb], end = srp[row - rb + 1];
        const TI *p = static_cast<const TI *>(S.pi);
        // gathers in flight per lane: as many as the registers allow
#pragma unroll(KP * sizeof(TI) >= 32 ? 4 : 8)
        for (int e = beg + h; e < end; e += L) {
            const int c = REL ? row + (int)scol[e - cb] : (int)scol[e - cb];
            const TI a = sval[e - vb];
            TI v[KP];
            vload<TI, KP>(p + (size_t)c * KP, v);
#pragma unroll
            for (int i = 0; i < KP; ++i) sum[i] = fma(a, v[i], sum[i]);
        }
    }
    for (int off = 1; off < L; off <<= 1)
#pragma unroll
        for (int i = 0; i < KP; ++i) sum[i] += __shfl_xor_sync(0xffffffffu, sum[i], off);
    if (act && h == 0) {
        TI pd[KP];
        vload<TI, KP>(static_cast<const TI *>(S.pi) + (size_t)row * KP, pd);
        vstore<TI, KP>(static_cast<TI *>(S.qi) + (size_t)row * KP, sum);
#pragma unroll
        for (int i = 0; i < KP; ++i) acc[i][0] += pd[i] * sum[i];
    }
}

// INNER step, a tile holding one row longer than GBS_WT_NNZ (read directly;
// lane-strided sums, fixed shuffle tree; lane 0 accumulates).
template <typename TI, int KP>
__device__ __forceinline__ void s_long_inner(const BSys &S, int4 d, TI (&acc)[KP][2], uint64_t ps)
{
    const int lane = threadIdx.x & 31;
    const int row = d.x, k0 = d.y, k1 = d.w;
    const TI *vals = bvals<TI>(S);
    const TI *p = static_cast<const TI *>(S.pi);
    TI sum[KP];
#pragma unroll
    for (int i = 0; i < KP; ++i) sum[i] = TI(0);
    for (int e = k0 + lane; e < k1; e += 32) {
        const int c = gbs_ld_stream(S.colidx + e, ps);
        const TI a = gbs_ld_stream(vals + e, ps);
        TI v[KP];
        vload<TI, KP>(p + (size_t)c * KP, v);
#pragma unroll
        for (int i = 0; i < KP; ++i) sum[i] = fma(a, v[i], sum[i]);
    }
#pragma unroll
    for (int i = 0; i < KP; ++i)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum[i] += __shfl_xor_sync(0xffffffffu, sum[i], off);
    if (lane == 0) {
        TI pd[KP];
        vload<TI, KP>(p + (size_t)row * KP, pd);
        vstore<TI, KP>(static_cast<TI *>(S.qi) + (size_t)row * KP, sum);
#pragma unroll
        for (int i = 0; i < KP; ++i) acc[i][0] += pd[i] * sum[i];
    }
}

// OUTER step (FP64, read directly): r64 = b - A x on the tile's rows;
// acc[c][0] += r.r, acc[c][1] += b.b.
template <int KP>
__device__ __forceinline__ void s_tile_outer(const BSys &S, int4 d, double (&acc)[KP][2], uint64_t ps)
{
    const int lane = threadIdx.x & 31;
    const int r0 = d.x, k0 = d.y, r1 = d.z, k1 = d.w;
    double sum[KP];
#pragma unroll
    for (int i = 0; i < KP; ++i) sum[i] = 0.0;
    int row = r0 + lane;
    bool own = false;
    if (k1 - k0 > GBS_WT_NNZ) {
        for (int e = k0 + lane; e < k1; e += 32) {
            const int c = gbs_ld_stream(S.colidx + e, ps);
            const double a = gbs_ld_stream(S.vals + e, ps);
            double v[KP];
            vload<double, KP>(S.x + (size_t)c * KP, v);
#pragma unroll
            for (int i = 0; i < KP; ++i) sum[i] = fma(a, v[i], sum[i]);
        }
#pragma unroll
        for (int i = 0; i < KP; ++i)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sum[i] += __shfl_xor_sync(0xffffffffu, sum[i], off);
        row = r0;
        own = lane == 0;
    } else if (lane < r1 - r0) {
        const int beg = __ldg(S.rowptr + row), end = __ldg(S.rowptr + row + 1);
#pragma unroll 4
        for (int e = beg; e < end; ++e) {
            const int c = gbs_ld_stream(S.colidx + e, ps);
            const double a = gbs_ld_stream(S.vals + e, ps);
            double v[KP];
            vload<double, KP>(S.x + (size_t)c * KP, v);
#pragma unroll
            for (int i = 0; i < KP; ++i) sum[i] = fma(a, v[i], sum[i]);
        }
        own = true;
    }
    if (own) {
        double bv[KP], rv[KP];
        vload<double, KP>(S.b + (size_t)row * KP, bv);
#pragma unroll
        for (int i = 0; i < KP; ++i) {
            rv[i] = bv[i] - sum[i];
            acc[i][0] += rv[i] * rv[i];
            acc[i][1] += bv[i] * bv[i];
        }
        vstore<double, KP>(S.r64 + (size_t)row * KP, rv);
    }
}

// ---------------------------------------------------------------------
// Reductions: per-unit partials, summed by the warp that completes them
// ---------------------------------------------------------------------

// Fixed-tree warp sums of entries [c][j], c < k, j < NJ; every lane gets them.
template <typename T, int NJ>
__device__ __forceinline__ void warp_tree(T (&acc)[GBS_KMAX][2], int k)
{
#pragma unroll
    for (int c = 0; c < GBS_KMAX; ++c) {
        if (c >= k) break;
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                acc[c][j] += __shfl_xor_sync(0xffffffffu, acc[c][j], off);
    }
}

// Sum entries [c][j] of the 16-value records [ua, ub) of src in type T, in
// a fixed order (lane l: records ua + l, ua + l + 32, ...; then a fixed
// shuffle tree); every lane gets the totals.
template <typename T, int NJ>
__device__ __forceinline__ void sum_records(const double *src, int ua, int ub, int k,
                                            T (&tot)[GBS_KMAX][2])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < GBS_KMAX; ++c) tot[c][0] = tot[c][1] = T(0);
    for (int u = ua + lane; u < ub; u += 32) {
        const double2 *s = reinterpret_cast<const double2 *>(src + (size_t)u * 2 * GBS_KMAX);
#pragma unroll
        for (int c = 0; c < GBS_KMAX; ++c) {
            if (c >= k) break;
            const double2 w = __ldcg(s + c);
            tot[c][0] += (T)w.x;
            if (NJ > 1) tot[c][1] += (T)w.y;
        }
    }
    warp_tree<T, NJ>(tot, k);
}

// Unit u of one system (units [u0, u0 + nu), chunks from c0) has stored its
// partials.  The warp that completes a chunk of GBS_RCHUNK units adds the
// chunk up; the warp that completes the system's last chunk adds the chunk
// sums up and returns true with the totals in every lane.  Both orders
// depend on the system alone, so the totals are the same in any batch.
template <typename T, int NJ>
__device__ __forceinline__ bool reduce_last(const double *part, double *cpart, int *ccnt,
                                            int *scnt, int u, int u0, int nu, int c0, int k,
                                            T (&tot)[GBS_KMAX][2])
{
    const int lane = threadIdx.x & 31;
    const int ch = (u - u0) / GBS_RCHUNK;
    const int ua = u0 + ch * GBS_RCHUNK, ub = min(ua + GBS_RCHUNK, u0 + nu);
    const int nch = (nu + GBS_RCHUNK - 1) / GBS_RCHUNK;
    int last = 0;
    if (lane == 0) {
        __threadfence();
        last = atomicAdd(&ccnt[c0 + ch], 1) == ub - ua - 1;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return false;
    __threadfence();
    sum_records<T, NJ>(part, ua, ub, k, tot);
    if (lane == 0) {
        double *dst = cpart + (size_t)(c0 + ch) * 2 * GBS_KMAX;
#pragma unroll
        for (int c = 0; c < GBS_KMAX; ++c) {
            if (c >= k) break;
            dst[2 * c] = (double)tot[c][0];
            dst[2 * c + 1] = NJ > 1 ? (double)tot[c][1] : 0.0;
        }
        ccnt[c0 + ch] = 0;
        __threadfence();
        last = atomicAdd(scnt, 1) == nch - 1;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return false;
    __threadfence();
    sum_records<T, NJ>(cpart, c0, c0 + nch, k, tot);
    if (lane == 0) *scnt = 0;
    return true;
}

// Lane 0 stores the warp-summed entries [c][j] as the unit's record.
template <typename T, int NJ>
__device__ __forceinline__ void store_record(double *part, int u, int k, const T (&acc)[GBS_KMAX][2])
{
    if ((threadIdx.x & 31) != 0) return;
    double *dst = part + (size_t)u * 2 * GBS_KMAX;
#pragma unroll
    for (int c = 0; c < GBS_KMAX; ++c) {
        if (c >= k) break;
        dst[2 * c] = (double)acc[c][0];
        dst[2 * c + 1] = NJ > 1 ? (double)acc[c][1] : 0.0;
    }
}

// The value of column `lane` (lanes < k) out of a register array.
template <typename T>
__device__ __forceinline__ T mine(const T (&tot)[GBS_KMAX][2], int j)
{
    const int lane = threadIdx.x & 31;
    T v = T(0);
#pragma unroll
    for (int c = 0; c < GBS_KMAX; ++c) v = c == lane ? tot[c][j] : v;
    return v;
}

// ---------------------------------------------------------------------
// Scalar steps, run by the warp that completes a system's reduction
// (lane c handles column c)
// ---------------------------------------------------------------------

// OUTER residual r = b - A x is complete: stopping test, refinement scale.
__device__ __noinline__ void s_finish_outer(const BArgs &a, int slot, double rr, double bb)
{
    const int lane = threadIdx.x & 31;
    const BSys &S = a.sys[slot];
    BPh &P = a.ph[slot];
    bool run = false;
    if (lane < S.k) {
        BCol &C = a.col[slot * GBS_KMAX + lane];
        if (C.status == GBS_RUNNING) {
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
                // FP64 inner solves aim below rtol ||b|| at once; FP32 ones
                // stop at the inner tolerance, or sooner where half the
                // outer target already suffices (the last refinement step)
                C.tol_inner = a.fp64 ? 0.5 * S.rtol * C.bnorm / rn
                                     : fmax(a.inner_rtol, 0.5 * S.rtol * C.bnorm / rn);
                P.scale[lane] = C.scale;
                P.rn[lane] = rn;
                run = true;
            }
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, run);
    if (lane == 0) {
        P.run = m;
        P.upd = m;
        a.dyn[slot].osteps += 1;
        if (!m) {
            a.dyn[slot].finished = 1;
            atomicAdd(a.nfin, 1);
        }
    }
}

// INNER p.q is complete: step length alpha, or breakdown.
template <typename TI>
__device__ __noinline__ void s_finish_inner(const BArgs &a, int slot, TI pq)
{
    const int lane = threadIdx.x & 31;
    const BSys &S = a.sys[slot];
    BPh &P = a.ph[slot];
    const unsigned upd = P.upd;
    bool bad = false;
    if (lane < S.k && ((upd >> lane) & 1u)) {
        BCol &C = a.col[slot * GBS_KMAX + lane];
        if (isnan(pq)) C.status = GBS_ERR_NAN;
        else if (pq <= TI(0)) C.status = GBS_ERR_INDEFINITE;
        else {
            const TI al = (TI)C.rho / pq;
            C.alpha = (double)al;
            ph_set(P, lane, al, al, true);
        }
        bad = C.status != GBS_RUNNING;
    }
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (lane == 0 && m) {
        P.upd = upd & ~m;
        P.run &= ~m;
        if (!P.run) {
            a.dyn[slot].finished = 1;
            atomicAdd(a.nfin, 1);
        }
    }
}

// OUTER start of an inner solve is complete: rho = r.z, inner tolerance.
template <typename TI>
__device__ __noinline__ void u_finish_outer(const BArgs &a, int slot, int nxt, TI rho, TI rr)
{
    const int lane = threadIdx.x & 31;
    const BSys &S = a.sys[slot];
    BPh &P = a.ph[slot];
    if (lane < S.k && ((P.run >> lane) & 1u)) {
        BCol &C = a.col[slot * GBS_KMAX + lane];
        C.rho = (double)rho;
        C.tol_inner = C.tol_inner * (double)sqrt(rr);
        C.kin = 0;
        C.inner_done = 0;
    }
    __syncwarp();
    if (lane == 0) {
        P.upd = P.run;
        a.dyn[slot].mode[nxt] = MODE_INNER;
    }
}

// INNER r.z and r.r are complete: beta, inner stopping test, next step.
template <typename TI>
__device__ __noinline__ void u_finish_inner(const BArgs &a, int slot, int nxt, TI rho_new, TI rr)
{
    const int lane = threadIdx.x & 31;
    const BSys &S = a.sys[slot];
    BPh &P = a.ph[slot];
    const unsigned upd = P.upd;
    bool fail = false, waiting = false;
    if (lane < S.k && ((upd >> lane) & 1u)) {
        BCol &C = a.col[slot * GBS_KMAX + lane];
        C.kin += 1;
        C.iters += 1;
        if (rho_new < TI(0)) {
            C.status = GBS_ERR_INDEFINITE;
        } else if (isnan(rr)) {
            C.status = GBS_ERR_NAN;
        } else {
            const TI be = rho_new / (TI)C.rho;
            C.beta = (double)be;
            C.rho = (double)rho_new;
            ph_set(P, lane, be, be, false);
            if ((double)sqrt(rr) <= C.tol_inner || C.iters >= S.maxit) C.inner_done = 1;
        }
        fail = C.status != GBS_RUNNING;
        waiting = !fail && !C.inner_done;
    }
    const unsigned mf = __ballot_sync(0xffffffffu, fail);
    const unsigned mw = __ballot_sync(0xffffffffu, waiting);
    if (lane == 0) {
        const unsigned run = P.run & ~mf;
        P.run = run;
        P.upd = mw;
        a.dyn[slot].isteps += 1;
        // refinement once every running column's inner solve has stopped
        if (!run) {
            a.dyn[slot].finished = 1;
            atomicAdd(a.nfin, 1);
        } else {
            a.dyn[slot].mode[nxt] = mw ? MODE_INNER : MODE_OUTER;
        }
    }
}

// ---------------------------------------------------------------------
// S phase: the warp's stage ring over the CTA's S units
// ---------------------------------------------------------------------

// Run the S unit whose first tile sits in stage m % NS (issued and
// checked): consume its tiles, which follow one another in the warp's ring,
// then store the unit's partials and take part in the system's reduction.
// Returns false if a copy did not complete in time (m then names the stage
// that failed).
template <typename TI, int KP, bool INNER, typename Issue>
__device__ __forceinline__ bool s_unit(const BArgs &a, BWarpQ &q, unsigned char *wsm,
                                       const GbsPipeCfg &cfg, int &m, uint32_t &parity, uint64_t ps,
                                       Issue &issue)
{
    using T = typename std::conditional<INNER, TI, double>::type;
    constexpr int NJ = INNER ? 1 : 2;
    const int lane = threadIdx.x & 31;
    const int NS = cfg.stages;
    const int unit = q.unit[m % NS], ai = q.ai[m % NS];
    const int slot = __ldg(a.act + ai);
    const BSys &S = a.sys[slot];
    T acc[KP][2];
#pragma unroll
    for (int i = 0; i < KP; ++i) acc[i][0] = acc[i][1] = T(0);
    for (;;) {
        const int j = m % NS;
        const int4 d = q.desc[j];
        const int flags = q.flags[j];
        if (flags & 1) {
            if (!gbs_mbar_wait(&q.bar[j], (parity >> j) & 1u, a.timeout_ns)) return false;
            parity ^= 1u << j;
        }
        if constexpr (INNER) {
            if (flags & 16) s_tile_inner<TI, KP, true>(S, wsm + (size_t)j * cfg.sbytes, cfg, d, acc);
            else if (flags & 1) s_tile_inner<TI, KP, false>(S, wsm + (size_t)j * cfg.sbytes, cfg, d, acc);
            else s_long_inner<TI, KP>(S, d, acc, ps);
        } else {
            s_tile_outer<KP>(S, d, acc, ps);
        }
        __syncwarp();
        ++m;
        if (flags & 4) break;   // the unit's last tile
        if (lane == 0) issue((m + NS - 1) % NS);
        __syncwarp();
    }
    const int k = S.k;
#pragma unroll
    for (int i = 0; i < KP; ++i)
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                acc[i][jj] += __shfl_xor_sync(0xffffffffu, acc[i][jj], off);
    if (lane == 0) {
        double *dst = a.partS + (size_t)unit * 2 * GBS_KMAX;
#pragma unroll
        for (int i = 0; i < KP; ++i) {
            if (i >= k) break;
            dst[2 * i] = (double)acc[i][0];
            dst[2 * i + 1] = NJ > 1 ? (double)acc[i][1] : 0.0;
        }
    }
    const int u0 = __ldg(a.scum + ai), nu = __ldg(a.scum + ai + 1) - u0;
    T tot[GBS_KMAX][2];
    if (reduce_last<T, NJ>(a.partS, a.cpartS, a.cntS, a.sysS + ai, unit, u0, nu, __ldg(a.ccs + ai), k,
                           tot)) {
        if constexpr (INNER) s_finish_inner<TI>(a, slot, mine(tot, 0));
        else s_finish_outer(a, slot, mine(tot, 0), mine(tot, 1));
    }
    return true;
}

// Active index of the system holding unit u: the last i with cum[i] <= u
// (cum: non-decreasing prefix sums of the active systems' units, n + 1
// entries), searched from i0 on; a warp's units only grow, so it keeps its
// last index.  One probe when u is still in system i0, else a binary search
// (late in a long launch most systems have finished and are passed over).
__device__ __forceinline__ int find_sys(const int *cum, int i0, int n, int u)
{
    if (__ldg(cum + i0 + 1) > u) return i0;
    int lo = i0 + 1, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(cum + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// A unit is `tg` consecutive warp tiles of one system.  Lane 0 of each warp
// claims the next unit of [gb, ge) from the counter *next (shared by the
// whole grid, so the work balances across SMs), keeps the next tile
// and its descriptor one step ahead, and copies the CSR slice of each INNER
// tile into the next free stage of the warp's ring (cfg.stages stages,
// cfg.stages - 1 in flight).  OUTER tiles (FP64, once per refinement step)
// and single rows longer than GBS_WT_NNZ are read directly.  After a unit's
// last tile the warp stores the unit's partials and takes part in the
// system's reduction.  Returns false if a copy did not complete within the
// time limit (the copies in flight are then waited for, again with a limit).
template <typename TI>
__device__ bool phase_s(const BArgs &a, int cur, int gb, int ge, int *next, unsigned char *wsm,
                        BWarpQ &q, uint32_t &parity, uint64_t ps)
{
    constexpr int E = 16 / (int)sizeof(TI);
    const int lane = threadIdx.x & 31;
    const GbsPipeCfg cfg = a.cfg;
    const int NS = cfg.stages;
    // lane 0: the pending tile (next to issue) with its descriptor
    int p_unit = -1, p_ai = 0, p_slot = 0, p_lt = 0, p_le = 0, p_mode = 0, p_first = 0;
    int2 d_lo = make_int2(0, 0), d_hi = make_int2(0, 0);
    int cai = 0;
    if (lane == 0 && gb < ge) {
        int lo = 0, hi = a.nact - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.scum + mid) <= gb) lo = mid;
            else hi = mid - 1;
        }
        cai = lo;
    }
    auto load_desc = [&]() {
        const int2 *td = reinterpret_cast<const int2 *>(a.sys[p_slot].tdesc);
        d_lo = __ldg(td + p_lt);
        d_hi = __ldg(td + p_lt + 1);
    };
    auto claim = [&]() {
        for (;;) {
            const int u = gb + atomicAdd(next, 1);
            if (u >= ge) {
                p_unit = -1;
                return;
            }
            cai = find_sys(a.scum, cai, a.nact, u);
            const int slot = __ldg(a.act + cai);
            const BSysDyn &D = a.dyn[slot];
            if (D.finished) {   // skip the rest of a finished system
                atomicMax(next, __ldg(a.scum + cai + 1) - gb);
                continue;
            }
            const BSys &S = a.sys[slot];
            p_unit = u;
            p_ai = cai;
            p_slot = slot;
            p_mode = D.mode[cur];
            p_lt = (u - __ldg(a.scum + cai)) * S.tg;
            p_le = min(p_lt + S.tg, S.ntiles);
            p_first = 1;
            load_desc();
            return;
        }
    };
    auto issue = [&](int j) {
        if (p_unit < 0) {
            q.unit[j] = -1;
            return;
        }
        const int r0 = d_lo.x, k0 = d_lo.y, r1 = d_hi.x, k1 = d_hi.y;
        const int staged = p_mode == MODE_INNER && k1 - k0 <= GBS_WT_NNZ;
        const BSys &S = a.sys[p_slot];
        const int16_t *rel = S.colrel16;
        const int rel16 = staged && rel != nullptr;
        q.unit[j] = p_unit;
        q.ai[j] = p_ai;
        q.desc[j] = make_int4(r0, k0, r1, k1);
        q.flags[j] = staged | (p_first << 1) | ((p_lt + 1 == p_le) << 2) |
                     ((p_mode == MODE_INNER) << 3) | (rel16 << 4);
        const TI *vals = bvals<TI>(S);
        const int32_t *colidx = S.colidx, *rowptr = S.rowptr;
        // the next tile: of this unit, or of the next claimed one
        if (p_lt + 1 < p_le) {
            ++p_lt;
            p_first = 0;
            load_desc();
        } else {
            claim();
        }
        if (!staged) return;
        const int vb = k0 & ~(E - 1), ve = (k1 + E - 1) & ~(E - 1);
        const int CE = rel16 ? 8 : 4;   // column indices per 16 bytes
        const int cb = k0 & ~(CE - 1), ce = (k1 + CE - 1) & ~(CE - 1);
        const int rb = r0 & ~3, re = (r1 + 4) & ~3;
        const uint32_t bv = (uint32_t)(sizeof(TI) * (ve - vb)),
                       bc = (uint32_t)((rel16 ? 2 : 4) * (ce - cb)), br = 4u * (uint32_t)(re - rb);
        unsigned char *st = wsm + (size_t)j * cfg.sbytes;
        gbs_mbar_expect_tx(&q.bar[j], bv + bc + br);
        gbs_bulk_g2s(st + cfg.rpoff, rowptr + rb, br, &q.bar[j], ps);
        if (bv) gbs_bulk_g2s(st, vals + vb, bv, &q.bar[j], ps);
        if (bc) {
            if (rel16) gbs_bulk_g2s(st + cfg.coloff, rel + cb, bc, &q.bar[j], ps);
            else gbs_bulk_g2s(st + cfg.coloff, colidx + cb, bc, &q.bar[j], ps);
        }
    };
    if (lane == 0) {
        claim();
        for (int j = 0; j < NS - 1; ++j) issue(j);
    }
    __syncwarp();
    bool ok = true;
    int m = 0;
    for (;;) {
        const int j = m % NS;
        if (lane == 0) issue((m + NS - 1) % NS);   // that stage was consumed at m - 1
        __syncwarp();
        if (q.unit[j] < 0) break;   // claims are monotonic: no later stage holds a tile either
        const int kp = a.sys[__ldg(a.act + q.ai[j])].kp;
        if (q.flags[j] & 8) {
            switch (kp) {
            case 1: ok = s_unit<TI, 1, true>(a, q, wsm, cfg, m, parity, ps, issue); break;
            case 2: ok = s_unit<TI, 2, true>(a, q, wsm, cfg, m, parity, ps, issue); break;
            case 4: ok = s_unit<TI, 4, true>(a, q, wsm, cfg, m, parity, ps, issue); break;
            default: ok = s_unit<TI, 8, true>(a, q, wsm, cfg, m, parity, ps, issue); break;
            }
        } else {
            switch (kp) {
            case 1: ok = s_unit<TI, 1, false>(a, q, wsm, cfg, m, parity, ps, issue); break;
            case 2: ok = s_unit<TI, 2, false>(a, q, wsm, cfg, m, parity, ps, issue); break;
            case 4: ok = s_unit<TI, 4, false>(a, q, wsm, cfg, m, parity, ps, issue); break;
            default: ok = s_unit<TI, 8, false>(a, q, wsm, cfg, m, parity, ps, issue); break;
            }
        }
        if (!ok) break;
    }
    if (!ok) {
        // wait (with a limit) for every copy still in flight, oldest first
        for (int dd = 0; dd < NS; ++dd) {
            const int jj = (m + dd) % NS;
            if (q.unit[jj] >= 0 && (q.flags[jj] & 1) &&
                gbs_mbar_wait(&q.bar[jj], (parity >> jj) & 1u, a.timeout_ns))
                parity ^= 1u << jj;
        }
    }
    __syncwarp();
    return ok;
}

// ---------------------------------------------------------------------
// U and P phases: flat passes over the interleaved vectors
// ---------------------------------------------------------------------

// A U/P unit is `usub` sub-blocks of GBS_SUB consecutive entries of the
// n x kp vectors; lane l handles entries l, l + 32, ... of each sub-block,
// all of one column c = l mod kp.

// U: x += alpha p, r -= alpha q, z = D^-1 r (INNER) or the start of an
// inner solve on r / ||r|| (OUTER); partials r.z and r.r per column.
// A lane takes its entries four at a time (offsets 0, 32, 64, 96 from
// the first); the row of the entry at offset 32 jj has its D^-1 at
// offset 32 jj / kp.
template <typename TI>
__device__ __forceinline__ void u_unit(const BArgs &a, int cur, int nxt, int slot, int ai, int u)
{
    const BSys &S = a.sys[slot];
    const BPh &P = a.ph[slot];
    const int KP = S.kp, lk = __ffs(KP) - 1, R = 32 >> lk;
    const int lane = threadIdx.x & 31, c = lane & (KP - 1), k = S.k;
    const int u0 = __ldg(a.ucum + ai);
    const int64_t nk = (int64_t)S.n * KP;
    const int64_t base = (int64_t)(u - u0) * S.usub * GBS_SUB + lane;
    const int mode = a.dyn[slot].mode[cur];
    TI s0 = TI(0), s1 = TI(0);
    if (mode == MODE_OUTER) {
        if (c < k && ((P.run >> c) & 1u)) {
            const double sc = P.scale[c];
            for (int sb = 0; sb < 2 * S.usub; ++sb) {
                const int64_t e0 = base + (int64_t)sb * (GBS_SUB / 2);
                const int64_t rem = nk - e0;
                if (rem <= 0) break;
                const double *rp = S.r64 + e0;
                const TI *dp = bdinv<TI>(S) + (e0 >> lk);
                TI *xp = static_cast<TI *>(S.xi) + e0, *r_ = static_cast<TI *>(S.ri) + e0,
                   *pp = static_cast<TI *>(S.pi) + e0;
                double rv[4];
                TI dg[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (32 * jj < rem) {
                        rv[jj] = rp[32 * jj];
                        dg[jj] = dp[R * jj];
                    }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (32 * jj < rem) {
                        const TI bi = (TI)(rv[jj] * sc);
                        const TI zi = rmul(dg[jj], bi);
                        xp[32 * jj] = TI(0);
                        r_[32 * jj] = bi;
                        pp[32 * jj] = zi;
                        s0 += bi * zi;
                        s1 += bi * bi;
                    }
            }
        }
    } else {
        if (c < k && ((P.upd >> c) & 1u)) {
            const TI al = ph_alpha(P, c, TI(0));
            for (int sb = 0; sb < 2 * S.usub; ++sb) {
                const int64_t e0 = base + (int64_t)sb * (GBS_SUB / 2);
                const int64_t rem = nk - e0;
                if (rem <= 0) break;
                const TI *dp = bdinv<TI>(S) + (e0 >> lk);
                TI *xp = static_cast<TI *>(S.xi) + e0, *r_ = static_cast<TI *>(S.ri) + e0;
                const TI *pp = static_cast<const TI *>(S.pi) + e0, *qp = static_cast<const TI *>(S.qi) + e0;
                TI xv[4], pv[4], rv[4], qv[4], dg[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (32 * jj < rem) {
                        xv[jj] = xp[32 * jj];
                        pv[jj] = pp[32 * jj];
                        rv[jj] = r_[32 * jj];
                        qv[jj] = qp[32 * jj];
                        dg[jj] = dp[R * jj];
                    }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (32 * jj < rem) {
                        xp[32 * jj] = xv[jj] + al * pv[jj];
                        const TI rn = rv[jj] - al * qv[jj];
                        const TI zn = rmul(dg[jj], rn);
                        r_[32 * jj] = rn;
                        s0 += rn * zn;
                        s1 += rn * rn;
                    }
            }
        }
    }
    // fixed tree over the lanes of one column; lane c then holds column c
    for (int off = 16; off >= KP; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    // lane 0 gathers the column sums and stores the unit's record
    for (int cc = 0; cc < KP; ++cc) {
        const TI v0 = __shfl_sync(0xffffffffu, s0, cc), v1 = __shfl_sync(0xffffffffu, s1, cc);
        if (lane == 0 && cc < k) {
            double *dst = a.partU + (size_t)u * 2 * GBS_KMAX;
            dst[2 * cc] = (double)v0;
            dst[2 * cc + 1] = (double)v1;
        }
    }
    TI tot[GBS_KMAX][2];
    if (reduce_last<TI, 2>(a.partU, a.cpartU, a.cntU, a.sysU + ai, u, u0, __ldg(a.ucum + ai + 1) - u0,
                           __ldg(a.ccu + ai), k, tot)) {
        const TI t0 = mine(tot, 0), t1 = mine(tot, 1);
        if (mode == MODE_OUTER) u_finish_outer<TI>(a, slot, nxt, t0, t1);
        else u_finish_inner<TI>(a, slot, nxt, t0, t1);
    }
}

// P: p = D^-1 r + beta p, or x += ||r|| d once the inner solve has stopped.
template <typename TI>
__device__ __forceinline__ void p_unit(const BArgs &a, int nxt, int slot, int ai, int u)
{
    const BSys &S = a.sys[slot];
    const BPh &P = a.ph[slot];
    const int KP = S.kp, lk = __ffs(KP) - 1, R = 32 >> lk;
    const int lane = threadIdx.x & 31, c = lane & (KP - 1), k = S.k;
    const int64_t nk = (int64_t)S.n * KP;
    const int64_t base = (int64_t)(u - __ldg(a.ucum + ai)) * S.usub * GBS_SUB + lane;
    if (a.dyn[slot].mode[nxt] == MODE_OUTER) {
        if (!(c < k && ((P.run >> c) & 1u))) return;
        const double rn = P.rn[c];
        for (int sb = 0; sb < 2 * S.usub; ++sb) {
            const int64_t e0 = base + (int64_t)sb * (GBS_SUB / 2);
            const int64_t rem = nk - e0;
            if (rem <= 0) break;
            const TI *dp_ = static_cast<const TI *>(S.xi) + e0;
            double *xp = S.x + e0;
            TI dv[4];
            double xv[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (32 * jj < rem) {
                    dv[jj] = dp_[32 * jj];
                    xv[jj] = xp[32 * jj];
                }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (32 * jj < rem) xp[32 * jj] = fma(rn, (double)dv[jj], xv[jj]);
        }
    } else {
        if (!(c < k && ((P.upd >> c) & 1u))) return;
        const TI be = ph_beta(P, c, TI(0));
        for (int sb = 0; sb < 2 * S.usub; ++sb) {
            const int64_t e0 = base + (int64_t)sb * (GBS_SUB / 2);
            const int64_t rem = nk - e0;
            if (rem <= 0) break;
            const TI *dp = bdinv<TI>(S) + (e0 >> lk);
            const TI *r_ = static_cast<const TI *>(S.ri) + e0;
            TI *pp = static_cast<TI *>(S.pi) + e0;
            TI rv[4], pv[4], dg[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (32 * jj < rem) {
                    rv[jj] = r_[32 * jj];
                    pv[jj] = pp[32 * jj];
                    dg[jj] = dp[R * jj];
                }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (32 * jj < rem) pp[32 * jj] = fma(be, pv[jj], rmul(dg[jj], rv[jj]));
        }
    }
}

// The warp's units of a U or P pass over [gb, ge), claimed from the grid-wide
// counter *next one unit ahead (the claim's latency overlaps a unit's work).
template <typename TI, bool U>
__device__ __forceinline__ void phase_up(const BArgs &a, int cur, int nxt, int gb, int ge, int *next)
{
    const int lane = threadIdx.x & 31;
    int cai = 0;
    int pend = 0;
    if (lane == 0) pend = gb + atomicAdd(next, 1);
    for (;;) {
        const int u = __shfl_sync(0xffffffffu, pend, 0);
        if (u >= ge) break;
        if (lane == 0) pend = gb + atomicAdd(next, 1);
        cai = find_sys(a.ucum, cai, a.nact, u);
        const int slot = __ldg(a.act + cai);
        const BSysDyn &D = a.dyn[slot];
        // nothing to do for a finished system, nor in P after an OUTER step
        if (D.finished || (!U && D.mode[cur] != MODE_INNER)) {
            if (lane == 0) atomicMax(next, __ldg(a.ucum + cai + 1) - gb);
            continue;
        }
        if (U) u_unit<TI>(a, cur, nxt, slot, cai, u);
        else p_unit<TI>(a, nxt, slot, cai, u);
    }
}

// One quantum of lockstep global iterations over the active systems:
// S (SpMV, p.q or the refinement residual), U (vector updates, r.z, r.r),
// P (direction update or solution update), a grid barrier after each.
// The warp completing a system's reduction in S or U computes the
// system's scalars for the next phase, so the barriers are the only
// global synchronisation.  Warps claim the units of each phase from
// grid-wide counters (one per phase and global iteration, zeroed before
// the launch), so SMs share the work evenly whatever the units cost.
template <typename TI, int NT>
__global__ void __launch_bounds__(NT, 1) k_batched(BArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ BWarpQ s_q[NT / 32];
    __shared__ int s_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wsm = smem + (size_t)warp * a.ring;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < GBS_MAX_STAGES; ++j) gbs_mbar_init(&s_q[warp].bar[j], 1);
        gbs_fence_mbar_init();
    }
    __syncthreads();
    const uint64_t ps = gbs_policy_stream();
    uint32_t parity = 0;
    int bno = 0;
    // The launch ends after `quantum` global iterations, or earlier once
    // every active system has finished.  Systems finish only in the S and U
    // phases (their scalar steps), so the count of finished systems read
    // between the U and P barriers is the same in every CTA, and all CTAs
    // leave after the same P barrier.  The claim counters rotate over 4
    // sets: the set of iteration q + 2 is zeroed in iteration q, two
    // barriers after its last use (all 4 are zeroed before the launch).
    __shared__ int s_done;
    for (int q = 0; q < a.quantum; ++q) {
        const int cur = (a.iter0 + q) & 1, nxt = cur ^ 1;
        int *ctr = a.claim + 3 * (q & 3);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            int *z = a.claim + 3 * ((q + 2) & 3);
            z[0] = z[1] = z[2] = 0;
        }
        if (!phase_s<TI>(a, cur, 0, a.nsu, ctr, wsm, s_q[warp], parity, ps) && lane == 0)
            atomicCAS(&a.bar->error, 0, GBS_ERR_TIMEOUT);
        if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) break;
        phase_up<TI, true>(a, cur, nxt, 0, a.nuu, ctr + 1);
        if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) break;
        if (threadIdx.x == 0) s_done = gbs_ld_relaxed_int(a.nfin) >= a.nact;
        phase_up<TI, false>(a, cur, nxt, 0, a.nuu, ctr + 2);
        if (!gbs_grid_sync(a.bar, a.timeout_ns, bno++, false, &s_flag)) break;
        if (s_done) break;
    }
}

// Column-major (c * n + i) <-> interleaved with padded stride kp
// (i * kp + c; padding entries are written as zeros).
__global__ void k_interleave(int64_t n, int k, int kp, const double *src, double *dst, int dir)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * kp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kp, cc = e % kp;
        if (dir == 0) dst[e] = cc < k ? src[cc * n + i] : 0.0;
        else if (cc < k) dst[cc * n + i] = src[e];
    }
}

// Many interleavings in one launch: job j moves n * kp entries (dir 0:
// column-major src -> interleaved dst; dir 1: back, padding dropped);
// off[j] is the first flat index of job j, off[njobs] the total.
struct IlvJob {
    const double *src;
    double *dst;
    int64_t n, off;
    int k, kp;
};

__global__ void k_interleave_many(const IlvJob *jobs, int njobs, int64_t total, int dir)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = njobs - 1;   // the job holding e: last j with off[j] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].off <= e) lo = mid;
            else hi = mid - 1;
        }
        const IlvJob J = jobs[lo];
        const int64_t le = e - J.off, i = le / J.kp, cc = le % J.kp;
        if (dir == 0) J.dst[le] = cc < J.k ? J.src[cc * J.n + i] : 0.0;
        else if (cc < J.k) J.dst[cc * J.n + i] = J.src[le];
    }
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// Global iterations per launch of gbs_ksp_solve_cg_batched.  Long quanta
// keep the launch count low; a single launch to the end was measured
// slower (512 systems: 2.82 against 2.35 s) because the units of finished
// systems are skipped one claim at a time until the host compacts the
// active list, which it does between launches.
constexpr int kBatchQuantum = 384;

// Threads per CTA of the batched kernel (one CTA per SM): 24 warps at 80
// registers in FP32, 20 warps at 96 in FP64.  The S phase is bound by the
// latency of its gathers, so more warps pay although the kernel spills a
// little more; measured on the 512-system C4 batch against 16 warps at 128
// registers: FP32 2.08 -> 1.89 s (20 warps 1.95 s), FP64 2.90 -> 2.85 s
// (24 warps 2.92 s: its spills, 1.3 KB, cost more than the warps gain).
constexpr int kBatchThreads32 = 768, kBatchThreads64 = 640;
inline int batch_threads(bool fp64) { return fp64 ? kBatchThreads64 : kBatchThreads32; }

// Column stride of a system with k right-hand sides: k rounded up to a power of two.
int padded_k(int k) { return k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : 8; }

// Reduction units of a system.  Large systems group more work per unit, so
// the per-unit completion count costs little; the grouping depends on the
// system alone (results do not depend on the batch).
// Units of work of one system: S units of up to 32 warp tiles, U/P units of
// up to 16 sub-blocks, at least 64 units per system where it is that large.
// Each claim of a unit costs a grid-wide atomic and a walk to its system's
// records; with 512 systems x 8 columns, units of at most 8 tiles / 4
// sub-blocks measured S 1090 -> 1000 us, U 931 -> 792 us per iteration.
// The sizes depend on the system alone (its reduction order with them).
int tiles_per_unit(int64_t ntiles) { return (int)std::min<int64_t>(32, std::max<int64_t>(1, ntiles / 64)); }
int subs_per_unit(int64_t nsub) { return (int)std::min<int64_t>(16, std::max<int64_t>(1, nsub / 64)); }

// ----------------------------------------------------------------------
// Host engine: a slot table of systems run by the kernel above.
// ----------------------------------------------------------------------

struct SlotHost {
    bool used = false;
    bool finished = false;
    gbs_mat A = nullptr;
    bool own_A = false;       // the engine created the matrix (serving) and frees it
    int k = 0, kp = 1;
    int li = 0;               // log2 of the lanes per row of its SpMV tiling
    int nsu = 0, nuu = 0;     // S units and U/P units
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
    BPh *d_ph = nullptr;
    BSysDyn *d_dyn = nullptr;
    int *d_idx = nullptr;     // act | scum | ucum | ccs | ccu
    int *d_cnt = nullptr;     // cntS | cntU | sysS | sysU | claim
    size_t cap_cnt = 0;
    double *d_partS = nullptr, *d_partU = nullptr, *d_cpartS = nullptr, *d_cpartU = nullptr;
    size_t cap_partS = 0, cap_partU = 0, cap_cpartS = 0, cap_cpartU = 0;
    gbs_grid_barrier *d_bar = nullptr;
    std::vector<SlotHost> slots;
    std::vector<BSysDyn> h_dyn;
    int64_t iter = 0;
    // graph of one quantum for the current active set
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    std::vector<int> g_act;   // active set the graph was captured for
    bool dirty = true;        // a slot was filled or released since the capture
    size_t cnt_bytes = 0;
    BArgs g_args;
    size_t g_smem = 0;       // dynamic shared memory of the captured launch
    int G = 0;
    // slots added since the last launch: their records (staged on the host
    // in h_sys / h_col / h_dyn) and their right-hand sides and initial
    // guesses go to the device together, before the next launch
    std::vector<BSys> h_sys;
    std::vector<BCol> h_col;
    std::vector<int> pending;
    std::vector<IlvJob> ilv_in;
    IlvJob *d_jobs = nullptr;
    size_t cap_jobs = 0;
};

void engine_free_graph(Engine &E)
{
    if (E.gexec) cudaGraphExecDestroy(E.gexec);
    if (E.graph) cudaGraphDestroy(E.graph);
    E.gexec = nullptr;
    E.graph = nullptr;
    E.g_act.clear();
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
    E.h_sys.assign(nslots, BSys());
    E.h_col.assign((size_t)nslots * GBS_KMAX, BCol());
    const size_t ns = (size_t)std::max(nslots, 1);
    GBS_CUDA_TRY(cudaMalloc(&E.d_sys, sizeof(BSys) * ns));
    GBS_CUDA_TRY(cudaMalloc(&E.d_col, sizeof(BCol) * ns * GBS_KMAX));
    GBS_CUDA_TRY(cudaMalloc(&E.d_ph, sizeof(BPh) * ns));
    GBS_CUDA_TRY(cudaMalloc(&E.d_dyn, sizeof(BSysDyn) * ns));
    GBS_CUDA_TRY(cudaMalloc(&E.d_idx, sizeof(int) * 5 * (ns + 2)));
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
    cudaFree(E.d_ph);
    cudaFree(E.d_dyn);
    cudaFree(E.d_idx);
    cudaFree(E.d_cnt);
    cudaFree(E.d_partS);
    cudaFree(E.d_partU);
    cudaFree(E.d_cpartS);
    cudaFree(E.d_cpartU);
    cudaFree(E.d_bar);
    cudaFree(E.d_jobs);
    E = Engine();
}

// Device bytes a system of n rows, nnz nonzeros and k columns holds.
size_t system_bytes(int64_t n, int64_t nnz, int k, int fp64)
{
    const size_t nk = (size_t)n * padded_k(k), tsz = fp64 ? 8 : 4;
    const size_t vecs = 3 * a256(nk * 8) + 4 * a256(nk * tsz);
    const size_t mat = 4 * (size_t)(n + 5) + 12 * (size_t)(nnz + 4) + (fp64 ? 0 : 4 * (size_t)(nnz + 4)) +
                       12 * (size_t)(n + 4) + 12 * (size_t)(n / 32 + 2) + 4096;
    return vecs + mat;
}

// Algorithmic bytes of the steps a slot's system has taken: an INNER step
// streams the inner-precision values and column indices (16-bit when the
// matrix has the compressed form), rowptr, the p gather and q written (S:
// 2 kp entries per row), x, p, r, q read and x, r written plus D^-1 (U:
// 6 kp + 1), r, p read and p written plus D^-1 (P: 3 kp + 1); an OUTER
// step streams the FP64 values and colidx, rowptr, the x gather, b and r64
// (S), r64 read, D^-1 and x_i, r_i, p_i written (U).  Vector entries count
// kp per row, once per pass that reads or writes them.
double slot_model_bytes(const Engine &E, int slot)
{
    const SlotHost &H = E.slots[slot];
    if (!H.used || !H.A) return 0.0;
    const BSysDyn &D = E.h_dyn[slot];
    const double n = (double)H.A->n, nnz = (double)H.A->nnz, kp = H.kp, tsz = E.fp64 ? 8 : 4;
    const double isz = H.A->colrel16 ? 2 : 4;   // index bytes of INNER tiles
    const double inner = (tsz + isz) * nnz + 4 * (n + 1) + tsz * n * (11 * kp + 2);
    const double outer = 12 * nnz + 4 * (n + 1) + 32 * n * kp + tsz * n * (3 * kp + 1);
    return D.isteps * inner + D.osteps * outer;
}

// Grow a device buffer to hold at least `need` elements (contents dropped).
template <typename T>
int ensure_cap(T *&p, size_t &cap, size_t need)
{
    if (need <= cap && p) return GBS_OK;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t n = need + need / 2 + 64;
    GBS_CUDA_TRY(cudaMalloc(&p, n * sizeof(T)));
    cap = n;
    return GBS_OK;
}

// Put a system into a free slot.  b and x0 are column-major device arrays
// (x0 may be NULL for zeros).  A failing matrix (no usable diagonal, n = 0)
// is admitted as finished with the corresponding column status.
int engine_add(Engine &E, int slot, gbs_mat A, int k, double rtol, int maxit, const double *b,
               const double *x0, bool own_A, uint64_t ticket, int li)
{
    gbs_ctx c = E.c;
    SlotHost &H = E.slots[slot];
    const int kp = padded_k(k);
    {
        const int st = gbs_mat_ensure_lane_tiling(A, li);
        if (st) return st;
    }
    const int64_t ntiles = A->ntiles_lanes[li];
    const size_t nk = (size_t)A->n * kp, tsz = E.fp64 ? 8 : 4;
    {   // FP32 values (mixed) and the 16-bit column offsets of the INNER tiles
        int st = E.fp64 ? gbs_mat_ensure_rel16(A) : gbs_mat_ensure_f32(A);
        if (st) return st;
    }
    const size_t bytes = 3 * a256(nk * 8) + 4 * a256(nk * tsz);
    char *p = nullptr;
    if (bytes) {
        // from the context's pool, in stream order (a slot's vectors come and
        // go with every served request)
        GBS_CUDA_TRY(gbs_mat_alloc(c, (void **)&p, bytes));
        // padding columns and unused entries hold zeros
        GBS_CUDA_TRY(cudaMemsetAsync(p, 0, bytes, c->stream));
    }
    // a reused slot may hold a system of another size: the active lists and
    // the captured launch must be rebuilt before the next quantum
    E.dirty = true;
    const int64_t nsub = ((int64_t)nk + GBS_SUB - 1) / GBS_SUB;
    const int tg = tiles_per_unit(ntiles), usub = subs_per_unit(nsub);
    H.used = true;
    H.finished = false;
    H.A = A;
    H.own_A = own_A;
    H.k = k;
    H.kp = kp;
    H.li = li;
    H.nsu = (int)((ntiles + tg - 1) / tg);
    H.nuu = (int)((nsub + usub - 1) / usub);
    H.work = p;
    H.bytes = bytes;
    H.ticket = ticket;
    BSys S;
    memset(&S, 0, sizeof(S));
    S.rowptr = A->rowptr;
    S.colidx = A->colidx;
    S.tdesc = A->tdesc_lanes[li];
    S.colrel16 = A->colrel16;
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
        S.pi = p; p += a256(nk * tsz);
        S.qi = p; p += a256(nk * tsz);
    }
    S.n = (int)A->n;
    S.k = k;
    S.kp = kp;
    S.ntiles = (int)ntiles;
    S.lanes_log = li;
    S.tg = tg;
    S.usub = usub;
    S.rtol = rtol;
    S.maxit = maxit;
    if (nk) {   // interleaved at the next flush, with every other added slot's
        E.ilv_in.push_back(IlvJob{b, (double *)S.b, A->n, 0, k, kp});
        if (x0) E.ilv_in.push_back(IlvJob{x0, S.x, A->n, 0, k, kp});
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
    E.h_sys[slot] = S;
    memcpy(&E.h_col[(size_t)slot * GBS_KMAX], C, sizeof(C));
    E.pending.push_back(slot);
    return GBS_OK;
}

// Send the records of the slots added since the last flush to the device
// (one copy per run of consecutive slots) and interleave all their
// right-hand sides and initial guesses in one launch.
int engine_flush(Engine &E)
{
    gbs_ctx c = E.c;
    if (!E.pending.empty()) {
        std::vector<int> ps = E.pending;
        std::sort(ps.begin(), ps.end());
        for (size_t i = 0; i < ps.size();) {
            size_t j = i + 1;
            while (j < ps.size() && ps[j] == ps[j - 1] + 1) ++j;
            const int s0 = ps[i], cnt = ps[j - 1] - s0 + 1;
            GBS_CUDA_TRY(cudaMemcpyAsync(E.d_sys + s0, &E.h_sys[s0], sizeof(BSys) * cnt,
                                         cudaMemcpyHostToDevice, c->stream));
            GBS_CUDA_TRY(cudaMemcpyAsync(E.d_col + (size_t)s0 * GBS_KMAX,
                                         &E.h_col[(size_t)s0 * GBS_KMAX],
                                         sizeof(BCol) * GBS_KMAX * cnt, cudaMemcpyHostToDevice,
                                         c->stream));
            GBS_CUDA_TRY(cudaMemsetAsync(E.d_ph + s0, 0, sizeof(BPh) * cnt, c->stream));
            GBS_CUDA_TRY(cudaMemcpyAsync(E.d_dyn + s0, &E.h_dyn[s0], sizeof(BSysDyn) * cnt,
                                         cudaMemcpyHostToDevice, c->stream));
            i = j;
        }
        E.pending.clear();
    }
    if (!E.ilv_in.empty()) {
        int64_t tot = 0;
        for (IlvJob &J : E.ilv_in) {
            J.off = tot;
            tot += J.n * J.kp;
        }
        int st = ensure_cap(E.d_jobs, E.cap_jobs, E.ilv_in.size());
        if (st) return st;
        GBS_CUDA_TRY(cudaMemcpyAsync(E.d_jobs, E.ilv_in.data(), sizeof(IlvJob) * E.ilv_in.size(),
                                     cudaMemcpyHostToDevice, c->stream));
        const int g = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 8);
        k_interleave_many<<<g, 256, 0, c->stream>>>(E.d_jobs, (int)E.ilv_in.size(), tot, 0);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
        // the job list is host memory the next flush rewrites
        GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        E.ilv_in.clear();
    }
    return GBS_OK;
}

// Copy a slot's results out (x column-major into x_out, device or host per
// memspace).
int engine_collect(Engine &E, int slot, double *x_out, int memspace, int *iters, double *rnorm,
                   int *status)
{
    gbs_ctx c = E.c;
    {
        const int st = engine_flush(E);
        if (st) return st;
    }
    SlotHost &H = E.slots[slot];
    BCol C[GBS_KMAX];
    GBS_CUDA_TRY(cudaMemcpyAsync(C, E.d_col + (size_t)slot * GBS_KMAX, sizeof(C),
                                 cudaMemcpyDeviceToHost, c->stream));
    const int64_t n = H.A->n;
    const int kp = H.kp;
    const size_t nk = (size_t)n * kp;
    if (nk && x_out) {
        const double *xil = (const double *)(H.work + a256(nk * 8));
        const int g = (int)std::min<int64_t>((int64_t)(nk + 255) / 256, (int64_t)c->num_sms * 8);
        if (memspace == GBS_MEM_DEVICE) {
            k_interleave<<<g, 256, 0, c->stream>>>(n, H.k, kp, xil, x_out, 1);
            gbs_count_launch(c);
            GBS_CUDA_TRY(cudaGetLastError());
        } else {
            // column-major on the device first (a pooled temporary), then
            // one copy to the host
            const size_t nkk = (size_t)n * H.k;
            double *tmp = nullptr;
            GBS_CUDA_TRY(gbs_mat_alloc(c, (void **)&tmp, nkk * 8));
            k_interleave<<<g, 256, 0, c->stream>>>(n, H.k, kp, xil, tmp, 1);
            gbs_count_launch(c);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(x_out, tmp, nkk * 8, cudaMemcpyDeviceToHost, c->stream);
            gbs_mat_release(c, tmp);
            if (e != cudaSuccess) return gbs_cuda_fail(e);
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

// Results of slots 0 .. ns-1 at once: every x (column-major, device
// arrays x_out[s]) in one launch, every column record in one copy.  Column
// j of slot s goes to position off[s] + j of iters / rnorm / status.
int engine_collect_all(Engine &E, int ns, double *const *x_out, const int64_t *off, int *iters,
                       double *rnorm, int *status)
{
    gbs_ctx c = E.c;
    int st = engine_flush(E);
    if (st) return st;
    std::vector<BCol> C((size_t)ns * GBS_KMAX);
    if (ns) GBS_CUDA_TRY(cudaMemcpyAsync(C.data(), E.d_col, sizeof(BCol) * C.size(),
                                         cudaMemcpyDeviceToHost, c->stream));
    std::vector<IlvJob> jobs;
    int64_t tot = 0;
    for (int s = 0; s < ns; ++s) {
        const SlotHost &H = E.slots[s];
        const int64_t nk = H.A->n * H.kp;
        if (!nk || !x_out[s]) continue;
        jobs.push_back(IlvJob{(const double *)(H.work + a256((size_t)nk * 8)), x_out[s], H.A->n, tot,
                              H.k, H.kp});
        tot += nk;
    }
    if (!jobs.empty()) {
        st = ensure_cap(E.d_jobs, E.cap_jobs, jobs.size());
        if (st) return st;
        GBS_CUDA_TRY(cudaMemcpyAsync(E.d_jobs, jobs.data(), sizeof(IlvJob) * jobs.size(),
                                     cudaMemcpyHostToDevice, c->stream));
        const int g = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 8);
        k_interleave_many<<<g, 256, 0, c->stream>>>(E.d_jobs, (int)jobs.size(), tot, 1);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < ns; ++s) {
        const SlotHost &H = E.slots[s];
        for (int cc = 0; cc < H.k; ++cc) {
            const BCol &B = C[(size_t)s * GBS_KMAX + cc];
            const int cs = B.status == GBS_RUNNING ? GBS_DIVERGED_ITS : B.status;
            if (iters) iters[off[s] + cc] = B.iters;
            if (rnorm) rnorm[off[s] + cc] = B.rn;
            if (status) status[off[s] + cc] = cs;
        }
    }
    return GBS_OK;
}

void engine_release(Engine &E, int slot)
{
    E.dirty = true;
    SlotHost &H = E.slots[slot];
    gbs_mat_release(E.c, H.work);
    if (H.own_A) gbs_mat_destroy(H.A);
    H = SlotHost();
}

// Stage geometry covering the tiles of every active system.
GbsPipeCfg engine_pipe_cfg(const Engine &E, const std::vector<int> &act)
{
    int v = 16, cl = 16, r = 16;
    for (int s : act) {
        const SlotHost &H = E.slots[s];
        // tiles may carry 16-bit or 32-bit indices: cover both geometries
        for (int w = 0; w < 2; ++w) {
            const GbsPipeCfg &p = E.fp64 ? (w == 0 ? H.A->pipe64_lanes[H.li] : H.A->pipe64r_lanes[H.li])
                                 : w == 0 ? H.A->pipe32_lanes[H.li] : H.A->pipe16_lanes[H.li];
            v = std::max(v, p.coloff);
            cl = std::max(cl, p.rpoff - p.coloff);
            r = std::max(r, p.sbytes - p.rpoff);
        }
    }
    GbsPipeCfg cfg;
    cfg.coloff = v;
    cfg.rpoff = v + cl;
    cfg.sbytes = v + cl + r;
    // two stages: the S phase is bound by the latency of its gathers, not of
    // its copies (4 and 8 stages measured 1.5 % and 6 % slower than 2), and
    // the smaller rings leave more of the SM's memory to L1
    cfg.stages = std::min(2, std::max(1, GBS_BWARP_BYTES / cfg.sbytes));
    return cfg;
}

// Run one quantum over the active slots; refresh the finished flags.
int engine_step(Engine &E, int *ran)
{
    gbs_ctx c = E.c;
    *ran = 0;
    {
        const int st = engine_flush(E);
        if (st) return st;
    }
    std::vector<int> act;
    for (int s = 0; s < E.nslots; ++s) {
        const SlotHost &H = E.slots[s];
        if (H.used && !H.finished && H.nsu > 0) act.push_back(s);
    }
    if (act.empty()) return GBS_OK;
    const int nact = (int)act.size();
    const int nt = batch_threads(E.fp64);
    const void *fn = E.fp64 ? (const void *)k_batched<double, kBatchThreads64>
                            : (const void *)k_batched<float, kBatchThreads32>;
    if (E.dirty || act != E.g_act) {
        engine_free_graph(E);
        E.dirty = false;
        // act | scum | ucum | ccs | ccu
        std::vector<int> idx(5 * (size_t)(nact + 1), 0);
        int *h_act = idx.data(), *scum = h_act + (nact + 1), *ucum = scum + (nact + 1),
            *ccs = ucum + (nact + 1), *ccu = ccs + (nact + 1);
        for (int i = 0; i < nact; ++i) {
            const SlotHost &H = E.slots[act[i]];
            h_act[i] = act[i];
            scum[i + 1] = scum[i] + H.nsu;
            ucum[i + 1] = ucum[i] + H.nuu;
            ccs[i + 1] = ccs[i] + (H.nsu + GBS_RCHUNK - 1) / GBS_RCHUNK;
            ccu[i + 1] = ccu[i] + (H.nuu + GBS_RCHUNK - 1) / GBS_RCHUNK;
        }
        const int nsu = scum[nact], nuu = ucum[nact], nchs = ccs[nact], nchu = ccu[nact];
        int st = ensure_cap(E.d_partS, E.cap_partS, (size_t)nsu * 2 * GBS_KMAX);
        if (!st) st = ensure_cap(E.d_partU, E.cap_partU, (size_t)nuu * 2 * GBS_KMAX);
        if (!st) st = ensure_cap(E.d_cpartS, E.cap_cpartS, (size_t)nchs * 2 * GBS_KMAX);
        if (!st) st = ensure_cap(E.d_cpartU, E.cap_cpartU, (size_t)nchu * 2 * GBS_KMAX);
        const size_t nclaim = 12;
        const size_t ncnt = (size_t)nchs + nchu + 2 * (size_t)nact + nclaim + 1;
        if (!st) st = ensure_cap(E.d_cnt, E.cap_cnt, ncnt);
        if (st) return st;
        E.cnt_bytes = ncnt * sizeof(int);
        GBS_CUDA_TRY(cudaMemcpyAsync(E.d_idx, idx.data(), sizeof(int) * idx.size(),
                                     cudaMemcpyHostToDevice, c->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));   // idx is a stack vector
        // the rings take only the stages the active tiles need; the rest of
        // the SM's on-chip memory stays L1, where the SpMV's gathers of p
        // (each entry read by every row that couples to it) find it
        const GbsPipeCfg cfg = engine_pipe_cfg(E, act);
        const int ring = (cfg.stages * cfg.sbytes + 127) & ~127;
        const size_t smem = (size_t)ring * (nt / 32);
        E.g_smem = smem;
        GBS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GBS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxL1));
        int per_sm = 0;
        GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
        if (per_sm < 1) return GBS_ERR_CUDA;
        // at most one CTA per warp-count units of the larger pass
        const int64_t need = ((int64_t)std::max(nsu, nuu) + nt / 32 - 1) / (nt / 32);
        E.G = (int)std::min<int64_t>((int64_t)per_sm * c->num_sms, std::max<int64_t>(need, 1));
        BArgs &a = E.g_args;
        memset(&a, 0, sizeof(a));
        a.sys = E.d_sys;
        a.col = E.d_col;
        a.ph = E.d_ph;
        a.dyn = E.d_dyn;
        a.act = E.d_idx;
        a.scum = E.d_idx + (nact + 1);
        a.ucum = E.d_idx + 2 * (nact + 1);
        a.ccs = E.d_idx + 3 * (nact + 1);
        a.ccu = E.d_idx + 4 * (nact + 1);
        a.nact = nact;
        a.nsu = nsu;
        a.nuu = nuu;
        a.partS = E.d_partS;
        a.partU = E.d_partU;
        a.cpartS = E.d_cpartS;
        a.cpartU = E.d_cpartU;
        a.cntS = E.d_cnt;
        a.cntU = E.d_cnt + nchs;
        a.sysS = E.d_cnt + nchs + nchu;
        a.sysU = E.d_cnt + nchs + nchu + nact;
        a.claim = E.d_cnt + nchs + nchu + 2 * nact;
        a.nfin = a.claim + nclaim;
        a.bar = E.d_bar;
        a.cfg = cfg;
        a.ring = ring;
        a.quantum = E.quantum;   // even: the parity of the global iteration is unchanged
        a.iter0 = 0;
        a.inner_rtol = E.inner_rtol;
        a.outer_maxit = E.outer_maxit;
        a.fp64 = E.fp64;
        a.timeout_ns = (unsigned long long)c->opts.barrier_timeout_ms * 1000000ull;
        // capture the counter and barrier reset and the cooperative launch
        // once for this active set
        cudaStream_t cap = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(E.d_cnt, 0, E.cnt_bytes, cap);
            cudaMemsetAsync(E.d_bar, 0, 256, cap);
            void *args[] = {&E.g_args};
            cudaLaunchCooperativeKernel(fn, dim3((unsigned)E.G), dim3((unsigned)nt), args, E.g_smem, cap);
            e = cudaStreamEndCapture(cap, &E.graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&E.gexec, E.graph, 0);
        if (cap) cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            engine_free_graph(E);   // launch directly below
        } else {
            E.g_act = act;
        }
    }
    if (E.gexec) {
        GBS_CUDA_TRY(cudaGraphLaunch(E.gexec, c->stream));
    } else {
        GBS_CUDA_TRY(cudaMemsetAsync(E.d_cnt, 0, E.cnt_bytes, c->stream));
        GBS_CUDA_TRY(cudaMemsetAsync(E.d_bar, 0, 256, c->stream));
        void *args[] = {&E.g_args};
        GBS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3((unsigned)E.G), dim3((unsigned)nt), args,
                                                 E.g_smem, c->stream));
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


// ----------------------------------------------------------------------
// Lanes-per-row autotuner
// ----------------------------------------------------------------------

__global__ void k_fill(int64_t n, double v, double *x)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

int ilog2(int64_t v)
{
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}

// Time one quantum of 16 global iterations of `rep` copies of the system
// (its own matrix, right-hand sides of ones, rtol 0 so nothing stops) with
// the tiling for 2^li lanes per row; the copies emulate a loaded engine.
int time_lanes(gbs_ctx c, gbs_mat A, int k, int fp64, int li, int rep, const double *b, float *ms)
{
    Engine T;
    int st = engine_init(T, c, rep, fp64, 16);
    for (int r = 0; r < rep && st == GBS_OK; ++r)
        st = engine_add(T, r, A, k, 0.0, 1 << 30, b, nullptr, false, 0, li);
    int ran = 0;
    if (st == GBS_OK) st = engine_step(T, &ran);   // capture, first refinement residual
    if (st == GBS_OK) {
        cudaEventRecord(c->ev0, c->stream);
        st = engine_step(T, &ran);
        cudaEventRecord(c->ev1, c->stream);
        cudaEventSynchronize(c->ev1);
        cudaEventElapsedTime(ms, c->ev0, c->ev1);
    }
    engine_destroy(T);
    return st;
}

// Lanes per row (as log2) for a system in a batched engine: the option's
// fixed value, else the context's decision for the system's class (row
// length, column stride, precision), made on first use by timing 1, 2 and
// 4 lanes per row on copies of the system that fill about 4 M rows (a
// loaded engine); more lanes are taken only when at least 10 % faster.
// The decision depends only on the class, so a system gets the same tiling
// alone and in any batch of the same context.
int choose_lanes(gbs_ctx c, gbs_mat A, int k, int fp64, int *li)
{
    *li = 0;
    if (c->opts.batched_lanes > 0) {
        *li = ilog2(c->opts.batched_lanes);
        return GBS_OK;
    }
    if (A->n == 0 || A->ntiles == 0 || !A->diag_ok) return GBS_OK;
    const int kp = padded_k(k);
    const int rb = std::min(7, ilog2(std::max<int64_t>(1, A->nnz / A->n)));
    signed char &slot = c->lane_choice[fp64 ? 1 : 0][ilog2(kp)][rb];
    if (slot > 0) {
        *li = slot - 1;
        return GBS_OK;
    }
    if (!fp64) {
        const int st = gbs_mat_ensure_f32(A);
        if (st) return st;
    }
    const int64_t nk = A->n * (int64_t)k;
    const int rep = (int)std::min<int64_t>(256, std::max<int64_t>(1, 4000000 / A->n));
    double *b = nullptr;
    GBS_CUDA_TRY(cudaMalloc(&b, sizeof(double) * (size_t)nk));
    const int g = (int)std::min<int64_t>((nk + 255) / 256, (int64_t)c->num_sms * 8);
    k_fill<<<g, 256, 0, c->stream>>>(nk, 1.0, b);
    gbs_count_launch(c);
    float t[3] = {INFINITY, INFINITY, INFINITY};
    int st = GBS_OK;
    for (int l = 0; l < 3 && st == GBS_OK; ++l) st = time_lanes(c, A, k, fp64, l, rep, b, &t[l]);
    cudaFree(b);
    if (st) return st;
    int pick = 0;
    for (int l = 1; l < 3; ++l)
        if (t[l] < 0.9f * t[pick]) pick = l;
    slot = (signed char)(pick + 1);
    *li = pick;
    return GBS_OK;
}

}  // namespace

// ----------------------------------------------------------------------
// gbs_batched_tune
// ----------------------------------------------------------------------

extern "C" int gbs_batched_tune(gbs_ctx c, gbs_mat A, int k, int mode, int *lanes)
{
    if (!c || !A || A->ctx != c || k < 1 || k > GBS_KMAX || A->n != A->ncols) return GBS_ERR_ARG;
    if (mode != GBS_MODE_FP64 && mode != GBS_MODE_MIXED) return GBS_ERR_ARG;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    int li = 0;
    const int st = choose_lanes(c, A, k, mode == GBS_MODE_FP64, &li);
    if (st == GBS_OK && lanes) *lanes = 1 << li;
    return st;
}

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
    int rc = engine_init(E, c, nsys, mode == GBS_MODE_FP64, kBatchQuantum);
    for (int s = 0; s < nsys && rc == GBS_OK; ++s) {
        int li = 0;
        rc = choose_lanes(c, A[s], nrhs[s], mode == GBS_MODE_FP64, &li);
        if (rc == GBS_OK)
            rc = engine_add(E, s, A[s], nrhs[s], rtol[s], maxit, (const double *)B[s]->data,
                            (const double *)X[s]->data, false, 0, li);
    }
    // the slots' set-up goes to the device in one flush, then launches of
    // up to kBatchQuantum global iterations each (the last ends as soon as
    // every system has finished); between launches the host drops finished
    // systems from the active list, so their units are not claimed again
    if (rc == GBS_OK) rc = engine_flush(E);
    if (rc == GBS_OK) {
        cudaEventRecord(c->ev0, c->stream);
        for (int ran = 1; rc == GBS_OK && ran;) rc = engine_step(E, &ran);
        cudaEventRecord(c->ev1, c->stream);
    }
    int first_bad = GBS_OK;
    double model = 0.0;
    for (int s = 0; s < nsys; ++s) model += slot_model_bytes(E, s);
    std::vector<int64_t> off(nsys + 1, 0);
    std::vector<double *> xo(nsys);
    for (int s = 0; s < nsys; ++s) {
        off[s + 1] = off[s] + nrhs[s];
        xo[s] = (double *)X[s]->data;
    }
    std::vector<int> stc(off[nsys]);
    if (rc == GBS_OK) rc = engine_collect_all(E, nsys, xo.data(), off.data(), iters, rnorm, stc.data());
    if (rc == GBS_OK) {
        for (int64_t o = 0; o < off[nsys]; ++o) {
            if (status) status[o] = stc[o];
            if (stc[o] != GBS_OK && first_bad == GBS_OK) first_bad = stc[o];
        }
    }
    memset(&c->last, 0, sizeof(c->last));
    c->last.status = rc != GBS_OK ? rc : first_bad;
    if (rc == GBS_OK) {
        cudaStreamSynchronize(c->stream);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->last.device_ms = ms;
        c->last.model_bytes = model;
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
    // the arrays in use: the copies above, or the caller's (borrowed)
    const int32_t *p_rowptr = nullptr, *p_colidx = nullptr;
    const double *p_vals = nullptr, *p_b = nullptr;
    size_t bytes;
    int slot = -1;
    bool done = false;
    double *x = nullptr;   // n x k column-major result, pinned (from the server's cache)
    size_t xn = 0, xcap = 0;
    std::vector<int> iters, status;
    std::vector<double> rnorm;
};

}  // namespace

// Pinned host buffers for the results: retirement copies a request's x
// into one at the link's rate (no page faults, no zero fill), the fetch
// copies it to the caller and returns the buffer here for the next request
// (best fit by capacity).
struct PinnedCache {
    std::multimap<size_t, double *> free_;
    double *take(size_t n, size_t *cap)
    {
        auto it = free_.lower_bound(n);
        if (it != free_.end()) {
            double *p = it->second;
            *cap = it->first;
            free_.erase(it);
            return p;
        }
        double *p = nullptr;
        if (cudaMallocHost((void **)&p, std::max<size_t>(n, 1) * sizeof(double)) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        *cap = std::max<size_t>(n, 1);
        return p;
    }
    void give(double *p, size_t cap)
    {
        if (p) free_.emplace(cap, p);
    }
    ~PinnedCache()
    {
        for (auto &kv : free_) cudaFreeHost(kv.second);
    }
};

struct gbs_server_s {
    gbs_ctx c;
    Engine E;
    PinnedCache pinned;
    size_t budget;
    size_t used = 0;
    int mode;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;                       // waiting for admission, FIFO
    std::unordered_map<uint64_t, Request> reqs;       // queued, running or done
    int running = 0, finished = 0;
    double t_admit = 0.0, t_quanta = 0.0, t_retire = 0.0;   // seconds spent in each step
    int64_t quanta = 0;
};

namespace {

double seconds_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

int server_submit(gbs_server srv, int64_t nrows, const int32_t *rowptr, const int32_t *colidx,
                  const double *vals, int k, const double *b, double rtol, int maxit, bool copy,
                  uint64_t *ticket)
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
    if (copy) {
        r.rowptr.assign(rowptr, rowptr + nrows + 1);
        r.colidx.assign(colidx, colidx + nnz);
        r.vals.assign(vals, vals + nnz);
        r.b.assign(b, b + nrows * k);
        r.p_rowptr = r.rowptr.data();
        r.p_colidx = r.colidx.data();
        r.p_vals = r.vals.data();
        r.p_b = r.b.data();
    } else {
        r.p_rowptr = rowptr;
        r.p_colidx = colidx;
        r.p_vals = vals;
        r.p_b = b;
    }
    r.bytes = bytes;
    *ticket = r.ticket;
    srv->queue.push_back(r.ticket);
    auto it = srv->reqs.emplace(r.ticket, std::move(r)).first;
    if (copy) {   // the vectors moved: point at their new storage
        Request &q = it->second;
        q.p_rowptr = q.rowptr.data();
        q.p_colidx = q.colidx.data();
        q.p_vals = q.vals.data();
        q.p_b = q.b.data();
    }
    return GBS_OK;
}

}  // namespace

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
    for (auto &kv : srv->reqs) srv->pinned.give(kv.second.x, kv.second.xcap);
    delete srv;
    return GBS_OK;
}

extern "C" int gbs_server_submit(gbs_server srv, int64_t nrows, const int32_t *rowptr,
                                 const int32_t *colidx, const double *vals, int k, const double *b,
                                 double rtol, int maxit, uint64_t *ticket)
{
    return server_submit(srv, nrows, rowptr, colidx, vals, k, b, rtol, maxit, true, ticket);
}

extern "C" int gbs_server_submit_borrowed(gbs_server srv, int64_t nrows, const int32_t *rowptr,
                                          const int32_t *colidx, const double *vals, int k,
                                          const double *b, double rtol, int maxit, uint64_t *ticket)
{
    return server_submit(srv, nrows, rowptr, colidx, vals, k, b, rtol, maxit, false, ticket);
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
        int st = gbs_mat_create_aij(srv->c, r.n, r.n, r.p_rowptr, r.p_colidx, r.p_vals,
                                    GBS_MEM_HOST, &A);
        if (st != GBS_OK) {
            // a malformed request finishes at once with that status
            r.done = true;
            r.xn = (size_t)r.n * r.k;
            r.x = srv->pinned.take(r.xn, &r.xcap);
            if (!r.x) return GBS_ERR_OOM;
            memset(r.x, 0, r.xn * sizeof(double));
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
                e = cudaMemcpyAsync(db, r.p_b, nb, cudaMemcpyHostToDevice, srv->c->stream);
            if (e != cudaSuccess) {
                cudaFree(db);
                gbs_mat_destroy(A);
                return gbs_cuda_fail(e);
            }
        }
        int li = 0;
        st = choose_lanes(srv->c, A, r.k, srv->mode == GBS_MODE_FP64, &li);
        if (st == GBS_OK) st = engine_add(E, slot, A, r.k, r.rtol, r.maxit, db, nullptr, true, r.ticket, li);
        // interleave b now: the flush synchronises the stream, so db can go
        if (st == GBS_OK) st = engine_flush(E);
        cudaFree(db);
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
        r.p_colidx = nullptr;
        r.p_vals = nullptr;
        r.p_b = nullptr;
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
        r.xn = (size_t)r.n * r.k;
        r.x = srv->pinned.take(r.xn, &r.xcap);
        if (!r.x) return GBS_ERR_OOM;
        r.iters.assign(r.k, 0);
        r.rnorm.assign(r.k, 0.0);
        r.status.assign(r.k, 0);
        const int st = engine_collect(E, s, r.x, GBS_MEM_HOST, r.iters.data(), r.rnorm.data(),
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
    auto t0 = std::chrono::steady_clock::now();
    int st = server_retire(srv, &n);   // systems that finished at admission
    srv->t_retire += seconds_since(t0);
    t0 = std::chrono::steady_clock::now();
    if (!st) st = server_admit(srv);
    srv->t_admit += seconds_since(t0);
    int ran = 0;
    t0 = std::chrono::steady_clock::now();
    if (!st) st = engine_step(srv->E, &ran);
    srv->t_quanta += seconds_since(t0);
    srv->quanta += ran;
    t0 = std::chrono::steady_clock::now();
    if (!st) st = server_retire(srv, &n);
    srv->t_retire += seconds_since(t0);
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
    if (x && r.xn) memcpy(x, r.x, r.xn * sizeof(double));
    for (int cc = 0; cc < r.k; ++cc) {
        if (iters) iters[cc] = r.iters[cc];
        if (rnorm) rnorm[cc] = r.rnorm[cc];
        if (status) status[cc] = r.status[cc];
    }
    srv->pinned.give(r.x, r.xcap);
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

extern "C" int gbs_server_times(gbs_server srv, double *admit_s, double *quanta_s, double *retire_s,
                                int64_t *quanta)
{
    if (!srv) return GBS_ERR_ARG;
    if (admit_s) *admit_s = srv->t_admit;
    if (quanta_s) *quanta_s = srv->t_quanta;
    if (retire_s) *retire_s = srv->t_retire;
    if (quanta) *quanta = srv->quanta;
    return GBS_OK;
}
