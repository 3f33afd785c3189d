// Jacobi-preconditioned CG solves (KSPCG + PCJACOBI, Sec. 5.5 / 5.3 of the
// paper) on one GPU.
//
// Persistent path: one cooperative kernel runs the whole solve.  Each CTA
// owns a contiguous range of warp tiles (rows); per iteration it
//   S: forms q = A p on its rows with the p.q partial fused in the SpMV
//      epilogue                                          -> grid barrier
//   U: alpha = rho / p.q; x += alpha p; r -= alpha q; z = D^-1 r, with the
//      r.z and r.r partials fused                         -> grid barrier
//   P: beta = rho'/rho; p = z + beta p                    -> grid barrier
// and tests convergence on the device (||r||_2 <= rtol ||b||_2 before each
// iteration), so the host is not involved until the end (Challenge A1:
// dot products otherwise force a host synchronisation each iteration).
// Every CTA reduces the per-CTA partials in the same fixed order, so all
// CTAs hold bitwise-identical scalars and take identical decisions.
// Matrix arrays stream through L2 with an evict-first policy; the solver
// vectors use evict-last so that they can stay in L2 across iterations.
//
// Mixed mode (Response A7: single precision on the GPU): the same kernel
// shape with an outer iterative-refinement loop inside it: FP64
// r = b - A x with ||r|| fused, FP32 inner PCG on r/||r|| (FP32 values,
// vectors and reductions), FP64 update x += ||r|| d.
//
// Per-op path: the same arithmetic as one kernel per operation with
// scalars kept on the device (the PETSc library-call-per-op pattern), and
// the same sequence captured in a CUDA graph (Challenge A1).

#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "gbs_impl.cuh"

namespace {

constexpr int kSlots = 8;   // partial-sum slots per CTA
constexpr size_t kPersistSmem = (size_t)GBS_WARP_STAGE_BYTES * GBS_PWARPS;

template <typename T>
struct PcgSmall {
    T out[8];                // totals and part sums of a CTA sum
};

// Control block written by thread 0 of each CTA after a grid reduction and
// read by the CTA's other threads.  All CTAs compute it from the same
// partials in the same order, so all take the same decisions.
template <typename T>
struct PcgCtl {
    T alpha, beta;
    T rn;        // square root of the stopping test, taken by warp 1
    int go;
    int need_rr;   // this iteration's update phase sums N(r)^2 as well
    int fallback;  // N(r)^2 is needed but was not summed: one extra pass
    int stale;     // the last N(r)^2 is not that of the current residual
    // the scalar recurrences, used by thread 0 only (kept in shared memory
    // rather than in registers that every thread would reserve)
    T rho, rr, bnorm, lbf, tol2;
    int k, st, rr_current;
};

// Arguments of the persistent kernels.
struct PcgArgs {
    int64_t n;
    int64_t ntiles;
    const int32_t *tdesc;   // {row start, nonzero start} per warp tile (the chosen tiling)
    const int32_t *rowptr;
    const int32_t *colidx;
    const int16_t *colrel16;   // col - row (FP32 inner loop, when the matrix has it)
    const double *vals;
    const float *vals32;
    const double *dinv;
    const float *dinv32;
    const double *b;
    double *x;
    // FP64 work vectors (FP64 mode: r, z, p, q; mixed: r holds b - A x)
    double *r, *z, *p, *q;
    // FP32 work vectors (mixed mode): rhs, solution, r, z, p, q
    float *b32, *x32, *r32, *z32, *p32, *q32;
    double *part64;   // kSlots * G
    float *part32;    // kSlots * G
    GbsPipeCfg pipe64, pipe32;
    gbs_grid_barrier *bar;
    gbs_result_dev *res;
    // grid-wide bounds of D^-1 as bit patterns of positive doubles (max of
    // the bits, max of the complemented bits = min), zeroed before the launch
    unsigned long long *dbound;
    double rtol;
    double inner_rtol;
    int maxit;
    int outer_maxit;
    int x0_zero;
    int norm;          // GBS_NORM_* of the stopping test (FP64 loop only)
    int skip_cta;
    unsigned long long timeout_ns;
};

// Warp tiles [t0, t1) of CTA c: an even split of the tile list.
__device__ __forceinline__ void cta_tiles(const PcgArgs &a, int64_t &t0, int64_t &t1)
{
    t0 = a.ntiles * blockIdx.x / gridDim.x;
    t1 = a.ntiles * (blockIdx.x + 1) / gridDim.x;
}

// Status of the stopping test taken before each iteration (-100: go on).
template <typename T>
__device__ __forceinline__ int pcg_check(T rn, T rho, T tol, int k, int maxit)
{
    if (isnan(rn) || isnan(rho)) return GBS_ERR_NAN;
    if (rn <= tol) return GBS_OK;
    if (k >= maxit) return GBS_DIVERGED_ITS;
    return -100;
}

// PCG loop on (vals_T, dinv_T) for rhs bT, solution xT (in/out), work
// vectors rT..qT, as described at the top of this file.  Returns a status,
// the same in every thread of every CTA.  The scalar recurrences (rho,
// ||r||, alpha, beta, the stopping test) run in thread 0 of each CTA only;
// *iters, *rnorm_out and *bnorm_out are valid in thread 0.
// NT: threads of the CTA; UNR: rows per thread per trip of the vector
// phases; `stage` holds the staged CTA sums: 3 NT values for a 512-thread
// CTA, 2 NT for a wider one.
template <typename T, typename IX, int NT, int UNR, int LOG_L>
__device__ int pcg_loop(const PcgArgs &a, const IX *colidx, const T *vals, const T *dinv, const T *bT,
                        T *xT, T *rT,
                        T *zT, T *pT, T *qT, T *part, T rtol, int maxit, bool x0_zero,
                        int *iters, T *rnorm_out, T *bnorm_out, int *barrier_no,
                        unsigned char *wsm, GbsWarpQ &wq, uint32_t &parity, int *s_next,
                        const GbsPipeCfg &cfg, PcgSmall<T> &sm, T *stage, PcgCtl<T> &ctl,
                        int *s_flag)
{
    const int G = gridDim.x, c = blockIdx.x, warp = threadIdx.x >> 5;
    const uint64_t ps = gbs_policy_stream(), pk = gbs_policy_keep();
    int64_t t0, t1;
    cta_tiles(a, t0, t1);
    const int64_t rb = t0 < t1 ? (int64_t)__ldg(a.tdesc + 2 * t0) : 0;
    const int64_t re = t0 < t1 ? (int64_t)__ldg(a.tdesc + 2 * t1) : 0;
    // scalar state, meaningful in thread 0 only
    T &rho = ctl.rho, &rr = ctl.rr, &bnorm = ctl.bnorm, &lbf = ctl.lbf, &tol2 = ctl.tol2;
    int &k = ctl.k, &status = ctl.st, &rr_current = ctl.rr_current;
    if (threadIdx.x == 0) {
        rho = rr = bnorm = lbf = tol2 = T(0);
        k = 0;
        status = GBS_DIVERGED_ITS;
        rr_current = 1;
    }
    // Stopping-test norm N: rr holds N(r)^2 (r.r, z.z, or r.z for the
    // natural norm), bnorm N(b).  ref_sq(b_i, i) is b_i's term of N(b)^2.
    const int norm = a.norm;
    auto ref_sq = [&](T bi, int64_t i) -> T {
        if (norm == GBS_NORM_UNPRECONDITIONED) return bi * bi;
        const T db = gbs_ld(dinv + i, pk) * bi;
        return norm == GBS_NORM_PRECONDITIONED ? db * db : bi * db;
    };

    // ---- set-up: r = b - A x, z = D^-1 r, p = z; partials r.z, r.r, b.b;
    // the extreme entries of D^-1 (their bit patterns: D^-1 > 0, so the
    // order of the bits is the order of the values)
    T acc[3] = {T(0), T(0), T(0)};
    unsigned long long dmx = 0ull, dmn_c = 0ull;
    auto dtrack = [&](T di) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong((double)di);
        dmx = bits > dmx ? bits : dmx;
        dmn_c = ~bits > dmn_c ? ~bits : dmn_c;
    };
    if (!x0_zero) {
        auto epi = [&](int64_t i, T s, T) {
            const T bi = gbs_ld(bT + i, pk);
            const T ri = bi - s;
            const T di = gbs_ld(dinv + i, pk);
            dtrack(di);
            const T zi = di * ri;
            gbs_st(rT + i, ri, pk);
            gbs_st(zT + i, zi, pk);
            gbs_st(pT + i, zi, pk);
            acc[0] += ri * zi;
            const T w = norm == GBS_NORM_PRECONDITIONED ? zi : ri;
            acc[1] += w * w;
            acc[2] += ref_sq(bi, i);
        };
        if (!gbs_spmv_pipe<T, IX, LOG_L>(a.tdesc, t0, t1, s_next, a.rowptr, colidx, vals, xT, wsm, wq,
                              parity, cfg, ps, pk, a.timeout_ns, epi) &&
            (threadIdx.x & 31) == 0)
            atomicCAS(&a.bar->error, 0, GBS_ERR_TIMEOUT);
    } else {
        for (int64_t i = rb + threadIdx.x; i < re; i += NT) {
            const T bi = gbs_ld(bT + i, pk);
            const T di = gbs_ld(dinv + i, pk);
            dtrack(di);
            const T zi = di * bi;
            gbs_st(xT + i, T(0), pk);
            gbs_st(rT + i, bi, pk);
            gbs_st(zT + i, zi, pk);
            gbs_st(pT + i, zi, pk);
            acc[0] += bi * zi;
            const T w = norm == GBS_NORM_PRECONDITIONED ? zi : bi;
            acc[1] += w * w;
            acc[2] += ref_sq(bi, i);
        }
    }
    if (NT <= GBS_PBLOCK) {
        gbs_block_sum_staged<T, 3, NT>(acc, stage, sm.out);
        if (threadIdx.x == 0) {
            part[0 * G + c] = sm.out[0];
            part[1 * G + c] = sm.out[1];
            part[2 * G + c] = sm.out[2];
        }
    } else {
        // a wide CTA stages at most two values at a time (`stage` holds 2 NT)
        const T a01[2] = {acc[0], acc[1]}, a2[1] = {acc[2]};
        gbs_block_sum_staged<T, 2, NT>(a01, stage, sm.out);
        if (threadIdx.x == 0) {
            part[0 * G + c] = sm.out[0];
            part[1 * G + c] = sm.out[1];
        }
        gbs_block_sum_staged<T, 1, NT>(a2, stage, sm.out);
        if (threadIdx.x == 0) part[2 * G + c] = sm.out[0];
    }
    if (threadIdx.x == 0) *s_next = 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long m = __shfl_xor_sync(0xffffffffu, dmx, off);
        const unsigned long long mc = __shfl_xor_sync(0xffffffffu, dmn_c, off);
        dmx = m > dmx ? m : dmx;
        dmn_c = mc > dmn_c ? mc : dmn_c;
    }
    if ((threadIdx.x & 31) == 0 && dmx != 0ull) {
        atomicMax(a.dbound, dmx);
        atomicMax(a.dbound + 1, dmn_c);
    }
    const bool skip = (a.skip_cta == c) && (*barrier_no == 0);
    if (!gbs_grid_sync(a.bar, a.timeout_ns, (*barrier_no)++, skip, s_flag)) return GBS_ERR_TIMEOUT;
    // Lower bound of N(r)^2 by r.z: r.r >= r.z / max(D^-1) and
    // ||D^-1 r||^2 >= min(D^-1) r.z (natural norm: N(r)^2 is r.z).  While
    // lbf * r.z alone shows the stopping test fails, the update phase skips
    // the N(r)^2 sum (one FP64 operation per row); the test itself is
    // unchanged: it is decided on the summed N(r)^2 whenever it could pass.
    // N(r)^2 of the current residual over the grid in an extra pass (thread
    // 0 gets it); false if a barrier timed out
    auto sum_nr2 = [&](T &out) -> bool {
        T w2[1] = {T(0)};
        for (int64_t i = rb + threadIdx.x; i < re; i += NT) {
            const T ri = gbs_ld(rT + i, pk);
            const T w = norm == GBS_NORM_PRECONDITIONED ? gbs_ld(dinv + i, pk) * ri : ri;
            w2[0] += w * w;
        }
        gbs_block_sum_staged<T, 1, NT>(w2, stage, sm.out);
        if (threadIdx.x == 0) part[5 * G + c] = sm.out[0];
        if (!gbs_grid_sync(a.bar, a.timeout_ns, (*barrier_no)++, false, s_flag)) return false;
        if (warp == 0) {
            T g1[1];
            gbs_warp_grid_sum<T, 1>(part + 5 * G, G, G, g1);
            if (threadIdx.x == 0) out = g1[0];
        }
        __syncthreads();
        return true;
    };
    if (warp == 0) {
        T g3[3];
        gbs_warp_grid_sum<T, 3>(part, G, G, g3);
        if (threadIdx.x == 0) {
            rho = g3[0];
            rr = norm == GBS_NORM_NATURAL ? g3[0] : g3[1];
            bnorm = sqrt(g3[2]);
            const T dmax = (T)__longlong_as_double((long long)__ldcg(a.dbound));
            const T dmin = (T)__longlong_as_double((long long)~__ldcg(a.dbound + 1));
            lbf = norm == GBS_NORM_UNPRECONDITIONED ? T(1) / dmax
                  : norm == GBS_NORM_PRECONDITIONED ? dmin : T(1);
            tol2 = (rtol * bnorm) * (rtol * bnorm);
            const int s = pcg_check<T>(sqrt(rr), rho, rtol * bnorm, 0, maxit);
            ctl.go = s == -100;
            if (!ctl.go) status = s;
        }
    }
    __syncthreads();

    // every thread also counts iterations itself, so the loop is finite even
    // if the shared control block were ever wrong
    for (int k_all = 0; ctl.go && k_all <= maxit; ++k_all) {
        // ---- S: q = A p, partial p.q
        T pq[1] = {T(0)};
        // p_i is the operand the row's diagonal entry gathered (every row
        // has one: the Jacobi set-up checked it)
        auto epi = [&](int64_t i, T s, T p_i) {
            gbs_st(qT + i, s, pk);
            pq[0] += p_i * s;
        };
        if (!gbs_spmv_pipe<T, IX, LOG_L>(a.tdesc, t0, t1, s_next, a.rowptr, colidx, vals, pT, wsm, wq,
                                  parity, cfg, ps, pk, a.timeout_ns, epi) &&
            (threadIdx.x & 31) == 0)
            atomicCAS(&a.bar->error, 0, GBS_ERR_TIMEOUT);
        gbs_block_sum_staged<T, 1, NT>(pq, stage, sm.out);
        if (threadIdx.x == 0) {
            *s_next = 0;
            part[3 * G + c] = sm.out[0];
        }
        if (!gbs_grid_sync(a.bar, a.timeout_ns, (*barrier_no)++, false, s_flag))
            return GBS_ERR_TIMEOUT;
        if (warp == 0) {
            T pi[1];
            gbs_warp_grid_sum<T, 1>(part + 3 * G, G, G, pi);
            if (threadIdx.x == 0) {
                if (isnan(pi[0])) status = GBS_ERR_NAN;
                else if (pi[0] <= T(0)) status = GBS_ERR_INDEFINITE;
                ctl.go = !(isnan(pi[0]) || pi[0] <= T(0));
                ctl.alpha = rho / pi[0];
                // sum N(r)^2 in this update unless the current r.z is well
                // clear of the test (a margin of 16 for one step's drop) and
                // the iteration limit is not next
                ctl.need_rr = norm != GBS_NORM_NATURAL &&
                              (k + 1 >= maxit || !(lbf * rho > T(16) * tol2));
                ctl.stale = !rr_current;
            }
        }
        __syncthreads();
        if (!ctl.go) {
            // breakdown: report N(r) of the current residual
            if (ctl.stale) {
                T t = T(0);
                if (!sum_nr2(t)) return GBS_ERR_TIMEOUT;
                if (threadIdx.x == 0) rr = t;
            }
            break;
        }
        const T alpha = ctl.alpha;

        // ---- U: r -= alpha q; z = D^-1 r; partials r.z (and r.r).  In
        // FP64 the solution update x += alpha p waits for the P phase, which
        // reads p anyway (8 bytes per row fewer than doing it here); an exit
        // right after U applies it in a pass of its own.  The FP32 inner loop
        // keeps it here: deferring it measured 14 % slower there (27-point
        // 96^3, two lanes per row: 22.5 against 19.8 ms).  (UNR rows per
        // thread per trip: all loads are issued before the first use.)
        constexpr bool kDeferX = sizeof(T) == 8;
        const bool need_rr = ctl.need_rr != 0;
        T u[2] = {T(0), T(0)};
        for (int64_t i0 = rb + threadIdx.x; i0 < re; i0 += UNR * NT) {
            T rv[UNR], qv[UNR], dv[UNR], pv[UNR], xv[UNR];
#pragma unroll
            for (int h = 0; h < UNR; ++h) {
                const int64_t i = i0 + h * NT;
                if (i < re) {
                    if constexpr (!kDeferX) {
                        pv[h] = gbs_ld(pT + i, pk);
                        xv[h] = gbs_ld(xT + i, pk);
                    }
                    rv[h] = gbs_ld(rT + i, pk);
                    qv[h] = gbs_ld(qT + i, pk);
                    dv[h] = gbs_ld(dinv + i, pk);
                }
            }
#pragma unroll
            for (int h = 0; h < UNR; ++h) {
                const int64_t i = i0 + h * NT;
                if (i < re) {
                    const T rn_ = rv[h] - alpha * qv[h], zn_ = dv[h] * rn_;
                    if constexpr (!kDeferX) gbs_st(xT + i, xv[h] + alpha * pv[h], pk);
                    gbs_st(rT + i, rn_, pk);
                    gbs_st(zT + i, zn_, pk);
                    u[0] += rn_ * zn_;
                    if (need_rr) {
                        const T w = norm == GBS_NORM_PRECONDITIONED ? zn_ : rn_;
                        u[1] += w * w;
                    }
                }
            }
        }
        if (need_rr) {
            gbs_block_sum_staged<T, 2, NT>(u, stage, sm.out);
            if (threadIdx.x == 0) {
                part[4 * G + c] = sm.out[0];
                part[5 * G + c] = sm.out[1];
            }
        } else {
            const T u0[1] = {u[0]};
            gbs_block_sum_staged<T, 1, NT>(u0, stage, sm.out);
            if (threadIdx.x == 0) part[4 * G + c] = sm.out[0];
        }
        if (!gbs_grid_sync(a.bar, a.timeout_ns, (*barrier_no)++, false, s_flag))
            return GBS_ERR_TIMEOUT;
        // warps 0 and 1 form the same grid sums (same order, same bits);
        // warp 0 divides for beta while warp 1 takes the stopping test's
        // square root, on different SM partitions: each is a long chain of
        // dependent FP64 steps
        T g2[2] = {T(0), T(0)};
        if (need_rr || norm == GBS_NORM_NATURAL) {
            if (warp < 2) {
                gbs_warp_grid_sum<T, 2>(part + 4 * G, G, G, g2);
                if (threadIdx.x == 32) ctl.rn = sqrt(norm == GBS_NORM_NATURAL ? g2[0] : g2[1]);
                if (threadIdx.x == 0) ctl.beta = g2[0] / rho;
            }
        } else if (warp == 0) {
            T g1[1];
            gbs_warp_grid_sum<T, 1>(part + 4 * G, G, G, g1);
            g2[0] = g1[0];
            if (threadIdx.x == 0) {
                ctl.beta = g1[0] / rho;
                // N(r)^2 was not summed: go on only if r.z proves the test
                // fails (with a margin of 2 for the rounding of both sums);
                // otherwise sum it in an extra pass below
                ctl.fallback = !(g1[0] >= T(0) && lbf * g1[0] > T(2) * tol2);
            }
        }
        __syncthreads();
        if (!need_rr && norm != GBS_NORM_NATURAL && ctl.fallback) {
            // extra pass (rare: the one-step prediction above missed)
            T t = T(0);
            if (!sum_nr2(t)) return GBS_ERR_TIMEOUT;
            if (threadIdx.x == 0) {
                g2[1] = t;
                ctl.rn = sqrt(t);
            }
        }
        if (threadIdx.x == 0) {
            ++k;
            const T rho_new = g2[0];
            const bool have_rr = need_rr || norm == GBS_NORM_NATURAL || ctl.fallback;
            rr_current = have_rr;
            if (have_rr) rr = norm == GBS_NORM_NATURAL ? g2[0] : g2[1];
            if (!have_rr) {
                // r.z proved the test fails; the limit was not reached
                // (need_rr is set for the last allowed iteration)
                rho = rho_new;
                ctl.go = 1;
            } else if (rho_new < T(0)) {
                status = GBS_ERR_INDEFINITE;
                ctl.go = 0;
            } else {
                rho = rho_new;
                const int s = pcg_check<T>(ctl.rn, rho, rtol * bnorm, k, maxit);
                ctl.go = s == -100;
                if (!ctl.go) status = s;
            }
        }
        __syncthreads();
        if (!ctl.go) {
            // the loop ends after this update: x += alpha p on own rows
            if constexpr (kDeferX)
                for (int64_t i = rb + threadIdx.x; i < re; i += NT)
                    gbs_st(xT + i, gbs_ld(xT + i, pk) + alpha * gbs_ld(pT + i, pk), pk);
            break;
        }
        const T beta = ctl.beta;

        // ---- P: (FP64: x += alpha p, the update U left) p = z + beta p
        for (int64_t i0 = rb + threadIdx.x; i0 < re; i0 += UNR * NT) {
            T zv[UNR], pv[UNR], xv[UNR];
#pragma unroll
            for (int h = 0; h < UNR; ++h) {
                const int64_t i = i0 + h * NT;
                if (i < re) {
                    zv[h] = gbs_ld(zT + i, pk);
                    pv[h] = gbs_ld(pT + i, pk);
                    if constexpr (kDeferX) xv[h] = gbs_ld(xT + i, pk);
                }
            }
#pragma unroll
            for (int h = 0; h < UNR; ++h) {
                const int64_t i = i0 + h * NT;
                if (i < re) {
                    if constexpr (kDeferX) gbs_st(xT + i, xv[h] + alpha * pv[h], pk);
                    gbs_st(pT + i, zv[h] + beta * pv[h], pk);
                }
            }
        }
        if (!gbs_grid_sync(a.bar, a.timeout_ns, (*barrier_no)++, false, s_flag))
            return GBS_ERR_TIMEOUT;
    }
    // the status decides the caller's control flow in every thread: every
    // thread takes thread 0's value (kept in shared memory) after a barrier
    __syncthreads();
    if (threadIdx.x == 0) {
        *iters = k;
        *rnorm_out = sqrt(rr);
        *bnorm_out = bnorm;
    }
    const int st_all = status;
    __syncthreads();
    return st_all;
}

// NT threads per CTA (one CTA per SM), WB bytes of copy ring per warp, UNR
// rows per thread per trip of the vector phases.  With 1024 threads (32
// warps, 64 registers, 6.4 KB rings) the SpMV hides its gathers' latency
// better; the staged CTA sums then live in dynamic shared memory after the
// rings.
// IX: the column indices the SpMV streams (int32, or the compressed 16-bit
// col - row when the matrix has them); 2^LOG_L lanes share a row of the
// SpMV (the tiling in a.tdesc has at most 32 / 2^LOG_L rows per tile).
template <int NT, int WB, int UNR, typename IX, int LOG_L>
__global__ void __launch_bounds__(NT, 1) k_pcg_fp64(PcgArgs a)
{
    constexpr bool WIDE = NT > GBS_PBLOCK;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PcgSmall<double> sm;
    __shared__ double s_stage[WIDE ? 1 : 3 * NT];
    __shared__ PcgCtl<double> ctl;
    __shared__ GbsWarpQ s_q[NT / 32];
    __shared__ int s_next;
    __shared__ int s_flag;
    const int warp = threadIdx.x >> 5;
    gbs_warpq_init(s_q[warp]);
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    uint32_t parity = 0;
    int iters = 0, barrier_no = 0;
    double rn = 0.0, bn = 0.0;
    double *stage = WIDE ? reinterpret_cast<double *>(smem + (size_t)WB * (NT / 32)) : s_stage;
    const IX *cols = sizeof(IX) == 2 ? (const IX *)(const void *)a.colrel16
                                     : (const IX *)(const void *)a.colidx;
    int st = pcg_loop<double, IX, NT, UNR, LOG_L>(
        a, cols, a.vals, a.dinv, a.b, a.x, a.r, a.z, a.p, a.q, a.part64, a.rtol, a.maxit,
        a.x0_zero != 0, &iters, &rn, &bn, &barrier_no, smem + (size_t)warp * WB, s_q[warp],
        parity, &s_next, a.pipe64, sm, stage, ctl, &s_flag);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->status = st;
        a.res->iters = iters;
        a.res->outer = 0;
        a.res->rnorm = rn;
        a.res->bnorm = bn;
        a.res->timeout_where = st == GBS_ERR_TIMEOUT ? a.bar->where : -1;
    }
}

// Mixed precision: FP64 iterative refinement around the FP32 inner loop.
// The refinement scalars live in thread 0 of each CTA, like the inner ones.
// IX: the column indices of the FP32 inner loop (int32, or the compressed
// 16-bit col - row); the FP64 residual always reads the int32 indices.
// 2^LOG_L lanes share a row of the inner SpMV (the FP64 residual takes one
// lane per row of the same tiles).
template <typename IX, int LOG_L>
__global__ void __launch_bounds__(GBS_PBLOCK) k_pcg_mixed(PcgArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PcgSmall<double> sm64;
    __shared__ double s_stage[3 * GBS_PBLOCK];
    __shared__ PcgCtl<float> ctl32;
    __shared__ GbsWarpQ s_q[GBS_PWARPS];
    __shared__ double s_scale;
    __shared__ double s_itol;
    __shared__ int s_go;
    __shared__ int s_next;
    __shared__ int s_flag;
    const int G = gridDim.x, c = blockIdx.x, warp = threadIdx.x >> 5;
    // the FP64 and FP32 pipelines share this warp's stage memory and mbarriers
    unsigned char *wsm = smem + (size_t)warp * GBS_WARP_STAGE_BYTES;
    PcgSmall<float> &sm32 = *reinterpret_cast<PcgSmall<float> *>(&sm64);
    gbs_warpq_init(s_q[warp]);
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    uint32_t parity = 0;
    const uint64_t ps = gbs_policy_stream(), pk = gbs_policy_keep();
    int64_t t0, t1;
    cta_tiles(a, t0, t1);
    const int64_t rb = t0 < t1 ? (int64_t)__ldg(a.tdesc + 2 * t0) : 0;
    const int64_t re = t0 < t1 ? (int64_t)__ldg(a.tdesc + 2 * t1) : 0;
    int barrier_no = 0, inner_total = 0, outer = 0, st = GBS_DIVERGED_ITS;
    double rn = 0.0, bnorm = 0.0, prev = INFINITY;   // thread 0
    for (int it = 0; it <= a.outer_maxit; ++it) {
        // ---- FP64 residual r = b - A x with r.r (and b.b once) fused
        double acc[2] = {0.0, 0.0};
        const bool first = it == 0;
        if (first && a.x0_zero) {
            for (int64_t i = rb + threadIdx.x; i < re; i += GBS_PBLOCK) {
                const double bi = gbs_ld(a.b + i, pk);
                gbs_st(a.x + i, 0.0, pk);
                gbs_st(a.r + i, bi, pk);
                acc[0] += bi * bi;
                acc[1] += bi * bi;
            }
        } else {
            auto epi = [&](int64_t i, double s, double) {
                const double bi = gbs_ld(a.b + i, pk);
                const double ri = bi - s;
                gbs_st(a.r + i, ri, pk);
                acc[0] += ri * ri;
                if (first) acc[1] += bi * bi;
            };
            if (!gbs_spmv_pipe<double, int32_t>(a.tdesc, t0, t1, &s_next, a.rowptr, a.colidx, a.vals, a.x,
                                       wsm, s_q[warp], parity, a.pipe64, ps, pk, a.timeout_ns,
                                       epi) &&
                (threadIdx.x & 31) == 0)
                atomicCAS(&a.bar->error, 0, GBS_ERR_TIMEOUT);
        }
        gbs_block_sum_staged<double, 2, GBS_PBLOCK>(acc, s_stage, sm64.out);
        double *part = a.part64 + (it & 1) * 2 * G;
        if (threadIdx.x == 0) {
            s_next = 0;
            part[c] = sm64.out[0];
            part[G + c] = sm64.out[1];
        }
        const bool skip = (a.skip_cta == c) && (barrier_no == 0);
        if (!gbs_grid_sync(a.bar, a.timeout_ns, barrier_no++, skip, &s_flag)) {
            st = GBS_ERR_TIMEOUT;
            break;
        }
        if (warp == 0) {
            double g2[2];
            gbs_warp_grid_sum<double, 2>(part, G, G, g2);
            if (threadIdx.x == 0) {
                rn = sqrt(g2[0]);
                if (first) bnorm = sqrt(g2[1]);
                outer = it;
                int s = -100;
                if (isnan(rn)) s = GBS_ERR_NAN;
                else if (rn <= a.rtol * bnorm) s = GBS_OK;
                else if (rn > 0.5 * prev) s = GBS_ERR_STAGNATION;
                else if (it >= a.outer_maxit) s = GBS_DIVERGED_ITS;
                s_go = s == -100;
                if (!s_go) st = s;
                prev = rn;
                s_scale = 1.0 / rn;
                // the inner tolerance: eta, or looser where half the outer
                // target already suffices (the last refinement step)
                s_itol = fmax(a.inner_rtol, 0.5 * a.rtol * bnorm / rn);
            }
        }
        __syncthreads();
        if (!s_go) break;
        // ---- scale to FP32 (own rows) and solve A d = r / ||r|| in FP32
        const double inv = s_scale;
        for (int64_t i = rb + threadIdx.x; i < re; i += GBS_PBLOCK)
            gbs_st(a.b32 + i, (float)(gbs_ld(a.r + i, pk) * inv), pk);
        int kin = 0;
        float rin = 0.f, bin = 0.f;
        const IX *col32 = sizeof(IX) == 2 ? (const IX *)(const void *)a.colrel16
                                          : (const IX *)(const void *)a.colidx;
        const int sti = pcg_loop<float, IX, GBS_PBLOCK, 4, LOG_L>(
            a, col32, a.vals32, a.dinv32, a.b32, a.x32, a.r32, a.z32, a.p32, a.q32, a.part32,
            (float)s_itol, a.maxit, true, &kin, &rin, &bin, &barrier_no, wsm, s_q[warp],
            parity, &s_next, a.pipe32, sm32, reinterpret_cast<float *>(s_stage), ctl32, &s_flag);
        inner_total += kin;
        if (sti < 0) { st = sti; break; }
        // ---- FP64 update x += ||r|| d (own rows), then a barrier so the next
        // residual SpMV sees every row of x
        if (threadIdx.x == 0) s_scale = rn;
        __syncthreads();
        const double scale = s_scale;
        for (int64_t i = rb + threadIdx.x; i < re; i += GBS_PBLOCK)
            gbs_st(a.x + i, gbs_ld(a.x + i, pk) + scale * (double)gbs_ld(a.x32 + i, pk), pk);
        if (!gbs_grid_sync(a.bar, a.timeout_ns, barrier_no++, false, &s_flag)) {
            st = GBS_ERR_TIMEOUT;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->status = st;
        a.res->iters = inner_total;
        a.res->outer = outer;
        a.res->rnorm = rn;
        a.res->bnorm = bnorm;
        a.res->timeout_where = st == GBS_ERR_TIMEOUT ? a.bar->where : -1;
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Cooperative grid for a persistent kernel: as many co-resident CTAs as
// fit, but no more than one CTA per GBS_PWARPS warp tiles (small systems
// run on few CTAs, so their barriers are cheap).
int coop_grid(gbs_ctx c, const void *fn, int64_t ntiles, int want = 0,
              size_t smem = kPersistSmem, int nt = GBS_PBLOCK)
{
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem) != cudaSuccess)
        return -1;
    if (per_sm < 1) return -1;
    int64_t g = (int64_t)per_sm * c->num_sms;
    if (want > 0) return (int)(want < g ? want : g);   // the caller's choice, within residency
    const int64_t need = (ntiles + nt / 32 - 1) / (nt / 32);
    if (g > need) g = need;
    return g < 1 ? 1 : (int)g;
}

// Algorithmic bytes of a persistent solve (gbs_solve_info.model_bytes): a
// nonzero streams its value and its column index (ib = 4 or 2 bytes); every
// vector entry is counted once per pass that reads or writes it.
//  FP64: the set-up pass (r = b - A x: matrix, row pointers, x gather, b
//  and D^-1 read, r, z, p written) and per iteration the S phase (matrix,
//  row pointers, p gather, q written: 4n + 16n), U (r, q, D^-1 read, r, z
//  written: 40n) and P (z, p, x read, p, x written: 40n), i.e.
//  (8 + ib) nnz + 100 n per iteration, and the final x += alpha p pass.
//  Mixed: per refinement step the FP64 residual (12 nnz with 32-bit
//  indices + 4n row pointers + 8n gather + 8n b read + 8n r written), the
//  scaling to FP32 (8n read, 4n written) and the FP64 update (16n x, 4n
//  FP32 solution); per inner solve its set-up (b32, D^-1 read, x, r, z, p
//  written: 24n) and per inner iteration (4 + ib) nnz + 56 n (the FP32
//  loop updates x in U).
double persistent_model_bytes(gbs_mat A, bool mixed, int ib, const gbs_solve_info &r)
{
    const double n = (double)A->n, nnz = (double)A->nnz;
    if (!mixed)
        return ((8.0 + ib) * nnz + 52.0 * n + 4.0) + (double)r.iters * ((8.0 + ib) * nnz + 100.0 * n) +
               (r.iters > 0 ? 24.0 * n : 0.0);
    const double outer = (double)r.outer_iters + 1.0;   // residual passes
    const double inner_solves = (double)r.outer_iters;
    return outer * (12.0 * nnz + 36.0 * n) + inner_solves * (12.0 * n + 20.0 * n + 24.0 * n) +
           (double)r.iters * ((4.0 + ib) * nnz + 56.0 * n);
}

// Launch a persistent kernel and read its result record (one host
// synchronisation per solve).
int launch_persistent(gbs_ctx c, const void *fn, int G, PcgArgs &a, gbs_solve_info *info,
                      size_t smem = kPersistSmem, int nt = GBS_PBLOCK)
{
    GBS_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    void *args[] = {&a};
    GBS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(nt), args, smem, c->stream));
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
    info->outer_iters = r.outer;
    info->rnorm = r.rnorm;
    info->bnorm = r.bnorm;
    info->device_ms = ms;
    return r.status;
}

// Tiling li (2^li lanes per row: tiles of at most 32 >> li rows) and its
// stage geometries.
void fill_matrix_args(PcgArgs &a, gbs_mat A, int li)
{
    a.n = A->n;
    a.ntiles = A->ntiles_lanes[li];
    a.tdesc = A->tdesc_lanes[li];
    a.rowptr = A->rowptr;
    a.colidx = A->colidx;
    a.vals = A->vals;
    a.vals32 = A->vals32;
    a.dinv = A->dinv;
    a.dinv32 = A->dinv32;
    a.pipe64 = A->pipe64_lanes[li];
    a.pipe32 = A->pipe32_lanes[li];
}

// Launch shapes of the persistent kernels.  FP64: one CTA of 16 warps per
// SM with 12.8 KB copy rings per warp (shape 1), or one CTA of 32 warps
// with 6.4 KB rings (shape 2: more warps hide the SpMV gathers' latency
// better, while the CTA-wide sums and barriers of a 1024-thread CTA cost
// more; it needs two stages of the largest tile in 6.4 KB).  The mixed
// kernel has shape 1 only.  Either runs the SpMV with 1 or 2 lanes per row
// (tilings of 32- and 16-row tiles).
struct PcgShape {
    const void *fn;
    size_t smem;
    int nt;
    GbsPipeCfg cfg;     // stage geometry of the SpMV the kernel's loop runs
};

template <typename IX, int LOG_L>
PcgShape fp64_shape_l(int shape, GbsPipeCfg cfg)
{
    constexpr int kSmallRing = GBS_WARP_STAGE_BYTES / 2;
    constexpr int kWide = 2 * GBS_PBLOCK;
    PcgShape s;
    s.cfg = cfg;
    if (shape == 2) {
        const int stages = kSmallRing / cfg.sbytes;
        s.cfg.stages = stages < GBS_MAX_STAGES ? stages : GBS_MAX_STAGES;
        s.fn = (const void *)k_pcg_fp64<kWide, kSmallRing, 2, IX, LOG_L>;
        s.smem = (size_t)kSmallRing * (kWide / 32) + 2 * kWide * sizeof(double);
        s.nt = kWide;
    } else {
        s.fn = (const void *)k_pcg_fp64<GBS_PBLOCK, GBS_WARP_STAGE_BYTES, 4, IX, LOG_L>;
        s.smem = kPersistSmem;
        s.nt = GBS_PBLOCK;
    }
    return s;
}

// The kernel and geometry for (mode, index width, shape, lanes 2^li).
PcgShape pcg_shape(gbs_mat A, bool mixed, bool rel, int shape, int li)
{
    if (mixed) {
        PcgShape s;
        s.fn = rel ? (li ? (const void *)k_pcg_mixed<int16_t, 1> : (const void *)k_pcg_mixed<int16_t, 0>)
                   : (li ? (const void *)k_pcg_mixed<int32_t, 1> : (const void *)k_pcg_mixed<int32_t, 0>);
        s.smem = kPersistSmem;
        s.nt = GBS_PBLOCK;
        s.cfg = rel ? A->pipe16_lanes[li] : A->pipe32_lanes[li];
        return s;
    }
    const GbsPipeCfg cfg = rel ? A->pipe64r_lanes[li] : A->pipe64_lanes[li];
    if (rel) return li ? fp64_shape_l<int16_t, 1>(shape, cfg) : fp64_shape_l<int16_t, 0>(shape, cfg);
    return li ? fp64_shape_l<int32_t, 1>(shape, cfg) : fp64_shape_l<int32_t, 0>(shape, cfg);
}

// Shape 2 is possible where two stages of the tiling's largest tile fit in
// a 6.4 KB ring and there are at least 32 tiles per SM.
bool wide_shape_fits(gbs_mat A, bool rel, int li)
{
    const GbsPipeCfg &cfg = rel ? A->pipe64r_lanes[li] : A->pipe64_lanes[li];
    if (!A->tdesc_lanes[li] || cfg.sbytes <= 0) return false;   // tiling not made
    return (GBS_WARP_STAGE_BYTES / 2) / cfg.sbytes >= 2 &&
           A->ntiles_lanes[li] >= (int64_t)A->ctx->num_sms * 32;
}

// The fixed rule used before a class is tuned and where tuning is not
// possible: the 32-warp shape wherever it fits, one lane per row.
void rule_shape(gbs_mat A, bool mixed, bool rel, int *shape, int *li)
{
    *li = 0;
    *shape = !mixed && wide_shape_fits(A, rel, 0) ? 2 : 1;
}

// Class of a system for the tuner's decisions: precision, index width,
// row length (at most 8, 16, 32 or more nonzeros) and log2 of the warp
// tiles per SM.
void pcg_class(gbs_mat A, bool mixed, bool rel, int *i0, int *i1, int *i2, int *i3)
{
    const int m = A->max_row_nnz;
    int64_t t = A->ntiles / (A->ctx->num_sms > 0 ? A->ctx->num_sms : 1);
    int lg = 0;
    while (t > 1 && lg < 11) {
        t >>= 1;
        ++lg;
    }
    *i0 = mixed ? 1 : 0;
    *i1 = rel ? 1 : 0;
    *i2 = m <= 8 ? 0 : m <= 16 ? 1 : m <= 32 ? 2 : 3;
    *i3 = lg;
}

// Launch a persistent solve of A with right-hand side b into x (device
// arrays of n entries) with the given shape and tiling; the caller made
// the FP32 copy and the compressed indices it asks for.
int persistent_run(gbs_mat A, const double *b, double *x, double rtol, int maxit, const gbs_opts *o,
                   bool mixed, bool rel16, int shape, int li, int outer_maxit, gbs_solve_info *info)
{
    gbs_ctx c = A->ctx;
    {
        const int st = gbs_mat_ensure_lane_tiling(A, li);
        if (st) return st;
    }
    const PcgShape sh = pcg_shape(A, mixed, rel16, shape, li);
    const int G = coop_grid(c, sh.fn, A->ntiles_lanes[li], o->persistent_ctas, sh.smem, sh.nt);
    if (G < 0) return GBS_ERR_CUDA;
    const int64_t n = A->n;
    // work vectors staggered by 4.25 KB: at power-of-two lengths (128^3)
    // their entries i would otherwise sit at the same offset modulo 16 MiB
    // (C2 82.46 -> 82.05 us per iteration, same box)
    const size_t vec64 = align256(sizeof(double) * (size_t)n) + 4352;
    const size_t vec32 = align256(sizeof(float) * (size_t)n) + 4352;
    const size_t part = align256(sizeof(double) * kSlots * (size_t)G);
    const size_t head = 512;  // barrier (offset 0), D^-1 bounds (128), result (256)
    const size_t total = head + 2 * part + (mixed ? vec64 + 6 * vec32 : 4 * vec64);
    void *scr = nullptr;
    int st = gbs_ctx_reserve(c, total, &scr);
    if (st) return st;
    char *base = (char *)scr;
    PcgArgs a;
    memset(&a, 0, sizeof(a));
    a.bar = (gbs_grid_barrier *)base;
    a.dbound = (unsigned long long *)(base + 128);
    a.res = (gbs_result_dev *)(base + 256);
    a.part64 = (double *)(base + head);
    a.part32 = (float *)(base + head + part);
    char *v = base + head + 2 * part;
    if (mixed) {
        a.r = (double *)v; v += vec64;
        a.b32 = (float *)v; v += vec32;
        a.x32 = (float *)v; v += vec32;
        a.r32 = (float *)v; v += vec32;
        a.z32 = (float *)v; v += vec32;
        a.p32 = (float *)v; v += vec32;
        a.q32 = (float *)v; v += vec32;
    } else {
        a.r = (double *)v; v += vec64;
        a.z = (double *)v; v += vec64;
        a.p = (double *)v; v += vec64;
        a.q = (double *)v; v += vec64;
    }
    fill_matrix_args(a, A, li);
    if (rel16) a.colrel16 = A->colrel16;   // the SpMV (FP64, or FP32 inner) streams 16-bit offsets
    if (mixed) a.pipe32 = sh.cfg;
    else a.pipe64 = sh.cfg;
    a.b = b;
    a.x = x;
    a.rtol = rtol;
    a.inner_rtol = o->inner_rtol;
    a.maxit = maxit;
    a.outer_maxit = outer_maxit;
    a.x0_zero = 0;
    a.norm = o->norm_type;
    a.skip_cta = o->fault_skip_arrival;
    a.timeout_ns = (unsigned long long)o->barrier_timeout_ms * 1000000ull;
    GBS_CUDA_TRY(cudaMemsetAsync(base, 0, head, c->stream));
    st = launch_persistent(c, sh.fn, G, a, info, sh.smem, sh.nt);
    info->model_bytes = persistent_model_bytes(A, mixed, rel16 ? 2 : 4, *info);
    info->cta_threads = sh.nt;
    info->lanes_per_row = 1 << li;
    return st;
}

// The tuner: for a class not yet decided on this context, time a solve
// capped at kTuneIters iterations (rtol 0, so none stops early; mixed: one
// refinement step) of every candidate (shape x lanes per row) on this
// system, median of three runs each, and keep the fastest; the rule's
// choice is kept unless another is at least 3 % faster.  The decision is
// cached per class, so every system of the class gets the same kernel.
constexpr int kTuneIters = 24;

int pcg_tune(gbs_mat A, bool mixed, bool rel16, const gbs_opts *o, int *shape, int *li)
{
    gbs_ctx c = A->ctx;
    int k0, k1, k2, k3;
    pcg_class(A, mixed, rel16, &k0, &k1, &k2, &k3);
    signed char &dec = c->pcg_choice[k0][k1][k2][k3];
    if (dec > 0) {
        *shape = 1 + ((dec - 1) >> 1);
        *li = (dec - 1) & 1;
        return GBS_OK;
    }
    int rshape, rli;
    rule_shape(A, mixed, rel16, &rshape, &rli);
    if (A->n == 0 || !A->diag_ok) {
        *shape = rshape;
        *li = rli;
        return GBS_OK;
    }
    double *bx = nullptr;   // b = D^-1 (any nonzero right-hand side), x
    GBS_CUDA_TRY(cudaMalloc(&bx, 2 * sizeof(double) * (size_t)A->n));
    GBS_CUDA_TRY(cudaMemcpyAsync(bx, A->dinv, sizeof(double) * A->n, cudaMemcpyDeviceToDevice,
                                 c->stream));
    float best = 0.f, rule_ms = 0.f;
    int bs = rshape, bl = rli, st = GBS_OK;
    gbs_opts to = *o;
    to.persistent_ctas = 0;
    to.fault_skip_arrival = -1;
    to.inner_rtol = 1e-300;   // mixed: the inner solve runs its kTuneIters iterations too
    for (int cl = 0; cl < 2 && st == GBS_OK; ++cl) {
        for (int cs = 1; cs <= (mixed ? 1 : 2) && st == GBS_OK; ++cs) {
            if (cs == 2 && !wide_shape_fits(A, rel16, cl)) continue;
            st = gbs_mat_ensure_lane_tiling(A, cl);
            float t[3];
            for (int r = 0; r < 3 && st == GBS_OK; ++r) {
                gbs_solve_info ti;
                memset(&ti, 0, sizeof(ti));
                cudaMemsetAsync(bx + A->n, 0, sizeof(double) * A->n, c->stream);
                const int rs = persistent_run(A, bx, bx + A->n, 0.0, kTuneIters, &to, mixed, rel16, cs,
                                              cl, 1, &ti);
                // a timing run's own status (limit reached, stagnation) is
                // of no interest; only a failure of the device stops tuning
                if (rs == GBS_ERR_CUDA || rs == GBS_ERR_OOM || rs == GBS_ERR_TIMEOUT ||
                    rs == GBS_ERR_UNSUPPORTED)
                    st = rs;
                t[r] = (float)ti.device_ms;
            }
            if (st != GBS_OK) break;
            std::sort(t, t + 3);
            if (cs == rshape && cl == rli) rule_ms = t[1];
            if (best == 0.f || t[1] < best) {
                best = t[1];
                bs = cs;
                bl = cl;
            }
        }
    }
    cudaFree(bx);
    if (st != GBS_OK) return st;
    if (rule_ms > 0.f && best > 0.97f * rule_ms) {
        bs = rshape;
        bl = rli;
    }
    dec = (signed char)(1 + 2 * (bs - 1) + bl);
    *shape = bs;
    *li = bl;
    return GBS_OK;
}

// Shape and lanes for a solve: the options' fixed choice, else the tuned
// decision of the class.
int pcg_choice(gbs_mat A, bool mixed, bool rel16, const gbs_opts *o, int *shape, int *li)
{
    if (o->persistent_shape == 0 || o->persistent_lanes == 0) {
        int st = pcg_tune(A, mixed, rel16, o, shape, li);
        if (st) return st;
    }
    if (o->persistent_shape != 0) *shape = mixed ? 1 : o->persistent_shape;
    if (o->persistent_lanes != 0) *li = o->persistent_lanes == 2 ? 1 : 0;
    // the check below reads the tiling's tile count: make it first (a
    // decision cached from another system of the class finds none here)
    const int st = gbs_mat_ensure_lane_tiling(A, *li);
    if (st) return st;
    if (*shape == 2 && !wide_shape_fits(A, rel16, *li)) *shape = 1;
    return GBS_OK;
}

}  // namespace

int gbs_solve_persistent(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                         const gbs_opts *o, gbs_solve_info *info)
{
    const bool mixed = o->mode == GBS_MODE_MIXED;
    if (mixed) {
        int st = gbs_mat_ensure_f32(A);
        if (st) return st;
    }
    if (!mixed && !o->no_rel16) {
        int st = gbs_mat_ensure_rel16(A);
        if (st) return st;
    }
    const bool rel16 = A->colrel16 && !o->no_rel16;
    int shape = 1, li = 0;
    int st = pcg_choice(A, mixed, rel16, o, &shape, &li);
    if (st) {   // the tuner's device failure is the solve's
        info->status = st;
        return st;
    }
    return persistent_run(A, (const double *)b->data, (double *)x->data, rtol, maxit, o, mixed,
                          rel16, shape, li, o->outer_maxit, info);
}

extern "C" int gbs_ksp_tune(gbs_mat A, int mode, int *shape, int *lanes)
{
    if (!A || !shape || !lanes || (mode != GBS_MODE_FP64 && mode != GBS_MODE_MIXED)) return GBS_ERR_ARG;
    gbs_ctx c = A->ctx;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    const bool mixed = mode == GBS_MODE_MIXED;
    int st = mixed ? gbs_mat_ensure_f32(A) : (c->opts.no_rel16 ? GBS_OK : gbs_mat_ensure_rel16(A));
    if (st) return st;
    const bool rel16 = A->colrel16 && !c->opts.no_rel16;
    gbs_opts o = c->opts;
    o.mode = mode;
    int sh = 1, li = 0;
    st = pcg_choice(A, mixed, rel16, &o, &sh, &li);
    if (st) return st;
    *shape = sh;
    *lanes = 1 << li;
    return GBS_OK;
}

// ----------------------------------------------------------------------
// Per-op path: one kernel per operation, scalars on the device.
// ----------------------------------------------------------------------

namespace {

constexpr size_t kOpSmem = sizeof(GbsWarpTile<double>) * GBS_WARPS;

struct OpScalars {
    double rho, rr, bnorm, pi, alpha, beta;
    int k, status, done, pad;
    unsigned int counter[4];
};

struct OpArgs {
    int64_t n, ntiles;
    const int32_t *tiles, *rowptr, *colidx;
    const double *vals, *dinv, *b;
    double *x, *r, *z, *p, *q;
    double *part;   // 3 * G
    OpScalars *s;
    double rtol;
    int maxit;
    int norm;      // GBS_NORM_*: s->rr holds N(r)^2 and s->bnorm N(b)
};

// Last-CTA-done reduction of K partials into tot (fixed order).  Returns
// true in the last CTA only.
template <int K>
__device__ bool op_reduce(double (&v)[K], double *part, unsigned int *counter, double *s_red,
                          double (&tot)[K], bool *s_last)
{
    const int G = gridDim.x;
    gbs_block_sum<double, K>(v, s_red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) part[k * G + blockIdx.x] = v[k];
        __threadfence();
        *s_last = atomicAdd(counter, 1u) == (unsigned)G - 1;
    }
    __syncthreads();
    if (!*s_last) return false;
    __threadfence();
    gbs_grid_sum<double, K>(part, G, G, tot, s_red);
    if (threadIdx.x == 0) *counter = 0;
    return true;
}

__device__ void op_check(OpScalars *s, double rtol, int maxit)
{
    const double rn = sqrt(s->rr);
    if (isnan(rn) || isnan(s->rho)) { s->status = GBS_ERR_NAN; s->done = 1; }
    else if (rn <= rtol * s->bnorm) { s->status = GBS_OK; s->done = 1; }
    else if (s->k >= maxit) { s->status = GBS_DIVERGED_ITS; s->done = 1; }
}

__global__ void __launch_bounds__(GBS_BLOCK) k_op_setup(OpArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[4 * GBS_WARPS];
    __shared__ bool s_last;
    GbsWarpTile<double> &wt = reinterpret_cast<GbsWarpTile<double> *>(smem)[threadIdx.x >> 5];
    const uint64_t ps = gbs_policy_stream(), pk = gbs_policy_keep();
    double acc[3] = {0.0, 0.0, 0.0};
    auto epi = [&](int64_t i, double s) {
        const double bi = a.b[i], di = a.dinv[i], ri = bi - s, zi = di * ri;
        a.r[i] = ri;
        a.z[i] = zi;
        a.p[i] = zi;
        acc[0] += ri * zi;
        const double w = a.norm == GBS_NORM_PRECONDITIONED ? zi : ri;
        acc[1] += w * w;
        if (a.norm == GBS_NORM_UNPRECONDITIONED) {
            acc[2] += bi * bi;
        } else {
            const double db = di * bi;
            acc[2] += a.norm == GBS_NORM_PRECONDITIONED ? db * db : bi * db;
        }
    };
    const int64_t nw = (int64_t)gridDim.x * GBS_WARPS;
    for (int64_t t = (int64_t)blockIdx.x * GBS_WARPS + (threadIdx.x >> 5); t < a.ntiles; t += nw)
        gbs_spmv_warp<double>(a.rowptr, a.colidx, a.vals, a.x, a.tiles[t], a.tiles[t + 1], wt, ps,
                              pk, epi);
    double tot[3];
    if (op_reduce<3>(acc, a.part, &a.s->counter[0], s_red, tot, &s_last) && threadIdx.x == 0) {
        a.s->rho = tot[0];
        a.s->rr = a.norm == GBS_NORM_NATURAL ? tot[0] : tot[1];
        a.s->bnorm = sqrt(tot[2]);
        a.s->k = 0;
        a.s->done = 0;
        a.s->status = GBS_DIVERGED_ITS;
        op_check(a.s, a.rtol, a.maxit);
    }
}

__global__ void __launch_bounds__(GBS_BLOCK) k_op_spmv_pq(OpArgs a)
{
    if (a.s->done) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[4 * GBS_WARPS];
    __shared__ bool s_last;
    GbsWarpTile<double> &wt = reinterpret_cast<GbsWarpTile<double> *>(smem)[threadIdx.x >> 5];
    const uint64_t ps = gbs_policy_stream(), pk = gbs_policy_keep();
    double pq[1] = {0.0};
    auto epi = [&](int64_t i, double s) {
        a.q[i] = s;
        pq[0] += a.p[i] * s;
    };
    const int64_t nw = (int64_t)gridDim.x * GBS_WARPS;
    for (int64_t t = (int64_t)blockIdx.x * GBS_WARPS + (threadIdx.x >> 5); t < a.ntiles; t += nw)
        gbs_spmv_warp<double>(a.rowptr, a.colidx, a.vals, a.p, a.tiles[t], a.tiles[t + 1], wt, ps,
                              pk, epi);
    double tot[1];
    if (op_reduce<1>(pq, a.part, &a.s->counter[1], s_red, tot, &s_last) && threadIdx.x == 0) {
        a.s->pi = tot[0];
        if (isnan(tot[0])) { a.s->status = GBS_ERR_NAN; a.s->done = 1; }
        else if (tot[0] <= 0.0) { a.s->status = GBS_ERR_INDEFINITE; a.s->done = 1; }
        else a.s->alpha = a.s->rho / tot[0];
    }
}

__global__ void __launch_bounds__(GBS_BLOCK) k_op_update(OpArgs a)
{
    if (a.s->done) return;
    __shared__ double s_red[4 * GBS_WARPS];
    __shared__ bool s_last;
    const double alpha = a.s->alpha;
    double u[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * GBS_BLOCK + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * GBS_BLOCK) {
        a.x[i] += alpha * a.p[i];
        const double ri = a.r[i] - alpha * a.q[i];
        const double zi = a.dinv[i] * ri;
        a.r[i] = ri;
        a.z[i] = zi;
        u[0] += ri * zi;
        const double w = a.norm == GBS_NORM_PRECONDITIONED ? zi : ri;
        u[1] += w * w;
    }
    double tot[2];
    if (op_reduce<2>(u, a.part, &a.s->counter[2], s_red, tot, &s_last) && threadIdx.x == 0) {
        a.s->k += 1;
        a.s->rr = a.norm == GBS_NORM_NATURAL ? tot[0] : tot[1];
        if (tot[0] < 0.0) {
            a.s->status = GBS_ERR_INDEFINITE;
            a.s->done = 1;
        } else {
            a.s->beta = tot[0] / a.s->rho;
            a.s->rho = tot[0];
            op_check(a.s, a.rtol, a.maxit);
        }
    }
}

__global__ void __launch_bounds__(GBS_BLOCK) k_op_pupdate(OpArgs a)
{
    if (a.s->done) return;
    const double beta = a.s->beta;
    for (int64_t i = (int64_t)blockIdx.x * GBS_BLOCK + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * GBS_BLOCK)
        a.p[i] = a.z[i] + beta * a.p[i];
}

void op_iteration(const OpArgs &a, int gt, int gv, cudaStream_t s)
{
    k_op_spmv_pq<<<gt, GBS_BLOCK, kOpSmem, s>>>(a);
    k_op_update<<<gv, GBS_BLOCK, 0, s>>>(a);
    k_op_pupdate<<<gv, GBS_BLOCK, 0, s>>>(a);
}

}  // namespace

int gbs_solve_perop(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit, const gbs_opts *o,
                    gbs_solve_info *info, int use_graph)
{
    gbs_ctx c = A->ctx;
    if (o->mode != GBS_MODE_FP64) return GBS_ERR_UNSUPPORTED;
    const int64_t n = A->n;
    GBS_CUDA_TRY(cudaFuncSetAttribute((const void *)k_op_setup,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOpSmem));
    GBS_CUDA_TRY(cudaFuncSetAttribute((const void *)k_op_spmv_pq,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOpSmem));
    const int64_t tiles_blocks = (A->ntiles + GBS_WARPS - 1) / GBS_WARPS;
    int gt = (int)(tiles_blocks < (int64_t)c->num_sms * 4 ? tiles_blocks : (int64_t)c->num_sms * 4);
    int gv = (int)((n + GBS_BLOCK - 1) / GBS_BLOCK);
    if (gv > c->num_sms * 4) gv = c->num_sms * 4;
    if (gt < 1) gt = 1;
    if (gv < 1) gv = 1;
    const int G = gt > gv ? gt : gv;
    const size_t vec64 = align256(sizeof(double) * (size_t)n);
    const size_t part = align256(sizeof(double) * 3 * (size_t)G);
    const size_t head = align256(sizeof(OpScalars));
    void *scr = nullptr;
    int st = gbs_ctx_reserve(c, head + part + 4 * vec64, &scr);
    if (st) return st;
    char *base = (char *)scr;
    OpArgs a;
    memset(&a, 0, sizeof(a));
    a.s = (OpScalars *)base;
    a.part = (double *)(base + head);
    char *v = base + head + part;
    a.r = (double *)v; v += vec64;
    a.z = (double *)v; v += vec64;
    a.p = (double *)v; v += vec64;
    a.q = (double *)v; v += vec64;
    a.n = n;
    a.ntiles = A->ntiles;
    a.tiles = A->tiles;
    a.rowptr = A->rowptr;
    a.colidx = A->colidx;
    a.vals = A->vals;
    a.dinv = A->dinv;
    a.b = (const double *)b->data;
    a.x = (double *)x->data;
    a.rtol = rtol;
    a.maxit = maxit;
    a.norm = o->norm_type;

    GBS_CUDA_TRY(cudaMemsetAsync(base, 0, head, c->stream));
    GBS_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    k_op_setup<<<gt, GBS_BLOCK, kOpSmem, c->stream>>>(a);
    gbs_count_launch(c);
    GBS_CUDA_TRY(cudaGetLastError());
    volatile OpScalars *hs = (volatile OpScalars *)c->pinned;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;
    int rc = GBS_OK;
    if (use_graph) {
        // capture graph_iters iterations once; the kernels are no-ops once done
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int i = 0; i < o->graph_iters; ++i) op_iteration(a, gt, gv, cap);
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) rc = gbs_cuda_fail(e);
    }
    for (int64_t it = 0; rc == GBS_OK;) {
        cudaError_t e = cudaMemcpyAsync(c->pinned, a.s, sizeof(OpScalars), cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { rc = gbs_cuda_fail(e); break; }
        if (hs->done) break;
        if (it > (int64_t)maxit + 1) { rc = GBS_ERR_CUDA; break; }  // device never finished
        if (use_graph) {
            e = cudaGraphLaunch(exec, c->stream);
            gbs_count_launch(c, 3 * o->graph_iters);
            if (e != cudaSuccess) { rc = gbs_cuda_fail(e); break; }
            it += o->graph_iters;
        } else {
            op_iteration(a, gt, gv, c->stream);
            gbs_count_launch(c, 3);
            e = cudaGetLastError();
            if (e != cudaSuccess) { rc = gbs_cuda_fail(e); break; }
            it += 1;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (rc != GBS_OK) return rc;
    GBS_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->status = hs->status;
    info->iters = hs->k;
    info->outer_iters = 0;
    info->rnorm = sqrt(hs->rr);
    info->bnorm = hs->bnorm;
    info->device_ms = ms;
    return hs->status;
}

// ----------------------------------------------------------------------
// Public solve entry points
// ----------------------------------------------------------------------

// Largest FP64 system GBS_ALG_AUTO gives to the one-cluster solve rather
// than to the grid-wide persistent kernel (the crossover measured on GB300).
constexpr int64_t kClusterAutoRows = GBS_CLUSTER_MAX_ROWS;

extern "C" int gbs_ksp_solve_cg_ex(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                                   const gbs_opts *opts, gbs_solve_info *info)
{
    if (!A || !b || !x) return GBS_ERR_ARG;
    gbs_ctx c = A->ctx;
    const gbs_opts *o = opts ? opts : &c->opts;
    if (b->ctx != c || x->ctx != c) return GBS_ERR_ARG;
    if (A->n != A->ncols || b->n != A->n || x->n != A->n) return GBS_ERR_ARG;
    if (b->dtype != GBS_F64 || x->dtype != GBS_F64) return GBS_ERR_ARG;
    if (b->data == x->data && A->n > 0) return GBS_ERR_ARG;
    if (!(rtol >= 0.0) || maxit < 0) return GBS_ERR_ARG;
    if (o->mode != GBS_MODE_FP64 && o->mode != GBS_MODE_MIXED) return GBS_ERR_ARG;
    if (o->norm_type < GBS_NORM_UNPRECONDITIONED || o->norm_type > GBS_NORM_NATURAL) return GBS_ERR_ARG;
    if (o->norm_type != GBS_NORM_UNPRECONDITIONED && o->mode == GBS_MODE_MIXED) return GBS_ERR_ARG;
    gbs_solve_info tmp;
    memset(&tmp, 0, sizeof(tmp));
    int st;
    if (A->n == 0) {
        st = GBS_OK;
        tmp.status = GBS_OK;
    } else if (!A->diag_ok) {
        st = GBS_ERR_DIAG;
        tmp.status = st;
    } else {
        GBS_CUDA_TRY(cudaSetDevice(c->device));
        int alg = o->algorithm;
        // AUTO: a small FP64 system runs in one thread-block cluster (no
        // grid barriers); anything else, or a device that cannot keep the
        // cluster resident, in the persistent grid kernel
        const bool fits = o->mode == GBS_MODE_FP64 && A->n <= GBS_CLUSTER_MAX_ROWS;
        const bool auto_cluster = alg == GBS_ALG_AUTO && fits && A->n <= kClusterAutoRows &&
                                  o->persistent_ctas == 0 && o->fault_skip_arrival < 0;
        if (alg == GBS_ALG_AUTO) alg = auto_cluster ? GBS_ALG_CLUSTER : GBS_ALG_PERSISTENT;
        st = GBS_ERR_UNSUPPORTED;
        if (alg == GBS_ALG_CLUSTER) {
            if (fits) st = gbs_solve_cluster(A, b, x, rtol, maxit, o->norm_type, &tmp);
            if (st == GBS_ERR_UNSUPPORTED && auto_cluster) alg = GBS_ALG_PERSISTENT;
        }
        if (alg == GBS_ALG_PERSISTENT)
            st = gbs_solve_persistent(A, b, x, rtol, maxit, o, &tmp);
        else if (alg == GBS_ALG_PEROP || alg == GBS_ALG_GRAPH)
            st = gbs_solve_perop(A, b, x, rtol, maxit, o, &tmp, alg == GBS_ALG_GRAPH);
        if (st == GBS_ERR_CUDA || st == GBS_ERR_OOM || st == GBS_ERR_UNSUPPORTED ||
            st == GBS_ERR_ARG)
            tmp.status = st;
    }
    c->last = tmp;
    if (info) *info = tmp;
    return st;
}

extern "C" int gbs_ksp_solve_cg(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                                int *iters, double *rnorm)
{
    gbs_solve_info info;
    const int st = gbs_ksp_solve_cg_ex(A, b, x, rtol, maxit, nullptr, &info);
    if (st >= GBS_OK || st == GBS_ERR_INDEFINITE || st == GBS_ERR_NAN ||
        st == GBS_ERR_STAGNATION || st == GBS_ERR_TIMEOUT) {
        if (iters) *iters = info.iters;
        if (rnorm) *rnorm = info.rnorm;
    }
    return st;
}

extern "C" int gbs_ksp_last_info(gbs_ctx c, gbs_solve_info *info)
{
    if (!c || !info) return GBS_ERR_ARG;
    *info = c->last;
    return GBS_OK;
}


// Allocation-free FP64 solve.
//
// Some callers cannot allocate device memory at solve time: latency-bound
// loops (cudaMalloc and cudaFree may synchronise the whole device and take
// unbounded time) and processes whose device memory is owned by another
// allocator's pool, where a fresh cudaMalloc can fail.  This entry point
// runs the same persistent FP64 kernel as gbs_ksp_solve_cg_ex, with its
// whole workspace (r, z, p, q, the per-CTA partial sums, the grid barrier
// and the result record) in the fixed array below instead of the
// context's scratch.  The array is part of this library's device image:
// every GPU that loads the library holds it until the process exits.
// ----------------------------------------------------------------------

namespace {

constexpr int64_t kNoAllocMaxRows = GBS_NOALLOC_MAX_ROWS;
constexpr int kNoAllocMaxCtas = 2048;
constexpr size_t kNoAllocHead = 512;  // barrier (offset 0), D^-1 bounds (128), result record (256)
constexpr size_t kNoAllocPart = sizeof(double) * kSlots * kNoAllocMaxCtas;
constexpr size_t kNoAllocVec = sizeof(double) * kNoAllocMaxRows;
constexpr size_t kNoAllocBytes = kNoAllocHead + kNoAllocPart + 4 * kNoAllocVec;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device, looked up once (under a
// lock, so concurrent first calls from several threads are safe).
struct NoAllocSetup {
    void *addr[64];
    bool done[64];
};
NoAllocSetup g_noalloc_setup = {};
std::mutex g_noalloc_lock;

int noalloc_address(int device, void **out)
{
    if (device < 0 || device >= 64) return GBS_ERR_ARG;
    std::lock_guard<std::mutex> guard(g_noalloc_lock);
    if (!g_noalloc_setup.done[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return gbs_cuda_fail(e);
        g_noalloc_setup.addr[device] = p;
        g_noalloc_setup.done[device] = true;
    }
    *out = g_noalloc_setup.addr[device];
    return GBS_OK;
}

}  // namespace

extern "C" int gbs_ksp_solve_cg_noalloc(gbs_mat A, const double *b, double *x, double rtol,
                                        int maxit, gbs_solve_info *info)
{
    if (!A || !info || !(rtol >= 0.0) || maxit < 0) return GBS_ERR_ARG;
    if (A->n != A->ncols) return GBS_ERR_ARG;
    if (A->n > kNoAllocMaxRows) return GBS_ERR_ARG;
    if (A->n > 0 && (!b || !x || b == x)) return GBS_ERR_ARG;
    memset(info, 0, sizeof(*info));
    if (A->n == 0) return GBS_OK;
    if (!A->diag_ok) {
        info->status = GBS_ERR_DIAG;
        return GBS_ERR_DIAG;
    }
    gbs_ctx c = A->ctx;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    void *scr = nullptr;
    int st = noalloc_address(c->device, &scr);
    if (st) return st;
    // the compressed column indices only if the matrix already has them
    // (making them would allocate)
    const bool rel16 = A->colrel16 && !c->opts.no_rel16;
    // the class's tuned shape and tiling if this context has decided it and
    // the tiling exists (tuning and making a tiling would allocate), else
    // the fixed rule
    int shp = 1, li = 0;
    {
        int k0, k1, k2, k3;
        pcg_class(A, false, rel16, &k0, &k1, &k2, &k3);
        const signed char dec = c->pcg_choice[k0][k1][k2][k3];
        if (dec > 0 && A->tdesc_lanes[(dec - 1) & 1]) {
            shp = 1 + ((dec - 1) >> 1);
            li = (dec - 1) & 1;
        } else {
            rule_shape(A, false, rel16, &shp, &li);
        }
        if (shp == 2 && !wide_shape_fits(A, rel16, li)) shp = 1;
    }
    const PcgShape shape = pcg_shape(A, false, rel16, shp, li);
    int G = coop_grid(c, shape.fn, A->ntiles_lanes[li], c->opts.persistent_ctas, shape.smem, shape.nt);
    if (G < 0) return GBS_ERR_CUDA;
    if (G > kNoAllocMaxCtas) G = kNoAllocMaxCtas;
    char *base = (char *)scr;
    PcgArgs a;
    memset(&a, 0, sizeof(a));
    a.bar = (gbs_grid_barrier *)base;
    a.dbound = (unsigned long long *)(base + 128);
    a.res = (gbs_result_dev *)(base + 256);
    a.part64 = (double *)(base + kNoAllocHead);
    char *v = base + kNoAllocHead + kNoAllocPart;
    a.r = (double *)v;
    a.z = (double *)(v + kNoAllocVec);
    a.p = (double *)(v + 2 * kNoAllocVec);
    a.q = (double *)(v + 3 * kNoAllocVec);
    fill_matrix_args(a, A, li);
    if (rel16) a.colrel16 = A->colrel16;
    a.b = b;
    a.x = x;
    a.rtol = rtol;
    a.maxit = maxit;
    a.skip_cta = -1;
    a.norm = c->opts.norm_type;
    a.timeout_ns = (unsigned long long)c->opts.barrier_timeout_ms * 1000000ull;
    // the barrier and the result record must start at zero; the vectors and
    // partial sums are written before they are read
    GBS_CUDA_TRY(cudaMemsetAsync(base, 0, kNoAllocHead, c->stream));
    a.pipe64 = shape.cfg;
    st = launch_persistent(c, shape.fn, G, a, info, shape.smem, shape.nt);
    if (st == GBS_ERR_CUDA) info->status = st;
    else info->model_bytes = persistent_model_bytes(A, false, rel16 ? 2 : 4, *info);
    info->cta_threads = shape.nt;
    info->lanes_per_row = 1 << li;
    c->last = *info;
    return st;
}
