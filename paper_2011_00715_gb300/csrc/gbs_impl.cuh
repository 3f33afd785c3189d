// Internal declarations of the GB300 Jacobi-PCG library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbs.h"

#define GBS_BLOCK 256          // threads per CTA of the standalone kernels
#define GBS_WARPS (GBS_BLOCK / 32)
#define GBS_PBLOCK 512         // threads per CTA of the persistent solver kernels
#define GBS_PWARPS (GBS_PBLOCK / 32)
#define GBS_WT_ROWS 32         // rows per warp tile at most
#define GBS_WT_NNZ 512         // nonzeros per warp tile at most (a longer row is a tile of its own)

#define GBS_CUDA_TRY(call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return gbs_cuda_fail(e_);     \
    } while (0)

int gbs_cuda_fail(cudaError_t e);

struct gbs_ctx_s {
    int device;
    cudaStream_t stream;
    gbs_opts opts;
    int num_sms;
    int coop_supported;
    void *scratch;              // device scratch for solves (grown on demand)
    size_t scratch_bytes;
    void *pinned;               // small pinned host buffer for results
    void *devsmall;             // small device buffer for flags and results (4 KB)
    gbs_solve_info last;
    int64_t launches;           // kernel launches issued by this library
    cudaEvent_t ev0, ev1;
    // stream-ordered pool for the matrices' device arrays: freed memory
    // stays reserved for the next matrix (no mapping or unmapping per
    // create / destroy)
    cudaMemPool_t pool;
    // batched engines' lanes-per-row decisions, per precision, column stride
    // and row-length class: 0 = not tuned yet, else 1 + log2(lanes)
    signed char lane_choice[2][4][8];
    // persistent single-system CG: the tuner's shape and tiling decisions,
    // per precision, index width, row-length class and log2 of the warp
    // tiles per SM: 0 = not tuned yet, else 1 + 2 (shape - 1) + log2(lanes)
    signed char pcg_choice[2][2][4][12];
};

// Geometry of the bulk-copy pipeline of one matrix for one value type,
// computed on the host from the tile list so that every stage holds the
// largest tile: GBS_WARP_STAGE_BYTES per warp divided into `stages` slots.
#define GBS_MAX_STAGES 4
#define GBS_WARP_STAGE_BYTES 12800
struct GbsPipeCfg {
    int stages;   // 2..GBS_MAX_STAGES
    int sbytes;   // stride of one stage in bytes (multiple of 16)
    int coloff;   // byte offset of the column indices in a stage
    int rpoff;    // byte offset of the row pointers in a stage
};

struct gbs_mat_s {
    gbs_ctx ctx;
    int64_t n, ncols, nnz;
    int32_t *rowptr;
    int32_t *colidx;
    double *vals;
    float *vals32;              // FP32 copy of vals (mixed precision)
    double *dinv;               // 1 / a_ii (valid if diag_ok)
    float *dinv32;
    int diag_ok;
    int32_t *tiles;             // row starts of the warp tiles, ntiles + 1 entries
    int32_t *tdesc;             // {row start, nonzero start} per tile, ntiles + 1 pairs
    GbsPipeCfg pipe64, pipe32;  // pipeline geometry for FP64 and FP32 values
    int64_t ntiles;
    int max_row_nnz;
    // tilings for 1, 2 and 4 lanes per row (warp tiles of at most 32, 16 and
    // 8 rows; made on first use; entry 0 is the tiling above)
    int32_t *tdesc_lanes[3];
    int64_t ntiles_lanes[3];
    GbsPipeCfg pipe64_lanes[3], pipe32_lanes[3];
    // compressed column indices: col - row as int16, made on first use
    // (rel16_state 0 = not yet, 1 = made, -1 = some |col - row| > 32767,
    // colrel16 NULL); their stage geometry per tiling for FP32 values
    // (pipe16) and for FP64 values (pipe64r)
    int16_t *colrel16;
    int rel16_state;
    GbsPipeCfg pipe16, pipe16_lanes[3], pipe64r, pipe64r_lanes[3];
    // made from coordinate triplets: their count, the triplet indices in
    // sorted (row, column, index) order and each entry's segment of them
    int64_t coo_m;
    int64_t *coo_seg;     // nnz + 1
    uint32_t *coo_perm;   // coo_m
};

struct gbs_vec_s {
    gbs_ctx ctx;
    void *data;
    int64_t n;
    int dtype;
    int owned;
};

struct gbs_pc_s {
    gbs_mat A;
};

// Scratch memory of a context, grown on demand (synchronises when it grows).
int gbs_ctx_reserve(gbs_ctx ctx, size_t bytes, void **out);
void gbs_count_launch(gbs_ctx ctx, int n = 1);

// Result record written by the solver kernels (device memory).
struct gbs_result_dev {
    int status;
    int iters;
    int outer;
    int timeout_where;   // barrier index that gave up (-1 none)
    double rnorm;
    double bnorm;
};

// Software grid barrier for cooperative persistent kernels.
struct gbs_grid_barrier {
    unsigned int count;  // arrivals since the launch (zeroed before it)
    unsigned int gen;    // unused
    int error;           // 0, or a negative GBS_ERR_* set by the CTA that gave up
    int where;
};

// Internal entry points shared between translation units.
int gbs_solve_persistent(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                         const gbs_opts *o, gbs_solve_info *info);
int gbs_solve_perop(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                    const gbs_opts *o, gbs_solve_info *info, int use_graph);
// FP64 solve of a small system in one thread-block cluster.
int gbs_solve_cluster(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit, int norm,
                      gbs_solve_info *info);
int gbs_mat_ensure_f32(gbs_mat A);
// Make the compressed 16-bit column indices if the matrix allows them.
int gbs_mat_ensure_rel16(gbs_mat A);
// Make the tiling for 2^li lanes per row (li = 0, 1, 2) if it does not exist.
int gbs_mat_ensure_lane_tiling(gbs_mat A, int li);
// Device arrays owned by a matrix: from its context's pool, in its stream's
// order (GBS_ERR via the returned cudaError_t); freed likewise.
cudaError_t gbs_mat_alloc(gbs_ctx c, void **p, size_t bytes);
void gbs_mat_release(gbs_ctx c, void *p);

// ------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ unsigned long long gbs_globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int gbs_ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void gbs_st_release(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int gbs_ld_relaxed_int(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// L2 cache policies: matrix data is streamed once per iteration (evict
// first, no L1 allocation); solver vectors are re-read every iteration and
// should stay in the 126 MB L2 (evict last).
__device__ __forceinline__ uint64_t gbs_policy_stream()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t gbs_policy_keep()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Read-only streaming loads (matrix arrays, unchanged during a launch).
__device__ __forceinline__ int32_t gbs_ld_stream(const int32_t *p, uint64_t pol)
{
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
                 : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int16_t gbs_ld_stream(const int16_t *p, uint64_t pol)
{
    short v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s16 %0, [%1], %2;"
                 : "=h"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double gbs_ld_stream(const double *p, uint64_t pol)
{
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
                 : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float gbs_ld_stream(const float *p, uint64_t pol)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
                 : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

// Coherent loads and stores of vectors with an L2 policy.  Vectors written
// inside a persistent launch are read back with these (never through the
// read-only path); the grid barrier's acquire makes other CTAs' writes
// visible.
__device__ __forceinline__ double gbs_ld(const double *p, uint64_t pol)
{
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float gbs_ld(const float *p, uint64_t pol)
{
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void gbs_st(double *p, double v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void gbs_st(float *p, float v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol)
                 : "memory");
}

// Sum v[0..K) over a CTA of NW warps with a fixed shuffle tree; every thread
// gets the totals.  s_red must hold K * NW values.  Deterministic.
template <typename T, int K, int NW = GBS_WARPS>
__device__ __forceinline__ void gbs_block_sum(T (&v)[K], T *s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) s_red[k * NW + warp] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T t = lane < NW ? s_red[k * NW + lane] : T(0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        v[k] = t;
    }
    __syncthreads();
}

// Sum v[0..K) over a CTA of NT threads with few FP64 instructions (an SM
// partition retires about one FP64 warp instruction per 76 cycles, useful
// lanes or not, so a shuffle tree in every warp is costly): every thread
// stages its values in s_buf (K * NT entries); W = 4/K warps per value
// (K = 3: one) each add their share of the entries per lane, left to
// right, and finish with a fixed shuffle tree; one lane per value adds the
// W part sums.  Deterministic.  s_out holds 8 entries: the totals are
// returned in s_out[0..K) after a CTA barrier, s_out[4..8) is scratch.
template <typename T, int K, int NT>
__device__ __forceinline__ void gbs_block_sum_staged(const T (&v)[K], T *s_buf, T *s_out)
{
    constexpr int W = K >= 3 ? 1 : 4 / K;
    constexpr int PER = NT / 32 / W;
    static_assert(W * K <= NT / 32 && W * K <= 4 && PER >= 1, "warps per value");
#pragma unroll
    for (int k = 0; k < K; ++k) s_buf[k * NT + threadIdx.x] = v[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < W * K) {
        const int k = warp / W, j = warp % W;
        const T *src = s_buf + k * NT + j * (NT / W) + lane;
        T t = src[0];
#pragma unroll
        for (int m = 1; m < PER; ++m) t += src[32 * m];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) {
            if (W == 1) s_out[k] = t;
            else s_out[4 + k * W + j] = t;
        }
    }
    if (W > 1) {
        __syncthreads();
        if (threadIdx.x < K) {
            const T *q = s_out + 4 + threadIdx.x * W;
            s_out[threadIdx.x] = W == 4 ? (q[0] + q[1]) + (q[2] + q[3]) : q[0] + q[1];
        }
    }
    __syncthreads();
}

// Warp-level version of gbs_grid_sum for warp 0 only: every lane of the
// calling warp gets the K totals (same fixed order, no CTA barrier).
template <typename T, int K>
__device__ __forceinline__ void gbs_warp_grid_sum(const T *partials, int stride, int G,
                                                  T (&out)[K])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T t = T(0);
        for (int c = lane; c < G; c += 32) t += __ldcg(partials + k * stride + c);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        out[k] = t;
    }
}

// Sum partials[k * stride + c] over c in [0, G) for k < K, in a fixed order
// that does not depend on which CTA calls it: lane l adds c = l, l+32, ...
// left to right, then a fixed shuffle tree.  Every thread gets the totals.
template <typename T, int K>
__device__ __forceinline__ void gbs_grid_sum(const T *partials, int stride, int G, T (&out)[K],
                                             T *s_bcast)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T t = T(0);
            for (int c = lane; c < G; c += 32) t += __ldcg(partials + k * stride + c);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) s_bcast[k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = s_bcast[k];
    __syncthreads();
}

// Grid-wide barrier with a bounded wait.  Returns false if this CTA or
// another one gave up (bar->error set); the caller must then leave its
// loop.  `skip` makes this CTA not arrive (fault-injection for tests).
//
// One monotonic arrival counter, zeroed before the launch: barrier number
// `where` (0, 1, 2, ... in the order every CTA meets them) is complete once
// the counter reaches (where + 1) * gridDim.x.  Thread 0 of each CTA
// arrives with one release add (the CTA's writes, ordered before it by the
// CTA barrier, become visible to every CTA that observes the count) and
// waits with acquire loads of the same word: no generation word to read
// before arriving and no reset, so a barrier costs one round trip to L2
// plus the polling (1.2 us on 152 CTAs, against 2.0 us for a counter plus a
// generation word).  Counts are compared by signed difference, so the
// 32-bit counter may wrap.
__device__ __forceinline__ void gbs_red_add_release(unsigned int *p, unsigned int v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool gbs_grid_sync(gbs_grid_barrier *bar, unsigned long long timeout_ns,
                                              int where, bool skip, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (!skip) gbs_red_add_release(&bar->count, 1u);
        const unsigned int target = (unsigned int)(where + 1) * gridDim.x;
        const unsigned long long t0 = gbs_globaltimer();
        for (unsigned int spin = 1; (int)(gbs_ld_acquire(&bar->count) - target) < 0; ++spin) {
            if ((spin & 15u) == 0) {
                if (gbs_ld_relaxed_int(&bar->error) != 0) { ok = 0; break; }
                if (gbs_globaltimer() - t0 > timeout_ns) {
                    if (atomicCAS(&bar->error, 0, GBS_ERR_TIMEOUT) == 0) bar->where = where;
                    ok = 0;
                    break;
                }
            }
            __nanosleep(20);
        }
        // a failure recorded by any CTA before it arrived (e.g. a bulk copy
        // that did not complete) fails the barrier for everyone
        if (ok && gbs_ld_relaxed_int(&bar->error) != 0) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Multiply-accumulate of one nonzero.  FP64 uses one fused multiply-add
// (FP64 issue rate is the scarce resource on this GPU); FP32 rounds the
// product and the sum separately, the operation order of the definition.
__device__ __forceinline__ double gbs_mac(double a, double x, double s) { return fma(a, x, s); }
__device__ __forceinline__ float gbs_mac(float a, float x, float s)
{
    return __fadd_rn(s, __fmul_rn(a, x));
}

// Shared memory of one warp tile.
template <typename V>
struct GbsWarpTile {
    int32_t col[GBS_WT_NNZ];
    V val[GBS_WT_NNZ];
};

// One warp tile: rows [r0, r1) (at most 32) of y = A v, computed by one
// warp.  The tile's colidx/vals (contiguous in CSR) are staged in the
// warp's shared memory with coalesced streaming loads, several in flight
// per lane; then lane l accumulates row r0 + l left to right in storage
// order and calls epi(row, sum).  A tile holding a single row longer than
// GBS_WT_NNZ is reduced by the warp with a fixed shuffle tree.  No CTA-wide
// synchronisation: warps progress independently.  The gathers of v are
// coherent loads (v may have been written earlier in the same launch).
template <typename V, typename Epi>
__device__ __forceinline__ void gbs_spmv_warp(const int32_t *__restrict__ rowptr,
                                              const int32_t *__restrict__ colidx,
                                              const V *__restrict__ vals, const V *v, int64_t r0,
                                              int64_t r1, GbsWarpTile<V> &wt, uint64_t pol_stream,
                                              uint64_t pol_keep, Epi &epi)
{
    const int lane = threadIdx.x & 31;
    const int nrows = (int)(r1 - r0);
    int beg = 0, end = 0;
    if (lane < nrows) {
        beg = gbs_ld_stream(rowptr + r0 + lane, pol_stream);
        end = gbs_ld_stream(rowptr + r0 + lane + 1, pol_stream);
    }
    const int k0 = __shfl_sync(0xffffffffu, beg, 0);
    const int k1 = __shfl_sync(0xffffffffu, end, nrows - 1);
    if (k1 - k0 <= GBS_WT_NNZ) {
        constexpr int U = 8;
        for (int base = k0 + lane; base < k1; base += 32 * U) {
            int c[U];
            V a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = base + 32 * u;
                c[u] = k < k1 ? gbs_ld_stream(colidx + k, pol_stream) : 0;
                a[u] = k < k1 ? gbs_ld_stream(vals + k, pol_stream) : V(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = base + 32 * u;
                if (k < k1) {
                    wt.col[k - k0] = c[u];
                    wt.val[k - k0] = a[u];
                }
            }
        }
        __syncwarp();
        if (lane < nrows) {
            V s = V(0);
            const int e = end - k0;
#pragma unroll 4
            for (int k = beg - k0; k < e; ++k) s = gbs_mac(wt.val[k], gbs_ld(v + wt.col[k], pol_keep), s);
            epi(r0 + lane, s);
        }
        __syncwarp();
    } else {
        V s = V(0);
        for (int k = k0 + lane; k < k1; k += 32)
            s = gbs_mac(gbs_ld_stream(vals + k, pol_stream),
                        gbs_ld(v + gbs_ld_stream(colidx + k, pol_stream), pol_keep), s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) epi(r0, s);
        __syncwarp();
    }
}

// ------------------------------------------------------------------------
// Bulk-copy (TMA) staging of warp tiles.
//
// A warp tile's CSR slice -- rowptr[r0..r1], colidx[k0..k1), vals[k0..k1) --
// is contiguous in memory.  Lane 0 copies the 16-byte-aligned superset of
// each array into one of two shared-memory stages with cp.async.bulk,
// completing on that stage's mbarrier, while the warp computes the other
// stage: the next tile is always in flight.  Allocations are padded so the
// rounded-up ranges never leave a buffer.
// ------------------------------------------------------------------------

__device__ __forceinline__ uint32_t gbs_smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void gbs_mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gbs_smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void gbs_fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void gbs_mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gbs_smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool gbs_mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(gbs_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with parity `parity` to complete, for at most
// timeout_ns.  Returns false on timeout.
__device__ __forceinline__ bool gbs_mbar_wait(uint64_t *bar, uint32_t parity,
                                              unsigned long long timeout_ns)
{
    if (gbs_mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gbs_globaltimer();
    while (!gbs_mbar_try_wait(bar, parity))
        if (gbs_globaltimer() - t0 > timeout_ns) return false;
    return true;
}

__device__ __forceinline__ void gbs_bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(gbs_smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(gbs_smem_u32(bar)), "l"(pol)
        : "memory");
}

// Per-warp pipeline bookkeeping in shared memory.
struct GbsWarpQ {
    uint64_t bar[GBS_MAX_STAGES];   // one mbarrier per stage (count 1)
    int4 desc[GBS_MAX_STAGES];      // {r0, k0, r1, k1} of the tile in each stage
    int tile[GBS_MAX_STAGES];       // tile held by each stage, relative to the range (-1: none)
};

__device__ __forceinline__ void gbs_warpq_init(GbsWarpQ &q)
{
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int j = 0; j < GBS_MAX_STAGES; ++j) gbs_mbar_init(&q.bar[j], 1);
        gbs_fence_mbar_init();
    }
    __syncwarp();
}

// Column of a stored index: 32-bit indices are absolute; 16-bit ones are
// relative to the row (col - row), the compressed form FP32 paths use when
// every |col - row| of the matrix fits.
__device__ __forceinline__ int gbs_col(int32_t c, int) { return c; }
__device__ __forceinline__ int gbs_col(int16_t c, int row) { return row + (int)c; }

// y = A v over the warp tiles [t_begin, t_end), shared by the warps of a
// CTA: lane 0 of each warp claims the next unclaimed tile from *s_next
// (a CTA-shared counter, zero on entry) one step ahead, loads its
// descriptor while the previous copy is issued, and copies the tile's CSR
// slice into the next free stage of the warp's ring (wsm, cfg.stages
// stages), keeping cfg.stages - 1 tiles in flight; the warp then computes
// the oldest stage: lane l accumulates row r0 + l left to right and calls
// epi(row, sum, vdiag), vdiag being the gathered v[row] (the row's
// diagonal entry's operand; 0 if the row has no diagonal entry).  A tile
// holding one row longer than GBS_WT_NNZ is read directly and reduced with
// a fixed shuffle tree.  parity carries the warp's mbarrier phase bits
// across calls.  Returns false if a copy did not complete within
// timeout_ns; the copies still in flight are then waited for (again with a
// limit) before returning.
//
// The column indices are int32 (absolute) or int16 (relative to the row).
// gbs_spmv_pipe_pre is the same with a per-row prefetch: pre(row) runs before
// the row's nonzeros are gathered (so the loads it issues are in flight with
// the gathers) and its value is handed to epi(row, sum, vdiag, pre_value).
template <typename V, typename IX, int LOG_L = 0, typename Pre, typename Epi>
__device__ __forceinline__ bool gbs_spmv_pipe_pre(const int32_t *__restrict__ tdesc, int64_t t_begin,
                                                  int64_t t_end, int *s_next,
                                                  const int32_t *__restrict__ rowptr,
                                                  const IX *__restrict__ colidx,
                                                  const V *__restrict__ vals, const V *v,
                                                  unsigned char *wsm, GbsWarpQ &q, uint32_t &parity,
                                                  const GbsPipeCfg &cfg, uint64_t pol_stream,
                                                  uint64_t pol_keep, unsigned long long timeout_ns,
                                                  Pre &pre, Epi &epi)
{
    constexpr int E = 16 / (int)sizeof(V);    // values per 16 bytes
    constexpr int CE = 16 / (int)sizeof(IX);  // column indices per 16 bytes
    const int lane = threadIdx.x & 31;
    const int NS = cfg.stages;
    // lane 0: the next claimed tile and its descriptor, fetched one step ahead
    int64_t t_pend = t_end;
    int2 d_lo = make_int2(0, 0), d_hi = make_int2(0, 0);
    auto claim = [&]() {
        t_pend = t_begin + atomicAdd(s_next, 1);
        if (t_pend < t_end) {
            d_lo = __ldg(reinterpret_cast<const int2 *>(tdesc) + t_pend);
            d_hi = __ldg(reinterpret_cast<const int2 *>(tdesc) + t_pend + 1);
        }
    };
    // lane 0 only: start the copy of the pending tile into stage j, claim the next
    auto issue = [&](int j) {
        if (t_pend >= t_end) {
            q.tile[j] = -1;
            return;
        }
        const int r0 = d_lo.x, k0 = d_lo.y, r1 = d_hi.x, k1 = d_hi.y;
        q.tile[j] = (int)(t_pend - t_begin);
        q.desc[j] = make_int4(r0, k0, r1, k1);
        claim();
        if (k1 - k0 > GBS_WT_NNZ) return;
        const int vb = k0 & ~(E - 1), ve = (k1 + E - 1) & ~(E - 1);
        const int cb = k0 & ~(CE - 1), ce = (k1 + CE - 1) & ~(CE - 1);
        const int rb = r0 & ~3, re = (r1 + 4) & ~3;
        const uint32_t bv = (uint32_t)(sizeof(V) * (ve - vb)),
                       bc = (uint32_t)(sizeof(IX) * (ce - cb)), br = 4u * (uint32_t)(re - rb);
        unsigned char *st = wsm + (size_t)j * cfg.sbytes;
        gbs_mbar_expect_tx(&q.bar[j], bv + bc + br);
        gbs_bulk_g2s(st + cfg.rpoff, rowptr + rb, br, &q.bar[j], pol_stream);
        if (bv) gbs_bulk_g2s(st, vals + vb, bv, &q.bar[j], pol_stream);
        if (bc) gbs_bulk_g2s(st + cfg.coloff, colidx + cb, bc, &q.bar[j], pol_stream);
    };
    if (lane == 0) {
        claim();
        for (int j = 0; j < NS - 1; ++j) issue(j);
    }
    __syncwarp();
    bool ok = true;
    int m = 0;
    for (;; ++m) {
        const int j = m % NS;
        if (lane == 0) issue((m + NS - 1) % NS);   // that stage was consumed at m - 1
        __syncwarp();
        if (q.tile[j] < 0) break;   // claims are monotonic: no later stage holds a tile either
        const int4 d = q.desc[j];
        const int r0 = d.x, k0 = d.y, r1 = d.z, k1 = d.w;
        if (k1 - k0 > GBS_WT_NNZ) {
            const auto pv = pre((int64_t)r0);
            V sum = V(0), vd = V(0);
            for (int k = k0 + lane; k < k1; k += 32) {
                const int c = gbs_col(gbs_ld_stream(colidx + k, pol_stream), r0);
                const V xv = gbs_ld(v + c, pol_keep);
                if (c == r0) vd = xv;
                sum = gbs_mac(gbs_ld_stream(vals + k, pol_stream), xv, sum);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                sum += __shfl_xor_sync(0xffffffffu, sum, off);
                vd += __shfl_xor_sync(0xffffffffu, vd, off);
            }
            if (lane == 0) epi((int64_t)r0, sum, vd, pv);
        } else {
            if (!gbs_mbar_wait(&q.bar[j], (parity >> j) & 1u, timeout_ns)) {
                ok = false;
                break;
            }
            parity ^= 1u << j;
            const unsigned char *st = wsm + (size_t)j * cfg.sbytes;
            const V *sval = reinterpret_cast<const V *>(st);
            const IX *scol = reinterpret_cast<const IX *>(st + cfg.coloff);
            const int32_t *srp = reinterpret_cast<const int32_t *>(st + cfg.rpoff);
            const int nrows = r1 - r0;
            if constexpr (LOG_L == 0) {
                if (lane < nrows) {
                    const int row = r0 + lane;
                    const int vb = k0 & ~(E - 1), cb = k0 & ~(CE - 1), rb = r0 & ~3;
                    const auto pv = pre((int64_t)row);
                    const int beg = srp[row - rb], end = srp[row - rb + 1];
                    V sum = V(0), vd = V(0);
#pragma unroll 8
                    for (int k = beg; k < end; ++k) {
                        const int c = gbs_col(scol[k - cb], row);
                        const V xv = gbs_ld(v + c, pol_keep);
                        if (c == row) vd = xv;
                        sum = gbs_mac(sval[k - vb], xv, sum);
                    }
                    epi((int64_t)row, sum, vd, pv);
                }
            } else {
                // L = 2^LOG_L lanes per row (tiles of at most 32 / L rows):
                // lane l takes row r0 + l / L and every L-th nonzero of it
                // from l mod L on; the L partial sums meet in a fixed
                // shuffle tree and the group's first lane finishes the row
                constexpr int L = 1 << LOG_L;
                const int sub = lane & (L - 1);
                const bool act = (lane >> LOG_L) < nrows;
                const int row = r0 + (lane >> LOG_L);
                V sum = V(0), vd = V(0);
                if (act) {
                    const int vb = k0 & ~(E - 1), cb = k0 & ~(CE - 1), rb = r0 & ~3;
                    const int beg = srp[row - rb], end = srp[row - rb + 1];
#pragma unroll 4
                    for (int k = beg + sub; k < end; k += L) {
                        const int c = gbs_col(scol[k - cb], row);
                        const V xv = gbs_ld(v + c, pol_keep);
                        if (c == row) vd = xv;
                        sum = gbs_mac(sval[k - vb], xv, sum);
                    }
                }
#pragma unroll
                for (int off = L / 2; off > 0; off >>= 1) {
                    sum += __shfl_xor_sync(0xffffffffu, sum, off);
                    vd += __shfl_xor_sync(0xffffffffu, vd, off);
                }
                if (act && sub == 0) {
                    const auto pv = pre((int64_t)row);
                    epi((int64_t)row, sum, vd, pv);
                }
            }
        }
        __syncwarp();
    }
    if (!ok) {
        // wait (with a limit) for every copy still in flight, oldest first
        for (int dd = 0; dd < NS; ++dd) {
            const int jj = (m + dd) % NS;
            if (q.tile[jj] >= 0 && q.desc[jj].w - q.desc[jj].y <= GBS_WT_NNZ &&
                gbs_mbar_wait(&q.bar[jj], (parity >> jj) & 1u, timeout_ns))
                parity ^= 1u << jj;
        }
    }
    __syncwarp();
    return ok;
}

// No per-row prefetch.
struct GbsNoPre {
    __device__ __forceinline__ int operator()(int64_t) const { return 0; }
};

template <typename V, typename IX, int LOG_L = 0, typename Epi>
__device__ __forceinline__ bool gbs_spmv_pipe(const int32_t *__restrict__ tdesc, int64_t t_begin,
                                              int64_t t_end, int *s_next,
                                              const int32_t *__restrict__ rowptr,
                                              const IX *__restrict__ colidx,
                                              const V *__restrict__ vals, const V *v,
                                              unsigned char *wsm, GbsWarpQ &q, uint32_t &parity,
                                              const GbsPipeCfg &cfg, uint64_t pol_stream,
                                              uint64_t pol_keep, unsigned long long timeout_ns,
                                              Epi &epi)
{
    GbsNoPre pre;
    auto e = [&](int64_t row, V sum, V vd, int) { epi(row, sum, vd); };
    return gbs_spmv_pipe_pre<V, IX, LOG_L>(
        tdesc, t_begin, t_end, s_next, rowptr, colidx, vals, v, wsm, q, parity, cfg, pol_stream,
        pol_keep, timeout_ns, pre, e);
}

#endif  // __CUDACC__
