// Internal declarations of the GB300 Jacobi-PCG library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbs.h"

#define GBS_BLOCK 256          // threads per CTA of the tile kernels
#define GBS_TILE_ROWS 256      // rows per CSR tile at most
#define GBS_TILE_NNZ 2048      // nonzeros per CSR tile at most (longer rows: own tile)
#define GBS_WARPS (GBS_BLOCK / 32)

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
    int32_t *tiles;             // row starts of the CSR tiles, ntiles + 1 entries
    int64_t ntiles;
    int max_row_nnz;
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
    unsigned int count;
    unsigned int gen;
    int error;           // 0, or a negative GBS_ERR_* set by the CTA that gave up
    int where;
};

// Internal entry points shared between translation units.
int gbs_solve_persistent(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                         const gbs_opts *o, gbs_solve_info *info);
int gbs_solve_perop(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                    const gbs_opts *o, gbs_solve_info *info, int use_graph);
int gbs_mat_ensure_f32(gbs_mat A);

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

// Streaming loads of matrix data: read once per iteration, not kept in L1.
template <typename T>
__device__ __forceinline__ T gbs_ld_stream(const T *p) { return __ldcs(p); }

// Sum v[0..K) over the CTA with a fixed shuffle tree; every thread gets the
// totals.  s_red must hold K * GBS_WARPS values.  Deterministic.
template <typename T, int K>
__device__ __forceinline__ void gbs_block_sum(T (&v)[K], T *s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) s_red[k * GBS_WARPS + warp] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T t = lane < GBS_WARPS ? s_red[k * GBS_WARPS + lane] : T(0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        v[k] = t;
    }
    __syncthreads();
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
__device__ __forceinline__ bool gbs_grid_sync(gbs_grid_barrier *bar, unsigned long long timeout_ns,
                                              int where, bool skip, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int gen = gbs_ld_acquire(&bar->gen);
        if (!skip) {
            __threadfence();
            const unsigned int arrived = atomicAdd(&bar->count, 1u);
            if (arrived == gridDim.x - 1) {
                atomicExch(&bar->count, 0u);
                __threadfence();
                gbs_st_release(&bar->gen, gen + 1);
            }
        }
        const unsigned long long t0 = gbs_globaltimer();
        while (gbs_ld_acquire(&bar->gen) == gen) {
            if (gbs_ld_relaxed_int(&bar->error) != 0) { ok = 0; break; }
            if (gbs_globaltimer() - t0 > timeout_ns) {
                if (atomicCAS(&bar->error, 0, GBS_ERR_TIMEOUT) == 0) bar->where = where;
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
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

// Shared memory of one CSR tile.
template <typename V>
struct GbsTile {
    int32_t rp[GBS_TILE_ROWS + 1];
    int32_t col[GBS_TILE_NNZ];
    V val[GBS_TILE_NNZ];
};

// One CSR tile: rows [r0, r1) of y = A v.  For each row, epi(row, sum) is
// called by exactly one thread.  The tile's colidx/vals (contiguous in
// CSR) are staged in shared memory with coalesced streaming loads; then
// one thread per row accumulates its row left to right in storage order.
// The gathers of v use ordinary coherent loads, never the read-only path:
// inside a persistent kernel v changes between iterations (made visible
// by the grid barrier's acquire).  A tile holding a single row longer than
// GBS_TILE_NNZ is reduced by the whole CTA with a fixed tree.
// s_red must hold GBS_WARPS values.
template <typename V, typename Epi>
__device__ __forceinline__ void gbs_spmv_tile(const int32_t *__restrict__ rowptr,
                                              const int32_t *__restrict__ colidx,
                                              const V *__restrict__ vals, const V *v, int64_t r0,
                                              int64_t r1, GbsTile<V> &tl, V *s_red, Epi &epi)
{
    const int nrows = (int)(r1 - r0);
    for (int t = threadIdx.x; t <= nrows; t += GBS_BLOCK) tl.rp[t] = rowptr[r0 + t];
    __syncthreads();
    const int k0 = tl.rp[0], k1 = tl.rp[nrows];
    if (k1 - k0 <= GBS_TILE_NNZ) {
        constexpr int U = 4;
        for (int base = k0 + threadIdx.x; base < k1; base += GBS_BLOCK * U) {
            int c[U];
            V a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = base + u * GBS_BLOCK;
                c[u] = k < k1 ? gbs_ld_stream(colidx + k) : 0;
                a[u] = k < k1 ? gbs_ld_stream(vals + k) : V(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = base + u * GBS_BLOCK;
                if (k < k1) {
                    tl.col[k - k0] = c[u];
                    tl.val[k - k0] = a[u];
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nrows; t += GBS_BLOCK) {
            const int e = tl.rp[t + 1] - k0;
            V s = V(0);
#pragma unroll 4
            for (int k = tl.rp[t] - k0; k < e; ++k) s = gbs_mac(tl.val[k], v[tl.col[k]], s);
            epi(r0 + t, s);
        }
        __syncthreads();
    } else {
        V s = V(0);
        for (int k = k0 + threadIdx.x; k < k1; k += GBS_BLOCK)
            s = gbs_mac(gbs_ld_stream(vals + k), v[gbs_ld_stream(colidx + k)], s);
        V tot[1] = {s};
        gbs_block_sum<V, 1>(tot, s_red);
        if (threadIdx.x == 0) epi(r0, tot[0]);
        __syncthreads();
    }
}

#endif  // __CUDACC__
