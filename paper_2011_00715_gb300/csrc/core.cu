// Contexts, CSR matrices, vectors, Jacobi preconditioner, vector kernels
// and MatMult of the GB300 Jacobi-PCG library.
//
// Objects follow the PETSc front-end the paper describes (Sec. 4: Mat of
// type MATAIJ, Vec; Sec. 2: create, fill, solve).  Every kernel here is
// bandwidth-bound: no tensor cores (the path is sparse), coalesced loads,
// grids sized in multiples of the SM count.

#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <memory>
#include <new>
#include <vector>

#include "gbs_impl.cuh"

static const char *kVersion = "gbs 0.1 (sm_103a)";

int gbs_cuda_fail(cudaError_t e)
{
    (void)cudaGetLastError();  // clear a sticky launch error where possible
    if (e == cudaErrorMemoryAllocation) return GBS_ERR_OOM;
    return GBS_ERR_CUDA;
}

extern "C" const char *gbs_version(void) { return kVersion; }

extern "C" const char *gbs_status_string(int s)
{
    switch (s) {
    case GBS_OK: return "converged";
    case GBS_DIVERGED_ITS: return "iteration limit reached";
    case GBS_ERR_ARG: return "bad argument";
    case GBS_ERR_OOM: return "out of memory";
    case GBS_ERR_CUDA: return "CUDA error";
    case GBS_ERR_DIAG: return "diagonal entry missing or not positive";
    case GBS_ERR_INDEFINITE: return "indefinite operator or preconditioner";
    case GBS_ERR_NAN: return "NaN in a solver scalar";
    case GBS_ERR_TIMEOUT: return "device-side wait timed out";
    case GBS_ERR_STAGNATION: return "iterative refinement stagnated";
    case GBS_ERR_BUDGET: return "request exceeds the memory budget";
    case GBS_ERR_CSR: return "malformed CSR matrix";
    case GBS_ERR_NOT_FOUND: return "unknown ticket";
    case GBS_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

extern "C" int gbs_opts_default(gbs_opts *o)
{
    if (!o) return GBS_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->mode = GBS_MODE_FP64;
    o->algorithm = GBS_ALG_AUTO;
    o->inner_rtol = 1e-4;
    o->outer_maxit = 30;
    o->barrier_timeout_ms = 2000;
    o->graph_iters = 16;
    o->fault_skip_arrival = -1;
    return GBS_OK;
}

static int opts_valid(const gbs_opts *o)
{
    if (o->mode != GBS_MODE_FP64 && o->mode != GBS_MODE_MIXED) return 0;
    if (o->algorithm < GBS_ALG_AUTO || o->algorithm > GBS_ALG_CLUSTER) return 0;
    if (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0)) return 0;
    if (o->outer_maxit < 0 || o->barrier_timeout_ms <= 0 || o->graph_iters <= 0) return 0;
    if (o->batched_lanes != 0 && o->batched_lanes != 1 && o->batched_lanes != 2 &&
        o->batched_lanes != 4)
        return 0;
    if (o->persistent_ctas < 0) return 0;
    if (o->norm_type < GBS_NORM_UNPRECONDITIONED || o->norm_type > GBS_NORM_NATURAL) return 0;
    if (o->norm_type != GBS_NORM_UNPRECONDITIONED && o->mode == GBS_MODE_MIXED) return 0;
    if (o->no_rel16 != 0 && o->no_rel16 != 1) return 0;
    if (o->persistent_shape < 0 || o->persistent_shape > 2) return 0;
    if (o->persistent_lanes != 0 && o->persistent_lanes != 1 && o->persistent_lanes != 2) return 0;
    if (o->spmv_lanes != 0 && o->spmv_lanes != 1 && o->spmv_lanes != 2 && o->spmv_lanes != 4)
        return 0;
    if (o->reserved[0] != 0) return 0;
    return 1;
}

void gbs_count_launch(gbs_ctx ctx, int n) { ctx->launches += n; }

// ------------------------------------------------------------------ ctx --

extern "C" int gbs_ctx_create(int device, void *stream, const gbs_opts *opts, gbs_ctx *out)
{
    if (!out) return GBS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    GBS_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return GBS_ERR_ARG;
    gbs_opts o;
    gbs_opts_default(&o);
    if (opts) {
        if (!opts_valid(opts)) return GBS_ERR_ARG;
        o = *opts;
    }
    GBS_CUDA_TRY(cudaSetDevice(device));
    gbs_ctx c = (gbs_ctx)calloc(1, sizeof(*c));
    if (!c) return GBS_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->opts = o;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess) {
        c->num_sms = prop.multiProcessorCount;
        c->coop_supported = prop.cooperativeLaunch;
        e = cudaMallocHost(&c->pinned, 4096);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->devsmall, 4096);
    // zero once: the dot products' arrival counter (word 5) is left at zero
    // by every launch that uses it
    if (e == cudaSuccess) e = cudaMemset(c->devsmall, 0, 4096);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&c->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = ~(uint64_t)0;   // never trim at synchronisation
            e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e != cudaSuccess) {
        if (c->pool) cudaMemPoolDestroy(c->pool);
        if (c->pinned) cudaFreeHost(c->pinned);
        if (c->devsmall) cudaFree(c->devsmall);
        free(c);
        return gbs_cuda_fail(e);
    }
    c->last.status = GBS_OK;
    *out = c;
    return GBS_OK;
}

extern "C" int gbs_ctx_destroy(gbs_ctx c)
{
    if (!c) return GBS_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->scratch) cudaFreeAsync(c->scratch, c->stream);
    cudaStreamSynchronize(c->stream);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->devsmall) cudaFree(c->devsmall);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    cudaEventDestroy(c->ev0);
    cudaEventDestroy(c->ev1);
    free(c);
    return GBS_OK;
}

extern "C" int gbs_ctx_set_stream(gbs_ctx c, void *stream)
{
    if (!c) return GBS_ERR_ARG;
    // the matrices' arrays are ordered on the stream they were made on:
    // finish its work before later work and frees go to the new one
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->stream = (cudaStream_t)stream;
    return GBS_OK;
}

extern "C" int gbs_ctx_set_opts(gbs_ctx c, const gbs_opts *o)
{
    if (!c || !o || !opts_valid(o)) return GBS_ERR_ARG;
    c->opts = *o;
    return GBS_OK;
}

extern "C" int gbs_ctx_synchronize(gbs_ctx c)
{
    if (!c) return GBS_ERR_ARG;
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    // word 1 of devsmall: set by an asynchronous MatMult whose bulk copy
    // did not complete in time; reported here and cleared
    GBS_CUDA_TRY(cudaMemcpy(c->pinned, (int *)c->devsmall + 1, sizeof(int),
                            cudaMemcpyDeviceToHost));
    if (*(volatile int *)c->pinned) {
        GBS_CUDA_TRY(cudaMemset((int *)c->devsmall + 1, 0, sizeof(int)));
        return GBS_ERR_TIMEOUT;
    }
    return GBS_OK;
}

extern "C" int gbs_ctx_launch_count(gbs_ctx c, int64_t *count)
{
    if (!c || !count) return GBS_ERR_ARG;
    *count = c->launches;
    return GBS_OK;
}

// FP64 FMA issue-rate probe: every thread runs 8 independent dependent
// chains of fused multiply-adds, enough for the FP64 pipe to stay busy.  The
// sum is stored only if it equals an impossible value, so nothing is
// written in practice but nothing can be elided either.
__global__ void __launch_bounds__(512) k_fp64_fma_rate(int iters, double m, double cst, double *sink)
{
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 1.0 + 1e-3 * (double)(threadIdx.x + 37 * j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fma(v[j], m, cst);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += v[j];
    if (s == -1.0) sink[blockIdx.x & 7] = s;
}

extern "C" int gbs_probe_fp64_rate(gbs_ctx c, int iters, double *fma_per_s)
{
    if (!c || !fma_per_s || iters <= 0 || iters > (1 << 24)) return GBS_ERR_ARG;
    *fma_per_s = 0.0;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    int per_sm = 0;
    GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma_rate, 512, 0));
    if (per_sm < 1) per_sm = 1;
    const int g = c->num_sms * per_sm;
    double *sink = (double *)c->devsmall + 32;   // bytes 256..319 of the context's small buffer
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // a warm-up launch, then the timed one
    for (int rep = 0; e == cudaSuccess && rep < 2; ++rep) {
        if (rep == 1) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) {
            k_fp64_fma_rate<<<g, 512, 0, c->stream>>>(iters, 0.999999999, 1e-9, sink);
            gbs_count_launch(c);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return gbs_cuda_fail(e);
    if (ms <= 0.f) return GBS_ERR_CUDA;
    *fma_per_s = (double)g * 512.0 * 8.0 * (double)iters / ((double)ms * 1e-3);
    return GBS_OK;
}

int gbs_ctx_reserve(gbs_ctx c, size_t bytes, void **out)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes > c->scratch_bytes) {
        // from the context's pool as well (stream-ordered)
        GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (c->scratch) cudaFreeAsync(c->scratch, c->stream);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
        GBS_CUDA_TRY(cudaMallocFromPoolAsync(&c->scratch, bytes, c->pool, c->stream));
        c->scratch_bytes = bytes;
    }
    *out = c->scratch;
    return GBS_OK;
}

// --------------------------------------------------------------- matrix --

// Per-row structure check and Jacobi set-up: one thread per row.
// flags bit 0: malformed CSR; bit 1: a diagonal missing or <= 0.
__global__ void k_csr_validate(int64_t n, int64_t ncols, int64_t nnz, const int32_t *rowptr,
                               const int32_t *colidx, const double *vals, double *dinv,
                               float *dinv32, int *flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bad = 0;
    const int32_t b = rowptr[i], e = rowptr[i + 1];
    if (i == 0 && b != 0) bad |= 1;
    if (e < b || b < 0 || (int64_t)e > nnz) bad |= 1;
    double d = 0.0;
    int found = 0;
    if (!(bad & 1)) {
        int32_t prev = -1;
        for (int32_t k = b; k < e; ++k) {
            const int32_t c = colidx[k];
            if (c < 0 || c >= ncols || c <= prev) { bad |= 1; break; }
            prev = c;
            if (c == i) { d = vals[k]; found = 1; }
        }
    }
    if (!found || !(d > 0.0)) {
        bad |= 2;
        dinv[i] = 0.0;
        dinv32[i] = 0.0f;
    } else {
        dinv[i] = 1.0 / d;
        dinv32[i] = (float)(1.0 / d);
    }
    if (bad) atomicOr(flags, bad);
}

__global__ void k_diag_refresh(int64_t n, const int32_t *rowptr, const int32_t *colidx,
                               const double *vals, double *dinv, float *dinv32, int *flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    int found = 0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
        if (colidx[k] == i) { d = vals[k]; found = 1; }
    if (!found || !(d > 0.0)) {
        dinv[i] = 0.0;
        dinv32[i] = 0.0f;
        atomicOr(flags, 2);
    } else {
        dinv[i] = 1.0 / d;
        dinv32[i] = (float)(1.0 / d);
    }
}

__global__ void k_f64_to_f32(int64_t n, const double *a, float *b)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// colidx - row as int16 for every nonzero; *overflow = 1 if some difference
// does not fit (the compressed copy is then discarded).
__global__ void k_make_rel16(int64_t n, const int32_t *rowptr, const int32_t *colidx, int16_t *rel,
                             int *overflow)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int64_t d = (int64_t)colidx[k] - i;
            if (d < -32768 || d > 32767) atomicExch(overflow, 1);
            else rel[k] = (int16_t)d;
        }
    }
}

static int grid_for(gbs_ctx c, int64_t n, int per_sm = 4)
{
    int64_t g = (n + GBS_BLOCK - 1) / GBS_BLOCK;
    const int64_t cap = (int64_t)c->num_sms * per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// Split rows into warp tiles: at most GBS_WT_ROWS rows and GBS_WT_NNZ
// nonzeros each; a longer row is a tile of its own.  Greedy from the first
// row; where the next rows_cap rows hold at most GBS_WT_NNZ nonzeros
// together (the common case) the greedy rule takes them all, so the tile is
// cut with one test instead of a walk over its rows.  Needs monotone row
// pointers.
static void make_tiles(const int32_t *rowptr, int64_t n, std::vector<int32_t> &tiles, int *maxrow,
                       int rows_cap = GBS_WT_ROWS)
{
    tiles.clear();
    tiles.reserve((size_t)(n / rows_cap) + 2);
    tiles.push_back(0);
    int mr = 0;   // longest row
    for (int64_t i = 0; i < n; ++i) {
        const int rn = rowptr[i + 1] - rowptr[i];
        mr = rn > mr ? rn : mr;
    }
    int64_t start = 0;
    while (start < n) {
        int64_t end = start + rows_cap < n ? start + rows_cap : n;
        if (rowptr[end] - rowptr[start] > GBS_WT_NNZ) {
            end = start;
            while (end < n && end - start < rows_cap) {
                const int64_t rn = rowptr[end + 1] - rowptr[end];
                if (end > start && rowptr[end + 1] - rowptr[start] > GBS_WT_NNZ) break;
                ++end;
                if (rn > GBS_WT_NNZ) break;  // a long row stays alone
            }
        }
        tiles.push_back((int32_t)end);
        start = end;
    }
    *maxrow = mr;
}

// Pipeline geometry: every stage must hold the largest copied tile (the
// 16-byte-aligned supersets of its values, column indices and row pointers).
static GbsPipeCfg make_pipe_cfg(const std::vector<int32_t> &tiles, const int32_t *rowptr,
                                int vsize, int isize = 4)
{
    const int E = 16 / vsize, CE = 16 / isize;
    int vcap = 0, ccap = 0, rcap = 0;
    for (size_t t = 0; t + 1 < tiles.size(); ++t) {
        const int r0 = tiles[t], r1 = tiles[t + 1], k0 = rowptr[r0], k1 = rowptr[r1];
        if (k1 - k0 > GBS_WT_NNZ) continue;
        const int v = ((k1 + E - 1) & ~(E - 1)) - (k0 & ~(E - 1));
        const int c = ((k1 + CE - 1) & ~(CE - 1)) - (k0 & ~(CE - 1));
        const int r = ((r1 + 4) & ~3) - (r0 & ~3);
        if (v > vcap) vcap = v;
        if (c > ccap) ccap = c;
        if (r > rcap) rcap = r;
    }
    auto r16 = [](int b) { return (b + 15) & ~15; };
    GbsPipeCfg cfg;
    cfg.coloff = r16(vsize * vcap);
    cfg.rpoff = cfg.coloff + r16(isize * ccap);
    cfg.sbytes = cfg.rpoff + r16(4 * rcap);
    if (cfg.sbytes < 16) cfg.sbytes = 16;
    cfg.stages = GBS_WARP_STAGE_BYTES / cfg.sbytes;
    if (cfg.stages > GBS_MAX_STAGES) cfg.stages = GBS_MAX_STAGES;
    return cfg;   // at least 2 stages: a full tile needs at most 6320 bytes
}

cudaError_t gbs_mat_alloc(gbs_ctx c, void **p, size_t bytes)
{
    return cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream);
}

void gbs_mat_release(gbs_ctx c, void *p)
{
    if (p) cudaFreeAsync(p, c->stream);
}

static void mat_free(gbs_mat A)
{
    if (!A) return;
    gbs_ctx c = A->ctx;
    gbs_mat_release(c, A->rowptr);
    gbs_mat_release(c, A->colidx);
    gbs_mat_release(c, A->vals);
    gbs_mat_release(c, A->vals32);
    gbs_mat_release(c, A->dinv);
    gbs_mat_release(c, A->dinv32);
    gbs_mat_release(c, A->tiles);
    gbs_mat_release(c, A->tdesc);
    gbs_mat_release(c, A->tdesc_lanes[1]);
    gbs_mat_release(c, A->tdesc_lanes[2]);
    gbs_mat_release(c, A->colrel16);
    // the coordinate maps come from the assembly's own allocations
    cudaFree(A->coo_seg);
    cudaFree(A->coo_perm);
    free(A);
}

int gbs_mat_ensure_lane_tiling(gbs_mat A, int li)
{
    if (li < 0 || li > 2) return GBS_ERR_ARG;
    if (li == 0) {
        A->tdesc_lanes[0] = A->tdesc;
        A->ntiles_lanes[0] = A->ntiles;
        A->pipe64_lanes[0] = A->pipe64;
        A->pipe32_lanes[0] = A->pipe32;
        A->pipe16_lanes[0] = A->pipe16;
        A->pipe64r_lanes[0] = A->pipe64r;
        return GBS_OK;
    }
    if (A->tdesc_lanes[li]) return GBS_OK;
    gbs_ctx c = A->ctx;
    std::vector<int32_t> hrp((size_t)A->n + 1), tiles;
    GBS_CUDA_TRY(cudaMemcpyAsync(hrp.data(), A->rowptr, sizeof(int32_t) * hrp.size(),
                                 cudaMemcpyDeviceToHost, c->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    int mr = 0;
    make_tiles(hrp.data(), A->n, tiles, &mr, GBS_WT_ROWS >> li);
    std::vector<int32_t> tdesc(2 * tiles.size());
    for (size_t t = 0; t < tiles.size(); ++t) {
        tdesc[2 * t] = tiles[t];
        tdesc[2 * t + 1] = hrp[tiles[t]];
    }
    int32_t *d = nullptr;
    GBS_CUDA_TRY(gbs_mat_alloc(c, (void **)&d, sizeof(int32_t) * tdesc.size()));
    cudaError_t e = cudaMemcpyAsync(d, tdesc.data(), sizeof(int32_t) * tdesc.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // tdesc is a stack vector
    if (e != cudaSuccess) {
        gbs_mat_release(c, d);
        return gbs_cuda_fail(e);
    }
    A->tdesc_lanes[li] = d;
    A->ntiles_lanes[li] = (int64_t)tiles.size() - 1;
    A->pipe64_lanes[li] = make_pipe_cfg(tiles, hrp.data(), 8);
    A->pipe32_lanes[li] = make_pipe_cfg(tiles, hrp.data(), 4);
    A->pipe16_lanes[li] = make_pipe_cfg(tiles, hrp.data(), 4, 2);
    A->pipe64r_lanes[li] = make_pipe_cfg(tiles, hrp.data(), 8, 2);
    return GBS_OK;
}

extern "C" int gbs_mat_create_aij(gbs_ctx c, int64_t nrows, int64_t ncols, const int32_t *rowptr,
                                  const int32_t *colidx, const double *vals, int memspace,
                                  gbs_mat *out)
{
    if (!c || !out || nrows < 0 || ncols < 0 || !rowptr) return GBS_ERR_ARG;
    if (memspace != GBS_MEM_HOST && memspace != GBS_MEM_DEVICE) return GBS_ERR_ARG;
    if (nrows >= (int64_t)INT32_MAX || ncols >= (int64_t)INT32_MAX) return GBS_ERR_ARG;
    *out = nullptr;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    // the row pointers are needed on the host for tiling: the caller's own
    // array when it is host memory (read, not copied), else a copy
    std::unique_ptr<int32_t[]> hrp_copy;
    const int32_t *hrp = rowptr;
    if (memspace == GBS_MEM_DEVICE) {
        hrp_copy.reset(new (std::nothrow) int32_t[(size_t)nrows + 1]);
        if (!hrp_copy) return GBS_ERR_OOM;
        GBS_CUDA_TRY(cudaMemcpyAsync(hrp_copy.get(), rowptr, sizeof(int32_t) * (nrows + 1),
                                     cudaMemcpyDeviceToHost, c->stream));
        GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        hrp = hrp_copy.get();
    }
    if (hrp[0] != 0) return GBS_ERR_CSR;
    // monotone row pointers (one pass without early exit), checked before
    // hrp[n] sizes any copy
    int bad = 0;
    for (int64_t i = 0; i < nrows; ++i) bad |= hrp[i + 1] < hrp[i];
    if (bad) return GBS_ERR_CSR;
    const int64_t nnz = hrp[nrows];
    if (nnz > 0 && (!colidx || !vals)) return GBS_ERR_ARG;

    gbs_mat A = (gbs_mat)calloc(1, sizeof(*A));
    if (!A) return GBS_ERR_OOM;
    A->ctx = c;
    A->n = nrows;
    A->ncols = ncols;
    A->nnz = nnz;
    // allocations padded to 16 bytes so vector loads never leave the buffer
    const size_t pad_nnz = (size_t)((nnz + 4) & ~(int64_t)3);
    const size_t pad_n = (size_t)((nrows + 4) & ~(int64_t)3);
    cudaError_t e = gbs_mat_alloc(c, (void **)&A->rowptr, sizeof(int32_t) * (pad_n + 1));
    if (e == cudaSuccess) e = gbs_mat_alloc(c, (void **)&A->colidx, sizeof(int32_t) * pad_nnz);
    if (e == cudaSuccess) e = gbs_mat_alloc(c, (void **)&A->vals, sizeof(double) * pad_nnz);
    if (e == cudaSuccess) e = gbs_mat_alloc(c, (void **)&A->dinv, sizeof(double) * pad_n);
    if (e == cudaSuccess) e = gbs_mat_alloc(c, (void **)&A->dinv32, sizeof(float) * pad_n);
    // the bulk of the matrix goes to the device first, so the copies run
    // while the host cuts the tiles
    const cudaMemcpyKind kind =
        memspace == GBS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(A->colidx, colidx, sizeof(int32_t) * nnz, kind, c->stream);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(A->vals, vals, sizeof(double) * nnz, kind, c->stream);
    // only the padding after the nnz entries needs zeros: the copies fill the rest
    if (e == cudaSuccess)
        e = cudaMemsetAsync(A->colidx + nnz, 0, sizeof(int32_t) * (pad_nnz - nnz), c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(A->vals + nnz, 0, sizeof(double) * (pad_nnz - nnz), c->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        mat_free(A);
        return gbs_cuda_fail(e);
    }
    std::vector<int32_t> tiles;
    make_tiles(hrp, nrows, tiles, &A->max_row_nnz);
    A->ntiles = (int64_t)tiles.size() - 1;
    A->pipe64 = make_pipe_cfg(tiles, hrp, 8);
    A->pipe32 = make_pipe_cfg(tiles, hrp, 4);
    A->pipe16 = make_pipe_cfg(tiles, hrp, 4, 2);
    A->pipe64r = make_pipe_cfg(tiles, hrp, 8, 2);
    std::vector<int32_t> tdesc(2 * tiles.size());
    for (size_t t = 0; t < tiles.size(); ++t) {
        tdesc[2 * t] = tiles[t];
        tdesc[2 * t + 1] = hrp[tiles[t]];
    }
    e = gbs_mat_alloc(c, (void **)&A->tiles, sizeof(int32_t) * tiles.size());
    if (e == cudaSuccess) e = gbs_mat_alloc(c, (void **)&A->tdesc, sizeof(int32_t) * tdesc.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(A->rowptr, hrp, sizeof(int32_t) * (nrows + 1),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(A->tiles, tiles.data(), sizeof(int32_t) * tiles.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(A->tdesc, tdesc.data(), sizeof(int32_t) * tdesc.size(),
                            cudaMemcpyHostToDevice, c->stream);
    int *devflags = (int *)c->devsmall;
    if (e == cudaSuccess) e = cudaMemsetAsync(devflags, 0, sizeof(int), c->stream);
    if (e == cudaSuccess && nrows > 0) {
        const int g = (int)((nrows + 255) / 256);
        k_csr_validate<<<g, 256, 0, c->stream>>>(nrows, ncols, nnz, A->rowptr, A->colidx,
                                                  A->vals, A->dinv, A->dinv32, devflags);
        gbs_count_launch(c);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->pinned, devflags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        mat_free(A);
        return gbs_cuda_fail(e);
    }
    const int flags = *(volatile int *)c->pinned;
    if (flags & 1) {
        mat_free(A);
        return GBS_ERR_CSR;
    }
    A->diag_ok = (flags & 2) ? 0 : 1;
    if (nrows != ncols) A->diag_ok = 0;
    // the creation tiling is the one-lane tiling: registered now, so every
    // launch-shape decision sees its tile count from the first solve on
    (void)gbs_mat_ensure_lane_tiling(A, 0);
    *out = A;
    return GBS_OK;
}

// The compressed column indices (Challenge A7: with 32-bit indices an FP64
// nonzero streams 12 bytes and an FP32 one 8; 16-bit offsets from the row
// make that 10 and 6) where every |col - row| of the matrix fits in int16.
int gbs_mat_ensure_rel16(gbs_mat A)
{
    if (A->rel16_state != 0) return GBS_OK;
    if (A->nnz == 0 || A->n > (int64_t)INT32_MAX) {
        A->rel16_state = -1;
        return GBS_OK;
    }
    gbs_ctx c = A->ctx;
    const size_t pad16 = (size_t)((A->nnz + 15) & ~(int64_t)7);
    int16_t *rel = nullptr;
    GBS_CUDA_TRY(gbs_mat_alloc(c, (void **)&rel, sizeof(int16_t) * pad16));
    int *flag = (int *)c->devsmall + 2;   // word 2 of the context's small device buffer
    cudaError_t e = cudaMemsetAsync(rel, 0, sizeof(int16_t) * pad16, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        k_make_rel16<<<grid_for(c, A->n), GBS_BLOCK, 0, c->stream>>>(A->n, A->rowptr, A->colidx, rel,
                                                                     flag);
        gbs_count_launch(c);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->pinned, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        gbs_mat_release(c, rel);
        return gbs_cuda_fail(e);
    }
    if (*(volatile int *)c->pinned) {
        gbs_mat_release(c, rel);
        A->rel16_state = -1;
    } else {
        A->colrel16 = rel;
        A->rel16_state = 1;
    }
    return GBS_OK;
}

int gbs_mat_ensure_f32(gbs_mat A)
{
    if (A->vals32 || A->nnz == 0) {
        if (!A->vals32) GBS_CUDA_TRY(gbs_mat_alloc(A->ctx, (void **)&A->vals32, 16));
        return gbs_mat_ensure_rel16(A);
    }
    gbs_ctx c = A->ctx;
    const size_t pad_nnz = (size_t)((A->nnz + 4) & ~(int64_t)3);
    GBS_CUDA_TRY(gbs_mat_alloc(A->ctx, (void **)&A->vals32, sizeof(float) * pad_nnz));
    GBS_CUDA_TRY(cudaMemsetAsync(A->vals32, 0, sizeof(float) * pad_nnz, c->stream));
    k_f64_to_f32<<<grid_for(c, A->nnz), GBS_BLOCK, 0, c->stream>>>(A->nnz, A->vals, A->vals32);
    gbs_count_launch(c);
    GBS_CUDA_TRY(cudaGetLastError());
    return gbs_mat_ensure_rel16(A);
}

extern "C" int gbs_mat_get_csr(gbs_mat A, int32_t *rowptr, int32_t *colidx, double *vals,
                               int memspace)
{
    if (!A) return GBS_ERR_ARG;
    if (memspace != GBS_MEM_HOST && memspace != GBS_MEM_DEVICE) return GBS_ERR_ARG;
    gbs_ctx c = A->ctx;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    const cudaMemcpyKind kind =
        memspace == GBS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (rowptr)
        GBS_CUDA_TRY(cudaMemcpyAsync(rowptr, A->rowptr, sizeof(int32_t) * (A->n + 1), kind, c->stream));
    if (colidx && A->nnz > 0)
        GBS_CUDA_TRY(cudaMemcpyAsync(colidx, A->colidx, sizeof(int32_t) * A->nnz, kind, c->stream));
    if (vals && A->nnz > 0)
        GBS_CUDA_TRY(cudaMemcpyAsync(vals, A->vals, sizeof(double) * A->nnz, kind, c->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GBS_OK;
}

extern "C" int gbs_mat_set_values(gbs_mat A, const double *vals, int memspace)
{
    if (!A || (!vals && A->nnz > 0)) return GBS_ERR_ARG;
    if (memspace != GBS_MEM_HOST && memspace != GBS_MEM_DEVICE) return GBS_ERR_ARG;
    gbs_ctx c = A->ctx;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    if (A->nnz > 0)
        GBS_CUDA_TRY(cudaMemcpyAsync(A->vals, vals, sizeof(double) * A->nnz,
                                     memspace == GBS_MEM_HOST ? cudaMemcpyHostToDevice
                                                              : cudaMemcpyDeviceToDevice,
                                     c->stream));
    int *devflags = (int *)c->devsmall;
    GBS_CUDA_TRY(cudaMemsetAsync(devflags, 0, sizeof(int), c->stream));
    if (A->n > 0) {
        k_diag_refresh<<<(int)((A->n + 255) / 256), 256, 0, c->stream>>>(
            A->n, A->rowptr, A->colidx, A->vals, A->dinv, A->dinv32, devflags);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    if (A->vals32 && A->nnz > 0) {
        k_f64_to_f32<<<grid_for(c, A->nnz), GBS_BLOCK, 0, c->stream>>>(A->nnz, A->vals,
                                                                       A->vals32);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    GBS_CUDA_TRY(cudaMemcpyAsync(c->pinned, devflags, sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream));
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    A->diag_ok = ((*(volatile int *)c->pinned) & 2) || A->n != A->ncols ? 0 : 1;
    return GBS_OK;
}

extern "C" int gbs_mat_get_info(gbs_mat A, int64_t *nrows, int64_t *ncols, int64_t *nnz)
{
    if (!A) return GBS_ERR_ARG;
    if (nrows) *nrows = A->n;
    if (ncols) *ncols = A->ncols;
    if (nnz) *nnz = A->nnz;
    return GBS_OK;
}

extern "C" int gbs_mat_get_device(gbs_mat A, int *device)
{
    if (!A || !device) return GBS_ERR_ARG;
    *device = A->ctx->device;
    return GBS_OK;
}

extern "C" int gbs_mat_destroy(gbs_mat A)
{
    if (!A) return GBS_OK;
    cudaSetDevice(A->ctx->device);
    cudaStreamSynchronize(A->ctx->stream);
    mat_free(A);
    return GBS_OK;
}

// ------------------------------------------------------------- MatMult --

template <typename V>
struct StoreEpi {
    V *y;
    uint64_t pol;
    __device__ __forceinline__ void operator()(int64_t row, V s, V) const { gbs_st(y + row, s, pol); }
};

// MatMult over warp tiles: CTA c takes an even share of the tiles, its
// warps claim them one by one through their bulk-copy pipelines of WB
// bytes each.  A copy that does not complete within 2 s sets *err, which
// gbs_ctx_synchronize reports as GBS_ERR_TIMEOUT.  Two launch shapes: 8
// warps per CTA with 12.8 KB rings (2 CTAs, 16 warps per SM), or with
// 6.4 KB rings and at most 64 registers (4 CTAs, 32 warps per SM) whenever
// a stage fits in 6.4 KB (every tile of at most 512 nonzeros does) — twice
// the warps hide the gather latency better than deeper rings, even with a
// single stage per warp (measured: 7-point 128^3 FP64 51 -> 41 us, 27-point
// 96^3 FP32 43 -> 37 us).  2^LOG_L lanes share a row (tiles of 32 / 2^LOG_L
// rows, from the matching lane tiling).
template <typename V, typename IX, int WB, int MINB, int LOG_L>
__global__ void __launch_bounds__(GBS_BLOCK, MINB) k_spmv(int64_t ntiles, const int32_t *tdesc,
                                                          const int32_t *rowptr, const IX *colidx,
                                                          const V *vals, const V *x, V *y,
                                                          GbsPipeCfg cfg, int *err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ GbsWarpQ s_q[GBS_WARPS];
    __shared__ int s_next;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    gbs_warpq_init(s_q[warp]);
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const uint64_t ps = gbs_policy_stream(), pk = gbs_policy_keep();
    StoreEpi<V> epi{y, pk};
    uint32_t parity = 0;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const bool ok = gbs_spmv_pipe<V, IX, LOG_L>(tdesc, t0, t1, &s_next, rowptr, colidx, vals, x,
                                         smem + (size_t)warp * WB, s_q[warp], parity, cfg, ps, pk,
                                         2000000000ull, epi);
    if (!ok && lane == 0) atomicExch(err, 1);
}

template <typename V, typename IX, int WB, int MINB, int LOG_L>
static int spmv_launch_shape(gbs_ctx c, gbs_mat A, const V *vals, const IX *colidx, const V *x, V *y,
                             GbsPipeCfg cfg)
{
    const void *fn = (const void *)k_spmv<V, IX, WB, MINB, LOG_L>;
    const size_t smem = (size_t)WB * GBS_WARPS;
    GBS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, GBS_BLOCK, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = A->ntiles_lanes[LOG_L];
    const int64_t need = (ntiles + GBS_WARPS - 1) / GBS_WARPS;
    const int64_t cap = (int64_t)c->num_sms * per_sm;
    const int g = (int)(need < cap ? need : cap);
    int *err = (int *)c->devsmall + 1;   // word 1 of the context's small device buffer
    k_spmv<V, IX, WB, MINB, LOG_L><<<g, GBS_BLOCK, smem, c->stream>>>(
        ntiles, A->tdesc_lanes[LOG_L], A->rowptr, colidx, vals, x, y, cfg, err);
    gbs_count_launch(c);
    GBS_CUDA_TRY(cudaGetLastError());
    return GBS_OK;
}

template <typename V, typename IX, int LOG_L>
static int spmv_launch_l(gbs_ctx c, gbs_mat A, const V *vals, const IX *colidx, GbsPipeCfg cfg,
                         const V *x, V *y)
{
    constexpr int kSmallRing = GBS_WARP_STAGE_BYTES / 2;
    const int small_stages = kSmallRing / cfg.sbytes;
    if (small_stages >= 1) {
        cfg.stages = small_stages < GBS_MAX_STAGES ? small_stages : GBS_MAX_STAGES;
        return spmv_launch_shape<V, IX, kSmallRing, 4, LOG_L>(c, A, vals, colidx, x, y, cfg);
    }
    return spmv_launch_shape<V, IX, GBS_WARP_STAGE_BYTES, 1, LOG_L>(c, A, vals, colidx, x, y, cfg);
}

// Lanes per row of MatMult (log2): the context's spmv_lanes, else two lanes
// for rows of more than 16 nonzeros (27-point stencils: half the lanes of a
// one-lane tile would idle on the tail of every row) and one otherwise.
static int spmv_log_lanes(gbs_mat A)
{
    const int o = A->ctx->opts.spmv_lanes;
    if (o > 0) return o == 1 ? 0 : o == 2 ? 1 : 2;
    return A->max_row_nnz > 16 ? 1 : 0;
}

// MatMult with the tiling for li = log2(lanes per row); cfgs[li] is the
// stage layout of that tiling for these values and indices.
template <typename V, typename IX>
static int spmv_launch(gbs_ctx c, gbs_mat A, const V *vals, const IX *colidx, const GbsPipeCfg *cfgs,
                       int li, const V *x, V *y)
{
    const int st = gbs_mat_ensure_lane_tiling(A, li);
    if (st) return st;
    if (li == 1) return spmv_launch_l<V, IX, 1>(c, A, vals, colidx, cfgs[1], x, y);
    if (li == 2) return spmv_launch_l<V, IX, 2>(c, A, vals, colidx, cfgs[2], x, y);
    return spmv_launch_l<V, IX, 0>(c, A, vals, colidx, cfgs[0], x, y);
}

extern "C" int gbs_mat_mult(gbs_mat A, gbs_vec x, gbs_vec y)
{
    if (!A || !x || !y) return GBS_ERR_ARG;
    if (x->n != A->ncols || y->n != A->n || x->dtype != y->dtype) return GBS_ERR_ARG;
    if (x->data == y->data && A->n > 0) return GBS_ERR_ARG;
    gbs_ctx c = A->ctx;
    if (A->n == 0) return GBS_OK;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    const int li = spmv_log_lanes(A);
    if (x->dtype == GBS_F64) {
        int st = gbs_mat_ensure_rel16(A);
        if (st) return st;
        if (A->colrel16 && !c->opts.no_rel16)
            return spmv_launch<double, int16_t>(c, A, A->vals, A->colrel16, A->pipe64r_lanes, li,
                                                (const double *)x->data, (double *)y->data);
        return spmv_launch<double, int32_t>(c, A, A->vals, A->colidx, A->pipe64_lanes, li,
                                            (const double *)x->data, (double *)y->data);
    }
    int st = gbs_mat_ensure_f32(A);
    if (st) return st;
    // FP32: the compressed 16-bit column indices where the matrix allows them
    if (A->colrel16 && !c->opts.no_rel16)
        return spmv_launch<float, int16_t>(c, A, A->vals32, A->colrel16, A->pipe16_lanes, li,
                                           (const float *)x->data, (float *)y->data);
    return spmv_launch<float, int32_t>(c, A, A->vals32, A->colidx, A->pipe32_lanes, li,
                                       (const float *)x->data, (float *)y->data);
}

// --------------------------------------------------------------- vector --

static size_t dsize(int dtype) { return dtype == GBS_F64 ? 8 : 4; }

extern "C" int gbs_vec_create(gbs_ctx c, int64_t n, int dtype, gbs_vec *out)
{
    if (!c || !out || n < 0 || (dtype != GBS_F64 && dtype != GBS_F32)) return GBS_ERR_ARG;
    *out = nullptr;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    gbs_vec v = (gbs_vec)calloc(1, sizeof(*v));
    if (!v) return GBS_ERR_OOM;
    const size_t bytes = dsize(dtype) * (size_t)((n + 4) & ~(int64_t)3);
    cudaError_t e = cudaMalloc(&v->data, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->data, 0, bytes, c->stream);
    if (e != cudaSuccess) {
        if (v->data) cudaFree(v->data);
        free(v);
        return gbs_cuda_fail(e);
    }
    v->ctx = c;
    v->n = n;
    v->dtype = dtype;
    v->owned = 1;
    *out = v;
    return GBS_OK;
}

extern "C" int gbs_vec_wrap(gbs_ctx c, void *ptr, int64_t n, int dtype, gbs_vec *out)
{
    if (!c || !out || n < 0 || (dtype != GBS_F64 && dtype != GBS_F32)) return GBS_ERR_ARG;
    if (n > 0 && !ptr) return GBS_ERR_ARG;
    if (((uintptr_t)ptr) % dsize(dtype) != 0) return GBS_ERR_ARG;
    gbs_vec v = (gbs_vec)calloc(1, sizeof(*v));
    if (!v) return GBS_ERR_OOM;
    v->ctx = c;
    v->data = ptr;
    v->n = n;
    v->dtype = dtype;
    v->owned = 0;
    *out = v;
    return GBS_OK;
}

extern "C" int gbs_vec_destroy(gbs_vec v)
{
    if (!v) return GBS_OK;
    if (v->owned && v->data) {
        cudaSetDevice(v->ctx->device);
        cudaStreamSynchronize(v->ctx->stream);
        cudaFree(v->data);
    }
    free(v);
    return GBS_OK;
}

extern "C" int gbs_vec_get_info(gbs_vec v, int64_t *n, int *dtype, void **p)
{
    if (!v) return GBS_ERR_ARG;
    if (n) *n = v->n;
    if (dtype) *dtype = v->dtype;
    if (p) *p = v->data;
    return GBS_OK;
}

extern "C" int gbs_vec_set_values(gbs_vec v, const void *src, int memspace)
{
    if (!v || (!src && v->n > 0)) return GBS_ERR_ARG;
    if (memspace != GBS_MEM_HOST && memspace != GBS_MEM_DEVICE) return GBS_ERR_ARG;
    if (v->n == 0) return GBS_OK;
    GBS_CUDA_TRY(cudaSetDevice(v->ctx->device));
    GBS_CUDA_TRY(cudaMemcpyAsync(v->data, src, dsize(v->dtype) * v->n,
                                 memspace == GBS_MEM_HOST ? cudaMemcpyHostToDevice
                                                          : cudaMemcpyDeviceToDevice,
                                 v->ctx->stream));
    return GBS_OK;
}

extern "C" int gbs_vec_get_values(gbs_vec v, void *dst, int memspace)
{
    if (!v || (!dst && v->n > 0)) return GBS_ERR_ARG;
    if (memspace != GBS_MEM_HOST && memspace != GBS_MEM_DEVICE) return GBS_ERR_ARG;
    if (v->n == 0) return GBS_OK;
    GBS_CUDA_TRY(cudaSetDevice(v->ctx->device));
    GBS_CUDA_TRY(cudaMemcpyAsync(dst, v->data, dsize(v->dtype) * v->n,
                                 memspace == GBS_MEM_HOST ? cudaMemcpyDeviceToHost
                                                          : cudaMemcpyDeviceToDevice,
                                 v->ctx->stream));
    if (memspace == GBS_MEM_HOST) GBS_CUDA_TRY(cudaStreamSynchronize(v->ctx->stream));
    return GBS_OK;
}

// Rounded product (never fused into an add).
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }

// Elementwise kernels.  op: 0 set, 1 copy(y=x), 2 axpy(y=a x+y), 3 aypx(y=x+a y),
// 4 pointwise (y = x * w), 5 jacobi (y = dinv * x).  AXPY and AYPX round the
// exact a x + y once (one fused multiply-add per entry): on this GPU FP64
// operations are scarce enough that a separate multiply and add would make
// an FP64 AXPY ALU-bound instead of bandwidth-bound.
template <typename TX, typename TY>
__global__ void k_elementwise(int op, int64_t n, double a, const TX *__restrict__ x,
                              const TY *__restrict__ w, TY *__restrict__ y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        switch (op) {
        case 0: y[i] = (TY)a; break;
        case 1: y[i] = (TY)x[i]; break;
        case 2: y[i] = fma((TY)a, (TY)x[i], y[i]); break;
        case 3: y[i] = fma((TY)a, y[i], (TY)x[i]); break;
        case 4: y[i] = rn_mul((TY)x[i], w[i]); break;
        }
    }
}

static int launch_elementwise(int op, gbs_vec y, double a, gbs_vec x, gbs_vec w)
{
    gbs_ctx c = y->ctx;
    if (y->n == 0) return GBS_OK;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    const int g = grid_for(c, y->n, 8);
    const void *xd = x ? x->data : nullptr;
    const void *wd = w ? w->data : nullptr;
    const int xt = x ? x->dtype : y->dtype;
    if (y->dtype == GBS_F64) {
        if (xt == GBS_F64)
            k_elementwise<double, double><<<g, GBS_BLOCK, 0, c->stream>>>(
                op, y->n, a, (const double *)xd, (const double *)wd, (double *)y->data);
        else
            k_elementwise<float, double><<<g, GBS_BLOCK, 0, c->stream>>>(
                op, y->n, a, (const float *)xd, (const double *)wd, (double *)y->data);
    } else {
        if (xt == GBS_F64)
            k_elementwise<double, float><<<g, GBS_BLOCK, 0, c->stream>>>(
                op, y->n, a, (const double *)xd, (const float *)wd, (float *)y->data);
        else
            k_elementwise<float, float><<<g, GBS_BLOCK, 0, c->stream>>>(
                op, y->n, a, (const float *)xd, (const float *)wd, (float *)y->data);
    }
    gbs_count_launch(c);
    GBS_CUDA_TRY(cudaGetLastError());
    return GBS_OK;
}

extern "C" int gbs_vec_set(gbs_vec v, double a)
{
    if (!v) return GBS_ERR_ARG;
    return launch_elementwise(0, v, a, nullptr, nullptr);
}

extern "C" int gbs_vec_copy(gbs_vec x, gbs_vec y)
{
    if (!x || !y || x->n != y->n || x->ctx != y->ctx) return GBS_ERR_ARG;
    if (x->data == y->data) return GBS_OK;
    return launch_elementwise(1, y, 0.0, x, nullptr);
}

extern "C" int gbs_vec_axpy(gbs_vec y, double a, gbs_vec x)
{
    if (!x || !y || x->n != y->n || x->dtype != y->dtype) return GBS_ERR_ARG;
    return launch_elementwise(2, y, a, x, nullptr);
}

extern "C" int gbs_vec_aypx(gbs_vec y, double b, gbs_vec x)
{
    if (!x || !y || x->n != y->n || x->dtype != y->dtype) return GBS_ERR_ARG;
    return launch_elementwise(3, y, b, x, nullptr);
}

extern "C" int gbs_vec_pointwise_mult(gbs_vec w, gbs_vec x, gbs_vec y)
{
    if (!w || !x || !y || w->n != x->n || x->n != y->n) return GBS_ERR_ARG;
    if (w->dtype != x->dtype || x->dtype != y->dtype) return GBS_ERR_ARG;
    return launch_elementwise(4, w, 0.0, x, y);
}

// Dot product in two fixed-order stages within one launch: each CTA sums a
// grid-stride slice (thread partials, then a shuffle tree), the last CTA to
// finish adds the CTA partials in index order.  out[0] (FP64) gets the
// total, or its square root (VecNorm), taken in T and then widened.
template <typename T>
__global__ void __launch_bounds__(GBS_BLOCK) k_dot(int64_t n, const T *__restrict__ x,
                                                   const T *__restrict__ y, T *partials,
                                                   unsigned int *counter, double *out, int root)
{
    __shared__ T s_red[GBS_WARPS];
    __shared__ bool s_last;
    T acc[1] = {T(0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc[0] += x[i] * y[i];
    gbs_block_sum<T, 1>(acc, s_red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = acc[0];
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        T tot[1];
        gbs_grid_sum<T, 1>(partials, 0, gridDim.x, tot, s_red);
        if (threadIdx.x == 0) {
            out[0] = (double)(root ? sqrt(tot[0]) : tot[0]);
            *counter = 0;
        }
    }
}

// Launch the dot product (or norm) of x and y into out (device memory, or
// the context's pinned host buffer, which the device writes through the
// unified address space) on the context's stream, without waiting for it.
// The per-CTA partials are in the context's scratch: every later user of
// the scratch is ordered after this launch on the same stream, and growing
// the scratch synchronises the stream first.  The arrival counter is word 5
// of the context's small device buffer, zero at creation and reset by the
// last CTA of every launch, so no clearing copy precedes the kernel.
static int vec_dot_launch(gbs_vec x, gbs_vec y, double *dev_out, int root)
{
    gbs_ctx c = x->ctx;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    if (x->n == 0) {
        GBS_CUDA_TRY(cudaMemsetAsync(dev_out, 0, sizeof(double), c->stream));
        return GBS_OK;
    }
    const int g = grid_for(c, x->n, 4);
    void *scr = nullptr;
    int st = gbs_ctx_reserve(c, 64 + 8 * (size_t)g, &scr);
    if (st) return st;
    unsigned int *counter = (unsigned int *)c->devsmall + 5;
    void *partials = (char *)scr + 64;
    if (x->dtype == GBS_F64)
        k_dot<double><<<g, GBS_BLOCK, 0, c->stream>>>(x->n, (const double *)x->data,
                                                      (const double *)y->data,
                                                      (double *)partials, counter, dev_out, root);
    else
        k_dot<float><<<g, GBS_BLOCK, 0, c->stream>>>(x->n, (const float *)x->data,
                                                     (const float *)y->data, (float *)partials,
                                                     counter, dev_out, root);
    gbs_count_launch(c);
    GBS_CUDA_TRY(cudaGetLastError());
    return GBS_OK;
}

// Synchronous form: the last CTA writes the result straight into the
// context's pinned host buffer (no copy operation after the kernel).
static int vec_dot_sync(gbs_vec x, gbs_vec y, double *out, int root)
{
    gbs_ctx c = x->ctx;
    if (x->n == 0) {
        *out = 0.0;
        return GBS_OK;
    }
    int st = vec_dot_launch(x, y, (double *)c->pinned, root);
    if (st) return st;
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *out = *(volatile double *)c->pinned;
    return GBS_OK;
}

extern "C" int gbs_vec_dot(gbs_vec x, gbs_vec y, double *out)
{
    if (!x || !y || !out || x->n != y->n || x->dtype != y->dtype) return GBS_ERR_ARG;
    return vec_dot_sync(x, y, out, 0);
}

extern "C" int gbs_vec_norm2(gbs_vec x, double *out)
{
    if (!x || !out) return GBS_ERR_ARG;
    return vec_dot_sync(x, x, out, 1);
}

extern "C" int gbs_vec_dot_async(gbs_vec x, gbs_vec y, double *dev_out)
{
    if (!x || !y || !dev_out || x->n != y->n || x->dtype != y->dtype) return GBS_ERR_ARG;
    if ((uintptr_t)dev_out % alignof(double)) return GBS_ERR_ARG;
    return vec_dot_launch(x, y, dev_out, 0);
}

extern "C" int gbs_vec_norm2_async(gbs_vec x, double *dev_out)
{
    if (!x || !dev_out) return GBS_ERR_ARG;
    if ((uintptr_t)dev_out % alignof(double)) return GBS_ERR_ARG;
    return vec_dot_launch(x, x, dev_out, 1);
}

// ------------------------------------------------------------- Jacobi --

extern "C" int gbs_pc_jacobi_create(gbs_mat A, gbs_pc *out)
{
    if (!A || !out) return GBS_ERR_ARG;
    *out = nullptr;
    if (!A->diag_ok) return GBS_ERR_DIAG;
    gbs_pc pc = (gbs_pc)calloc(1, sizeof(*pc));
    if (!pc) return GBS_ERR_OOM;
    pc->A = A;
    *out = pc;
    return GBS_OK;
}

template <typename T>
__global__ void k_jacobi(int64_t n, const T *__restrict__ dinv, const T *__restrict__ r,
                         T *__restrict__ z)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        z[i] = dinv[i] * r[i];
}

extern "C" int gbs_pc_apply(gbs_pc pc, gbs_vec r, gbs_vec z)
{
    if (!pc || !r || !z || r->n != pc->A->n || z->n != r->n || r->dtype != z->dtype)
        return GBS_ERR_ARG;
    gbs_ctx c = pc->A->ctx;
    if (r->n == 0) return GBS_OK;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    const int g = grid_for(c, r->n, 8);
    if (r->dtype == GBS_F64)
        k_jacobi<double><<<g, GBS_BLOCK, 0, c->stream>>>(r->n, pc->A->dinv,
                                                         (const double *)r->data,
                                                         (double *)z->data);
    else
        k_jacobi<float><<<g, GBS_BLOCK, 0, c->stream>>>(r->n, pc->A->dinv32,
                                                        (const float *)r->data,
                                                        (float *)z->data);
    gbs_count_launch(c);
    GBS_CUDA_TRY(cudaGetLastError());
    return GBS_OK;
}

extern "C" int gbs_pc_destroy(gbs_pc pc)
{
    free(pc);
    return GBS_OK;
}
