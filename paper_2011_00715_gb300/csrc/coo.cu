// Device-side assembly of a CSR matrix from coordinate triplets
// (MatSetPreallocationCOO + MatSetValuesCOO, Sec. 4): triplet k adds v[k] at
// (i[k], j[k]); duplicates are summed in triplet order, so the result does
// not depend on thread scheduling.
//
//   1. validate the indices and count the triplets of each row (atomics;
//      the counts do not depend on the order)
//   2. exclusive scan of the counts: each row's segment
//   3. scatter key = (column << 32) | k into the row's segment (any order)
//   4. sort each segment by key: by column, equal columns by triplet index
//      (rank sort: a warp per row up to 64 entries, a CTA per row up to
//      4096, the host for longer rows)
//   5. merge: one CSR entry per distinct column, its value the left-to-right
//      sum of its triplets' values; the sorted triplet indices and the
//      segment of each entry are kept, so new values for the same triplets
//      (gbs_mat_set_values_coo) are summed the same way
//   6. the CSR goes through gbs_mat_create_aij (validation, tiling, Jacobi)

#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gbs_impl.cuh"

namespace {

constexpr int kShortRow = 64;     // rank-sorted by one warp
constexpr int kMediumRow = 4096;  // rank-sorted by one CTA in shared memory

int grid(gbs_ctx c, int64_t n)
{
    const int64_t g = (n + 255) / 256, cap = (int64_t)c->num_sms * 8;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

__global__ void k_coo_count(int64_t m, const int32_t *ti, const int32_t *tj, int64_t nrows,
                            int64_t ncols, int *cnt, int *bad)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = ti[k], c = tj[k];
        if (r < 0 || r >= nrows || c < 0 || c >= ncols) atomicExch(bad, 1);
        else atomicAdd(&cnt[r], 1);
    }
}

// Exclusive scan of n counts into out[0..n] (out[n] = total), in three
// passes over chunks of 2048 entries: chunk sums, a scan of the chunk sums
// by one CTA, then each chunk's own scan from its offset.
constexpr int kChunk = 2048;

__global__ void k_chunk_sums(int64_t n, const int *in, int64_t *sums)
{
    __shared__ int64_t red[256];
    const int64_t c0 = (int64_t)blockIdx.x * kChunk;
    int64_t s = 0;
    for (int64_t i = c0 + threadIdx.x; i < n && i < c0 + kChunk; i += 256) s += in[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

__global__ void k_scan_sums(int64_t nb, int64_t *sums)
{
    // one CTA of 1024 threads: each thread scans a contiguous run, then the
    // run totals are scanned by thread 0
    __shared__ int64_t tot[1024];
    const int64_t per = (nb + 1023) / 1024;
    const int64_t a = threadIdx.x * per, b = a + per < nb ? a + per : nb;
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += sums[i];
    tot[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < 1024; ++t) {
            const int64_t x = tot[t];
            tot[t] = run;
            run += x;
        }
    }
    __syncthreads();
    s = tot[threadIdx.x];
    for (int64_t i = a; i < b; ++i) {
        const int64_t x = sums[i];
        sums[i] = s;
        s += x;
    }
}

__global__ void k_chunk_scan(int64_t n, const int *in, const int64_t *offs, int64_t *out)
{
    if (threadIdx.x != 0) return;   // one thread per chunk: sequential, simple and cheap
    const int64_t c0 = (int64_t)blockIdx.x * kChunk;
    int64_t s = offs[blockIdx.x];
    for (int64_t i = c0; i < n && i < c0 + kChunk; ++i) {
        out[i] = s;
        s += in[i];
    }
    if (c0 + kChunk >= n) out[n] = s;
}

__global__ void k_coo_scatter(int64_t m, const int32_t *ti, const int32_t *tj, const int64_t *start,
                              int *fill, uint64_t *keys)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = ti[k];
        const int64_t pos = start[r] + atomicAdd(&fill[r], 1);
        keys[pos] = ((uint64_t)(uint32_t)tj[k] << 32) | (uint64_t)(uint32_t)k;
    }
}

// Rows of at most kShortRow keys: warp w sorts row w (keys are distinct, so
// a key's rank is the number of smaller keys).
__global__ void k_sort_short(int64_t nrows, const int64_t *start, uint64_t *keys)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < nrows; r += nw) {
        const int64_t a = start[r];
        const int len = (int)(start[r + 1] - a);
        if (len <= 1 || len > kShortRow) continue;
        const uint64_t k0 = lane < len ? keys[a + lane] : ~0ull;
        const uint64_t k1 = lane + 32 < len ? keys[a + lane + 32] : ~0ull;
        int r0 = 0, r1 = 0;
        for (int t = 0; t < len; ++t) {
            const uint64_t o = __shfl_sync(0xffffffffu, t < 32 ? k0 : k1, t & 31);
            r0 += o < k0;
            r1 += o < k1;
        }
        __syncwarp();
        if (lane < len) keys[a + r0] = k0;
        if (lane + 32 < len) keys[a + r1] = k1;
        __syncwarp();
    }
}

// Rows of kShortRow < len <= kMediumRow keys: CTA b sorts row rows[b] in
// shared memory by rank.
__global__ void k_sort_medium(const int64_t *rows, const int64_t *start, uint64_t *keys)
{
    __shared__ uint64_t s[kMediumRow];
    const int64_t r = rows[blockIdx.x];
    const int64_t a = start[r];
    const int len = (int)(start[r + 1] - a);
    for (int t = threadIdx.x; t < len; t += blockDim.x) s[t] = keys[a + t];
    __syncthreads();
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const uint64_t x = s[t];
        int rank = 0;
        for (int u = 0; u < len; ++u) rank += s[u] < x;
        keys[a + rank] = x;
    }
}

// Distinct columns per row (sorted segments).
__global__ void k_coo_unique(int64_t nrows, const int64_t *start, const uint64_t *keys, int *ucnt)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int u = 0;
        uint32_t prev = 0;
        for (int64_t p = start[r]; p < start[r + 1]; ++p) {
            const uint32_t c = (uint32_t)(keys[p] >> 32);
            u += (p == start[r] || c != prev);
            prev = c;
        }
        ucnt[r] = u;
    }
}

// CSR entries of each row: column, left-to-right sum of its triplets'
// values, the segment of its triplets in the sorted order; perm[p] = the
// triplet index at sorted position p.
__global__ void k_coo_write(int64_t nrows, const int64_t *start, const uint64_t *keys,
                            const int64_t *rowoff, const double *v, int32_t *colidx, double *vals,
                            int64_t *seg, uint32_t *perm)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = rowoff[r] - 1;
        uint32_t prev = 0;
        for (int64_t p = start[r]; p < start[r + 1]; ++p) {
            const uint32_t c = (uint32_t)(keys[p] >> 32), k = (uint32_t)keys[p];
            perm[p] = k;
            if (p == start[r] || c != prev) {
                ++u;
                colidx[u] = (int32_t)c;
                vals[u] = v[k];
                seg[u] = p;
            } else {
                vals[u] = vals[u] + v[k];
            }
            prev = c;
        }
    }
}

// New values for the same triplets: entry u sums v over its segment of the
// sorted triplet order, left to right.
__global__ void k_coo_refill(int64_t nnz, const int64_t *seg, const uint32_t *perm, const double *v,
                             double *vals)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nnz;
         u += (int64_t)gridDim.x * blockDim.x) {
        double s = v[perm[seg[u]]];
        for (int64_t p = seg[u] + 1; p < seg[u + 1]; ++p) s = s + v[perm[p]];
        vals[u] = s;
    }
}

int scan_counts(gbs_ctx c, int64_t n, const int *in, int64_t *out, int64_t *sums)
{
    const int64_t nb = (n + kChunk - 1) / kChunk;
    if (nb == 0) {
        GBS_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream));
        return GBS_OK;
    }
    k_chunk_sums<<<(unsigned)nb, 256, 0, c->stream>>>(n, in, sums);
    k_scan_sums<<<1, 1024, 0, c->stream>>>(nb, sums);
    k_chunk_scan<<<(unsigned)nb, 32, 0, c->stream>>>(n, in, sums, out);
    gbs_count_launch(c, 3);
    GBS_CUDA_TRY(cudaGetLastError());
    return GBS_OK;
}

// Device buffers of one assembly, freed together.
struct Bufs {
    std::vector<void *> p;
    template <typename T>
    int get(T **out, size_t count)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            (void)cudaGetLastError();
            return GBS_ERR_OOM;
        }
        p.push_back(q);
        *out = (T *)q;
        return GBS_OK;
    }
    void release(void *q)
    {
        auto it = std::find(p.begin(), p.end(), q);
        if (it != p.end()) p.erase(it);
    }
    ~Bufs()
    {
        for (void *q : p) cudaFree(q);
    }
};

}  // namespace

extern "C" int gbs_mat_create_coo(gbs_ctx c, int64_t nrows, int64_t ncols, int64_t m,
                                  const int32_t *ti, const int32_t *tj, const double *v,
                                  int memspace, gbs_mat *out)
{
    if (!c || !out || nrows < 0 || ncols < 0 || m < 0) return GBS_ERR_ARG;
    if (memspace != GBS_MEM_HOST && memspace != GBS_MEM_DEVICE) return GBS_ERR_ARG;
    if (nrows >= (int64_t)INT32_MAX || ncols >= (int64_t)INT32_MAX || m >= (int64_t)UINT32_MAX)
        return GBS_ERR_ARG;
    if (m > 0 && (!ti || !tj || !v)) return GBS_ERR_ARG;
    *out = nullptr;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = c->stream;
    Bufs B;
    int rc = GBS_OK;
    // triplets on the device
    const int32_t *di = ti, *dj = tj;
    const double *dv = v;
    if (memspace == GBS_MEM_HOST && m > 0) {
        int32_t *a, *b;
        double *w;
        if ((rc = B.get(&a, m)) || (rc = B.get(&b, m)) || (rc = B.get(&w, m))) return rc;
        GBS_CUDA_TRY(cudaMemcpyAsync(a, ti, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
        GBS_CUDA_TRY(cudaMemcpyAsync(b, tj, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
        GBS_CUDA_TRY(cudaMemcpyAsync(w, v, sizeof(double) * m, cudaMemcpyHostToDevice, st));
        di = a;
        dj = b;
        dv = w;
    }
    int *cnt, *fill;
    int64_t *start, *sums;
    const int64_t nb = (nrows + kChunk - 1) / kChunk;
    if ((rc = B.get(&cnt, nrows)) || (rc = B.get(&fill, nrows)) || (rc = B.get(&start, nrows + 1)) ||
        (rc = B.get(&sums, nb)))
        return rc;
    int *bad = (int *)c->devsmall + 3;   // word 3 of the context's small device buffer
    GBS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * std::max<int64_t>(nrows, 1), st));
    GBS_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int) * std::max<int64_t>(nrows, 1), st));
    GBS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    if (m > 0) {
        k_coo_count<<<grid(c, m), 256, 0, st>>>(m, di, dj, nrows, ncols, cnt, bad);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    GBS_CUDA_TRY(cudaMemcpyAsync(c->pinned, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBS_CUDA_TRY(cudaStreamSynchronize(st));
    if (*(volatile int *)c->pinned) return GBS_ERR_CSR;
    if ((rc = scan_counts(c, nrows, cnt, start, sums))) return rc;
    uint64_t *keys;
    if ((rc = B.get(&keys, m))) return rc;
    if (m > 0) {
        k_coo_scatter<<<grid(c, m), 256, 0, st>>>(m, di, dj, start, fill, keys);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    // row lengths on the host: which rows need the CTA or the host sort
    std::vector<int64_t> hs((size_t)nrows + 1);
    GBS_CUDA_TRY(cudaMemcpyAsync(hs.data(), start, sizeof(int64_t) * (nrows + 1),
                                 cudaMemcpyDeviceToHost, st));
    GBS_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> medium, longrows;
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t len = hs[r + 1] - hs[r];
        if (len > kMediumRow) longrows.push_back(r);
        else if (len > kShortRow) medium.push_back(r);
    }
    if (nrows > 0 && m > 0) {
        k_sort_short<<<grid(c, nrows * 32), 256, 0, st>>>(nrows, start, keys);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    if (!medium.empty()) {
        int64_t *dm;
        if ((rc = B.get(&dm, medium.size()))) return rc;
        GBS_CUDA_TRY(cudaMemcpyAsync(dm, medium.data(), sizeof(int64_t) * medium.size(),
                                     cudaMemcpyHostToDevice, st));
        k_sort_medium<<<(unsigned)medium.size(), 256, 0, st>>>(dm, start, keys);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
        GBS_CUDA_TRY(cudaStreamSynchronize(st));   // medium is a host vector
    }
    for (int64_t r : longrows) {   // rare: rows longer than a CTA sorts in shared memory
        const int64_t a = hs[r], len = hs[r + 1] - a;
        std::vector<uint64_t> h((size_t)len);
        GBS_CUDA_TRY(cudaMemcpyAsync(h.data(), keys + a, sizeof(uint64_t) * len,
                                     cudaMemcpyDeviceToHost, st));
        GBS_CUDA_TRY(cudaStreamSynchronize(st));
        std::sort(h.begin(), h.end());
        GBS_CUDA_TRY(cudaMemcpyAsync(keys + a, h.data(), sizeof(uint64_t) * len,
                                     cudaMemcpyHostToDevice, st));
        GBS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // distinct columns -> row offsets of the CSR
    int *ucnt;
    int64_t *rowoff;
    if ((rc = B.get(&ucnt, nrows)) || (rc = B.get(&rowoff, nrows + 1))) return rc;
    if (nrows > 0) {
        k_coo_unique<<<grid(c, nrows), 256, 0, st>>>(nrows, start, keys, ucnt);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    if ((rc = scan_counts(c, nrows, ucnt, rowoff, sums))) return rc;
    std::vector<int64_t> hro((size_t)nrows + 1);
    GBS_CUDA_TRY(cudaMemcpyAsync(hro.data(), rowoff, sizeof(int64_t) * (nrows + 1),
                                 cudaMemcpyDeviceToHost, st));
    GBS_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t nnz = hro[nrows];
    if (nnz >= (int64_t)INT32_MAX) return GBS_ERR_ARG;
    std::vector<int32_t> hrp((size_t)nrows + 1);
    for (int64_t r = 0; r <= nrows; ++r) hrp[r] = (int32_t)hro[r];
    int32_t *drp;
    if ((rc = B.get(&drp, nrows + 1))) return rc;
    GBS_CUDA_TRY(cudaMemcpyAsync(drp, hrp.data(), sizeof(int32_t) * (nrows + 1), cudaMemcpyHostToDevice,
                                 st));
    int32_t *ci;
    double *vals;
    int64_t *seg;
    uint32_t *perm;
    if ((rc = B.get(&ci, nnz)) || (rc = B.get(&vals, nnz)) || (rc = B.get(&seg, nnz + 1)) ||
        (rc = B.get(&perm, m)))
        return rc;
    if (nrows > 0 && m > 0) {
        k_coo_write<<<grid(c, nrows), 256, 0, st>>>(nrows, start, keys, rowoff, dv, ci, vals, seg, perm);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    GBS_CUDA_TRY(cudaMemcpyAsync(seg + nnz, &m, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    GBS_CUDA_TRY(cudaStreamSynchronize(st));   // &m is on the stack
    // the assembled CSR, on the device
    gbs_mat A = nullptr;
    rc = gbs_mat_create_aij(c, nrows, ncols, drp, ci, vals, GBS_MEM_DEVICE, &A);
    if (rc) return rc;
    A->coo_m = m;
    A->coo_seg = seg;
    A->coo_perm = perm;
    B.release(seg);
    B.release(perm);
    *out = A;
    return GBS_OK;
}

extern "C" int gbs_mat_set_values_coo(gbs_mat A, const double *v, int memspace)
{
    if (!A || (!v && A->coo_m > 0)) return GBS_ERR_ARG;
    if (memspace != GBS_MEM_HOST && memspace != GBS_MEM_DEVICE) return GBS_ERR_ARG;
    if (!A->coo_seg) return GBS_ERR_ARG;   // not made by gbs_mat_create_coo
    gbs_ctx c = A->ctx;
    GBS_CUDA_TRY(cudaSetDevice(c->device));
    Bufs B;
    int rc = GBS_OK;
    const double *dv = v;
    if (memspace == GBS_MEM_HOST && A->coo_m > 0) {
        double *w;
        if ((rc = B.get(&w, A->coo_m))) return rc;
        GBS_CUDA_TRY(cudaMemcpyAsync(w, v, sizeof(double) * A->coo_m, cudaMemcpyHostToDevice,
                                     c->stream));
        dv = w;
    }
    double *vals;
    if ((rc = B.get(&vals, A->nnz))) return rc;
    if (A->nnz > 0) {
        k_coo_refill<<<grid(c, A->nnz), 256, 0, c->stream>>>(A->nnz, A->coo_seg, A->coo_perm, dv, vals);
        gbs_count_launch(c);
        GBS_CUDA_TRY(cudaGetLastError());
    }
    rc = gbs_mat_set_values(A, vals, GBS_MEM_DEVICE);
    GBS_CUDA_TRY(cudaStreamSynchronize(c->stream));   // before the buffers are freed
    return rc;
}
