/*
 * gbs.h -- C ABI of the GB300 Jacobi-preconditioned CG library.
 *
 * The library solves A x = b for a sparse symmetric positive definite A in
 * compressed sparse row (AIJ) form with the conjugate-gradient method and a
 * Jacobi (diagonal) preconditioner, entirely on one GPU.  The objects and
 * calls follow the PETSc usage the paper describes: objects are created,
 * filled with data, then handed to a solver (Sec. 2, Listing 1); every call
 * returns an error code and passes outputs through pointers (Sec. 2,
 * Listing 4: VecAXPY(rk,-1.0,r), VecNorm(rk,NORM_2,&norm)); a Mat of type
 * MATAIJ holds CSR data and Vec holds a dense vector (Sec. 4).
 *
 * Conventions for every function below:
 *  - Return value: GBS_OK (0) on success, a positive status for a solve that
 *    ended without converging but left valid output, or a negative GBS_ERR_*
 *    code.  On a negative code no output argument is written unless stated.
 *  - Handles are opaque pointers owned by the library; *_destroy frees them
 *    and accepts NULL.  A handle must not be used after its context is
 *    destroyed.
 *  - Index arrays are int32 (rowptr has nrows+1 entries, colidx nnz
 *    entries); vector lengths and sizes are int64.
 *  - "memspace" says where a caller pointer lives: GBS_MEM_HOST (pageable or
 *    pinned host memory) or GBS_MEM_DEVICE (device memory of the context's
 *    GPU).  The library never queries pointer attributes (Sec. 3, Challenge
 *    A5: those queries cost about 0.3 us each); the caller states it.
 *  - Work is queued on the context's CUDA stream.  Calls that return host
 *    scalars (dot, norm, solve results) synchronise that stream; all others
 *    are asynchronous with respect to the host.
 *  - Not thread-safe per context: one host thread drives a context at a time.
 */
#ifndef GBS_H
#define GBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status --- */
enum {
    GBS_OK = 0,
    GBS_DIVERGED_ITS = 1,      /* iteration limit reached; x holds the last iterate */
    GBS_ERR_ARG = -1,          /* bad argument: NULL, size mismatch, aliasing, dtype */
    GBS_ERR_OOM = -2,          /* device or pinned host allocation failed */
    GBS_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    GBS_ERR_DIAG = -4,         /* Jacobi: a diagonal entry is missing or <= 0 */
    GBS_ERR_INDEFINITE = -5,   /* CG breakdown: p.Ap <= 0 or r.z < 0 */
    GBS_ERR_NAN = -6,          /* a NaN appeared in a solver scalar */
    GBS_ERR_TIMEOUT = -7,      /* a device-side wait gave up (cooperative barrier) */
    GBS_ERR_STAGNATION = -8,   /* mixed mode: an outer step reduced ||r|| by less than 2x */
    GBS_ERR_BUDGET = -9,       /* server: the request alone exceeds the memory budget */
    GBS_ERR_CSR = -10,         /* malformed CSR: rowptr, column range or order */
    GBS_ERR_NOT_FOUND = -11,   /* server: unknown ticket */
    GBS_ERR_UNSUPPORTED = -12  /* valid request the library does not implement */
};

enum { GBS_MEM_HOST = 0, GBS_MEM_DEVICE = 1 };
enum { GBS_F64 = 0, GBS_F32 = 1 };

/* Precision of a solve (Response A7, Sec. 4: single precision on the GPU,
 * with the flags carried by the solve). */
enum {
    GBS_MODE_FP64 = 0,   /* every step in FP64 */
    GBS_MODE_MIXED = 1   /* FP32 inner PCG (FP32 SpMV, vectors and reductions)
                            inside FP64 iterative refinement: FP64 is kept
                            for r = b - A x, the update x += s d and the
                            convergence norms */
};

/* How a solve is launched. */
enum {
    GBS_ALG_AUTO = 0,        /* library choice */
    GBS_ALG_PERSISTENT = 1,  /* one cooperative kernel per solve; the iteration
                                loop, reductions and convergence test run on
                                the device (Challenge A1: no host round trip
                                per dot product) */
    GBS_ALG_PEROP = 2,       /* one kernel per vector/matrix operation, scalars
                                kept on the device, convergence read by the
                                host every iteration: the library-call-per-op
                                pattern of PETSc's GPU back-end */
    GBS_ALG_GRAPH = 3,       /* GBS_ALG_PEROP's kernels captured once into a
                                CUDA graph of several iterations and replayed
                                (Challenge A1: CUDA graphs) */
    GBS_ALG_CLUSTER = 4      /* FP64, n <= GBS_CLUSTER_MAX_ROWS: the whole solve
                                in one thread-block cluster of up to 16 CTAs,
                                the vectors in shared memory, hardware cluster
                                barriers instead of grid barriers (Challenge A1:
                                small problems are latency-bound).  GBS_ALG_AUTO
                                takes it for small FP64 systems.
                                GBS_ERR_UNSUPPORTED for a larger system, for
                                GBS_MODE_MIXED, or where the device cannot
                                keep such a cluster resident */
};

/* Norm of the CG stopping test.  The paper names KSPCG (Sec. 5.5) but does
 * not fix the norm of its test; the test runs before each iteration as
 * N(r) <= rtol N(b). */
enum {
    GBS_NORM_UNPRECONDITIONED = 0,  /* N(v) = ||v||_2 (default) */
    GBS_NORM_PRECONDITIONED = 1,    /* N(v) = ||D^-1 v||_2 */
    GBS_NORM_NATURAL = 2            /* N(v) = sqrt(v . D^-1 v); for the residual
                                       this is sqrt(r . z), already computed */
};

typedef struct gbs_ctx_s *gbs_ctx;
typedef struct gbs_mat_s *gbs_mat;
typedef struct gbs_vec_s *gbs_vec;
typedef struct gbs_pc_s *gbs_pc;
typedef struct gbs_server_s *gbs_server;

/* Solver options.  gbs_opts_default fills the defaults noted per field. */
typedef struct {
    int mode;                /* GBS_MODE_FP64 (default) or GBS_MODE_MIXED */
    int algorithm;           /* GBS_ALG_* (default GBS_ALG_AUTO) */
    double inner_rtol;       /* MIXED: relative tolerance eta of each FP32 inner
                                solve (default 1e-4); a refinement step j with
                                outer residual r_j stops its inner solve at
                                max(eta, rtol ||b|| / (2 ||r_j||)), so the last
                                step does only the work that finishes the solve */
    int outer_maxit;         /* MIXED: refinement steps at most (default 30) */
    int barrier_timeout_ms;  /* device-side waits give up after this many
                                milliseconds with GBS_ERR_TIMEOUT (default 2000) */
    int graph_iters;         /* GBS_ALG_GRAPH: iterations per captured graph (default 16) */
    int fault_skip_arrival;  /* testing only: if >= 0, that CTA of the next
                                persistent solve does not arrive at its first
                                grid barrier, so the barrier times out (default -1) */
    int batched_lanes;       /* batched and serving engines: lanes per matrix row
                                in the SpMV (1, 2 or 4), or 0 (default) to let the
                                autotuner pick per class of systems (row length,
                                right-hand-side count, precision), timing the
                                candidates once per context on the first system
                                of the class */
    int persistent_ctas;     /* persistent solves: CTAs of the launch (at most one per
                                SM), or 0 (default) for the library's choice */
    int norm_type;           /* GBS_NORM_* of the stopping test of the FP64
                                single-system CG solves (every algorithm, and
                                gbs_ksp_solve_cg_noalloc through the context's
                                options); GBS_MODE_MIXED, the batched and serving
                                engines and Chebyshev test the unpreconditioned
                                norm, and a solve in GBS_MODE_MIXED with another
                                norm is refused with GBS_ERR_ARG.
                                Default GBS_NORM_UNPRECONDITIONED */
    int no_rel16;            /* 1: single-system MatMult, CG and Chebyshev solves
                                stream the 32-bit column indices; 0 (default):
                                they stream 16-bit offsets col - row instead
                                wherever every |col - row| of the matrix is at
                                most 32767 (made on the first such use; Sec. 3,
                                Challenge A7: the index bytes cap what narrower
                                values save) */
    int persistent_shape;    /* persistent single-system CG solves: 1 = one CTA of
                                16 warps per SM (12.8 KB copy rings), 2 = one CTA of
                                32 warps (6.4 KB rings; FP64 only, where two stages
                                of the largest tile fit), 0 (default) = the tuner's
                                choice for the system's class (gbs_ksp_tune) */
    int persistent_lanes;    /* persistent single-system CG solves: lanes per matrix
                                row in the SpMV, 1 (warp tiles of 32 rows) or 2 (16
                                rows), or 0 (default) for the tuner's choice */
    int spmv_lanes;          /* gbs_mat_mult: lanes per matrix row (1, 2 or 4: warp
                                tiles of 32, 16 or 8 rows), or 0 (default): 2 where
                                a row has more than 16 nonzeros, else 1.  The
                                partial sums of a row are added in a fixed order
                                for a given setting */
    int reserved[1];         /* must be 0 */
} gbs_opts;

/* Result of the last solve on a context. */
typedef struct {
    int status;          /* GBS_OK, GBS_DIVERGED_ITS or a negative GBS_ERR_* */
    int iters;           /* CG iterations (SpMVs after set-up); MIXED: summed
                            over all inner solves */
    int outer_iters;     /* MIXED: refinement steps; FP64: 0 */
    double rnorm;        /* final ||r||_2: recurrence residual in FP64 mode,
                            true FP64 residual ||b - A x||_2 in MIXED mode;
                            N(r) in the chosen norm_type */
    double bnorm;        /* ||b||_2; N(b) in the chosen norm_type */
    double device_ms;    /* device time of the solve (CUDA events) */
    double model_bytes;  /* algorithmic bytes the solve moved by the library's
                            byte model: persistent single-system CG solves
                            (FP64 and MIXED; a nonzero counts its value and
                            the column index width actually streamed) and
                            batched solves; 0 where not computed */
    int cta_threads;     /* persistent single-system CG solves: threads per CTA
                            of the launch (one CTA per SM: 512 or 1024); 0 for
                            other algorithms */
    int lanes_per_row;   /* persistent single-system CG solves: lanes sharing a
                            matrix row in the SpMV (1 or 2); 0 otherwise */
} gbs_solve_info;

/* Library version string (static storage). */
const char *gbs_version(void);

/* Human-readable name of a status code (static storage). */
const char *gbs_status_string(int status);

/* Fill *opts with the defaults.  GBS_ERR_ARG if opts is NULL. */
int gbs_opts_default(gbs_opts *opts);

/* ----------------------------------------------------------- context --- */

/* Create a context bound to CUDA device `device` and the CUDA stream
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * stream is borrowed: the caller keeps it alive until gbs_ctx_destroy.
 * `opts` may be NULL for defaults.  Errors: GBS_ERR_ARG, GBS_ERR_CUDA,
 * GBS_ERR_OOM. */
int gbs_ctx_create(int device, void *cuda_stream, const gbs_opts *opts, gbs_ctx *out);

/* Destroy a context and the scratch memory it owns.  Matrices, vectors,
 * preconditioners and servers created on it must be destroyed first. */
int gbs_ctx_destroy(gbs_ctx ctx);

/* Replace the context's stream (borrowed, as above). */
int gbs_ctx_set_stream(gbs_ctx ctx, void *cuda_stream);

/* Replace the context's default solver options (copied). */
int gbs_ctx_set_opts(gbs_ctx ctx, const gbs_opts *opts);

/* Block until all work queued on the context's stream has finished. */
int gbs_ctx_synchronize(gbs_ctx ctx);

/* Number of this library's kernel launches on the context so far (a
 * counter kept by the host code; used to report launch counts). */
int gbs_ctx_launch_count(gbs_ctx ctx, int64_t *count);

/* Measure the device's FP64 fused multiply-add rate (the denominator of the
 * FP64 arithmetic roofline of the CG kernels): one warm-up and one timed
 * launch of a kernel in which every thread of a full grid runs 8
 * independent chains of `iters` FMAs (1 <= iters <= 2^24; 4096 takes a few
 * milliseconds).  *fma_per_s receives the FMAs per second of the timed
 * launch (CUDA events on the context's stream).  Synchronises the stream.
 * GBS_ERR_ARG for a NULL pointer or iters out of range, GBS_ERR_CUDA. */
int gbs_probe_fp64_rate(gbs_ctx ctx, int iters, double *fma_per_s);

/* ------------------------------------------------------------ matrix --- */

/* MatCreate + MatSetType(MATAIJ) + fill (Sec. 4): copy a CSR matrix into
 * library-owned device memory.  rowptr[nrows+1], colidx[nnz] (int32),
 * vals[nnz] (FP64), nnz = rowptr[nrows]; all three arrays in `memspace`
 * (host arrays are staged through pinned memory).  The caller keeps
 * ownership of its arrays; the library keeps none of their pointers.
 * Validation on the device: rowptr[0] = 0, rowptr non-decreasing, every
 * column in [0, ncols), columns strictly increasing within a row
 * (GBS_ERR_CSR otherwise).  The Jacobi diagonal D^-1 and the FP32 copy
 * of the values (for GBS_MODE_MIXED) are prepared here as well.
 * Errors: GBS_ERR_ARG, GBS_ERR_CSR, GBS_ERR_OOM, GBS_ERR_CUDA. */
int gbs_mat_create_aij(gbs_ctx ctx, int64_t nrows, int64_t ncols, const int32_t *rowptr,
                       const int32_t *colidx, const double *vals, int memspace, gbs_mat *out);

/* Replace the values of an existing matrix (same sparsity pattern), e.g. a
 * new Jacobian with the old structure.  vals[nnz] in `memspace`. */
int gbs_mat_set_values(gbs_mat A, const double *vals, int memspace);

/* Sizes of a matrix; any output pointer may be NULL. */
int gbs_mat_get_info(gbs_mat A, int64_t *nrows, int64_t *ncols, int64_t *nnz);

/* CUDA device ordinal of the context the matrix belongs to (where its
 * arrays live and its solves run).  GBS_ERR_ARG for a NULL argument. */
int gbs_mat_get_device(gbs_mat A, int *device);

/* Free a matrix (NULL is allowed). */
int gbs_mat_destroy(gbs_mat A);

/* MatMult: y = A x.  x has ncols entries, y has nrows entries, same dtype
 * (GBS_F64 uses the FP64 values, GBS_F32 the FP32 copy).  y must not alias
 * x (GBS_ERR_ARG).  Asynchronous. */
int gbs_mat_mult(gbs_mat A, gbs_vec x, gbs_vec y);

/* Assemble a matrix on the device from nnz_in coordinate triplets
 * (MatSetPreallocationCOO + MatSetValuesCOO, Sec. 4): triplet k adds v[k]
 * at row i[k], column j[k] (int32 indices, FP64 values; any order, repeats
 * allowed).  Repeated (row, column) pairs are summed in triplet order (k
 * increasing, left to right), so the result does not depend on thread
 * scheduling.  The arrays live in memspace (host or device) and are not
 * kept.  The matrix is then set up as by gbs_mat_create_aij (validation,
 * Jacobi diagonal, tiling) and remembers the triplet-to-entry map, so
 * gbs_mat_set_values_coo can refill its values.  GBS_ERR_CSR if an index
 * is out of range; GBS_ERR_ARG for bad arguments or more than 2^31 - 1
 * distinct entries; GBS_ERR_OOM. */
int gbs_mat_create_coo(gbs_ctx ctx, int64_t nrows, int64_t ncols, int64_t nnz_in, const int32_t *i,
                       const int32_t *j, const double *v, int memspace, gbs_mat *out);

/* New values for the triplets of a matrix made by gbs_mat_create_coo (the
 * same count and order as at creation), summed the same way; the Jacobi
 * diagonal and the FP32 copy follow.  GBS_ERR_ARG if A was not made from
 * triplets. */
int gbs_mat_set_values_coo(gbs_mat A, const double *v, int memspace);

/* Copy the matrix's CSR out (MatGetRowIJ / MatSeqAIJGetArray, Sec. 4):
 * rowptr (nrows + 1), colidx and vals (nnz entries each, see
 * gbs_mat_get_info) into caller buffers in memspace; any pointer may be
 * NULL to skip that array.  Blocks until the copies are done. */
int gbs_mat_get_csr(gbs_mat A, int32_t *rowptr, int32_t *colidx, double *vals, int memspace);

/* ------------------------------------------------------------ vector --- */

/* VecCreate: a device vector of n entries of `dtype`, owned by the library,
 * zero-filled.  Errors: GBS_ERR_ARG, GBS_ERR_OOM. */
int gbs_vec_create(gbs_ctx ctx, int64_t n, int dtype, gbs_vec *out);

/* Wrap caller-owned device memory (n entries of `dtype`) without copying
 * (VecCreate...WithArray, Sec. 2).  The caller keeps ownership and must keep
 * the memory alive until gbs_vec_destroy.  dev_ptr must be aligned to the
 * element size (GBS_ERR_ARG otherwise). */
int gbs_vec_wrap(gbs_ctx ctx, void *dev_ptr, int64_t n, int dtype, gbs_vec *out);

/* Free a vector handle (and its memory if the library owns it). */
int gbs_vec_destroy(gbs_vec v);

/* Length and device pointer of a vector (outputs may be NULL). */
int gbs_vec_get_info(gbs_vec v, int64_t *n, int *dtype, void **dev_ptr);

/* Copy n entries of the vector's dtype from `src` (in `memspace`) into v.
 * Asynchronous for device and pinned host sources. */
int gbs_vec_set_values(gbs_vec v, const void *src, int memspace);

/* Copy the vector's n entries into `dst` (in `memspace`).  Synchronises the
 * stream when dst is host memory. */
int gbs_vec_get_values(gbs_vec v, void *dst, int memspace);

/* VecSet: v_i = alpha. */
int gbs_vec_set(gbs_vec v, double alpha);

/* VecCopy: y <- x (same length; dtypes may differ, converting on the GPU). */
int gbs_vec_copy(gbs_vec x, gbs_vec y);

/* VecAXPY: y <- alpha x + y (Sec. 5.1: 2 flops, 3 memory accesses per entry). */
int gbs_vec_axpy(gbs_vec y, double alpha, gbs_vec x);

/* VecAYPX: y <- x + beta y. */
int gbs_vec_aypx(gbs_vec y, double beta, gbs_vec x);

/* VecPointwiseMult: w_i = x_i y_i. */
int gbs_vec_pointwise_mult(gbs_vec w, gbs_vec x, gbs_vec y);

/* VecDot: *out = x . y, reduced on the device in a fixed order (so repeated
 * calls give identical bits).  FP32 vectors accumulate in FP32.
 * Synchronises the stream. */
int gbs_vec_dot(gbs_vec x, gbs_vec y, double *out);

/* VecNorm(NORM_2): *out = ||x||_2.  Synchronises the stream. */
int gbs_vec_norm2(gbs_vec x, double *out);

/* VecDot and VecNorm without a host synchronisation (Challenge A1: a
 * scalar returned to the host stalls the kernel queue): the result is
 * written, in stream order on the context's stream, to dev_out, a DEVICE
 * pointer to one 8-byte-aligned double that the caller owns and keeps valid
 * until the stream has passed the write.  Same bits as gbs_vec_dot /
 * gbs_vec_norm2 (an FP32 vector's FP32 result is widened to double).
 * GBS_ERR_ARG for NULL or misaligned pointers or mismatched vectors; the
 * pointer's memory space is not checked. */
int gbs_vec_dot_async(gbs_vec x, gbs_vec y, double *dev_out);
int gbs_vec_norm2_async(gbs_vec x, double *dev_out);

/* ---------------------------------------------------- preconditioner --- */

/* PCJACOBI (Sec. 5.3): z = D^-1 r with D = diag(A).  GBS_ERR_DIAG if a
 * diagonal entry is missing or not positive.  The pc borrows A. */
int gbs_pc_jacobi_create(gbs_mat A, gbs_pc *out);

/* PCApply: z = D^-1 r (vectors of A's size, same dtype). */
int gbs_pc_apply(gbs_pc pc, gbs_vec r, gbs_vec z);

int gbs_pc_destroy(gbs_pc pc);

/* ------------------------------------------------------------ solver --- */

/* KSPSolve with KSPCG + PCJACOBI (Sec. 5.5, Sec. 5.3), using the context's
 * options.  b (FP64, nrows) is read; x (FP64, nrows) is the initial guess on
 * entry and the solution on exit.  Stops when ||r||_2 <= rtol ||b||_2 (the
 * test is taken before each iteration) or after maxit iterations.
 * Returns GBS_OK (converged), GBS_DIVERGED_ITS (limit reached, x valid) or
 * GBS_ERR_DIAG / GBS_ERR_INDEFINITE / GBS_ERR_NAN / GBS_ERR_TIMEOUT /
 * GBS_ERR_STAGNATION / GBS_ERR_ARG / GBS_ERR_CUDA.  iters and rnorm may be
 * NULL.  Synchronises the stream once, at the end. */
int gbs_ksp_solve_cg(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit, int *iters,
                     double *rnorm);

/* The same with explicit options (NULL = the context's) and the full
 * result in *info (may be NULL). */
int gbs_ksp_solve_cg_ex(gbs_mat A, gbs_vec b, gbs_vec x, double rtol, int maxit,
                        const gbs_opts *opts, gbs_solve_info *info);

/* Result of the last solve issued on the context. */
int gbs_ksp_last_info(gbs_ctx ctx, gbs_solve_info *info);

/* Jacobi-preconditioned Chebyshev iteration (KSPCHEBYSHEV with PCJACOBI,
 * the paper's multigrid smoother, Sec. 5.3; Chebyshev acceleration as in
 * Saad, Iterative Methods for Sparse Linear Systems, Algorithm 12.1, with
 * D^-1 r where the direction is formed) for A x = b in FP64, given an
 * interval [emin, emax] that holds the spectrum of D^-1 A (0 < emin <=
 * emax < inf; for a Dirichlet Laplacian it is known in closed form, and a
 * wider interval still converges, more slowly).  x holds the initial guess
 * on entry and the solution on return.  Same stopping test and statuses as
 * gbs_ksp_solve_cg (no inner products inside the iteration, so no
 * GBS_ERR_INDEFINITE); info (may be NULL) gets iterations, the final
 * ||r||_2 (recurrence residual), ||b||_2, device time and the algorithmic
 * bytes moved.  GBS_ERR_ARG for a bad interval or arguments, GBS_ERR_DIAG
 * for a missing or non-positive diagonal.  One persistent launch, one grid
 * barrier per iteration. */
int gbs_ksp_solve_chebyshev(gbs_mat A, gbs_vec b, gbs_vec x, double emin, double emax,
                            double rtol, int maxit, gbs_solve_info *info);

/* Autotuner of the persistent single-system CG kernels (the library's
 * own; the paper has no counterpart: its kernels come from vendor
 * libraries).  For the class of A (mode, column index width, row length up
 * to 8 / 16 / 32 / more nonzeros, log2 of the warp tiles per SM) it times a
 * solve capped at 24 iterations of every candidate launch shape (one CTA of
 * 16 or of 32 warps per SM; FP64 only for the latter) and SpMV tiling (1 or
 * 2 lanes per row: warp tiles of 32 or 16 rows) on A itself, median of
 * three, and keeps the fastest (the fixed rule's choice unless another is
 * at least 3 % faster).  The decision is cached in the context, so every
 * system of the class gets the same kernel; GBS_ALG_PERSISTENT and AUTO
 * solves call it on first use of a class unless gbs_opts fixes the shape
 * and lanes.  Outputs: *shape (1 or 2) and *lanes (1 or 2).  Allocates two
 * vectors of nrows entries while tuning.  GBS_ERR_ARG for a NULL argument
 * or an unknown mode. */
int gbs_ksp_tune(gbs_mat A, int mode, int *shape, int *lanes);

/* Largest system GBS_ALG_CLUSTER takes (rows): 8 CTAs (the portable
 * cluster size) of 4096 rows, x, r, p, A p and D^-1 in FP64 shared memory. */
#define GBS_CLUSTER_MAX_ROWS 32768

/* Largest system gbs_ksp_solve_cg_noalloc accepts (rows). */
#define GBS_NOALLOC_MAX_ROWS 262144

/* FP64 Jacobi-PCG solve that allocates nothing (the paper has no
 * counterpart: this is a library service).  It is meant for callers that
 * cannot allocate device memory while they solve: latency-bound loops,
 * where cudaMalloc/cudaFree may synchronise the whole device and take
 * unbounded time, and processes whose device memory is held by another
 * allocator's pool, where a fresh cudaMalloc can fail.  The matrix must
 * have been created beforehand (that allocates, once).
 *
 * Same arithmetic, stopping rule and statuses as gbs_ksp_solve_cg_ex with
 * GBS_MODE_FP64 and GBS_ALG_PERSISTENT, with the context's options
 * (stopping norm, barrier time limit, persistent_ctas capped at 2048 CTAs);
 * the result is also kept as the context's last solve (gbs_ksp_last_info).
 * b (read) and x (initial guess in, solution out) are caller-owned FP64
 * device arrays of nrows entries on the context's device: the C entry
 * point receives bare pointers and cannot check their length or device,
 * so the caller must (the Python binding does, from the tensors).
 * *info receives the result.  The solver's workspace (four FP64 vectors of
 * GBS_NOALLOC_MAX_ROWS entries, per-CTA partial sums, barrier and result
 * record: about 8.6 MB) is one fixed array in the library's device image;
 * every GPU that loads the library holds it until the process exits.
 * Limits and behaviour:
 *  - GBS_ERR_ARG if nrows > GBS_NOALLOC_MAX_ROWS, the matrix is not
 *    square, b or x is NULL, or b == x.
 *  - Every call on a device uses the same array and leaves its contents
 *    behind; the call clears the parts that must start at zero.  Calls that
 *    overlap on the GPU (other streams or threads of the same device) race
 *    on the array: serialise them.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; later calls reuse it.
 *  - Calls no cudaMalloc, no cudaFree and no other allocating routine; it
 *    uses the context's stream, events and pinned result buffer (created
 *    with the context) and synchronises the stream once, at the end, to
 *    read the result record. */
int gbs_ksp_solve_cg_noalloc(gbs_mat A, const double *b, double *x, double rtol, int maxit,
                             gbs_solve_info *info);

/* Block Jacobi-preconditioned CG for k right-hand sides of one matrix at
 * once (Sec. 3, Challenge F2: Krylov methods with multiple right-hand sides
 * raise arithmetic intensity and converge in fewer iterations; the block
 * method is O'Leary's block CG, which the paper reaches through KSPHPDDM).
 * The k columns share one search space: per iteration Q = A P (one pass
 * over the matrix for all columns), alpha = (P^T Q)^-1 (Z^T R),
 * X += P alpha, R -= Q alpha, Z = D^-1 R, beta = (Z^T R)_old^-1 (Z^T R),
 * P = Z + P beta, with the k x k systems solved by LDL^T.  FP64.
 * B (read) and X (initial guess in, solution out): vectors of nrows * k
 * entries, column-major (column j at offset j * nrows); 1 <= k <= 8.
 * Stopping test before each iteration: every column ||R_j||_2 <= rtol
 * ||B_j||_2.  info->iters = block iterations; info->rnorm / bnorm = the
 * largest column norms; rnorm[k] (may be NULL) receives each column's
 * final ||R_j||_2 (recurrence residual).  One cooperative launch.
 * Statuses: GBS_OK, GBS_DIVERGED_ITS, GBS_ERR_INDEFINITE (P^T A P or
 * Z^T R not positive definite: A indefinite, or the columns of B, or of
 * the residual block, linearly dependent), GBS_ERR_NAN, GBS_ERR_DIAG,
 * GBS_ERR_TIMEOUT; GBS_ERR_ARG for bad sizes or k out of range. */
int gbs_ksp_solve_cg_block(gbs_mat A, int k, gbs_vec B, gbs_vec X, double rtol, int maxit,
                           gbs_solve_info *info, double *rnorm);

/* Batched solve of independent systems in one persistent launch (Response
 * A6, Sec. 4: many different-size problems at once; Challenge F2 / Sec. 4:
 * multiple right-hand sides raise arithmetic intensity).  System s has
 * matrix A[s] (all on ctx), right-hand sides B[s] and solutions X[s]:
 * FP64 vectors of nrows(A[s]) * nrhs[s] entries, column-major (column c at
 * offset c * nrows).  X[s] holds the initial guesses on entry.  Each
 * column is an independent CG solve with tolerance rtol[s].  Results per
 * (system, column), flattened in system order: iters[], rnorm[], status[]
 * each with sum(nrhs) entries (any may be NULL).  Returns GBS_OK if every
 * column converged, else the first non-zero column status.  `mode` is
 * GBS_MODE_FP64 or GBS_MODE_MIXED.  Each column's result is independent of
 * the other systems in the batch. */
int gbs_ksp_solve_cg_batched(gbs_ctx ctx, int nsys, const gbs_mat *A, const gbs_vec *B,
                             gbs_vec *X, const int *nrhs, const double *rtol, int maxit,
                             int mode, int *iters, double *rnorm, int *status);

/* Autotune the batched engines for systems like A with k right-hand sides
 * in `mode` (GBS_MODE_FP64 or GBS_MODE_MIXED): the lanes per matrix row of
 * the SpMV (1, 2 or 4) for A's class (row length, column stride,
 * precision) is chosen by timing the candidates on copies of A, once per
 * context; later batched solves and servers on ctx use the decision.  The
 * chosen lanes go to *lanes (may be NULL).  With gbs_opts.batched_lanes set
 * (non-zero), nothing is timed and that value is reported.  Lets a caller
 * pay the tuning before its first timed solve. */
int gbs_batched_tune(gbs_ctx ctx, gbs_mat A, int k, int mode, int *lanes);

/* ----------------------------------------------------------- serving --- */

/* A serving engine: solve requests are admitted against a device-memory
 * budget, their CSR and Krylov state stay on the device, and a persistent
 * batched kernel advances all admitted requests together; requests that
 * arrive while others run join as slots and memory free up (continuous
 * batching).  hbm_budget_bytes bounds the device memory held by admitted
 * requests.  max_slots bounds concurrent requests (0 = library default). */
int gbs_server_create(gbs_ctx ctx, size_t hbm_budget_bytes, int max_slots, int mode,
                      gbs_server *out);

int gbs_server_destroy(gbs_server srv);

/* Submit a request: host CSR (rowptr/colidx/vals as in gbs_mat_create_aij),
 * k right-hand sides b[nrows * k] (host, column-major), tolerance rtol,
 * iteration limit maxit.  The arrays are copied before return.  Returns a
 * ticket in *ticket.  GBS_ERR_BUDGET if the request alone can never fit the
 * budget; otherwise it is queued until memory and a slot are free. */
int gbs_server_submit(gbs_server srv, int64_t nrows, const int32_t *rowptr, const int32_t *colidx,
                      const double *vals, int k, const double *b, double rtol, int maxit,
                      uint64_t *ticket);

/* As gbs_server_submit, but the arrays are borrowed instead of copied: the
 * caller keeps rowptr, colidx, vals and b valid and unchanged until
 * gbs_server_poll reports the request done (they are read when the request
 * is admitted).  Saves a host copy of every request. */
int gbs_server_submit_borrowed(gbs_server srv, int64_t nrows, const int32_t *rowptr,
                               const int32_t *colidx, const double *vals, int k, const double *b,
                               double rtol, int maxit, uint64_t *ticket);

/* Advance the engine without blocking for long: admit queued requests,
 * launch or continue device work, retire finished requests.  Returns the
 * number of requests retired by this call in *retired (may be NULL). */
int gbs_server_progress(gbs_server srv, int *retired);

/* *done = 1 if the request has finished (its result can be fetched). */
int gbs_server_poll(gbs_server srv, uint64_t ticket, int *done);

/* Drive the engine until the request has finished. */
int gbs_server_wait(gbs_server srv, uint64_t ticket);

/* Copy a finished request's solution (host, nrows * k, column-major) and
 * per-column iters/rnorm/status (k entries each; any may be NULL), then
 * release it.  A finished request's solution waits in a pinned host buffer
 * of the server (reused by later requests once fetched), so results that
 * are never fetched hold pinned memory until gbs_server_destroy.  The
 * server's calls are not thread-safe: one thread drives a server.
 * GBS_ERR_NOT_FOUND for unknown or already fetched tickets. */
int gbs_server_fetch(gbs_server srv, uint64_t ticket, double *x, int *iters, double *rnorm,
                     int *status);

/* Engine counters: queued, running and finished requests, device bytes in
 * use (outputs may be NULL). */
int gbs_server_stats(gbs_server srv, int *queued, int *running, int *finished,
                     size_t *bytes_in_use);

/* Host wall time the engine has spent since creation, in seconds: admitting
 * requests (matrix upload and set-up), running quanta (launch to
 * completion), retiring requests (results to the host); and the number of
 * quanta run (outputs may be NULL). */
int gbs_server_times(gbs_server srv, double *admit_s, double *quanta_s, double *retire_s,
                     int64_t *quanta);

#ifdef __cplusplus
}
#endif

#endif /* GBS_H */
