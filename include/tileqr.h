/*
 * tileqr.h -- C ABI of the GB300 tiled Householder QR library (libtileqr.so).
 *
 * The library factors A = QR with the tiled algorithm of Buttari, Langou,
 * Kurzak and Dongarra, "A Class of Parallel Tiled Linear Algebra Algorithms
 * for Multicore Architectures": A is stored as a p x q grid of nb x nb tiles
 * (Sec. 3, Block Data Layout), each tile is processed by the DGEQRT, DLARFB,
 * DTSQRT and DSSRFB tasks of Sec. 3.2.1 with inner block size ib (Sec. 3.2.3),
 * in the order of Algorithm 2 as its dependencies clear (Sec. 4).
 *
 * Conventions for every entry point:
 *  - Matrices are FP64, column-major, with a leading dimension >= rows.
 *  - Pointers named A, B, R, X are DEVICE pointers owned by the caller.
 *  - All device memory the library uses is the caller's `workspace`; the
 *    library allocates no device memory.  The descriptor filled in by
 *    tileqr_factor points into that workspace, so the workspace must stay
 *    allocated and untouched while the descriptor is used.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) unless stated otherwise.  Device-side failures (watchdog, non-
 *    finite input) are recorded in the workspace and returned by
 *    tileqr_status(), which synchronises the stream.
 *  - Return codes follow LAPACK: 0 = success, -i = argument i is illegal,
 *    positive = one of the TILEQR_ERR_* codes below.
 *  - Every scheduler wait is bounded: a persistent kernel that sees no
 *    progress for 10 s (or TILEQR_WATCHDOG_MS milliseconds, if that
 *    environment variable is set when a call is made) gives up and records
 *    TILEQR_ERR_TIMEOUT.
 *  - Threads and devices: calls work on the device current in the calling
 *    thread.  The one-time launch set-up (shared-memory opt-in, persistent
 *    grid size) is made per device and kernel under a lock, so several host
 *    threads and several devices may use the library at once; calls that
 *    share a workspace (or tileqr_factor_noalloc's scratch) must not overlap
 *    on the GPU.  The instrumentation hooks below (trace buffer, profile
 *    events) are process-wide settings.
 */
#ifndef TILEQR_H
#define TILEQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tileqr_stream_t; /* identical to cudaStream_t */

/* Arithmetic of the trailing updates (DLARFB/DSSRFB, and DTTMQR in the tree
 * form).  Panels (DGEQRT, DTSQRT, DTTQRT: norms, tau, T factors) are always
 * FP64; with TILEQR_TF32 their in-tile trailing updates run in FP32. */
enum {
    TILEQR_FP64 = 0,       /* every task in FP64 */
    TILEQR_TF32 = 1,       /* updates as 3xTF32 tensor-core products (tcgen05),
                              FP32 accumulation; nb 128, ib 16 or 32, task graph only.
                              The FP32 operands are scaled per matrix column by a
                              power of two taken from the column's largest entry,
                              so any magnitude of A is handled (column norms in
                              [2^-1000, 2^1000]); each update's output column is
                              within ~2^-21 of its norm (tileqr_mixed_update_tile) */
    TILEQR_SPLIT_BF16 = 2  /* split-BF16 updates: NOT BUILT in this library; every
                              call that asks for it returns TILEQR_ERR_UNSUPPORTED */
};

/* How the task graph is executed. */
enum {
    TILEQR_SCHED_DAG = 0,  /* one persistent kernel: per-task dependency counters and
                              device ready queues in the priority order of Sec. 4 */
    TILEQR_SCHED_BULK = 1  /* fork-join comparator: per step k, one launch per task
                              kind (GEQRT; LARFB row; TSQRT chain; SSRFB columns) */
};

/* Flags for tileqr_factor. */
enum {
    TILEQR_FLAG_NONE = 0,
    /* Fault injection for tests of the watchdog: the scheduler never releases
     * the final task, so the persistent kernel must give up after the watchdog
     * limit and report TILEQR_ERR_TIMEOUT.  No device fault is involved. */
    TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK = 1,
    /* Stress test of the task-graph schedule (TILEQR_SCHED_DAG): every task
     * sleeps a pseudo-random time (up to ~40 us, from a hash of the task and
     * a seed) before it runs and before it releases its successors, so the
     * tasks finish in orders the natural timing rarely produces.  The seed is
     * flags >> 8.  The results must not change: every tile is written by a
     * fixed sequence of tasks (Sec. 4). */
    TILEQR_FLAG_TEST_RANDOM_DELAYS = 2
};

/* Positive error codes. */
enum {
    TILEQR_ERR_CUDA = 1001,      /* a CUDA runtime call failed */
    TILEQR_ERR_TIMEOUT = 1002,   /* the scheduler's watchdog saw no progress */
    TILEQR_ERR_NONFINITE = 1003, /* A holds a NaN or an infinity; nothing was factored */
    TILEQR_ERR_WORKSPACE = 1004, /* workspace too small or misaligned (256 B) */
    TILEQR_ERR_SINGULAR = 1005,  /* R has an exact zero on its diagonal (solve) */
    TILEQR_ERR_UNSUPPORTED = 1006, /* (nb, ib, precision) combination not built */
    TILEQR_ERR_SCRATCH_LIMIT = 1007, /* problem too large for tileqr_factor_noalloc's fixed scratch */
    TILEQR_ERR_NOT_SPD = 1008       /* tileqr_cholesky: the matrix is not positive definite */
};

/* Factorization descriptor, filled in by tileqr_factor.  Plain data; the
 * device pointers point into the caller's workspace.
 *
 * tiles: p*q tiles of nb*nb doubles, tile (i,j) at offset ((j*p)+i)*nb*nb,
 *   column-major inside the tile; partial edge tiles are zero-padded.  After
 *   the factorization tile (i,j) holds R_ij for i < j, R_kk on and above the
 *   diagonal of diagonal tiles with V_kk (unit lower, implicit 1s) below it,
 *   and the full reflector tile V_ik for i > k (Sec. 3.2.1: "no extra
 *   storage is required for the V and R tiles").
 * T: one strip of ib*nb doubles per tile, strip (i,k) at offset
 *   ((k*p)+i)*ib*nb, column-major ib x nb: t = nb/ib upper-triangular ib x ib
 *   blocks side by side (the s x s T_i of Sec. 3.2.3), lower parts zero.
 * Tree form (tileqr_factor_tree, domain < p): at step k the tile rows
 *   k..p-1 form domains of `domain` rows from row k; tile (i,k) of a domain
 *   head i holds its DGEQRT reflectors below the diagonal and, for i > k,
 *   the reflectors of the merge DTTQRT(i,k) on and above it (upper
 *   triangular); their T strips are in T2, laid out like T.  T2 is NULL for
 *   the flat form (domain == p: Algorithm 2). */
typedef struct tileqr_desc {
    int64_t m, n;
    int32_t nb, ib;
    int32_t p, q;
    int32_t precision;
    int32_t schedule;
    double *tiles;
    double *T;
    void *sched;          /* scheduler state (device) */
    size_t sched_bytes;
    void *workspace;
    size_t workspace_bytes;
    int32_t domain;       /* domain size of the elimination tree (p: flat) */
    int32_t reserved;
    double *T2;           /* DTTQRT T strips (tree form), else NULL */
} tileqr_desc;

/* Bytes of device workspace tileqr_factor needs for an m x n matrix (the
 * tiles, the T strips of Sec. 3.2.1, and the scheduler state).  Returns 0 or
 * -i for an illegal argument i.  Host only; no CUDA call. */
int tileqr_workspace_size(int64_t m, int64_t n, int nb, int ib, int precision, size_t *bytes);

/* Tiled QR factorization, Algorithm 2 (Sec. 3.2.1) with inner blocking
 * (Sec. 3.2.3), executed as a task graph (Sec. 4).
 *   m, n      matrix shape (m, n >= 0; any aspect ratio, min(p,q) steps)
 *   A, lda    device, column-major, lda >= max(1,m); read only
 *   nb, ib    tile size b and inner block size s; ib must divide nb.  Built
 *             combinations: nb in {64,128,256}, ib in {16,32}
 *   precision TILEQR_FP64, or TILEQR_TF32 (nb 128, TILEQR_SCHED_DAG);
 *             TILEQR_SPLIT_BF16 and other combinations: TILEQR_ERR_UNSUPPORTED
 *   schedule  TILEQR_SCHED_DAG or TILEQR_SCHED_BULK
 *   flags     TILEQR_FLAG_*
 *   workspace device, 256-byte aligned, >= tileqr_workspace_size() bytes
 *   out       host descriptor, filled in on success
 * Asynchronous.  Returns 0, -i, TILEQR_ERR_WORKSPACE, TILEQR_ERR_UNSUPPORTED
 * or TILEQR_ERR_CUDA (launch failure).  Device-side outcome: tileqr_status. */
int tileqr_factor(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib,
                  int precision, int schedule, int flags, void *workspace, size_t ws_bytes,
                  tileqr_stream_t stream, tileqr_desc *out);

/* Tree form of the factorization, for tall matrices: the panel column of
 * step k is eliminated in domains of `domain` tile rows (each a DGEQRT plus
 * the DTSQRT chain of Algorithm 2 into the domain head), and the domain heads
 * are merged pairwise (binary tree, log2 depth) by the triangle-on-triangle
 * kernels DTTQRT / DTTMQR.  This shortens Algorithm 2's serial DTSQRT chain
 * of p - k tasks per step (the critical path of Sec. 4 for p >> q) to about
 * domain + log2(p / domain); it is a variant beyond the paper's flat
 * elimination order.  R is the same matrix up to rounding and row signs;
 * Q is a different product of reflectors (see tileqr_desc).
 *   domain  1 <= domain; domain >= p (or 0) gives exactly tileqr_factor
 *   other arguments as tileqr_factor (task-graph schedule only)
 * Returns 0, -i, TILEQR_ERR_WORKSPACE, TILEQR_ERR_UNSUPPORTED or
 * TILEQR_ERR_CUDA. */
int tileqr_workspace_size_tree(int64_t m, int64_t n, int nb, int ib, int precision, int domain, size_t *bytes);
int tileqr_factor_tree(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib, int domain,
                       int precision, int flags, void *workspace, size_t ws_bytes, tileqr_stream_t stream,
                       tileqr_desc *out);

/* tileqr_factor_noalloc -- the same FP64 factorization (persistent task-graph
 * kernel, same results as tileqr_factor with TILEQR_SCHED_DAG) for callers
 * that cannot allocate device memory.  The paper has no counterpart: it is an
 * interface for deployments, not part of the method.
 *
 * Who it is for: services that reserve all of their device memory when they
 * start and may not allocate afterwards (a cudaMalloc can stall the device and
 * can fail at an arbitrary later time), and plug-ins whose host framework owns
 * every device allocation and passes them only the buffers they read and
 * write.  Such a caller passes the input and the outputs; nothing else.
 *
 *   m, n, A, lda, nb, ib  as for tileqr_factor (FP64; same built (nb, ib))
 *   tiles, tiles_bytes    device output, >= p*q*nb*nb*8 bytes: the factored
 *                         tiles, same layout as tileqr_desc.tiles
 *   T, T_bytes            device output, >= p*q*ib*nb*8 bytes: the T strips,
 *                         same layout as tileqr_desc.T
 *   out                   filled in; usable with tileqr_status, tileqr_get_R,
 *                         tileqr_get_factors, tileqr_apply_qt, tileqr_solve_ls
 *
 * The scheduler's scratch (dependency counters, ready queues, status word)
 * is one fixed 4 MiB device array inside the library; every GPU that loads
 * the library holds it until the process exits.  Problems whose scratch would
 * exceed it (tile grids beyond roughly 80 x 80, e.g. n > 10240 at nb 128)
 * return TILEQR_ERR_SCRATCH_LIMIT before any device work.  Allocates nothing:
 * no cudaMalloc, cudaFree or allocating library call.
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * on a device share the array, which keeps the previous call's contents; each
 * call clears it on its stream before use.  Calls whose executions overlap on
 * the GPU (other streams, other host threads) race on it, and the device-side
 * status read by tileqr_status(out) is only valid until the next call of this
 * entry point on the same device.  The looked-up address is kept for the
 * life of the process: do not call this entry point on a device after
 * cudaDeviceReset (or any other reset of its primary context), which reloads
 * the library's module at another address.  The scheduler watchdog honours
 * TILEQR_WATCHDOG_MS like tileqr_factor; the task trace (tileqr_set_trace)
 * and the profile events (tileqr_set_profile_events) are not recorded by this
 * entry point.  Asynchronous; returns 0, -i, TILEQR_ERR_UNSUPPORTED,
 * TILEQR_ERR_SCRATCH_LIMIT or TILEQR_ERR_CUDA. */
int tileqr_factor_noalloc(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib,
                          double *tiles, size_t tiles_bytes, double *T, size_t T_bytes,
                          tileqr_stream_t stream, tileqr_desc *out);

/* One update task of the TILEQR_TF32 factorization on caller tiles, for
 * checking the accuracy of a single DLARFB or DSSRFB (Sec. 3.2.1) against
 * FP64 tile kernels.  It runs the code the factorization runs for that task:
 * the panel's full T built from V and its T strip, then three 3xTF32 tcgen05
 * products with FP32 accumulation, tiles FP64, columns scaled by powers of
 * two from the largest exponent of each column of [B; C].
 *   kind  TILEQR_UPDATE_LARFB: C <- (I - V T V^T)^T C, V the unit lower part
 *         of a DGEQRT tile (the entries on and above its diagonal, R, are
 *         not read);
 *         TILEQR_UPDATE_SSRFB: [B; C] <- (I - V T V^T)^T [B; C] with the
 *         reflectors [I; V], V a full DTSQRT reflector tile
 *   ib    16 or 32 (nb is 128)
 *   V, T  device: the 128 x 128 reflector tile (column-major) and its
 *         ib x 128 T strip (column-major, ld ib), as in tileqr_desc
 *   B, C  device 128 x 128 column-major tiles, 16-byte aligned (else -5 /
 *         -6), updated in place (B is not read for TILEQR_UPDATE_LARFB and
 *         may be NULL)
 *   workspace  device, 256-byte aligned, >= TILEQR_MIXED_UPDATE_WS_BYTES
 * Synchronous.  Returns 0, -i, TILEQR_ERR_UNSUPPORTED, TILEQR_ERR_WORKSPACE,
 * TILEQR_ERR_TIMEOUT (a tensor-core wait gave up) or TILEQR_ERR_CUDA. */
enum { TILEQR_UPDATE_LARFB = 0, TILEQR_UPDATE_SSRFB = 1 };
#define TILEQR_MIXED_UPDATE_WS_BYTES (388u * 1024u)
int tileqr_mixed_update_tile(int kind, int ib, const double *V, const double *T, double *B, double *C,
                             void *workspace, size_t ws_bytes, tileqr_stream_t stream);

/* Synchronises `stream` and returns the device-side status of the last
 * factorization run on `d`: 0, TILEQR_ERR_TIMEOUT or TILEQR_ERR_NONFINITE
 * (or TILEQR_ERR_CUDA if the stream reports an error). */
int tileqr_status(const tileqr_desc *d, tileqr_stream_t stream);

/* Copies the min(m,n) x n upper-trapezoidal R (zeros below the diagonal) to
 * the device array R (column-major, ldr >= max(1,min(m,n))). */
int tileqr_get_R(const tileqr_desc *d, double *R, int64_t ldr, tileqr_stream_t stream);

/* Copies the factored matrix in LAPACK's in-place form: m x n column-major
 * AV (ldav >= max(1,m)) with R on and above the diagonal of the tile rows and
 * the reflectors below, exactly the tile contents without padding; and, if T
 * is not NULL, the T strips as a (p*ib) x n column-major array (ldt >= p*ib),
 * strip (i,k) at rows i*ib.., columns k*nb.. . Both device pointers. */
int tileqr_get_factors(const tileqr_desc *d, double *AV, int64_t ldav, double *T, int64_t ldt,
                       tileqr_stream_t stream);

/* Copies the DTTQRT T strips of a tree-form factorization as a (p*ib) x n
 * column-major device array (ldt >= p*ib), strip (i,k) at rows i*ib..,
 * columns k*nb.. (zero for rows that are not merged at step k).  Returns
 * TILEQR_ERR_UNSUPPORTED for a flat factorization. */
int tileqr_get_tree_T(const tileqr_desc *d, double *T2, int64_t ldt, tileqr_stream_t stream);

/* B <- Q^T B for the Q of a factorization (Sec. 3.2.1: the DLARFB and DSSRFB
 * transformations replayed on the columns of B in the order of Algorithm 2;
 * for the tree form also the DTTMQR merges).
 *   B, ldb    device, column-major m x nrhs, ldb >= max(1,m), in place
 *   workspace device scratch of tileqr_apply_workspace_size() bytes
 * Asynchronous. */
int tileqr_apply_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes);
int tileqr_apply_qt(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                    size_t ws_bytes, tileqr_stream_t stream);

/* B <- Q B (Q itself): the same transformations in the reverse order, each
 * with its inner blocks reversed and T_l in place of T_l^T.  Arguments,
 * workspace and returns as tileqr_apply_qt. */
int tileqr_apply_q(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace, size_t ws_bytes,
                   tileqr_stream_t stream);

/* B <- Q^T B (trans = 1) or Q B (trans = 0) on the tensor cores, for a
 * TILEQR_TF32 factorization with nb 128: the same task graphs as
 * tileqr_apply_qt / tileqr_apply_q (Sec. 3.2.1, Algorithm 2's order and its
 * reverse), each update applied with the full T and the pre-split operands
 * the factorization kept (3xTF32 products, FP32 accumulation, columns of B
 * scaled by powers of two), on column chunks of 128.  Not FP64: each column
 * comes out within about 2^-19 of the exact product relative to its norm;
 * the FP64 refinement of tileqr_solve_ls_refine uses it for its corrections.
 *   trans      1: Q^T B;  0: Q B (T is first transposed into the workspace)
 *   B, ldb     device, column-major m x nrhs, ldb >= max(1,m), in place
 *   workspace  device, 256-byte aligned, tileqr_apply_mixed_workspace_size()
 *              bytes (the factorization's workspace must be intact)
 * Synchronous.  Returns 0, -i, TILEQR_ERR_UNSUPPORTED (not TILEQR_TF32 or
 * nb != 128), TILEQR_ERR_WORKSPACE, TILEQR_ERR_TIMEOUT (a tensor-core or
 * copy wait gave up) or TILEQR_ERR_CUDA. */
int tileqr_apply_mixed_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes);
int tileqr_apply_mixed(const tileqr_desc *d, int trans, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                       size_t ws_bytes, tileqr_stream_t stream);

/* The leading ncols columns of Q (0 <= ncols <= m; ncols = min(m,n) gives
 * the thin factor with A = Q R), written to Q (device, column-major m x
 * ncols, ldq >= max(1,m)): Q applied to the identity's first columns.
 *   workspace  tileqr_apply_workspace_size(d, ncols) bytes
 * Asynchronous.  Returns 0, -i, TILEQR_ERR_WORKSPACE, TILEQR_ERR_CUDA. */
int tileqr_form_q(const tileqr_desc *d, double *Q, int64_t ldq, int64_t ncols, void *workspace, size_t ws_bytes,
                  tileqr_stream_t stream);

/* Least-squares solve min ||A X - B||_F for m >= n with the factorization d
 * of A: B <- Q^T B, then R X = (Q^T B)(0:n-1, :) by tiled back substitution.
 *   B, ldb    device m x nrhs, in place; on return X is in B(0:n-1, :)
 *   workspace device scratch of tileqr_apply_workspace_size() bytes
 * Synchronous (returns after the solve has finished).  Returns 0, -i,
 * TILEQR_ERR_SINGULAR (exact zero on diag R), TILEQR_ERR_CUDA. */
int tileqr_solve_ls(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                    size_t ws_bytes, tileqr_stream_t stream);

/* Batched form: many independent factorizations (shapes may all differ) in
 * one persistent launch.  tileqr_batched_prepare lays the batch out in the
 * caller's workspace and uploads a per-matrix table (synchronous);
 * tileqr_factor_batched then only enqueues a memset and two kernels (layout
 * conversion of every matrix, then one task-graph kernel over all tasks of
 * all matrices, Sec. 4 priorities shared across the batch), so it can be
 * captured in a CUDA graph and replayed.  Call it once outside any capture
 * first (it sets kernel attributes on first use).  The paper factors one
 * matrix at a time; batching is an addition of this library. */
typedef struct tileqr_batch {
    int count, nb, ib, precision;
    uint64_t total_tasks;
    uint32_t cap[4];
    size_t off_ctrl, off_cnt, off_q[4], off_mats, sched_bytes;
    void *workspace;
    size_t workspace_bytes;
    double flops;   /* LAPACK operation count of the whole batch */
} tileqr_batch;

/* Workspace bytes for a batch of `count` matrices m[b] x n[b] (host arrays). */
int tileqr_batched_workspace_size(int count, const int64_t *m, const int64_t *n, int nb, int ib, int precision,
                                  size_t *bytes);
/* A[b]: device pointer of matrix b (column-major, lda[b] >= m[b]); host
 * arrays of `count` entries. Fills *out. Synchronous on `stream`. */
int tileqr_batched_prepare(int count, const int64_t *m, const int64_t *n, const double *const *A,
                           const int64_t *lda, int nb, int ib, int precision, void *workspace, size_t ws_bytes,
                           tileqr_stream_t stream, tileqr_batch *out);
/* Factor every matrix of a prepared batch (asynchronous, graph-capturable). */
int tileqr_factor_batched(const tileqr_batch *bt, tileqr_stream_t stream);
/* Synchronise and return the batch's device-side status (as tileqr_status). */
int tileqr_batched_status(const tileqr_batch *bt, tileqr_stream_t stream);
/* Descriptor of matrix `index` of a factored batch (usable with tileqr_get_R,
 * tileqr_get_factors, tileqr_apply_qt, tileqr_solve_ls). */
int tileqr_batched_get(const tileqr_batch *bt, int index, tileqr_desc *out);

/* Outcome of tileqr_solve_refine. */
typedef struct tileqr_refine_info {
    int iterations;             /* refinement steps taken */
    int inner_iterations;       /* GMRES iterations in total (method 2) */
    int method;                 /* 1 = classical refinement, 2 = flexible GMRES-IR */
    int converged;              /* rel_residual <= tol */
    double initial_rel_residual; /* ||b - A x0|| / ||b||, x0 from the factors alone */
    double rel_residual;        /* final ||b - A x|| / ||b|| (FP64) */
} tileqr_refine_info;

/* Bytes of workspace tileqr_solve_refine needs for the factorization d. */
int tileqr_refine_workspace_size(const tileqr_desc *d, size_t *bytes);

/* Solve A x = b (square, or tall and consistent: m >= n) to relative
 * residual ||b - A x||_2 / ||b||_2 <= tol with FP64 iterative refinement on
 * top of a factorization d of A (nb 128; any precision, meant for
 * TILEQR_TF32).  The correction solves use an FP32 copy of the factors
 * (Q^T applied as the task graph of Algorithm 2 on one column, R^{-1} by a
 * tiled back substitution with inverted diagonal tiles); residuals, x and the
 * Krylov vectors are FP64.  Classical refinement x += M^{-1} r runs first; if
 * it stops converging (kappa(A) u_factor not small) the remaining steps are
 * restarted flexible GMRES(40) on A d = r with M^{-1} as right
 * preconditioner.  This mixed-precision refinement is an addition to the
 * paper's method (it is not in the paper).
 *   A, lda   the original matrix (device, column-major, FP64)
 *   b        device, m entries;   x  device, n entries (output)
 *   max_iter refinement steps (outer iterations) at most
 * Works on flat and tree-form factorizations (the correction solve replays
 * the factorization's apply graph), nb 128.  The FP32 correction solve works
 * on power-of-two scaled quantities (b, each corrected residual, and R's
 * columns), so any magnitude of A and b is handled.
 * Synchronous.  Returns 0 (also when not converged: see info), -i,
 * TILEQR_ERR_SINGULAR, TILEQR_ERR_WORKSPACE, TILEQR_ERR_UNSUPPORTED (nb other
 * than 128), TILEQR_ERR_CUDA. */
int tileqr_solve_refine(const tileqr_desc *d, const double *A, int64_t lda, const double *b, double *x,
                        int max_iter, double tol, void *workspace, size_t ws_bytes, tileqr_stream_t stream,
                        tileqr_refine_info *info);

/* Least squares for every matrix of a factored batch (one right-hand side
 * per matrix, m_b >= n_b), refined in FP64 on the augmented system as in
 * tileqr_solve_ls_refine, all matrices in one persistent launch: one CTA
 * runs the whole refinement of one matrix (Q^T and Q replayed on the vector
 * in Algorithm 2's order and its reverse, R^-1 and R^-T by blocked
 * substitution, the FP64 residuals), largest matrices first.  max_iter = 1
 * gives the plain solve x = R^-1 (Q^T b)(0:n) (Sec. 3.2.1).  An addition to
 * the paper (which factors one matrix at a time).
 *   B, X      host arrays of bt->count device pointers: b_k (m_k entries,
 *             read only) and x_k (n_k entries, output)
 *   workspace tileqr_batched_ls_workspace_size(bt) bytes, 256-aligned
 *   summary   (optional) iterations = the most any matrix took; method 3;
 *             converged = every matrix stopped by the rule (||dx|| <= tol
 *             ||x||, ||dx|| no longer halving, or the rate of the last two
 *             steps putting the next correction below tol ||x||);
 *             rel_residual = the largest last ||dx|| / ||x||
 * Synchronous.  Returns 0, -i, TILEQR_ERR_WORKSPACE, TILEQR_ERR_SINGULAR,
 * TILEQR_ERR_UNSUPPORTED or TILEQR_ERR_CUDA. */
int tileqr_batched_ls_workspace_size(const tileqr_batch *bt, size_t *bytes);
int tileqr_batched_solve_ls(const tileqr_batch *bt, const double *const *B, double *const *X, int max_iter,
                            double tol, void *workspace, size_t ws_bytes, tileqr_stream_t stream,
                            tileqr_refine_info *summary);

/* Least squares min ||A X - B||_F (m >= n, inconsistent systems included)
 * to FP64 accuracy on top of a factorization d of A that may be inexact (a
 * TILEQR_TF32 one, flat or tree form): iterative refinement of the
 * augmented system [I A; A^T 0] [r; x] = [b; 0] (Bjorck, 1967; an addition
 * to the paper).  Each step forms u = b - r - A x and w = -A^T r in FP64
 * and solves for the correction with the factors: h = R^-T w,
 * [d1; d2] = Q^T u (the DLARFB / DSSRFB graph of Sec. 3.2.1),
 * dx = R^-1 (d1 - h), dr = Q [h; d2] (the same graph reversed); x += dx,
 * r += dr.  It starts from x = 0, r = 0, so the first step is the plain
 * solve of tileqr_solve_ls.  For a TILEQR_TF32 factorization with nb 128
 * the two applications of Q run on the tensor cores as in
 * tileqr_apply_mixed (they only form corrections; the residuals are FP64).
 * A column stops when ||dx|| <= tol ||x||, when ||dx|| no longer halves (the
 * rounding level of the FP64 residuals), or when the rate of its last two
 * steps puts the next correction below tol ||x||.
 *   A, lda    the original matrix (device, column-major, FP64)
 *   B, ldb    device m x nrhs right-hand sides (not modified)
 *   X, ldx    device n x nrhs solution (output)
 *   Rres, ldr device m x nrhs residuals b - A x (output; NULL to skip)
 *   max_iter  steps at most (>= 1);  tol  stopping tolerance (> 0)
 *   workspace tileqr_ls_refine_workspace_size(d, nrhs) bytes, 256-aligned
 *   info      iterations; method 3; converged = every column stopped;
 *             initial_rel_residual = the largest ||dx||/||x|| of the first
 *             correction after the plain solve, rel_residual = that of the
 *             last step
 * Synchronous.  Returns 0, -i, TILEQR_ERR_WORKSPACE, TILEQR_ERR_SINGULAR,
 * TILEQR_ERR_TIMEOUT or TILEQR_ERR_CUDA. */
int tileqr_ls_refine_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes);
int tileqr_solve_ls_refine(const tileqr_desc *d, const double *A, int64_t lda, const double *B, int64_t ldb,
                           int64_t nrhs, double *X, int64_t ldx, double *Rres, int64_t ldr, int max_iter,
                           double tol, void *workspace, size_t ws_bytes, tileqr_stream_t stream,
                           tileqr_refine_info *info);

/* Tiled Cholesky factorization A = L L^T of a symmetric positive definite
 * matrix (Sec. 3.1, Algorithm 1): the tasks DPOTF2 (Cholesky of a diagonal
 * tile), DTRSM (L_ik = A_ik L_kk^{-T}) and DGSMM (A_ij -= L_ik L_jk^T, lower
 * triangle only on diagonal tiles) run as a task graph in one persistent
 * kernel (FP64).
 *   n, A, lda  device, column-major; only the lower triangle is read
 *   nb         tile size: 64 or 128 (others: TILEQR_ERR_UNSUPPORTED)
 *   flags      reserved (0)
 *   workspace  device, 256-byte aligned, >= tileqr_cholesky_workspace_size()
 *   out        host descriptor (m = n; tiles hold L in the lower tiles)
 * Asynchronous.  Returns 0, -i, TILEQR_ERR_WORKSPACE, TILEQR_ERR_UNSUPPORTED,
 * TILEQR_ERR_CUDA.  tileqr_status() then reports 0, TILEQR_ERR_NOT_SPD (the
 * factorization stopped at a pivot that was not positive; see
 * tileqr_cholesky_info), TILEQR_ERR_NONFINITE or TILEQR_ERR_TIMEOUT. */
int tileqr_cholesky_workspace_size(int64_t n, int nb, size_t *bytes);
int tileqr_cholesky(int64_t n, const double *A, int64_t lda, int nb, int flags, void *workspace, size_t ws_bytes,
                    tileqr_stream_t stream, tileqr_desc *out);
/* L (n x n lower triangular, zeros above the diagonal) to the device array
 * L (column-major, ldl >= max(1,n)).  Asynchronous. */
int tileqr_cholesky_get_L(const tileqr_desc *d, double *L, int64_t ldl, tileqr_stream_t stream);
/* *info = 0, or the 1-based column of the first pivot that was not positive
 * (synchronises the stream). */
int tileqr_cholesky_info(const tileqr_desc *d, tileqr_stream_t stream, int64_t *info);

/* Tiled LU factorization with tiled pairwise pivoting (Sec. 3.2.2,
 * Algorithm 3; inner blocking of Sec. 3.2.3): the tasks DGETRF (LU with
 * partial pivoting of a diagonal tile), DGESSM (its interchanges and L^{-1}
 * applied to a tile of its row), DTSTRF (LU with pairwise pivoting of the
 * stacked [U_kk; A_ik]) and DSSSSM (its transformations applied to the
 * stacked pair [U_kj; A_ij]) run as a task graph in one persistent kernel
 * (FP64).  The graph is that of Algorithm 2's flat tree, kernel for kernel.
 * The result is N U = A (Sec. 3.2.4), N the inverse of the recorded
 * transformations: not the P A = L U of partial pivoting.
 *   n, A, lda  device, column-major, FP64; A is not modified
 *   nb, ib     tile size 64 or 128, inner block 16 or 32 (else
 *              TILEQR_ERR_UNSUPPORTED).  n need not be a multiple of nb:
 *              the padding is the identity and stays the identity.
 *   flags      0, or TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK (watchdog test)
 *   workspace  device, 256-byte aligned, >= tileqr_lu_workspace_size()
 *   out        host descriptor (m = n, T = the L1 strips)
 * Pivots are the first entry of largest magnitude among the candidates.  An
 * exactly zero pivot does not stop the factorization (U then has a zero on
 * its diagonal); tileqr_lu_info reports the smallest such column.
 * Asynchronous.  Returns 0, -i, TILEQR_ERR_WORKSPACE, TILEQR_ERR_UNSUPPORTED,
 * TILEQR_ERR_CUDA; tileqr_status() then reports 0, TILEQR_ERR_NONFINITE
 * (nothing factored) or TILEQR_ERR_TIMEOUT. */
int tileqr_lu_workspace_size(int64_t n, int nb, int ib, size_t *bytes);
int tileqr_lu(int64_t n, const double *A, int64_t lda, int nb, int ib, int flags, void *workspace,
              size_t ws_bytes, tileqr_stream_t stream, tileqr_desc *out);
/* *info = 0, or the smallest 1-based column at which an exactly zero pivot
 * was met (synchronises the stream). */
int tileqr_lu_info(const tileqr_desc *d, tileqr_stream_t stream, int64_t *info);
/* The factors, to device arrays (asynchronous; NULL skips Lx / piv):
 *   F    n x n (ldf >= n): U on and above the diagonal; below it the
 *        multipliers: DGETRF's in the diagonal tiles, DTSTRF's L2 blocks in
 *        the tiles below (tile (i, k), column block l = ib columns)
 *   Lx   (p*ib) x n (ldlx >= p*ib): the unit lower ib x ib blocks L1 of the
 *        DTSTRF of tile (i, k) at rows i*ib.., columns k*nb + l*ib..
 *        (unit diagonal stored; zero for i <= k)
 *   piv  p x n int (ldpiv >= p): entry (i, k*nb + c) = pivot c of DGETRF
 *        (i == k: the tile row swapped with row c, >= c, LAPACK's
 *        convention) or DTSTRF (i > k: < nb a row of U_kk, else row
 *        piv - nb of tile (i, k)); 0 for i < k.
 * Returns 0, -i, TILEQR_ERR_CUDA. */
int tileqr_lu_get_factors(const tileqr_desc *d, double *F, int64_t ldf, double *Lx, int64_t ldlx, int *piv,
                          int64_t ldpiv, tileqr_stream_t stream);
/* Solve A X = B in place (B: device, n x nrhs, ldb >= n): the recorded
 * transformations applied to B in Algorithm 3's order as a task graph
 * (DGESSM / DSSSSM on column chunks of B), then the tiled back substitution
 * with U.  Synchronous.  Returns 0, -i, TILEQR_ERR_WORKSPACE,
 * TILEQR_ERR_SINGULAR (U has an exact zero on its diagonal),
 * TILEQR_ERR_TIMEOUT, TILEQR_ERR_CUDA. */
int tileqr_lu_solve_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes);
int tileqr_lu_solve(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace, size_t ws_bytes,
                    tileqr_stream_t stream);

/* Microbenchmarks of this GPU's FP64 rates (diagnostic; not part of the
 * method): *dfma_gflops from independent FP64 fused multiply-add chains on
 * every SM, *dmma_gflops from FP64 mma.sync m16n8k16 on every SM, both in
 * GFLOP/s from CUDA-event times.  The FP64 tile kernels use the faster of
 * the two pipes.  Synchronous.  Returns 0, -1 or TILEQR_ERR_CUDA. */
int tileqr_measure_fp64_rates(double *dfma_gflops, double *dmma_gflops, tileqr_stream_t stream);

/* Human-readable text for a return code (static storage). */
const char *tileqr_strerror(int code);

/* Instrumentation for benchmarks.  tileqr_launch_count: kernels the library
 * launched since the last reset (host only).  tileqr_set_profile_events: if
 * both are non-NULL (cudaEvent_t handles), every later tileqr_factor records
 * `before` just before and `after` just after the launches of the task-graph
 * execution proper (after the layout conversion), on the call's stream; NULL
 * disables it. */
uint64_t tileqr_launch_count(void);
void tileqr_reset_launch_count(void);
void tileqr_set_profile_events(void *before, void *after);

/* Task trace (the execution-flow view of Sec. 4, Fig. 6): if `records` is a
 * device buffer of `capacity` records of 4 uint64 each, every later
 * tileqr_factor with TILEQR_SCHED_DAG writes one record per executed task:
 * {task code (tt << 63 | k << 42 | i << 21 | j; tt = 1 for the tree form's
 * DTTQRT / DTTMQR), start ns, end ns (%globaltimer), SM id}.
 * Records beyond `capacity` are dropped; the number written is readable with
 * tileqr_trace_count after the factorization (synchronises the stream).
 * NULL disables tracing. Host only. */
void tileqr_set_trace(void *records, uint64_t capacity);
int tileqr_trace_count(const tileqr_desc *d, tileqr_stream_t stream, uint64_t *count);

/* Task-graph introspection (host only, no CUDA call): the graph that the
 * persistent kernel executes (Sec. 4's dependency-driven schedule) for an
 * m x n matrix, tile size nb and domain size `domain` (0: flat).
 *   what      0 = the factorization; 1 = Q^T applied to one column chunk
 *             of right-hand sides (tileqr_apply_qt / tileqr_solve_ls);
 *             2 = Q applied to one chunk (tileqr_apply_q / tileqr_form_q);
 *             3 = the tiled Cholesky of an m x m matrix (tileqr_cholesky;
 *             n and domain ignored; kinds 0 DPOTF2, 1 DTRSM, 2 DGSMM)
 *             4 = the tiled LU of an m x m matrix (tileqr_lu; n and domain
 *             ignored; kinds 0 DGETRF, 1 DGESSM, 2 DTSTRF, 3 DSSSSM)
 *   tasks     ntasks rows {kind, i, j, k}: kind 0 DGEQRT, 1 DTSQRT, 2 DLARFB,
 *             3 DSSRFB, 4 DTTQRT, 5 DTTMQR; j = -1 for what = 1
 *   ndeps     per task, the number of predecessors that release it
 *   succ_ptr  ntasks + 1 offsets into succ (CSR); succ: successor indices
 *             (kinds for what >= 1: 2 DLARFB, 3 DSSRFB, 5 DTTMQR)
 * Call with tasks == NULL to get *ntasks and *nedges, then again with
 * buffers of that size (4*ntasks, ntasks, ntasks+1, nedges entries).
 * Returns 0 or -i (-99: a successor outside the graph, an internal error). */
int tileqr_task_graph(int64_t m, int64_t n, int nb, int domain, int what, int32_t *tasks, int32_t *ndeps,
                      int64_t *succ_ptr, int64_t *succ, int64_t *ntasks, int64_t *nedges);

#ifdef __cplusplus
}
#endif
#endif /* TILEQR_H */
