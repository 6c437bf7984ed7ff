// ls_refine.cu -- least squares min ||A X - B|| (m >= n, several right-hand
// sides) refined in FP64 on top of a factorization of A that may be inexact
// (a TILEQR_TF32 one): iterative refinement of the augmented system
//   [I  A; A^T  0] [r; x] = [b; 0]
// (A. Bjorck, "Iterative refinement of linear least squares solutions I",
// BIT 7, 1967).  Each step forms the augmented residuals in FP64,
//   u = b - r - A x,   w = -A^T r,
// and solves for the correction with the factors (A ~ Q [R; 0]):
//   h = R^-T w,  [d1; d2] = Q^T u,  dx = R^-1 (d1 - h),  dr = Q [h; d2],
// x += dx, r += dr.  The Q^T and Q applications are the task graphs of the
// factorization (Sec. 3.2.1, Algorithm 2 order, and its reverse); R^-1 and
// R^-T are tiled triangular solves.  Refining x alone stalls at an error
// proportional to the factors' error times the residual; this form converges
// to the FP64 least-squares solution.  The refinement is an addition to the
// paper.  Starting from x = 0, r = 0, the first step is the plain solve.
#include <cmath>
#include <cstring>
#include <vector>

#include "factor.h"

namespace tqr {

// U = B - Rr - A X for nrhs columns: one thread per row, RHS in groups of
// 16 accumulators, X staged 64 columns at a time.
__global__ void __launch_bounds__(256) k_ls_resid(const double *__restrict__ A, int64_t lda, int64_t m,
                                                  int64_t n, const double *__restrict__ X, int64_t ldx,
                                                  const double *__restrict__ B, int64_t ldb,
                                                  const double *__restrict__ Rr, int64_t ldr, double *U,
                                                  int64_t ldu, int nrhs)
{
    __shared__ double xs[64][17];
    const int tid = threadIdx.x;
    const int64_t row = (int64_t)blockIdx.x * 256 + tid;
    for (int k0 = 0; k0 < nrhs; k0 += 16) {
        const int nk = nrhs - k0 < 16 ? nrhs - k0 : 16;
        double acc[16];
#pragma unroll
        for (int k = 0; k < 16; k++)
            acc[k] = 0.0;
        for (int64_t c0 = 0; c0 < n; c0 += 64) {
            const int nc = (int)(n - c0 < 64 ? n - c0 : 64);
            __syncthreads();
            for (int idx = tid; idx < 64 * 16; idx += 256) {
                const int c = idx >> 4, k = idx & 15;
                xs[c][k] = (c < nc && k < nk) ? X[(size_t)(k0 + k) * ldx + c0 + c] : 0.0;
            }
            __syncthreads();
            if (row < m) {
                for (int c = 0; c < nc; c++) {
                    const double a = A[(size_t)(c0 + c) * lda + row];
#pragma unroll
                    for (int k = 0; k < 16; k++)
                        acc[k] = fma(a, xs[c][k], acc[k]);
                }
            }
        }
        if (row < m)
            for (int k = 0; k < nk; k++) {
                const size_t kk = (size_t)(k0 + k);
                U[kk * ldu + row] = (B[kk * ldb + row] - Rr[kk * ldr + row]) - acc[k];
            }
    }
}

// Partial sums of A^T Rr: block (column group g of 8 columns, row split s);
// warp w takes column 8 g + w over rows [s * rows, (s + 1) * rows), lanes
// along the rows; part[(s * n + c) * nrhs + k].  A fixed reduction order, so
// the result does not depend on scheduling.
__global__ void __launch_bounds__(256) k_ls_atr(const double *__restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                const double *__restrict__ Rr, int64_t ldr, int nrhs,
                                                int64_t rows, double *part)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * 8 + warp;
    const int64_t r0 = (int64_t)blockIdx.y * rows;
    const int64_t r1 = r0 + rows < m ? r0 + rows : m;
    if (c >= n)
        return;
    for (int k0 = 0; k0 < nrhs; k0 += 16) {
        const int nk = nrhs - k0 < 16 ? nrhs - k0 : 16;
        double acc[16];
#pragma unroll
        for (int k = 0; k < 16; k++)
            acc[k] = 0.0;
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            const double a = A[(size_t)c * lda + r];
#pragma unroll
            for (int k = 0; k < 16; k++)
                if (k < nk)
                    acc[k] = fma(a, Rr[(size_t)(k0 + k) * ldr + r], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const double s = warp_allsum(acc[k]);
            if (lane == 0 && k < nk)
                part[((size_t)blockIdx.y * n + c) * nrhs + k0 + k] = s;
        }
    }
}
// W = -sum over the splits (n x nrhs, ld n)
__global__ void k_ls_atr_reduce(const double *__restrict__ part, int nsplit, int64_t n, int nrhs, double *W)
{
    const int64_t total = n * nrhs;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e % n, k = e / n;
        double s = 0.0;
        for (int sp = 0; sp < nsplit; sp++)
            s += part[((size_t)sp * n + c) * nrhs + k];
        W[(size_t)k * n + c] = -s;
    }
}

// Tiled forward substitution R^T H = W on the first q row blocks of a
// tile-row layout (nb x ncp per block).  For j = 0 .. q-1: H_j = R_jj^-T W_j
// (k_trsmt_diag), then W_i -= R_ji^T H_j for i > j (k_trsmt_update).  One CTA
// per 32-column chunk (and row block).
__global__ void __launch_bounds__(NT) k_trsmt_diag(const double *__restrict__ tiles, double *Bt, int nb, int p,
                                                   int64_t ncp, int j, int64_t n, int *flag)
{
    extern __shared__ double ys[];  // nb x 32, [r][c] ld 33
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cb = blockIdx.x;
    const double *R = tiles + ((size_t)j * p + j) * (size_t)nb * nb;
    double *Y = Bt + ((size_t)j * ncp + (size_t)cb * 32) * nb;
    for (int idx = threadIdx.x; idx < nb * 32; idx += NT) {
        const int c = idx / nb, r = idx - c * nb;
        ys[r * 33 + c] = Y[(size_t)c * nb + r];
    }
    __syncthreads();
    const int64_t col0 = (int64_t)j * nb;
    int last = nb - 1;
    if (col0 + last >= n)
        last = (int)(n - 1 - col0);
    // row c of R^T is column c of R: h(c) = (w(c) - sum_{r<c} R(r,c) h(r)) / R(c,c)
    for (int c = 0; c <= last; c++) {
        const double d = ldcg(R + (size_t)c * nb + c);
        double x = 0.0;
        if (d != 0.0)
            x = ys[c * 33 + lane] / d;
        else if (threadIdx.x == 0)
            atomicCAS(flag, 0, (int)(col0 + c + 1));
        __syncthreads();
        if (warp == 0)
            ys[c * 33 + lane] = x;
        // rows r > c of the transposed system use R(c, r)
        for (int r = c + 1 + warp; r <= last; r += NWARP)
            ys[r * 33 + lane] = fma(-ldcg(R + (size_t)r * nb + c), x, ys[r * 33 + lane]);
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * 32; idx += NT) {
        const int c = idx / nb, r = idx - c * nb;
        Y[(size_t)c * nb + r] = (r <= last) ? ys[r * 33 + c] : 0.0;
    }
}

__global__ void __launch_bounds__(NT) k_trsmt_update(const double *__restrict__ tiles, double *Bt, int nb, int p,
                                                     int64_t ncp, int j)
{
    extern __shared__ double xs[];  // nb x 32, [r][c] ld 33
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = j + 1 + blockIdx.x, cb = blockIdx.y;
    const double *R = tiles + ((size_t)i * p + j) * (size_t)nb * nb;   // tile (j, i)
    const double *X = Bt + ((size_t)j * ncp + (size_t)cb * 32) * nb;
    double *Y = Bt + ((size_t)i * ncp + (size_t)cb * 32) * nb;
    for (int idx = threadIdx.x; idx < nb * 32; idx += NT) {
        const int c = idx / nb, r = idx - c * nb;
        xs[r * 33 + c] = X[(size_t)c * nb + r];
    }
    __syncthreads();
    // Y(r) -= sum_c R_ji(c, r) X(c): column r of the tile, contiguous
    for (int r = warp; r < nb; r += NWARP) {
        const double *col = R + (size_t)r * nb;
        double acc0 = Y[(size_t)lane * nb + r], acc1 = 0.0;
        int c = 0;
        for (; c + 1 < nb; c += 2) {
            acc0 = fma(-ldcg(col + c), xs[c * 33 + lane], acc0);
            acc1 = fma(-ldcg(col + c + 1), xs[(c + 1) * 33 + lane], acc1);
        }
        if (c < nb)
            acc0 = fma(-ldcg(col + c), xs[c * 33 + lane], acc0);
        Y[(size_t)lane * nb + r] = acc0 + acc1;
    }
}

// Row-layout helpers on the first n rows (q blocks of nb x ncp):
// mode 0: Y -= H; mode 1: Y = H.
__global__ void k_rows_combine(double *Y, const double *__restrict__ H, int nb, int q, int64_t ncp, int64_t n,
                               int mode)
{
    const size_t total = (size_t)q * ncp * nb;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % nb);
        const int64_t blk = (int64_t)(e / ((size_t)ncp * nb));
        if (blk * nb + r >= n)
            continue;
        Y[e] = mode == 0 ? Y[e] - H[e] : H[e];
    }
}

// Y (rows x ncols, ld) += D (ld same), column-major
__global__ void k_add_cm(double *Y, int64_t ldy, const double *__restrict__ D, int64_t ldd, int64_t rows,
                         int64_t ncols)
{
    const int64_t total = rows * ncols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % rows, c = e / rows;
        Y[c * ldy + r] += D[c * ldd + r];
    }
}

// Sum of squares of each column (one CTA per column, fixed order).
__global__ void __launch_bounds__(256) k_colsumsq(const double *__restrict__ M, int64_t ld, int64_t rows, double *out)
{
    __shared__ double red[8];
    const int64_t c = blockIdx.x;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += 256)
        acc = fma(M[c * ld + r], M[c * ld + r], acc);
    acc = warp_allsum(acc);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; w++)
            s += red[w];
        out[c] = s;
    }
}

}  // namespace tqr

// ---------------------------------------------------------------------------
// Host side.
namespace tqr {
namespace {

constexpr int64_t ATR_ROWS = 8192;   // rows per partial sum of A^T r

struct LsLayout {
    int64_t ncp, nsplit;
    size_t Bt, Ct, Wt, sched, flag, Rr, U, DX, DR, W, part, colsq, end;
};

LsLayout ls_layout(const tileqr_desc *d, int64_t nrhs)
{
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain);
    LsLayout S{};
    S.ncp = ((nrhs + APPLY_W - 1) / APPLY_W) * APPLY_W;
    S.nsplit = (d->m + ATR_ROWS - 1) / ATR_ROWS;
    if (S.nsplit < 1)
        S.nsplit = 1;
    const size_t rows_p = (size_t)L.p * L.nb * S.ncp * 8, rows_q = (size_t)L.q * L.nb * S.ncp * 8;
    size_t off = 0;
    S.Bt = off;
    off += align256(rows_p);
    S.Ct = off;
    off += align256(rows_p);
    S.Wt = off;
    off += align256(rows_q);
    S.sched = off;
    off += align256(apply_sched_bytes(L, (int)(S.ncp / APPLY_W)));
    S.flag = off;
    off += 256;
    const size_t mcols = (size_t)d->m * nrhs * 8, ncols = (size_t)d->n * nrhs * 8;
    S.Rr = off;
    off += align256(mcols);
    S.U = off;
    off += align256(mcols);
    S.DR = off;
    off += align256(mcols);
    S.DX = off;
    off += align256(ncols);
    S.W = off;
    off += align256(ncols);
    S.part = off;
    off += align256((size_t)S.nsplit * ncols);
    S.colsq = off;
    off += align256((size_t)2 * nrhs * 8);
    S.end = off;
    return S;
}

}  // namespace
}  // namespace tqr

using namespace tqr;

extern "C" int tileqr_ls_refine_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes)
{
    if (d == nullptr)
        return -1;
    if (nrhs < 0)
        return -2;
    if (bytes == nullptr)
        return -3;
    *bytes = ls_layout(d, nrhs).end;
    return 0;
}

extern "C" int tileqr_solve_ls_refine(const tileqr_desc *d, const double *A, int64_t lda, const double *B,
                                      int64_t ldb, int64_t nrhs, double *X, int64_t ldx, double *Rres,
                                      int64_t ldr, int max_iter, double tol, void *workspace, size_t ws_bytes,
                                      tileqr_stream_t stream, tileqr_refine_info *info)
{
    if (d == nullptr || d->m < d->n)
        return -1;
    if (A == nullptr && d->m > 0 && d->n > 0)
        return -2;
    if (lda < (d->m > 1 ? d->m : 1))
        return -3;
    if (B == nullptr && nrhs > 0 && d->m > 0)
        return -4;
    if (ldb < (d->m > 1 ? d->m : 1))
        return -5;
    if (nrhs < 0)
        return -6;
    if (X == nullptr && nrhs > 0 && d->n > 0)
        return -7;
    if (ldx < (d->n > 1 ? d->n : 1))
        return -8;
    if (Rres != nullptr && ldr < (d->m > 1 ? d->m : 1))
        return -10;
    if (max_iter < 1)
        return -11;
    if (!(tol > 0.0))
        return -12;
    const LsLayout S = ls_layout(d, nrhs);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < S.end)
        return TILEQR_ERR_WORKSPACE;
    tileqr_refine_info loc{};
    if (info == nullptr)
        info = &loc;
    std::memset(info, 0, sizeof(*info));
    info->method = 3;
    if (nrhs == 0 || d->n == 0)
        return 0;
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    double *Bt = (double *)(ws + S.Bt), *Ct = (double *)(ws + S.Ct), *Wt = (double *)(ws + S.Wt);
    char *sched = ws + S.sched;
    int *flag = (int *)(ws + S.flag);
    double *Rr = (double *)(ws + S.Rr), *U = (double *)(ws + S.U), *DR = (double *)(ws + S.DR);
    double *DX = (double *)(ws + S.DX), *W = (double *)(ws + S.W), *part = (double *)(ws + S.part);
    double *colsq = (double *)(ws + S.colsq);
    const int64_t m = d->m, n = d->n, ncp = S.ncp;
    const int nchunk = (int)(ncp / 32);
    const size_t tsm = (size_t)L.nb * 33 * sizeof(double);
    if (kernel_smem_optin((const void *)k_trsmt_diag, 256 * 33 * 8) != 0 ||
        kernel_smem_optin((const void *)k_trsmt_update, 256 * 33 * 8) != 0)
        return TILEQR_ERR_CUDA;
    const unsigned long long wd = watchdog_ns_default();
    // x = 0, r = 0: the first step is the plain solve
    for (int64_t k = 0; k < nrhs; k++)
        if (cudaMemsetAsync(X + k * ldx, 0, (size_t)n * 8, st) != cudaSuccess)
            return TILEQR_ERR_CUDA;
    if (cudaMemsetAsync(Rr, 0, (size_t)m * nrhs * 8, st) != cudaSuccess ||
        cudaMemsetAsync(flag, 0, 256, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    std::vector<double> prev(nrhs, INFINITY), hsq(2 * nrhs);
    std::vector<char> done(nrhs, 0);
    int rc = 0;
    int it = 0;
    for (it = 1; it <= max_iter; it++) {
        // u = b - r - A x ;  w = -A^T r (zero while r = 0)
        k_ls_resid<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(A, lda, m, n, X, ldx, B, ldb, Rr, m, U, m,
                                                               (int)nrhs);
        count_launch();
        if (it > 1) {
            k_ls_atr<<<dim3((unsigned)((n + 7) / 8), (unsigned)S.nsplit), 256, 0, st>>>(A, lda, m, n, Rr, m,
                                                                                       (int)nrhs, ATR_ROWS, part);
            k_ls_atr_reduce<<<152, 256, 0, st>>>(part, (int)S.nsplit, n, (int)nrhs, W);
            count_launch(2);
        } else if (cudaMemsetAsync(W, 0, (size_t)n * nrhs * 8, st) != cudaSuccess) {
            return TILEQR_ERR_CUDA;
        }
        // h = R^-T w, in the tile-row layout of the first q blocks
        if ((rc = launch_cm2rows(W, n, n, nrhs, Wt, L.nb, L.q, ncp, st)) != 0)
            return rc;
        for (int j = 0; j < L.q; j++) {
            k_trsmt_diag<<<nchunk, NT, tsm, st>>>(d->tiles, Wt, L.nb, L.p, ncp, j, n, flag);
            count_launch();
            if (j + 1 < L.q) {
                k_trsmt_update<<<dim3(L.q - j - 1, nchunk), NT, tsm, st>>>(d->tiles, Wt, L.nb, L.p, ncp, j);
                count_launch();
            }
        }
        // [d1; d2] = Q^T u; keep a copy for dr
        if ((rc = launch_cm2rows(U, m, m, nrhs, Bt, L.nb, L.p, ncp, st)) != 0)
            return rc;
        if ((rc = launch_apply(L, d->tiles, d->T, d->T2, Bt, ncp, sched, st, wd, false)) != 0)
            return rc;
        if (cudaMemcpyAsync(Ct, Bt, (size_t)L.p * L.nb * ncp * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return TILEQR_ERR_CUDA;
        // dx = R^-1 (d1 - h)
        k_rows_combine<<<4 * 152, 256, 0, st>>>(Bt, Wt, L.nb, L.q, ncp, n, 0);
        count_launch();
        if ((rc = launch_trsm(L, d->tiles, Bt, ncp, flag, st)) != 0)
            return rc;
        if ((rc = launch_rows2cm(Bt, L.nb, L.q, ncp, n, nrhs, DX, n, st)) != 0)
            return rc;
        // dr = Q [h; d2]
        k_rows_combine<<<4 * 152, 256, 0, st>>>(Ct, Wt, L.nb, L.q, ncp, n, 1);
        count_launch();
        if ((rc = launch_apply(L, d->tiles, d->T, d->T2, Ct, ncp, sched, st, wd, true)) != 0)
            return rc;
        if ((rc = launch_rows2cm(Ct, L.nb, L.p, ncp, m, nrhs, DR, m, st)) != 0)
            return rc;
        // x += dx, r += dr
        for (int64_t k = 0; k < nrhs; k++) {
            k_add_cm<<<152, 256, 0, st>>>(X + k * ldx, ldx, DX + k * n, n, n, 1);
            count_launch();
        }
        k_add_cm<<<4 * 152, 256, 0, st>>>(Rr, m, DR, m, m, nrhs);
        k_colsumsq<<<(unsigned)nrhs, 256, 0, st>>>(DX, n, n, colsq);
        count_launch(2);
        for (int64_t k = 0; k < nrhs; k++) {
            k_colsumsq<<<1, 256, 0, st>>>(X + k * ldx, ldx, n, colsq + nrhs + k);
            count_launch();
        }
        if (cudaMemcpyAsync(hsq.data(), colsq, (size_t)2 * nrhs * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return TILEQR_ERR_CUDA;
        int hflag = 0;
        SchedCtrl c;
        if (cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&c, sched, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
            return TILEQR_ERR_CUDA;
        if (c.error)
            return c.error;
        if (hflag)
            return TILEQR_ERR_SINGULAR;
        // per column: stop once the correction is negligible or no longer
        // halves (the rounding level of the FP64 residuals)
        double worst = 0.0;
        bool all = true;
        for (int64_t k = 0; k < nrhs; k++) {
            const double ndx = std::sqrt(hsq[k]), nx = std::sqrt(hsq[nrhs + k]);
            const double ratio = nx > 0.0 ? ndx / nx : ndx;
            if (it > 1 && !done[k] && (ratio <= tol || ndx > 0.5 * prev[k]))
                done[k] = 1;
            if (it > 1)
                worst = ratio > worst ? ratio : worst;
            prev[k] = ndx;
            all = all && done[k];
        }
        if (it == 2)
            info->initial_rel_residual = worst;
        if (it > 1)
            info->rel_residual = worst;
        if (all)
            break;
    }
    info->iterations = it > max_iter ? max_iter : it;
    info->converged = 1;
    for (int64_t k = 0; k < nrhs; k++)
        info->converged &= done[k] ? 1 : 0;
    if (Rres != nullptr)
        for (int64_t k = 0; k < nrhs; k++)
            if (cudaMemcpyAsync(Rres + k * ldr, Rr + k * m, (size_t)m * 8, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
                return TILEQR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}
