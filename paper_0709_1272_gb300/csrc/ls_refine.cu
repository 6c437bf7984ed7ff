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
// For a TILEQR_TF32 factorization (nb 128) the two applications of Q run on
// the tensor cores (launch_apply_mixed: 3xTF32, about 2^-19 relative per
// column, the same order of error as the factors), since they only form the
// corrections; the residuals stay FP64, so the fixed point is the same.
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

// The same on buffers of different widths, for the tensor-core form: Y
// (ncpy columns) over the first q blocks.  mode 0: Y = X - H on the first n
// rows and ncols columns, 0 elsewhere; mode 1: Y = H there, Y kept elsewhere.
__global__ void k_rows_combine2(double *Y, int64_t ncpy, const double *__restrict__ X, int64_t ncpx,
                                const double *__restrict__ H, int64_t ncph, int nb, int q, int64_t n, int64_t ncols,
                                int mode)
{
    const size_t total = (size_t)q * ncpy * nb;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % nb);
        const int64_t c = (int64_t)((e / nb) % (size_t)ncpy), i = (int64_t)(e / ((size_t)ncpy * nb));
        const bool in = i * nb + r < n && c < ncols;
        const double h = in ? H[((size_t)i * ncph + c) * nb + r] : 0.0;
        if (mode == 0)
            Y[e] = in ? X[((size_t)i * ncpx + c) * nb + r] - h : 0.0;
        else if (in)
            Y[e] = h;
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
    size_t Bt, Ct, Wt, sched, sched2, flag, Rr, U, DX, DR, W, part, colsq, end;
    // tensor-core form (TILEQR_TF32 factorization, nb 128): the applications
    // on ncpm = nrhs rounded up to 128 columns, T transposed for Q
    bool mixed;
    int64_t ncpm;
    size_t BtM, CtM, TN, cexpm;
};

LsLayout ls_layout(const tileqr_desc *d, int64_t nrhs)
{
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain, d->precision);
    LsLayout S{};
    S.mixed = d->precision == TILEQR_TF32 && d->nb == 128 && L.off_TF2 > L.off_TF;
    S.ncpm = ((nrhs + 127) / 128) * 128;
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
    size_t sb = apply_sched_bytes(L, (int)(S.ncp / APPLY_W));
    if (S.mixed && apply_sched_bytes(L, (int)(S.ncpm / 128)) > sb)
        sb = apply_sched_bytes(L, (int)(S.ncpm / 128));
    off += align256(sb);
    S.sched2 = off;   // the application of Q, so that both report errors
    off += align256(sb);
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
    if (S.mixed) {
        const size_t rows_m = (size_t)L.p * L.nb * S.ncpm * 8;
        S.BtM = off;
        off += align256(rows_m);
        S.CtM = off;
        off += align256(rows_m);
        S.TN = off;
        off += align256(mixed_tn_bytes(L));
        S.cexpm = off;
        off += align256((size_t)(S.ncpm ? S.ncpm : 1) * sizeof(int));
    }
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
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain, d->precision);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    double *Bt = (double *)(ws + S.Bt), *Ct = (double *)(ws + S.Ct), *Wt = (double *)(ws + S.Wt);
    char *sched = ws + S.sched, *sched2 = ws + S.sched2;
    int *flag = (int *)(ws + S.flag);
    double *Rr = (double *)(ws + S.Rr), *U = (double *)(ws + S.U), *DR = (double *)(ws + S.DR);
    double *DX = (double *)(ws + S.DX), *W = (double *)(ws + S.W), *part = (double *)(ws + S.part);
    double *colsq = (double *)(ws + S.colsq);
    const int64_t m = d->m, n = d->n, ncp = S.ncp;
    const unsigned long long wd = watchdog_ns_default();
    // x = 0, r = 0: the first step is the plain solve
    for (int64_t k = 0; k < nrhs; k++)
        if (cudaMemsetAsync(X + k * ldx, 0, (size_t)n * 8, st) != cudaSuccess)
            return TILEQR_ERR_CUDA;
    if (cudaMemsetAsync(Rr, 0, (size_t)m * nrhs * 8, st) != cudaSuccess ||
        cudaMemsetAsync(flag, 0, 256, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    // tensor-core form: the operand blocks of the factorization, T transposed once
    MixedOperands M;
    double *BtM = nullptr, *CtM = nullptr;
    int *cexpm = nullptr;
    if (S.mixed) {
        BtM = (double *)(ws + S.BtM);
        CtM = (double *)(ws + S.CtM);
        cexpm = (int *)(ws + S.cexpm);
        const int rcm = mixed_operands(d, L, (unsigned char *)(ws + S.TN), st, &M);
        if (rcm)
            return rcm;
    }
    std::vector<double> prev(nrhs, INFINITY), hsq(2 * nrhs);
    std::vector<char> done(nrhs, 0);
    int rc = 0;
    int it = 0;
    for (it = 1; it <= max_iter; it++) {
        if (it == 1) {
            // x = 0, r = 0: u = b and w = 0, so h = 0 (the plain solve)
            if (cudaMemcpy2DAsync(U, (size_t)m * 8, B, (size_t)ldb * 8, (size_t)m * 8, (size_t)nrhs,
                                  cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaMemsetAsync(Wt, 0, (size_t)L.q * L.nb * ncp * 8, st) != cudaSuccess)
                return TILEQR_ERR_CUDA;
        } else {
            // u = b - r - A x ;  w = -A^T r
            k_ls_resid<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(A, lda, m, n, X, ldx, B, ldb, Rr, m, U, m,
                                                                   (int)nrhs);
            k_ls_atr<<<dim3((unsigned)((n + 7) / 8), (unsigned)S.nsplit), 256, 0, st>>>(A, lda, m, n, Rr, m,
                                                                                       (int)nrhs, ATR_ROWS, part);
            k_ls_atr_reduce<<<152, 256, 0, st>>>(part, (int)S.nsplit, n, (int)nrhs, W);
            count_launch(3);
            // h = R^-T w, in the tile-row layout of the first q blocks
            if ((rc = launch_cm2rows(W, n, n, nrhs, Wt, L.nb, L.q, ncp, st)) != 0 ||
                (rc = launch_trsm(L, d->tiles, Wt, ncp, flag, st, true, nrhs)) != 0)
                return rc;
        }
        if (S.mixed) {
            // [d1; d2] = Q^T u on the tensor cores; keep a copy for dr
            const int64_t ncpm = S.ncpm;
            const size_t rows_m = (size_t)L.p * L.nb * ncpm * 8;
            if ((rc = launch_cm2rows(U, m, m, nrhs, BtM, L.nb, L.p, ncpm, st)) != 0 ||
                (rc = launch_rows_cexp(BtM, L.nb, L.p, ncpm, cexpm, st)) != 0 ||
                (rc = launch_apply_mixed(L, M, BtM, ncpm, nrhs, cexpm, sched, st, wd, false)) != 0)
                return rc;
            if (cudaMemcpyAsync(CtM, BtM, rows_m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return TILEQR_ERR_CUDA;
            // dx = R^-1 (d1 - h), in the narrow layout of the triangular solves
            k_rows_combine2<<<4 * 152, 256, 0, st>>>(Bt, ncp, BtM, ncpm, Wt, ncp, L.nb, L.q, n, nrhs, 0);
            count_launch();
            if ((rc = launch_trsm(L, d->tiles, Bt, ncp, flag, st, false, nrhs)) != 0)
                return rc;
            if ((rc = launch_rows2cm(Bt, L.nb, L.q, ncp, n, nrhs, DX, n, st)) != 0)
                return rc;
            // dr = Q [h; d2] on the tensor cores
            k_rows_combine2<<<4 * 152, 256, 0, st>>>(CtM, ncpm, nullptr, 0, Wt, ncp, L.nb, L.q, n, nrhs, 1);
            count_launch();
            if ((rc = launch_rows_cexp(CtM, L.nb, L.p, ncpm, cexpm, st)) != 0 ||
                (rc = launch_apply_mixed(L, M, CtM, ncpm, nrhs, cexpm, sched2, st, wd, true)) != 0)
                return rc;
            if ((rc = launch_rows2cm(CtM, L.nb, L.p, ncpm, m, nrhs, DR, m, st)) != 0)
                return rc;
        } else {
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
            if ((rc = launch_trsm(L, d->tiles, Bt, ncp, flag, st, false, nrhs)) != 0)
                return rc;
            if ((rc = launch_rows2cm(Bt, L.nb, L.q, ncp, n, nrhs, DX, n, st)) != 0)
                return rc;
            // dr = Q [h; d2]
            k_rows_combine<<<4 * 152, 256, 0, st>>>(Ct, Wt, L.nb, L.q, ncp, n, 1);
            count_launch();
            if ((rc = launch_apply(L, d->tiles, d->T, d->T2, Ct, ncp, sched2, st, wd, true)) != 0)
                return rc;
            if ((rc = launch_rows2cm(Ct, L.nb, L.p, ncp, m, nrhs, DR, m, st)) != 0)
                return rc;
        }
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
        SchedCtrl c, c2;
        if (cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&c, sched, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&c2, sched2, sizeof(c2), cudaMemcpyDeviceToHost) != cudaSuccess)
            return TILEQR_ERR_CUDA;
        if (c.error)
            return c.error;
        if (c2.error)
            return c2.error;
        if (hflag)
            return TILEQR_ERR_SINGULAR;
        // per column: stop once the correction is negligible, or no longer
        // halves (the rounding level of the FP64 residuals), or once the
        // linear rate of the last two steps puts the next correction below
        // tol (the error left in x is about that next correction)
        double worst = 0.0;
        bool all = true;
        for (int64_t k = 0; k < nrhs; k++) {
            const double ndx = std::sqrt(hsq[k]), nx = std::sqrt(hsq[nrhs + k]);
            const double ratio = nx > 0.0 ? ndx / nx : ndx;
            const bool predicted = it > 2 && ndx <= 0.5 * prev[k] && ratio * (ndx / prev[k]) <= tol;
            if (it > 1 && !done[k] && (ratio <= tol || ndx > 0.5 * prev[k] || predicted))
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
