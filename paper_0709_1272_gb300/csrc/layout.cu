// layout.cu -- conversion between column-major storage and the Block Data
// Layout of contiguous nb x nb tiles (Sec. 3: tiles stored contiguously so
// each task touches a few compact blocks).  Pure copies, bound by HBM
// bandwidth: each warp moves one tile column (nb contiguous doubles on both
// sides), so loads and stores are fully coalesced.
#include "factor.h"

namespace tqr {

static int grid_for(size_t warps_needed)
{
    int nsm = 1;
    if (device_sm_count(&nsm) != 0)
        nsm = 1;   // a failed query only shrinks the grid; the launch reports the error
    const size_t per_cta = 8;  // 256 threads
    size_t ctas = (warps_needed + per_cta - 1) / per_cta;
    const size_t cap = (size_t)nsm * 16;
    if (ctas > cap)
        ctas = cap;
    return (int)(ctas ? ctas : 1);
}

// One warp per tile column segment (nb contiguous doubles on both sides).
// With cexp, also the largest biased exponent of every matrix column
// (integer atomicMax per segment; cexp cleared beforehand).
__global__ void k_cm2tile(const double *__restrict__ A, int64_t lda, int64_t m, int64_t n,
                          double *__restrict__ tiles, int nb, int p, int q, int *nonfinite, int *cexp)
{
    const int lane = threadIdx.x & 31;
    const size_t nseg = (size_t)p * q * nb;
    const size_t wstride = (size_t)gridDim.x * (blockDim.x >> 5);
    bool bad = false;
    for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += wstride) {
        const int c = (int)(s % nb);
        const size_t t = s / nb;
        const int i = (int)(t % p), j = (int)(t / p);
        const int64_t col = (int64_t)j * nb + c, row0 = (int64_t)i * nb;
        int valid = 0;
        if (col < n) {
            const int64_t rem = m - row0;
            valid = rem < nb ? (int)rem : nb;
        }
        const double *src = A + col * lda + row0;
        double *dst = tiles + (t * nb + c) * nb;
        unsigned int emax = 0;
        for (int r = lane; r < nb; r += 32) {
            double v = 0.0;
            if (r < valid) {
                v = __ldg(src + r);
                bad |= !isfinite(v);
                emax = max(emax, (unsigned int)(__double2hiint(v) >> 20) & 0x7FFu);
            }
            dst[r] = v;
        }
        if (cexp != nullptr) {
            emax = __reduce_max_sync(0xffffffffu, emax);
            if (lane == 0 && emax > 0 && col < n)
                atomicMax(cexp + col, (int)emax);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0)
        atomicExch(nonfinite, 1);
}

__global__ void k_tile2cm(const double *__restrict__ tiles, int nb, int p, int q, int64_t m, int64_t n,
                          double *__restrict__ A, int64_t lda, int upper_only, int64_t rows_out)
{
    const int lane = threadIdx.x & 31;
    const size_t nseg = (size_t)p * n;  // (tile row i, output column col)
    const size_t wstride = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += wstride) {
        const int i = (int)(s % p);
        const int64_t col = (int64_t)(s / p);
        const int j = (int)(col / nb), c = (int)(col % nb);
        const int64_t row0 = (int64_t)i * nb;
        const double *src = tiles + (((size_t)j * p + i) * nb + c) * nb;
        for (int r = lane; r < nb; r += 32) {
            const int64_t row = row0 + r;
            if (row >= rows_out)
                break;
            double v = src[r];
            if (upper_only && row > col)
                v = 0.0;
            A[col * lda + row] = v;
        }
    }
}

__global__ void k_strips2cm(const double *__restrict__ T, int nb, int ib, int p, int q, int64_t n,
                            double *__restrict__ Tout, int64_t ldt)
{
    const int steps = p < q ? p : q;
    const size_t rows = (size_t)p * ib;
    const size_t total = rows * (size_t)n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e % rows;
        const int64_t col = (int64_t)(e / rows);
        const int i = (int)(r / ib), b = (int)(r % ib);
        const int k = (int)(col / nb), c = (int)(col % nb);
        double v = 0.0;
        if (k < steps && i >= k)
            v = T[(((size_t)k * p + i) * nb + c) * ib + b];
        Tout[col * ldt + r] = v;
    }
}

__global__ void k_cm2rows(const double *__restrict__ B, int64_t ldb, int64_t m, int64_t ncols,
                          double *__restrict__ Bt, int nb, int p, int64_t ncp)
{
    const int lane = threadIdx.x & 31;
    const size_t nseg = (size_t)p * ncp;
    const size_t wstride = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += wstride) {
        const int i = (int)(s % p);
        const int64_t c = (int64_t)(s / p);
        const int64_t row0 = (int64_t)i * nb;
        double *dst = Bt + ((size_t)i * ncp + c) * nb;
        for (int r = lane; r < nb; r += 32) {
            const int64_t row = row0 + r;
            dst[r] = (c < ncols && row < m) ? B[c * ldb + row] : 0.0;
        }
    }
}

__global__ void k_rows2cm(const double *__restrict__ Bt, int nb, int p, int64_t ncp, int64_t m,
                          int64_t ncols, double *__restrict__ B, int64_t ldb)
{
    const int lane = threadIdx.x & 31;
    const size_t nseg = (size_t)p * ncols;
    const size_t wstride = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += wstride) {
        const int i = (int)(s % p);
        const int64_t c = (int64_t)(s / p);
        const int64_t row0 = (int64_t)i * nb;
        const double *src = Bt + ((size_t)i * ncp + c) * nb;
        for (int r = lane; r < nb; r += 32) {
            const int64_t row = row0 + r;
            if (row < m)
                B[c * ldb + row] = src[r];
        }
    }
}

int launch_cm2tile(const double *A, int64_t lda, int64_t m, int64_t n, double *tiles, int nb, int p,
                   int q, SchedCtrl *ctrl, int *cexp, cudaStream_t st)
{
    const size_t segs = (size_t)p * q * nb;
    k_cm2tile<<<grid_for(segs), 256, 0, st>>>(A, lda, m, n, tiles, nb, p, q, &ctrl->nonfinite, cexp);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_tile2cm(const double *tiles, int nb, int p, int q, int64_t m, int64_t n, double *A,
                   int64_t lda, int upper_only, int64_t rows_out, cudaStream_t st)
{
    const size_t segs = (size_t)p * n;
    if (segs == 0)
        return 0;
    k_tile2cm<<<grid_for(segs), 256, 0, st>>>(tiles, nb, p, q, m, n, A, lda, upper_only, rows_out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_strips2cm(const double *T, int nb, int ib, int p, int q, int64_t n, double *Tout,
                     int64_t ldt, cudaStream_t st)
{
    const size_t total = (size_t)p * ib * n;
    if (total == 0)
        return 0;
    k_strips2cm<<<grid_for(total / 32 + 1), 256, 0, st>>>(T, nb, ib, p, q, n, Tout, ldt);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_cm2rows(const double *B, int64_t ldb, int64_t m, int64_t ncols, double *Bt, int nb, int p,
                   int64_t ncp, cudaStream_t st)
{
    const size_t segs = (size_t)p * ncp;
    if (segs == 0)
        return 0;
    k_cm2rows<<<grid_for(segs), 256, 0, st>>>(B, ldb, m, ncols, Bt, nb, p, ncp);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_rows2cm(const double *Bt, int nb, int p, int64_t ncp, int64_t m, int64_t ncols, double *B,
                   int64_t ldb, cudaStream_t st)
{
    const size_t segs = (size_t)p * ncols;
    if (segs == 0)
        return 0;
    k_rows2cm<<<grid_for(segs), 256, 0, st>>>(Bt, nb, p, ncp, m, ncols, B, ldb);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

// B (m x ncols, ld ldb) <- the leading ncols columns of the identity; one
// warp per column, grid-stride.
__global__ void __launch_bounds__(256) k_eye(double *B, int64_t ldb, int64_t m, int64_t ncols)
{
    const int64_t warps = (int64_t)gridDim.x * 8;
    const int lane = threadIdx.x & 31;
    for (int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); c < ncols; c += warps)
        for (int64_t r = lane; r < m; r += 32)
            B[c * ldb + r] = (r == c) ? 1.0 : 0.0;
}

int launch_eye(double *B, int64_t ldb, int64_t m, int64_t ncols, cudaStream_t st)
{
    if (m == 0 || ncols == 0)
        return 0;
    k_eye<<<grid_for((size_t)ncols), 256, 0, st>>>(B, ldb, m, ncols);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

}  // namespace tqr
