// trsm.cu -- tiled triangular solves with the R of a factorization (the
// upper triangles of the first q tile rows), on right-hand sides in the
// tile-row layout (p blocks of nb x ncp, ld nb):
//   R X = Y    (back substitution: the least-squares solve after Q^T B)
//   R^T X = Y  (forward substitution: h = R^-T w of the refinement)
// block by block: the diagonal tile's solve (k_trsm_diag), then the
// off-diagonal tiles' updates of the block rows still to solve
// (k_trsm_update).
//
// Each right-hand-side column is solved by one warp, with no block barrier
// per column: the columns of R are staged in shared memory 32 at a time
// and each warp runs its column's recurrence on them.  The solves are
// FP64; on GB300 the FP64 pipe (about 2 DFMA per clock per SM) bounds
// them, so a CTA takes 4 columns and the grid spreads the columns (and for
// the updates, 32-row groups of each tile) over the SMs.  x = y / R(c,c) is
// taken as y times the reciprocal of R(c,c), formed once per column.
#include "factor.h"

namespace tqr {
namespace {

constexpr int TRSM_CW = 4;    // right-hand-side columns per CTA, one warp each
constexpr int TRSM_CB = 32;   // columns (rows, for R^T) of R staged per round

size_t diag_smem(int nb) { return ((size_t)TRSM_CW * nb + (size_t)TRSM_CB * (nb + 1) + TRSM_CB) * sizeof(double); }
size_t update_smem(int nb) { return ((size_t)nb * 33 + (size_t)TRSM_CW * nb) * sizeof(double); }

}  // namespace

// Diagonal block j: Y_j <- R_jj^-1 Y_j (TRANS: R_jj^-T Y_j) for the first
// ncols columns; rows and columns past n are not part of the system (zero
// on output).  An exact zero R(c,c) sets *flag to its global index + 1 and
// gives x = 0 there.
template <bool TRANS>
__global__ void __launch_bounds__(32 * TRSM_CW) k_trsm_diag(const double *__restrict__ tiles, double *Bt, int nb,
                                                            int p, int64_t ncp, int j, int64_t n, int64_t ncols,
                                                            int *flag)
{
    extern __shared__ double sm[];
    double *ys = sm;                                // [TRSM_CW][nb]: the warps' columns
    double *rs = ys + TRSM_CW * nb;                 // [TRSM_CB][nb + 1]: staged R
    double *rcp = rs + (size_t)TRSM_CB * (nb + 1);  // [TRSM_CB]: 1 / R(c,c)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col = (int64_t)blockIdx.x * TRSM_CW + warp;
    const bool active = col < ncols;
    const double *R = tiles + ((size_t)j * p + j) * (size_t)nb * nb;
    double *Y = Bt + ((size_t)j * ncp + (size_t)(active ? col : 0)) * nb;
    double *y = ys + warp * nb;
    for (int r = lane; r < nb; r += 32)
        y[r] = active ? Y[r] : 0.0;
    const int64_t col0 = (int64_t)j * nb;
    int last = nb - 1;
    if (col0 + last >= n)
        last = (int)(n - 1 - col0);
    const int nblk = (last + TRSM_CB) / TRSM_CB;
    for (int bi = 0; bi < nblk; bi++) {
        const int b = TRANS ? bi : nblk - 1 - bi;
        const int c0 = b * TRSM_CB;
        const int cend = c0 + TRSM_CB < last + 1 ? c0 + TRSM_CB : last + 1;
        __syncthreads();
        // rs[cc][r] = R(r, c0 + cc) (column c0 + cc), or R(c0 + cc, r) (row);
        // consecutive threads read consecutive addresses of R
        for (int e = threadIdx.x; e < TRSM_CB * nb; e += blockDim.x) {
            int cc, r;
            if (TRANS) {
                r = e / TRSM_CB;
                cc = e - r * TRSM_CB;
            } else {
                cc = e / nb;
                r = e - cc * nb;
            }
            const int c = c0 + cc;
            rs[cc * (nb + 1) + r] =
                c < cend ? ldcg(R + (TRANS ? (size_t)r * nb + c : (size_t)c * nb + r)) : 0.0;
        }
        if (threadIdx.x < TRSM_CB) {
            const int c = c0 + threadIdx.x;
            const double d = c < cend ? ldcg(R + (size_t)c * nb + c) : 1.0;
            if (d == 0.0)
                atomicCAS(flag, 0, (int)(col0 + c + 1));
            rcp[threadIdx.x] = d != 0.0 ? 1.0 / d : 0.0;
        }
        __syncthreads();
        for (int t = 0; t < cend - c0; t++) {
            const int cc = TRANS ? t : cend - c0 - 1 - t, c = c0 + cc;
            const double x = y[c] * rcp[cc];
            __syncwarp();
            if (lane == 0)
                y[c] = x;
            const double *rc = rs + cc * (nb + 1);
            if (TRANS) {
                for (int r = c + 1 + lane; r <= last; r += 32)
                    y[r] = fma(-rc[r], x, y[r]);
            } else {
                for (int r = lane; r < c; r += 32)
                    y[r] = fma(-rc[r], x, y[r]);
            }
            __syncwarp();
        }
    }
    if (active)
        for (int r = lane; r < nb; r += 32)
            Y[r] = r <= last ? y[r] : 0.0;
}

// Y_i -= R_ij X_j for the block rows i < j (TRANS: Y_i -= R_ji^T X_j for
// i > j), X_j the solved block row j.  Block (x, y, z): block row i (x), 32
// rows of it (y), 4 right-hand-side columns (z); warp q takes column q and
// its lanes the 32 rows, with the 32 x nb rows of the product's matrix
// staged in shared memory as [k][r].
template <bool TRANS>
__global__ void __launch_bounds__(32 * TRSM_CW) k_trsm_update(const double *__restrict__ tiles, double *Bt, int nb,
                                                              int p, int64_t ncp, int j, int64_t ncols)
{
    extern __shared__ double sm[];
    double *ms = sm;                 // [nb][33]
    double *xs = ms + (size_t)nb * 33;   // [TRSM_CW][nb]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = TRANS ? j + 1 + (int)blockIdx.x : (int)blockIdx.x;
    const int r0 = 32 * (int)blockIdx.y;
    const int64_t col = (int64_t)blockIdx.z * TRSM_CW + warp;
    const bool active = col < ncols;
    // NOTRANS: tile (i, j), M(r, k) = R_ij(r, k); TRANS: tile (j, i), M(r, k) = R_ji(k, r)
    const double *Rt = tiles + (TRANS ? ((size_t)i * p + j) : ((size_t)j * p + i)) * (size_t)nb * nb;
    const double *X = Bt + ((size_t)j * ncp + (size_t)(active ? col : 0)) * nb;
    double *Y = Bt + ((size_t)i * ncp + (size_t)(active ? col : 0)) * nb;
    for (int k = lane; k < nb; k += 32)
        xs[warp * nb + k] = active ? X[k] : 0.0;
    for (int e = threadIdx.x; e < 32 * nb; e += blockDim.x) {
        int rr, k;
        if (TRANS) {   // R_ji(k, r0 + rr): column r0 + rr of the tile, k consecutive
            rr = e / nb;
            k = e - rr * nb;
            ms[k * 33 + rr] = ldcg(Rt + (size_t)(r0 + rr) * nb + k);
        } else {       // R_ij(r0 + rr, k): column k of the tile, rr consecutive
            k = e >> 5;
            rr = e & 31;
            ms[k * 33 + rr] = ldcg(Rt + (size_t)k * nb + r0 + rr);
        }
    }
    __syncthreads();
    if (!active)
        return;
    const double *x = xs + warp * nb;
    double acc0 = Y[r0 + lane], acc1 = 0.0;
    int k = 0;
    for (; k + 1 < nb; k += 2) {
        acc0 = fma(-ms[k * 33 + lane], x[k], acc0);
        acc1 = fma(-ms[(k + 1) * 33 + lane], x[k + 1], acc1);
    }
    if (k < nb)
        acc0 = fma(-ms[k * 33 + lane], x[k], acc0);
    Y[r0 + lane] = acc0 + acc1;
}

template <bool TRANS>
static int launch_trsm_t(const WsLayout &L, const double *tiles, double *Bt, int64_t ncp, int *flag,
                         cudaStream_t st, int64_t ncols)
{
    const int nb = L.nb;
    if (kernel_smem_optin((const void *)k_trsm_diag<TRANS>, diag_smem(nb)) != 0 ||
        kernel_smem_optin((const void *)k_trsm_update<TRANS>, update_smem(nb)) != 0)
        return TILEQR_ERR_CUDA;
    const unsigned int gc = (unsigned int)((ncols + TRSM_CW - 1) / TRSM_CW);
    for (int t = 0; t < L.q; t++) {
        const int j = TRANS ? t : L.q - 1 - t;
        k_trsm_diag<TRANS><<<gc, 32 * TRSM_CW, diag_smem(nb), st>>>(tiles, Bt, nb, L.p, ncp, j, L.n, ncols, flag);
        count_launch();
        const int rows = TRANS ? L.q - 1 - j : j;   // block rows still to update
        if (rows > 0) {
            k_trsm_update<TRANS><<<dim3((unsigned)rows, (unsigned)(nb / 32), gc), 32 * TRSM_CW, update_smem(nb), st>>>(
                tiles, Bt, nb, L.p, ncp, j, ncols);
            count_launch();
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_trsm(const WsLayout &L, const double *tiles, double *Bt, int64_t ncp, int *flag, cudaStream_t st,
                bool trans, int64_t ncols)
{
    if (ncols < 0 || ncols > ncp)
        ncols = ncp;
    if (ncols == 0 || L.q == 0)
        return 0;
    return trans ? launch_trsm_t<true>(L, tiles, Bt, ncp, flag, st, ncols)
                 : launch_trsm_t<false>(L, tiles, Bt, ncp, flag, st, ncols);
}

}  // namespace tqr
