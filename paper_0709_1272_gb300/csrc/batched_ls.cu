// batched_ls.cu -- least-squares solves of a factored batch (the batched
// form of the factorization), one right-hand side per matrix, refined in
// FP64 on the augmented system [I A; A^T 0] [r; x] = [b; 0] (Bjorck, 1967;
// an addition to the paper), all matrices in one persistent launch.
//
// One CTA owns one matrix at a time (largest first, claimed with a ticket)
// and runs the whole refinement on it: u = b - r - A x, w = -A^T r,
// h = R^-T w, d = Q^T u, dx = R^-1 (d1 - h), dr = Q [h; d2], x += dx,
// r += dr, until ||dx|| <= tol ||x||, ||dx|| stops halving, or the rate of
// the last two steps puts the next correction below tol.  Q^T replays
// the factorization's DLARFB / DSSRFB transformations on the vector in the
// order of Algorithm 2 (Sec. 3.2.1), inner blocks in order (Sec. 3.2.3); Q
// replays them in reverse with T_l in place of T_l^T.  Starting from x = 0,
// r = 0, one step is the plain solve x = R^-1 (Q^T b)(0:n).  Everything is
// FP64; the factors may come from a TILEQR_TF32 factorization.
#include <cmath>
#include <cstring>
#include <vector>

#include "dag.cuh"
#include "factor.h"

namespace tqr {

struct BlsEntry {
    const double *b;
    double *x;
    double *u, *r, *h, *dx;   // per-matrix vectors: m, m, n, n entries
};
struct BlsInfo {
    int iterations;
    int status;   // 1 stopped by the rule, 0 step limit reached, -1 exact zero on diag R
    double correction;
};

constexpr int BLS_CHUNK = 1024;

// Reductions over the CTA (256 threads): all threads get the result.
__device__ __forceinline__ double cta_sum(double v, double *red)
{
    v = warp_allsum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NWARP; w++)
        s += red[w];
    return s;
}

// Element (r, c) of R, r <= c, in the tiles of a matrix.
template <int NB>
__device__ __forceinline__ double r_elem(const MatInfo &mi, int r, int c)
{
    return mi.tiles[(((size_t)(c / NB) * mi.p + r / NB) * NB + (c % NB)) * NB + (r % NB)];
}

// The DSSRFB (tile (i, k): full reflectors) or DLARFB (i == k: unit lower
// reflectors of the diagonal tile) transformation of step k on the vector v,
// as Q^T (NOTRANS false: blocks in order, T_l^T) or Q (reverse, T_l).
template <int NB, int S, bool NOTRANS>
__device__ void bls_task(const MatInfo &mi, int i, int k, double *v, double *vk, double *vi, double *y,
                         double *w)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool lb = i == k;
    const double *V = mi.tiles + ((size_t)k * mi.p + i) * NB * NB;
    const double *T = mi.T + ((size_t)k * mi.p + i) * S * NB;
    const int64_t rk = (int64_t)k * NB, ri = (int64_t)i * NB;
    for (int r = tid; r < NB; r += NT) {
        vk[r] = rk + r < mi.m ? v[rk + r] : 0.0;
        if (!lb)
            vi[r] = ri + r < mi.m ? v[ri + r] : 0.0;
    }
    __syncthreads();
    for (int lb_ = 0; lb_ < NB / S; lb_++) {
        const int l0 = (NOTRANS ? NB / S - 1 - lb_ : lb_) * S;
        // y = V_l^T x (+ the identity rows of vk for DSSRFB)
        for (int a = warp; a < S; a += NWARP) {
            const int j = l0 + a;
            const double *col = V + (size_t)j * NB;
            double s = 0.0;
            if (lb) {
                for (int r = lane; r < NB; r += 32)
                    s = fma(r < j ? 0.0 : (r == j ? 1.0 : col[r]), vk[r], s);
            } else {
                for (int r = lane; r < NB; r += 32)
                    s = fma(col[r], vi[r], s);
            }
            s = warp_allsum(s);
            if (lane == 0)
                y[a] = lb ? s : vk[j] + s;
        }
        __syncthreads();
        // w = T_l^T y (Q^T) or T_l y (Q); T_l upper, T_l(b, a) at T[(l0 + a) S + b]
        if (tid < S) {
            const int a = tid;
            double s = 0.0;
            if (!NOTRANS) {
                for (int b = 0; b <= a; b++)
                    s = fma(T[(size_t)(l0 + a) * S + b], y[b], s);
            } else {
                for (int b = a; b < S; b++)
                    s = fma(T[(size_t)(l0 + b) * S + a], y[b], s);
            }
            w[a] = s;
        }
        __syncthreads();
        if (lb) {
            for (int r = tid; r < NB; r += NT) {
                double s = 0.0;
                for (int a = 0; a < S; a++) {
                    const int j = l0 + a;
                    const double vv = r < j ? 0.0 : (r == j ? 1.0 : V[(size_t)j * NB + r]);
                    s = fma(vv, w[a], s);
                }
                vk[r] -= s;
            }
        } else {
            if (tid < S)
                vk[l0 + tid] -= w[tid];
            for (int r = tid; r < NB; r += NT) {
                double s = 0.0;
                for (int a = 0; a < S; a++)
                    s = fma(V[(size_t)(l0 + a) * NB + r], w[a], s);
                vi[r] -= s;
            }
        }
        __syncthreads();
    }
    for (int r = tid; r < NB; r += NT) {
        if (rk + r < mi.m)
            v[rk + r] = vk[r];
        if (!lb && ri + r < mi.m)
            v[ri + r] = vi[r];
    }
    __syncthreads();
}

template <int NB, int S>
__device__ void bls_apply_qt(const MatInfo &mi, double *v, double *vk, double *vi, double *y, double *w)
{
    for (int k = 0; k < mi.steps; k++)
        for (int i = k; i < mi.p; i++)
            bls_task<NB, S, false>(mi, i, k, v, vk, vi, y, w);
}
template <int NB, int S>
__device__ void bls_apply_q(const MatInfo &mi, double *v, double *vk, double *vi, double *y, double *w)
{
    for (int k = mi.steps - 1; k >= 0; k--)
        for (int i = mi.p - 1; i >= k; i--)
            bls_task<NB, S, true>(mi, i, k, v, vk, vi, y, w);
}

// x (n entries, in place) = R^-1 x by blocks of 32 columns from the last;
// returns false if R has an exact zero on its diagonal.
template <int NB>
__device__ bool bls_rsolve(const MatInfo &mi, double *x)
{
    const int n = (int)mi.n, tid = threadIdx.x, lane = tid & 31;
    bool ok = true;
    for (int c1 = n; c1 > 0; c1 -= 32) {
        const int c0 = c1 > 32 ? c1 - 32 : 0;
        if (tid < 32) {
            double yv = c0 + lane < c1 ? x[c0 + lane] : 0.0;
            for (int c = c1 - 1; c >= c0; c--) {
                const int j = c - c0;
                const double d = r_elem<NB>(mi, c, c);
                const double xc = d != 0.0 ? __shfl_sync(0xffffffffu, yv, j) / d : 0.0;
                ok &= d != 0.0;
                if (lane == j)
                    yv = xc;
                else if (lane < j)
                    yv = fma(-r_elem<NB>(mi, c0 + lane, c), xc, yv);
            }
            if (c0 + lane < c1)
                x[c0 + lane] = yv;
        }
        __syncthreads();
        for (int r = tid; r < c0; r += NT) {
            double s = 0.0;
            for (int c = c0; c < c1; c++)
                s = fma(r_elem<NB>(mi, r, c), x[c], s);
            x[r] -= s;
        }
        __syncthreads();
    }
    return __syncthreads_and(ok);
}

// h (n entries, in place) = R^-T h by blocks of 32 columns from the first.
template <int NB>
__device__ bool bls_rtsolve(const MatInfo &mi, double *h)
{
    const int n = (int)mi.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    bool ok = true;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int c1 = c0 + 32 < n ? c0 + 32 : n;
        // h_c -= sum_{r < c0} R(r, c) h_r for the block's columns (warp per column)
        for (int c = c0 + warp; c < c1; c += NWARP) {
            double s = 0.0;
            for (int r = lane; r < c0; r += 32)
                s = fma(r_elem<NB>(mi, r, c), h[r], s);
            s = warp_allsum(s);
            if (lane == 0)
                h[c] -= s;
        }
        __syncthreads();
        if (tid < 32) {
            double wv = c0 + lane < c1 ? h[c0 + lane] : 0.0;
            for (int c = c0; c < c1; c++) {
                const int j = c - c0;
                const double d = r_elem<NB>(mi, c, c);
                const double hc = d != 0.0 ? __shfl_sync(0xffffffffu, wv, j) / d : 0.0;
                ok &= d != 0.0;
                if (lane == j)
                    wv = hc;
                else if (lane > j && c0 + lane < c1)
                    wv = fma(-r_elem<NB>(mi, c, c0 + lane), hc, wv);
            }
            if (c0 + lane < c1)
                h[c0 + lane] = wv;
        }
        __syncthreads();
    }
    return __syncthreads_and(ok);
}

// The refinement of one matrix by one CTA (see the file comment).
template <int NB, int S>
__device__ void bls_refine(const MatInfo &mi, const BlsEntry &e, int max_iter, double tol, BlsInfo *out,
                           double *sm)
{
    double *vk = sm, *vi = sm + NB, *y = sm + 2 * NB, *w = y + 32, *red = w + 32, *xs = red + 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m = mi.m, n = mi.n;
    for (int64_t r = tid; r < m; r += NT)
        e.r[r] = 0.0;
    for (int64_t c = tid; c < n; c += NT)
        e.x[c] = 0.0;
    __syncthreads();
    double prev = INFINITY, ratio = 0.0;
    int it = 0, status = 0;
    for (it = 1; it <= max_iter; it++) {
        // u = b - r - A x (x staged in chunks)
        {
            double acc[8];
            for (int64_t rb = 0; rb < m; rb += 8 * NT) {
#pragma unroll
                for (int q = 0; q < 8; q++)
                    acc[q] = 0.0;
                for (int64_t c0 = 0; c0 < n; c0 += BLS_CHUNK) {
                    const int nc = (int)(n - c0 < BLS_CHUNK ? n - c0 : BLS_CHUNK);
                    __syncthreads();
                    for (int c = tid; c < nc; c += NT)
                        xs[c] = e.x[c0 + c];
                    __syncthreads();
                    for (int c = 0; c < nc; c++) {
                        const double *col = mi.A + (size_t)(c0 + c) * mi.lda;
#pragma unroll
                        for (int q = 0; q < 8; q++) {
                            const int64_t r = rb + q * NT + tid;
                            if (r < m)
                                acc[q] = fma(col[r], xs[c], acc[q]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int64_t r = rb + q * NT + tid;
                    if (r < m)
                        e.u[r] = (e.b[r] - e.r[r]) - acc[q];
                }
            }
        }
        // h = -A^T r (warp per column), then h = R^-T h
        for (int64_t c = warp; c < n; c += NWARP) {
            double s = 0.0;
            if (it > 1) {
                const double *col = mi.A + (size_t)c * mi.lda;
                for (int64_t r = lane; r < m; r += 32)
                    s = fma(col[r], e.r[r], s);
                s = warp_allsum(s);
            }
            if (lane == 0)
                e.h[c] = -s;
        }
        __syncthreads();
        bool ok = bls_rtsolve<NB>(mi, e.h);
        // d = Q^T u (in u); dx = R^-1 (d1 - h); then u(0:n) = h, u = Q u (= dr)
        bls_apply_qt<NB, S>(mi, e.u, vk, vi, y, w);
        for (int64_t c = tid; c < n; c += NT) {
            e.dx[c] = e.u[c] - e.h[c];
            e.u[c] = e.h[c];
        }
        __syncthreads();
        ok &= bls_rsolve<NB>(mi, e.dx);
        bls_apply_q<NB, S>(mi, e.u, vk, vi, y, w);
        // x += dx, r += dr; the sizes of dx and x
        double sdx = 0.0, sx = 0.0;
        for (int64_t c = tid; c < n; c += NT) {
            const double xn = e.x[c] + e.dx[c];
            e.x[c] = xn;
            sdx = fma(e.dx[c], e.dx[c], sdx);
            sx = fma(xn, xn, sx);
        }
        for (int64_t r = tid; r < m; r += NT)
            e.r[r] += e.u[r];
        sdx = cta_sum(sdx, red);
        sx = cta_sum(sx, red);
        __syncthreads();
        if (!ok) {
            status = -1;
            break;
        }
        const double ndx = sqrt(sdx), nx = sqrt(sx);
        ratio = nx > 0.0 ? ndx / nx : ndx;
        // as tileqr_solve_ls_refine: also stop once the rate of the last two
        // steps puts the next correction below tol
        const bool predicted = it > 2 && ndx <= 0.5 * prev && ratio * (ndx / prev) <= tol;
        if (it > 1 && (ratio <= tol || ndx > 0.5 * prev || predicted)) {
            status = 1;
            break;
        }
        prev = ndx;
    }
    if (tid == 0) {
        out->iterations = it > max_iter ? max_iter : it;
        out->status = status;
        out->correction = ratio;
    }
}

template <int NB, int S>
__global__ void __launch_bounds__(NT) k_batched_ls(const MatInfo *__restrict__ mats, int count,
                                                   const BlsEntry *__restrict__ ent, int max_iter, double tol,
                                                   BlsInfo *info, unsigned int *ticket)
{
    __shared__ double sm[2 * NB + 32 + 32 + 8 + BLS_CHUNK];
    __shared__ int s_b;
    const int *order = (const int *)(mats + count);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int t = atomicAdd(ticket, 1u);
            s_b = t < (unsigned int)count ? order[t] : -1;
        }
        __syncthreads();
        const int b = s_b;
        __syncthreads();
        if (b < 0)
            break;
        const MatInfo mi = mats[b];
        if (mi.n > 0 && mi.m >= mi.n)
            bls_refine<NB, S>(mi, ent[b], max_iter, tol, info + b, sm);
        __syncthreads();
    }
}

}  // namespace tqr

using namespace tqr;

namespace {

struct BlsLayout {
    size_t ticket, ent, info, vecs, end;
};

BlsLayout bls_layout(const tileqr_batch *bt, const int64_t *m, const int64_t *n)
{
    BlsLayout L{};
    size_t off = 0;
    L.ticket = off;
    off += 256;
    L.ent = off;
    off += align256((size_t)(bt->count ? bt->count : 1) * sizeof(BlsEntry));
    L.info = off;
    off += align256((size_t)(bt->count ? bt->count : 1) * sizeof(BlsInfo));
    L.vecs = off;
    size_t v = 0;
    for (int b = 0; b < bt->count; b++)
        v += (size_t)(2 * m[b] + 2 * n[b]) * 8;
    off += align256(v);
    L.end = off;
    return L;
}

// The shapes of a prepared batch, from its table on the device.
int batch_shapes(const tileqr_batch *bt, std::vector<int64_t> &m, std::vector<int64_t> &n)
{
    std::vector<MatInfo> infos(bt->count);
    if (bt->count > 0 &&
        cudaMemcpy(infos.data(), (char *)bt->workspace + bt->off_mats, (size_t)bt->count * sizeof(MatInfo),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    m.resize(bt->count);
    n.resize(bt->count);
    for (int b = 0; b < bt->count; b++) {
        m[b] = infos[b].m;
        n[b] = infos[b].n;
    }
    return 0;
}

}  // namespace

extern "C" int tileqr_batched_ls_workspace_size(const tileqr_batch *bt, size_t *bytes)
{
    if (bt == nullptr)
        return -1;
    if (bytes == nullptr)
        return -2;
    std::vector<int64_t> m, n;
    const int rc = batch_shapes(bt, m, n);
    if (rc)
        return rc;
    *bytes = bls_layout(bt, m.data(), n.data()).end;
    return 0;
}

extern "C" int tileqr_batched_solve_ls(const tileqr_batch *bt, const double *const *B, double *const *X,
                                       int max_iter, double tol, void *workspace, size_t ws_bytes,
                                       tileqr_stream_t stream, tileqr_refine_info *summary)
{
    if (bt == nullptr)
        return -1;
    if (bt->count > 0 && B == nullptr)
        return -2;
    if (bt->count > 0 && X == nullptr)
        return -3;
    if (max_iter < 1)
        return -4;
    if (!(tol > 0.0))
        return -5;
    std::vector<int64_t> m, n;
    int rc = batch_shapes(bt, m, n);
    if (rc)
        return rc;
    for (int b = 0; b < bt->count; b++) {
        if (m[b] < n[b])
            return -1;
        if ((B[b] == nullptr && m[b] > 0) || (X[b] == nullptr && n[b] > 0))
            return B[b] == nullptr ? -2 : -3;
    }
    const BlsLayout L = bls_layout(bt, m.data(), n.data());
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.end)
        return TILEQR_ERR_WORKSPACE;
    tileqr_refine_info loc{};
    if (summary == nullptr)
        summary = &loc;
    std::memset(summary, 0, sizeof(*summary));
    summary->method = 3;
    if (bt->count == 0)
        return 0;
    char *ws = (char *)workspace;
    std::vector<BlsEntry> ent(bt->count);
    double *v = (double *)(ws + L.vecs);
    for (int b = 0; b < bt->count; b++) {
        ent[b].b = B[b];
        ent[b].x = X[b];
        ent[b].u = v;
        ent[b].r = v + m[b];
        ent[b].h = v + 2 * m[b];
        ent[b].dx = v + 2 * m[b] + n[b];
        v += 2 * m[b] + 2 * n[b];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws + L.ticket, 0, 256, st) != cudaSuccess ||
        cudaMemsetAsync(ws + L.info, 0, (size_t)bt->count * sizeof(BlsInfo), st) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.ent, ent.data(), ent.size() * sizeof(BlsEntry), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return TILEQR_ERR_CUDA;
    const MatInfo *mats = (const MatInfo *)((char *)bt->workspace + bt->off_mats);
    int grid = 0;
#define TQR_CASE(NB_, S_)                                                                                  \
    if (bt->nb == NB_ && bt->ib == S_) {                                                                   \
        if ((rc = kernel_grid((const void *)k_batched_ls<NB_, S_>, NT, 0, &grid)) != 0)                    \
            return rc;                                                                                     \
        k_batched_ls<NB_, S_><<<grid, NT, 0, st>>>(mats, bt->count, (const BlsEntry *)(ws + L.ent), max_iter, \
                                                   tol, (BlsInfo *)(ws + L.info), (unsigned int *)(ws + L.ticket)); \
    } else
    TQR_CASE(64, 16)
    TQR_CASE(64, 32)
    TQR_CASE(128, 16)
    TQR_CASE(128, 32)
    TQR_CASE(256, 16)
    TQR_CASE(256, 32)
#undef TQR_CASE
    return TILEQR_ERR_UNSUPPORTED;
    count_launch();
    if (cudaGetLastError() != cudaSuccess)
        return TILEQR_ERR_CUDA;
    std::vector<BlsInfo> info(bt->count);
    if (cudaMemcpyAsync(info.data(), ws + L.info, info.size() * sizeof(BlsInfo), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    summary->converged = 1;
    for (int b = 0; b < bt->count; b++) {
        if (n[b] == 0)
            continue;
        if (info[b].status < 0)
            return TILEQR_ERR_SINGULAR;
        summary->iterations = info[b].iterations > summary->iterations ? info[b].iterations : summary->iterations;
        summary->converged &= info[b].status == 1 ? 1 : 0;
        summary->rel_residual = info[b].correction > summary->rel_residual ? info[b].correction
                                                                             : summary->rel_residual;
    }
    return 0;
}
