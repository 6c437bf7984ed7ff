// refine.cu -- solve of A x = b with FP64 iterative refinement for the
// mixed-precision factorization (square A, or tall A with b in its range; one
// right-hand side).  The stopping test is the FP64 residual ||b - A x||.
//
// The correction solves use an FP32 copy of the factors: M^{-1} v =
// R^{-1} (Q^T v)(0:n) with Q^T applied as the factorization's task graph
// restricted to one column (DLARFB / DSSRFB, and DTTMQR for the tree form, on
// vectors, single precision; the apply graph of graph.cuh) and R^{-1} as a
// tiled back substitution with precomputed inverses of R's diagonal tiles.  Residuals r = b - A x, the Krylov vectors and x are FP64.
// Classical refinement (x += M^{-1} r) is tried first; if the residual stops
// shrinking, the solve continues with restarted flexible GMRES on A d = r
// with M^{-1} as the right preconditioner (GMRES-IR).
#include <cmath>
#include <cstring>
#include <vector>

#include "factor.h"
#include "graph.cuh"
#include "sched.cuh"
#include "tile_mixed.cuh"

namespace tqr {

// ---------------------------------------------------------------------------
// Range: the correction solve runs in FP32, whose range (1e-38 .. 3e38) is
// far narrower than FP64's.  So it works on scaled quantities, every scaling
// a power of two (exact):
//  - b enters as b' = b 2^-sb (largest entry in [1, 2)), x' solves A x' = b'
//    and x = x' 2^sb at the end;
//  - each vector v handed to M^{-1} is scaled by 2^-sv the same way;
//  - the FP32 copy of R is R' = R D^-1, D = diag(2^s_c) with s_c from the
//    largest exponent of column c of R (||R(:,c)|| = ||a_c|| <= 2^s_c, see
//    col_shift), and its diagonal-tile inverses are D_j U_j^{-1};
// so M^{-1} v = 2^sv D^-1 R'^{-1} (Q^T v 2^-sv)(0:n) with every FP32
// quantity of moderate size.  The reflectors and T are scale-free.

// FP64 -> FP32 copy (integer conversion), for the T strips.
__global__ void k_to_f32(const double *__restrict__ src, float *__restrict__ dst, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = f64_to_f32_bits(src[i]);
}

// Largest biased exponent of the entries of R's column c (the tiles on and
// above the diagonal, rows <= c in the diagonal tile), into cexp[c] (cleared
// beforehand); one warp per tile column segment.
__global__ void k_r_colexp(const double *__restrict__ tiles, int p, int q, int *cexp)
{
    const int lane = threadIdx.x & 31;
    const size_t nseg = (size_t)q * 128 * q;   // (column, tile row i < q)
    for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg;
         s += (size_t)gridDim.x * (blockDim.x >> 5)) {
        const int i = (int)(s % q);
        const int col = (int)(s / q), j = col >> 7, c = col & 127;
        if (i > j)
            continue;
        const double *src = tiles + (((size_t)j * p + i) * 128 + c) * 128;
        unsigned int e = 0;
        for (int r = lane; r < 128; r += 32)
            if (i < j || r <= c)
                e = max(e, (unsigned int)(__double2hiint(ldcg(src + r)) >> 20) & 0x7FFu);
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0 && e > 0)
            atomicMax(cexp + col, (int)e);
    }
}

// FP32 copy of the factored tiles: R' = R D^-1 (tiles i < j, and rows <= c
// of diagonal tile j), the reflectors as they are.
__global__ void k_tiles_to_f32(const double *__restrict__ tiles, int p, int q, const int *__restrict__ cexp,
                               int lm, float *__restrict__ dst)
{
    const size_t n = (size_t)p * q * 128 * 128;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t t = e >> 14;
        const int i = (int)(t % p), j = (int)(t / p), c = (int)((e >> 7) & 127), r = (int)(e & 127);
        const bool is_r = i < j || (i == j && r <= c);
        dst[e] = f64_to_f32_sc(tiles[e], is_r ? col_shift(cexp[j * 128 + c], lm) : 0);
    }
}

// Largest biased exponent of a vector's entries, into *out (cleared
// beforehand).
__global__ void k_vec_maxexp(const double *__restrict__ v, int64_t n, int *out)
{
    unsigned int e = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        e = max(e, (unsigned int)(__double2hiint(v[i]) >> 20) & 0x7FFu);
    e = __reduce_max_sync(0xffffffffu, e);
    if ((threadIdx.x & 31) == 0 && e > 0)
        atomicMax(out, (int)e);
}
// The power-of-two exponent that brings a largest biased exponent e to [1, 2).
__device__ __forceinline__ int unit_shift(int e) { return e > 0 ? e - 1023 : 0; }

// y = x 2^(sign * unit_shift(*e))  (exact)
__global__ void k_scale_pow2(const double *__restrict__ x, double *y, int64_t n, const int *e, int sign)
{
    const int k = sign * unit_shift(*e);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = ldexp(x[i], k);
}

// Inverse of the upper triangle of diagonal tile j (nb = 128), written as
// FP32 tile Rinv_j (column-major).  Padded columns (beyond n) get a zero
// column and row.  One CTA per tile, thread c computes column c of the
// inverse by back substitution in FP64.
__global__ void __launch_bounds__(128) k_inv_diag(const double *__restrict__ tiles, int p, int q, int64_t n,
                                                  const int *__restrict__ cexp, int lm, float *__restrict__ rinv,
                                                  int *singular)
{
    extern __shared__ double U[];   // 128 x 129, [r][c] row-major padded
    double *rcp = U + 128 * 129;
    const int j = blockIdx.x, c = threadIdx.x;
    const double *T = tiles + ((size_t)j * p + j) * 128 * 128;
    for (int idx = c; idx < 128 * 128; idx += 128) {
        const int cc = idx >> 7, r = idx & 127;
        U[r * 129 + cc] = ldcg(T + idx);
    }
    __syncthreads();
    const int nvalid = (int)((n - (int64_t)j * 128) < 128 ? (n - (int64_t)j * 128) : 128);
    if (c < nvalid) {
        const double d = U[c * 129 + c];
        if (d == 0.0)
            atomicCAS(singular, 0, j * 128 + c + 1);
        rcp[c] = d != 0.0 ? 1.0 / d : 0.0;
    } else {
        rcp[c] = 0.0;
    }
    __syncthreads();
    // column c of X = U^{-1}: X(c,c) = 1/U(c,c); X(r,c) = -(sum_{k=r+1..c} U(r,k) X(k,c)) / U(r,r)
    double x[128];
#pragma unroll 1
    for (int r = 0; r < 128; r++)
        x[r] = 0.0;
    float *out = rinv + (size_t)j * 128 * 128 + (size_t)c * 128;
    if (c < nvalid) {
        x[c] = rcp[c];
#pragma unroll 1
        for (int r = c - 1; r >= 0; r--) {
            double acc = 0.0;
#pragma unroll 1
            for (int k = r + 1; k <= c; k++)
                acc = fma(U[r * 129 + k], x[k], acc);
            x[r] = -acc * rcp[r];
        }
    }
    // the inverse of the column-scaled tile U D_j^-1 is D_j U^-1: row r
    // scaled by 2^s_r
#pragma unroll 1
    for (int r = 0; r < 128; r++)
        out[r] = r < nvalid ? f64_to_f32_sc(x[r], -col_shift(cexp[j * 128 + r], lm)) : 0.0f;
}

// ---------------------------------------------------------------------------
// Q^T v in FP32 for single columns: the task graph LB(k) / SB(i,k) per
// column (same dependencies as the FP64 apply), one 128-thread CTA per task.
struct Apply32Args {
    const float *tiles;   // FP32 copy of the factored tiles
    const float *T;       // FP32 copy of the T strips
    const float *T2;      // FP32 copy of the DTTQRT T strips (tree form), else nullptr
    float *X;             // p row blocks of 128 x ncol (ld 128)
    int p, steps, ncol, S;
    TGraph G;
};

__device__ __forceinline__ size_t apply32_cnt(const Apply32Args &A, int tt, int k, int i, int col)
{
    return (((size_t)tt * A.steps + k) * A.p + i) * A.ncol + col;
}

// One task: LB = DLARFB with a domain head's unit-lower V on its own block;
// SB = DSSRFB of row i into its domain head's block (full V); TB = DTTMQR
// merging head i into its partner's block (upper-triangular V, T2 strips).
// TREE = false is Algorithm 2's flat graph (heads = the diagonal), with its
// successors written out; TREE = true runs the graph functions of graph.cuh.
template <bool TREE>
__global__ void __launch_bounds__(128) k_apply32_dag(Apply32Args A, Queues Q)
{
    __shared__ float Vs[128 * 33];   // V_l as [r][a], ld s+1 (s <= 32)
    __shared__ float Ts[32 * 32];
    __shared__ float xk[128], xi[128];
    __shared__ float part[4][32];
    __shared__ float yw[32];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = A.S;
    const TGraph &G = A.G;
    if (blockIdx.x == 0) {
        const int nd0 = TREE ? g_ndom(G, 0) : 1;
        for (int u = tid; u < A.ncol * nd0; u += 128)
            q_push(Q, 0, encode_task(0, TREE ? g_head(G, 0, u / A.ncol) : 0, u % A.ncol));
    }
    unsigned int ticket = NO_TICKET;   // thread 0's bulk-level claim
    for (;;) {
        if (tid == 0)
            s_cmd = q_acquire(Q, s_code, ticket);
        __syncthreads();
        if (s_cmd != CMD_RUN)
            break;
        int k, i, col;
        decode_task(s_code, k, i, col);
        const int tt = decode_tt(s_code);
        const int kind = TREE ? ga_kind(G, tt, k, i) : (i == k ? K_LARFB : K_SSRFB);
        const bool lb = kind == K_LARFB, tri = TREE && kind == K_TTMQR;
        const int top = !TREE ? k : (lb ? i : (tri ? g_partner(G, k, i) : g_head(G, k, g_dom(G, k, i))));
        const float *Vt = A.tiles + ((size_t)k * A.p + i) * 128 * 128;
        const float *Tt = (tri ? A.T2 : A.T) + ((size_t)k * A.p + i) * (size_t)S * 128;
        float *gxk = A.X + ((size_t)top * A.ncol + col) * 128;
        float *gxi = A.X + ((size_t)i * A.ncol + col) * 128;
        // other CTAs write these blocks in this launch: read them from L2
        xk[tid] = __ldcg(gxk + tid);
        if (!lb)
            xi[tid] = __ldcg(gxi + tid);
        for (int l0 = 0; l0 < 128; l0 += S) {
            __syncthreads();
            for (int idx = tid; idx < 128 * S; idx += 128) {
                const int a = idx >> 7, r = idx & 127;
                const int jj = l0 + a;
                float v = Vt[(size_t)jj * 128 + r];
                if (lb)
                    v = (r < jj) ? 0.0f : (r == jj ? 1.0f : v);
                else if (tri && r > jj)
                    v = 0.0f;
                Vs[r * 33 + a] = v;
            }
            for (int idx = tid; idx < S * S; idx += 128)
                Ts[idx] = Tt[(size_t)l0 * S + idx];
            __syncthreads();
            // y(a) = [x_top(l0+a)] + sum_r V(r,a) x(r)   (x = x_i for SB / TB, x_top for LB)
            const float *xv = lb ? xk : xi;
            float acc = 0.0f;
            if (lane < S) {
#pragma unroll 4
                for (int r = warp * 32; r < warp * 32 + 32; r++)
                    acc = fmaf(Vs[r * 33 + lane], xv[r], acc);
                part[warp][lane] = acc;
            }
            __syncthreads();
            if (tid < S) {
                float y = part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid];
                if (!lb)
                    y += xk[l0 + tid];
                yw[tid] = y;
            }
            __syncthreads();
            float w = 0.0f;
            if (tid < S)
                for (int b = 0; b <= tid; b++)
                    w = fmaf(Ts[tid * S + b], yw[b], w);
            __syncthreads();
            if (tid < S) {
                yw[tid] = w;
                if (!lb)
                    xk[l0 + tid] -= w;
            }
            __syncthreads();
            float d = 0.0f;
            for (int a = 0; a < S; a++)
                d = fmaf(Vs[tid * 33 + a], yw[a], d);
            if (lb)
                xk[tid] -= d;
            else
                xi[tid] -= d;
        }
        __syncthreads();
        __stcg(gxk + tid, xk[tid]);
        if (!lb)
            __stcg(gxi + tid, xi[tid]);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            if (TREE) {
                GTask sp[2];
                const int ns = ga_specific(G, kind, k, i, sp);
                for (int s2 = 0; s2 < ns; s2++) {
                    const int sk = ga_kind(G, sp[s2].tt, sp[s2].k, sp[s2].i);
                    q_signal(Q, apply32_cnt(A, sp[s2].tt, sp[s2].k, sp[s2].i, col), ga_ndeps(sk, sp[s2].k),
                             sk == K_LARFB ? 0 : 1, encode_task(sp[s2].k, sp[s2].i, col, sp[s2].tt));
                }
            } else if (lb) {
                // LB(k) -> SB(k+1, k)
                if (k + 1 < A.p)
                    q_signal(Q, apply32_cnt(A, 0, k, k + 1, col), 1 + (k > 0 ? 1 : 0), 1, encode_task(k, k + 1, col));
            } else {
                // SB(i, k) -> SB(i+1, k); the step-(k+1) task on row i (LB if i == k+1)
                if (i + 1 < A.p)
                    q_signal(Q, apply32_cnt(A, 0, k, i + 1, col), 1 + (k > 0 ? 1 : 0), 1, encode_task(k, i + 1, col));
                if (k + 1 < A.steps) {
                    if (i == k + 1)
                        q_signal(Q, apply32_cnt(A, 0, k + 1, i, col), 1, 0, encode_task(k + 1, i, col));
                    else
                        q_signal(Q, apply32_cnt(A, 0, k + 1, i, col), 2, 1, encode_task(k + 1, i, col));
                }
            }
            __threadfence();
            atomicAdd(&Q.ctrl->completed, 1u);
        }
    }
}

// Tiled back substitution in FP32 with inverted diagonal tiles, for block
// column j: x_j = Rinv_j y_j (one CTA per column), then y_i -= R_ij x_j
// (one CTA per (i < j, column)).
__global__ void __launch_bounds__(128) k_trsv32_diag(const float *__restrict__ rinv, float *X, int ncol, int j)
{
    __shared__ float y[128];
    const int col = blockIdx.x, r = threadIdx.x;
    float *xj = X + ((size_t)j * ncol + col) * 128;
    y[r] = xj[r];
    __syncthreads();
    const float *Ri = rinv + (size_t)j * 128 * 128;
    float acc0 = 0.0f, acc1 = 0.0f;
    for (int c = 0; c < 128; c += 2) {
        acc0 = fmaf(Ri[(size_t)c * 128 + r], y[c], acc0);
        acc1 = fmaf(Ri[(size_t)(c + 1) * 128 + r], y[c + 1], acc1);
    }
    xj[r] = acc0 + acc1;
}
__global__ void __launch_bounds__(128) k_trsv32_update(const float *__restrict__ tiles, float *X, int p, int ncol,
                                                       int j)
{
    __shared__ float x[128];
    const int i = blockIdx.x, col = blockIdx.y, r = threadIdx.x;
    x[r] = X[((size_t)j * ncol + col) * 128 + r];
    __syncthreads();
    const float *R = tiles + ((size_t)j * p + i) * 128 * 128;
    float acc0 = 0.0f, acc1 = 0.0f;
    for (int c = 0; c < 128; c += 2) {
        acc0 = fmaf(R[(size_t)c * 128 + r], x[c], acc0);
        acc1 = fmaf(R[(size_t)(c + 1) * 128 + r], x[c + 1], acc1);
    }
    X[((size_t)i * ncol + col) * 128 + r] -= acc0 + acc1;
}

// ---------------------------------------------------------------------------
// FP64 vector kernels.
// r = b - A x  (A column-major m x n); one thread per row, columns split
// across blockIdx.y with atomic accumulation into r (pre-set to b).
__global__ void k_residual(const double *__restrict__ A, int64_t lda, int64_t m, int64_t n,
                           const double *__restrict__ x, double *r, int64_t cols_per_block)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.y * cols_per_block;
    const int64_t c1 = c0 + cols_per_block < n ? c0 + cols_per_block : n;
    if (row >= m)
        return;
    double a0 = 0.0, a1 = 0.0;
    int64_t c = c0;
    for (; c + 1 < c1; c += 2) {
        a0 = fma(A[c * lda + row], x[c], a0);
        a1 = fma(A[(c + 1) * lda + row], x[c + 1], a1);
    }
    if (c < c1)
        a0 = fma(A[c * lda + row], x[c], a0);
    atomicAdd(r + row, -(a0 + a1));
}

// partial sums of x.y into out[blockIdx.x]
__global__ void k_dot(const double *__restrict__ x, const double *__restrict__ y, int64_t n, double *out)
{
    __shared__ double red[8];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(x[i], y[i], acc);
    acc = warp_allsum(acc);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++)
            s += red[w];
        out[blockIdx.x] = s;
    }
}

// y += alpha * x, alpha read from device memory (alpha_scale * *alpha_ptr)
__global__ void k_axpy(double alpha, const double *__restrict__ x, double *y, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(alpha, x[i], y[i]);
}
__global__ void k_scale_copy(double alpha, const double *__restrict__ x, double *y, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = alpha * x[i];
}
// FP64 vector (length m) scaled by 2^-sv -> FP32 row blocks X (p x 128,
// zero-padded); and back (first n rows): v_c = X_c 2^(sv - s_c), undoing the
// vector's scaling and R's column scaling (sv = unit_shift(*vexp)).
__global__ void k_vec_to_blocks(const double *__restrict__ v, int64_t m, float *X, int p, const int *vexp)
{
    const int sv = unit_shift(*vexp);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)p * 128;
         i += (int64_t)gridDim.x * blockDim.x)
        X[i] = i < m ? f64_to_f32_sc(v[i], sv) : 0.0f;
}
__global__ void k_blocks_to_vec(const float *__restrict__ X, int64_t n, double *v, const int *vexp,
                                const int *__restrict__ cexp, int lm)
{
    const int sv = unit_shift(*vexp);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = f32_to_f64_sc(X[i], sv - col_shift(cexp[i], lm));
}

}  // namespace tqr

// ---------------------------------------------------------------------------
// Host side.
namespace tqr {

// multi-dot: out[c * nb + b] = partial over block b of V(:,c) . w
__global__ void k_multidot(const double *__restrict__ V, int64_t ldv, int ncols, const double *__restrict__ w,
                           int64_t n, double *out)
{
    __shared__ double red[8];
    for (int c = 0; c < ncols; c++) {
        double acc = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            acc = fma(V[(size_t)c * ldv + i], w[i], acc);
        acc = warp_allsum(acc);
        if ((threadIdx.x & 31) == 0)
            red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ww++)
                s += red[ww];
            out[(size_t)c * gridDim.x + blockIdx.x] = s;
        }
        __syncthreads();
    }
}
// w -= V h (h on the device, ncols entries)
__global__ void k_multiaxpy(const double *__restrict__ V, int64_t ldv, int ncols, const double *__restrict__ h,
                            double *w, int64_t n, double sign)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = w[i];
        for (int c = 0; c < ncols; c++)
            acc = fma(sign * h[c], V[(size_t)c * ldv + i], acc);
        w[i] = acc;
    }
}

namespace {

constexpr int DOT_BLOCKS = 152;
constexpr int GMRES_RESTART = 40;

struct RefineLayout {
    size_t tiles32, T32, T2_32, rinv, X, sched, vecs, dots, flag, cexp, end;
    size_t sched_bytes, cnt_bytes;
    unsigned long long nlb, nsb;   // queue capacities: DLARFB; DSSRFB + DTTMQR
    int64_t m, n;
    int p, q, steps, S;
    TGraph G;
};

RefineLayout refine_layout(const tileqr_desc *d)
{
    RefineLayout R{};
    R.m = d->m;
    R.n = d->n;
    R.p = d->p;
    R.q = d->q;
    R.steps = d->p < d->q ? d->p : d->q;
    R.S = d->ib;
    size_t off = 0;
    R.tiles32 = off;
    off += align256((size_t)d->p * d->q * 128 * 128 * 4);
    R.T32 = off;
    off += align256((size_t)d->p * d->q * d->ib * 128 * 4);
    R.T2_32 = off;
    if (d->T2 != nullptr)
        off += align256((size_t)d->p * d->q * d->ib * 128 * 4);
    R.rinv = off;
    off += align256((size_t)d->q * 128 * 128 * 4);
    R.X = off;
    off += align256((size_t)d->p * 128 * 4);
    // scheduler of the one-column FP32 apply: control block, counters (a
    // second bank for the tree's merges), 2 queues
    R.G = make_graph(d->p, d->q, d->T2 != nullptr ? d->domain : 0);
    unsigned long long cnt[2];
    ga_count(R.G, cnt);
    R.nlb = cnt[0];
    R.nsb = cnt[1];
    R.cnt_bytes = align256((size_t)(R.G.H < R.G.p ? 2 : 1) * R.steps * d->p * 4);
    R.sched = off;
    R.sched_bytes = 256 + R.cnt_bytes + align256((R.nlb ? R.nlb : 1) * 8) + align256((R.nsb ? R.nsb : 1) * 8);
    off += R.sched_bytes;
    // FP64 vectors: r (m), b copy (m), d (n), w (m), V (m x (restart+1)), Z (n x restart)
    const int64_t mm = d->m > d->n ? d->m : d->n;
    R.vecs = off;
    off += align256((size_t)mm * 8 * (4 + (GMRES_RESTART + 1) + GMRES_RESTART));
    R.dots = off;
    off += align256((size_t)(GMRES_RESTART + 2) * DOT_BLOCKS * 8);
    R.flag = off;   // [0] singular column + 1, [1] exponent of b, [2] exponent of the preconditioned vector
    off += 256;
    R.cexp = off;   // largest exponent per column of R (q * 128 ints)
    off += align256((size_t)d->q * 128 * 4);
    R.end = off;
    return R;
}

struct Refiner {
    const tileqr_desc *d;
    RefineLayout L;
    char *ws;
    cudaStream_t st;
    int grid_apply = 0;
    const double *A;
    int64_t lda;
    double *r, *bc, *dv, *w, *V, *Z, *dots;
    int64_t mm;
    std::vector<double> hdots;

    int gemv_residual(const double *x, double *out, const double *rhs, bool negate_only)
    {
        // out = rhs - A x   (rhs == nullptr: out = -A x)
        if (rhs)
            cudaMemcpyAsync(out, rhs, (size_t)L.m * 8, cudaMemcpyDeviceToDevice, st);
        else
            cudaMemsetAsync(out, 0, (size_t)L.m * 8, st);
        // rows over threads (coalesced), columns over 8 blocks (8 atomics per row)
        const int64_t cpb = (L.n + 7) / 8 > 0 ? (L.n + 7) / 8 : 1;
        dim3 grid((unsigned)((L.m + 255) / 256), (unsigned)((L.n + cpb - 1) / cpb));
        k_residual<<<grid, 256, 0, st>>>(A, lda, L.m, L.n, x, out, cpb);
        count_launch();
        (void)negate_only;
        return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
    }

    double dot(const double *x, const double *y, int64_t n)
    {
        k_dot<<<DOT_BLOCKS, 256, 0, st>>>(x, y, n, dots);
        count_launch();
        double h[DOT_BLOCKS];
        cudaMemcpyAsync(h, dots, sizeof(h), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        double s = 0.0;
        for (int b = 0; b < DOT_BLOCKS; b++)
            s += h[b];
        return s;
    }

    // z (n, FP64) = R^{-1} (Q^T v)(0:n) with the FP32 factors; v has m entries
    int precond(const double *v, double *z)
    {
        float *X = (float *)(ws + L.X);
        int *vexp = (int *)(ws + L.flag) + 2;
        if (cudaMemsetAsync(vexp, 0, sizeof(int), st) != cudaSuccess)
            return TILEQR_ERR_CUDA;
        k_vec_maxexp<<<DOT_BLOCKS, 256, 0, st>>>(v, L.m, vexp);
        k_vec_to_blocks<<<DOT_BLOCKS, 256, 0, st>>>(v, L.m, X, L.p, vexp);
        count_launch(2);
        // Q^T on one column
        char *sched = ws + L.sched;
        if (cudaMemsetAsync(sched, 0, L.sched_bytes, st) != cudaSuccess)
            return TILEQR_ERR_CUDA;
        Apply32Args a;
        a.tiles = (const float *)(ws + L.tiles32);
        a.T = (const float *)(ws + L.T32);
        a.T2 = d->T2 != nullptr ? (const float *)(ws + L.T2_32) : nullptr;
        a.X = X;
        a.p = L.p;
        a.steps = L.steps;
        a.ncol = 1;
        a.S = L.S;
        a.G = L.G;
        const size_t cnt_bytes = L.cnt_bytes;
        const unsigned long long nlb = L.nlb, nsb = L.nsb;
        Queues Q;
        Q.ctrl = (SchedCtrl *)sched;
        Q.cnt = (unsigned int *)(sched + 256);
        Q.slot[0] = (unsigned long long *)(sched + 256 + cnt_bytes);
        Q.slot[1] = (unsigned long long *)(sched + 256 + cnt_bytes + align256((nlb ? nlb : 1) * 8));
        Q.slot[2] = Q.slot[3] = nullptr;
        Q.cap[0] = (unsigned int)nlb;
        Q.cap[1] = (unsigned int)nsb;
        Q.cap[2] = Q.cap[3] = 0;
        Q.total = (unsigned int)(nlb + nsb);
        Q.watchdog_ns = watchdog_ns_default();
        Q.withheld = ~0ull;
        Q.trace = nullptr;
        Q.trace_cap = 0;
        int grid = grid_apply;
        if ((unsigned)grid > Q.total)
            grid = (int)Q.total;
        if (grid > 0) {
            if (L.G.H < L.G.p)
                k_apply32_dag<true><<<grid, 128, 0, st>>>(a, Q);
            else
                k_apply32_dag<false><<<grid, 128, 0, st>>>(a, Q);
            count_launch();
        }
        // R^{-1} on the first q blocks
        const float *rinv = (const float *)(ws + L.rinv);
        const float *t32 = (const float *)(ws + L.tiles32);
        for (int j = L.q - 1; j >= 0; j--) {
            k_trsv32_diag<<<1, 128, 0, st>>>(rinv, X, 1, j);
            count_launch();
            if (j > 0) {
                k_trsv32_update<<<dim3(j, 1), 128, 0, st>>>(t32, X, L.p, 1, j);
                count_launch();
            }
        }
        k_blocks_to_vec<<<DOT_BLOCKS, 256, 0, st>>>(X, L.n, z, vexp, (const int *)(ws + L.cexp),
                                                    ceil_log2_sqrt(L.n));
        count_launch();
        return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
    }
};

}  // namespace
}  // namespace tqr

using namespace tqr;

extern "C" int tileqr_refine_workspace_size(const tileqr_desc *d, size_t *bytes)
{
    if (d == nullptr)
        return -1;
    if (bytes == nullptr)
        return -2;
    *bytes = refine_layout(d).end;
    return 0;
}

extern "C" int tileqr_solve_refine(const tileqr_desc *d, const double *A, int64_t lda, const double *b, double *x,
                                   int max_iter, double tol, void *workspace, size_t ws_bytes,
                                   tileqr_stream_t stream, tileqr_refine_info *info)
{
    if (d == nullptr)
        return -1;
    if (d->m < d->n)
        return -1;
    if (A == nullptr && d->m > 0)
        return -2;
    if (lda < (d->m > 1 ? d->m : 1))
        return -3;
    if (b == nullptr && d->m > 0)
        return -4;
    if (x == nullptr && d->n > 0)
        return -5;
    if (max_iter < 0)
        return -6;
    if (!(tol > 0.0))
        return -7;
    if (d->nb != 128)
        return TILEQR_ERR_UNSUPPORTED;
    const RefineLayout L = refine_layout(d);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.end)
        return TILEQR_ERR_WORKSPACE;
    tileqr_refine_info loc{};
    if (info == nullptr)
        info = &loc;
    std::memset(info, 0, sizeof(*info));
    if (d->n == 0)
        return 0;
    Refiner R;
    R.d = d;
    R.L = L;
    R.ws = (char *)workspace;
    R.st = (cudaStream_t)stream;
    R.A = A;
    R.lda = lda;
    R.mm = d->m;
    double *vecs = (double *)(R.ws + L.vecs);
    R.r = vecs;
    R.bc = vecs + R.mm;
    R.dv = vecs + 2 * R.mm;
    R.w = vecs + 3 * R.mm;
    R.V = vecs + 4 * R.mm;
    R.Z = R.V + (size_t)(GMRES_RESTART + 1) * R.mm;
    R.dots = (double *)(R.ws + L.dots);
    cudaStream_t st = R.st;
    {
        int grid = 0;
        if (kernel_grid((const void *)k_apply32_dag<true>, 128, 0, &grid) != 0 ||
            kernel_smem_optin((const void *)k_inv_diag, (128 * 129 + 128) * 8) != 0)
            return TILEQR_ERR_CUDA;
        R.grid_apply = grid;
    }
    // FP32 factors (R column-scaled) and inverted diagonal tiles of R
    int *flag = (int *)(R.ws + L.flag);
    int *cexp = (int *)(R.ws + L.cexp);
    const int lm = ceil_log2_sqrt(d->n);
    cudaMemsetAsync(flag, 0, 256, st);
    cudaMemsetAsync(cexp, 0, (size_t)d->q * 128 * 4, st);
    const size_t nT = (size_t)d->p * d->q * d->ib * 128;
    k_r_colexp<<<4 * DOT_BLOCKS, 256, 0, st>>>(d->tiles, d->p, d->q, cexp);
    k_tiles_to_f32<<<4 * DOT_BLOCKS, 256, 0, st>>>(d->tiles, d->p, d->q, cexp, lm, (float *)(R.ws + L.tiles32));
    k_to_f32<<<DOT_BLOCKS, 256, 0, st>>>(d->T, (float *)(R.ws + L.T32), nT);
    if (d->T2 != nullptr) {
        k_to_f32<<<DOT_BLOCKS, 256, 0, st>>>(d->T2, (float *)(R.ws + L.T2_32), nT);
        count_launch();
    }
    k_inv_diag<<<d->q, 128, (128 * 129 + 128) * 8, st>>>(d->tiles, d->p, d->q, d->n, cexp, lm,
                                                        (float *)(R.ws + L.rinv), flag);
    count_launch(4);
    if (cudaGetLastError() != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int hflag = 0;
    cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (hflag)
        return TILEQR_ERR_SINGULAR;

    // b' = b 2^-sb (largest entry in [1, 2)); the loop solves A x' = b'
    int *bexp = flag + 1;
    k_vec_maxexp<<<DOT_BLOCKS, 256, 0, st>>>(b, d->m, bexp);
    k_scale_pow2<<<DOT_BLOCKS, 256, 0, st>>>(b, R.bc, d->m, bexp, -1);
    count_launch(2);
    const double *bs = R.bc;
    const double bnorm = std::sqrt(R.dot(bs, bs, d->m));
    if (bnorm == 0.0) {
        cudaMemsetAsync(x, 0, (size_t)d->n * 8, st);
        info->converged = 1;
        return 0;
    }
    // x0 = M^{-1} b'
    int rc = R.precond(bs, x);
    if (rc)
        return rc;
    rc = R.gemv_residual(x, R.r, bs, false);
    if (rc)
        return rc;
    double rnorm = std::sqrt(R.dot(R.r, R.r, d->m));
    info->initial_rel_residual = rnorm / bnorm;
    info->method = 1;
    int outer = 0;
    bool use_gmres = false;
    while (rnorm / bnorm > tol && outer < max_iter) {
        outer++;
        if (!use_gmres) {
            // classical refinement: x += M^{-1} r
            rc = R.precond(R.r, R.dv);
            if (rc)
                return rc;
            k_axpy<<<DOT_BLOCKS, 256, 0, st>>>(1.0, R.dv, x, d->n);
            count_launch();
        } else {
            // flexible GMRES(restart) on A d = r, right preconditioner M^{-1}
            info->method = 2;
            const double beta = rnorm;
            k_scale_copy<<<DOT_BLOCKS, 256, 0, st>>>(1.0 / beta, R.r, R.V, d->m);
            count_launch();
            const int mr = GMRES_RESTART;
            std::vector<double> H((size_t)(mr + 1) * mr, 0.0), cs(mr), sn(mr), g(mr + 1, 0.0);
            g[0] = beta;
            int jdone = 0;
            for (int j = 0; j < mr; j++) {
                double *vj = R.V + (size_t)j * R.mm, *zj = R.Z + (size_t)j * R.mm;
                rc = R.precond(vj, zj);
                if (rc)
                    return rc;
                rc = R.gemv_residual(zj, R.w, nullptr, true);   // w = -A z_j
                if (rc)
                    return rc;
                k_scale_copy<<<DOT_BLOCKS, 256, 0, st>>>(-1.0, R.w, R.w, d->m);
                count_launch();
                // classical Gram-Schmidt, twice
                std::vector<double> h(j + 1, 0.0);
                double *hdev = R.dots + (size_t)(GMRES_RESTART + 1) * DOT_BLOCKS;
                for (int pass = 0; pass < 2; pass++) {
                    k_multidot<<<DOT_BLOCKS, 256, 0, st>>>(R.V, R.mm, j + 1, R.w, d->m, R.dots);
                    count_launch();
                    std::vector<double> part((size_t)(j + 1) * DOT_BLOCKS);
                    cudaMemcpyAsync(part.data(), R.dots, part.size() * 8, cudaMemcpyDeviceToHost, st);
                    cudaStreamSynchronize(st);
                    std::vector<double> hp(j + 1, 0.0);
                    for (int c = 0; c <= j; c++)
                        for (int bb = 0; bb < DOT_BLOCKS; bb++)
                            hp[c] += part[(size_t)c * DOT_BLOCKS + bb];
                    for (int c = 0; c <= j; c++)
                        h[c] += hp[c];
                    cudaMemcpyAsync(hdev, hp.data(), (j + 1) * 8, cudaMemcpyHostToDevice, st);
                    k_multiaxpy<<<DOT_BLOCKS, 256, 0, st>>>(R.V, R.mm, j + 1, hdev, R.w, d->m, -1.0);
                    count_launch();
                }
                const double hn = std::sqrt(R.dot(R.w, R.w, d->m));
                for (int c = 0; c <= j; c++)
                    H[(size_t)j * (mr + 1) + c] = h[c];
                H[(size_t)j * (mr + 1) + j + 1] = hn;
                // apply previous Givens rotations to column j, then a new one
                for (int c = 0; c < j; c++) {
                    double *hc = &H[(size_t)j * (mr + 1) + c];
                    const double t = cs[c] * hc[0] + sn[c] * hc[1];
                    hc[1] = -sn[c] * hc[0] + cs[c] * hc[1];
                    hc[0] = t;
                }
                double *hj = &H[(size_t)j * (mr + 1) + j];
                const double den = std::hypot(hj[0], hj[1]);
                cs[j] = den > 0 ? hj[0] / den : 1.0;
                sn[j] = den > 0 ? hj[1] / den : 0.0;
                hj[0] = den;
                hj[1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                jdone = j + 1;
                info->inner_iterations++;
                if (std::fabs(g[j + 1]) <= 0.1 * tol * bnorm || hn == 0.0)
                    break;
                if (j + 1 < mr)
                    k_scale_copy<<<DOT_BLOCKS, 256, 0, st>>>(1.0 / hn, R.w, R.V + (size_t)(j + 1) * R.mm, d->m);
            }
            // y = H^{-1} g (upper triangular jdone x jdone), d = Z y
            std::vector<double> y(jdone, 0.0);
            for (int rr = jdone - 1; rr >= 0; rr--) {
                double acc = g[rr];
                for (int c = rr + 1; c < jdone; c++)
                    acc -= H[(size_t)c * (mr + 1) + rr] * y[c];
                y[rr] = acc / H[(size_t)rr * (mr + 1) + rr];
            }
            double *hdev = R.dots + (size_t)(GMRES_RESTART + 1) * DOT_BLOCKS;
            cudaMemcpyAsync(hdev, y.data(), jdone * 8, cudaMemcpyHostToDevice, st);
            k_multiaxpy<<<DOT_BLOCKS, 256, 0, st>>>(R.Z, R.mm, jdone, hdev, x, d->n, 1.0);
            count_launch();
        }
        rc = R.gemv_residual(x, R.r, bs, false);
        if (rc)
            return rc;
        const double rn = std::sqrt(R.dot(R.r, R.r, d->m));
        if (!use_gmres && rn > 0.5 * rnorm)
            use_gmres = true;   // classical refinement stalls: kappa * u_factor is not small
        rnorm = rn;
    }
    info->iterations = outer;
    info->rel_residual = rnorm / bnorm;
    info->converged = rnorm / bnorm <= tol;
    // x = x' 2^sb
    k_scale_pow2<<<DOT_BLOCKS, 256, 0, st>>>(x, x, d->n, bexp, 1);
    count_launch();
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}
