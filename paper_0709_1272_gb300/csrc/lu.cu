// lu.cu -- the tiled LU factorization with tiled pairwise pivoting (Sec.
// 3.2.2, Algorithm 3) on the GPU: layout conversion with identity padding,
// one persistent kernel running the task graph of DGETRF / DGESSM / DTSTRF /
// DSSSSM (the graph of Algorithm 2's flat tree, graph.cuh) with the
// scheduler of the QR factorization, the solve A X = B (the transformations
// replayed on B as a task graph, then the tiled back substitution with U),
// and the C entry points.
#include <cstring>

#include "factor.h"
#include "graph.cuh"
#include "lu.cuh"
#include "release.cuh"
#include "sched.cuh"

namespace tqr {

// Workspace: tiles (p x p), the L1 strips of every DTSTRF (S x NB per tile
// pair (i, k), laid out like the QR T strips), the pivots (NB ints per tile
// pair), control block, task counters and the four ready queues.
struct LuLayout {
    int64_t n;
    int nb, ib, p;
    size_t off_tiles, off_L, off_piv, off_ctrl, off_cnt, off_q[K_NKIND], end;
    unsigned int cap[K_NKIND], total;
};

static LuLayout lu_layout(int64_t n, int nb, int ib)
{
    LuLayout L{};
    L.n = n;
    L.nb = nb;
    L.ib = ib;
    L.p = (int)((n + nb - 1) / nb);
    const size_t pp = (size_t)L.p * L.p;
    L.off_tiles = 0;
    L.off_L = align256(pp * nb * nb * sizeof(double));
    L.off_piv = L.off_L + align256(pp * ib * nb * sizeof(double));
    L.off_ctrl = L.off_piv + align256(pp * nb * sizeof(int));
    L.off_cnt = L.off_ctrl + 256;
    size_t off = L.off_cnt + align256(pp * L.p * sizeof(unsigned int));
    // queue levels of the QR kinds (GETRF as DGEQRT, TSTRF as DTSQRT, ...)
    unsigned long long cnt[K_NKIND];
    g_level_counts(make_graph(L.p, L.p, 0), cnt);
    unsigned long long tot = 0;
    for (int t = 0; t < K_NKIND; t++) {
        L.cap[t] = (unsigned int)cnt[t];
        tot += cnt[t];
        L.off_q[t] = off;
        off += align256((size_t)(cnt[t] ? cnt[t] : 1) * sizeof(unsigned long long));
    }
    L.total = (unsigned int)tot;
    L.end = off;
    return L;
}

static bool lu_supported(int nb, int ib)
{
    return (nb == 64 || nb == 128) && (ib == 16 || ib == 32);
}

// Column-major n x n A into tiles; the padding beyond n is the identity on
// the diagonal, zero elsewhere, so the padded matrix is diag(A, I): no
// padded row is ever a strictly larger pivot candidate, and the factors are
// diag(L, I), diag(U, I).  Non-finite entries are flagged.
__global__ void k_cm2tile_eye(const double *__restrict__ A, int64_t lda, int64_t n, double *__restrict__ tiles,
                              int nb, int p, int *nonfinite)
{
    const int lane = threadIdx.x & 31;
    const size_t nseg = (size_t)p * p * nb;
    const size_t wstride = (size_t)gridDim.x * (blockDim.x >> 5);
    bool bad = false;
    for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += wstride) {
        const int c = (int)(s % nb);
        const size_t t = s / nb;
        const int i = (int)(t % p), j = (int)(t / p);
        const int64_t col = (int64_t)j * nb + c, row0 = (int64_t)i * nb;
        double *dst = tiles + (t * nb + c) * nb;
        for (int r = lane; r < nb; r += 32) {
            const int64_t row = row0 + r;
            double v;
            if (row < n && col < n) {
                v = __ldg(A + col * lda + row);
                bad |= !isfinite(v);
            } else {
                v = row == col ? 1.0 : 0.0;
            }
            dst[r] = v;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0)
        atomicExch(nonfinite, 1);
}

// The pivots as a p x n int matrix (ld ldp): entry (i, k*nb + c) = pivot c of
// DGETRF (i == k) or DTSTRF (i > k) at step k; 0 for i < k.
__global__ void k_piv2cm(const int *__restrict__ piv, int nb, int p, int64_t n, int *__restrict__ out, int64_t ldp)
{
    const size_t total = (size_t)p * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % p);
        const int64_t col = (int64_t)(e / p);
        const int k = (int)(col / nb), c = (int)(col % nb);
        out[col * ldp + i] = i >= k ? piv[((size_t)k * p + i) * nb + c] : 0;
    }
}

struct LuArgs {
    double *tiles;
    double *L;   // L1 strips
    int *piv;
    int p;
    TGraph G;
};

template <int NB, int S>
__device__ __forceinline__ double *lu_tile(const LuArgs &F, int i, int j)
{
    return F.tiles + ((size_t)j * F.p + i) * (size_t)NB * NB;
}
template <int NB, int S>
__device__ __forceinline__ double *lu_strip(const LuArgs &F, int i, int k)
{
    return F.L + ((size_t)k * F.p + i) * (size_t)S * NB;
}
template <int NB, int S>
__device__ __forceinline__ int *lu_piv(const LuArgs &F, int i, int k)
{
    return F.piv + ((size_t)k * F.p + i) * NB;
}

// Record an exactly zero pivot at global column col (1-based): the smallest
// such column is kept (stored complemented, so the maximum wins).
__device__ __forceinline__ void lu_note_zero(const Queues &Q, unsigned long long col)
{
    atomicMax(&Q.ctrl->info, ~col);
}

template <int NB, int S>
__global__ void __launch_bounds__(NT, (LuCfg<NB, S>::CTAS_PER_SM)) k_lu_dag(LuArgs F, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (ld_relaxed_s32(&Q.ctrl->nonfinite) != 0)
            atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_NONFINITE);
        else
            q_push(Q, kind_prio(K_GEQRT), encode_task(0, 0, 0));
    }
    unsigned int ticket = NO_TICKET;   // thread 0's bulk-level claim
    for (;;) {
        if (threadIdx.x == 0)
            s_cmd = q_acquire(Q, s_code, ticket);
        __syncthreads();
        if (s_cmd != CMD_RUN)
            break;
        int k, i, j;
        decode_task(s_code, k, i, j);
        const int kind = g_kind(F.G, 0, k, i, j);
        const unsigned long long t0 = Q.trace ? globaltimer_ns() : 0ull;
        int z = 0;
        switch (kind) {
        case K_GEQRT: {
            // DGETRF has no L1 strip: keep strip (k, k) zero
            double *st = lu_strip<NB, S>(F, k, k);
            for (int e = threadIdx.x; e < S * NB; e += NT)
                stcg(st + e, 0.0);
            z = lu_task_getrf<NB, S>(sm, lu_tile<NB, S>(F, k, k), lu_piv<NB, S>(F, k, k));
            break;
        }
        case K_LARFB:
            lu_task_gessm<NB, S>(sm, lu_tile<NB, S>(F, k, j), lu_tile<NB, S>(F, k, k), lu_piv<NB, S>(F, k, k));
            break;
        case K_TSQRT:
            z = lu_task_tstrf<NB, S>(sm, lu_tile<NB, S>(F, k, k), lu_tile<NB, S>(F, i, k), lu_strip<NB, S>(F, i, k),
                                     lu_piv<NB, S>(F, i, k));
            break;
        default:
            lu_task_ssssm<NB, S>(sm, lu_tile<NB, S>(F, i, j), lu_tile<NB, S>(F, k, j), lu_tile<NB, S>(F, i, k),
                                 lu_strip<NB, S>(F, i, k), lu_piv<NB, S>(F, i, k));
            break;
        }
        if (z != 0 && threadIdx.x == 0)
            lu_note_zero(Q, (unsigned long long)k * NB + z);
        __syncthreads();
        release_graph(Q, F.G, kind, k, i, j);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (Q.trace)
                trace_record(Q, s_code, t0, globaltimer_ns());
            __threadfence();
            atomicAdd(&Q.ctrl->completed, 1u);
        }
    }
}

static void lu_queues(const LuLayout &L, char *ws, Queues &Q, unsigned long long watchdog_ns,
                      unsigned long long *trace, unsigned int trace_cap)
{
    Q.ctrl = (SchedCtrl *)(ws + L.off_ctrl);
    Q.cnt = (unsigned int *)(ws + L.off_cnt);
    for (int t = 0; t < K_NKIND; t++) {
        Q.slot[t] = (unsigned long long *)(ws + L.off_q[t]);
        Q.cap[t] = L.cap[t];
    }
    Q.total = L.total;
    Q.watchdog_ns = watchdog_ns;
    Q.withheld = ~0ull;
    Q.trace = trace;
    Q.trace_cap = trace_cap;
}

template <int NB, int S>
static int launch_lu_t(const LuLayout &L, char *ws, int flags, cudaStream_t st, unsigned long long watchdog_ns,
                       unsigned long long *trace, unsigned int trace_cap)
{
    constexpr size_t smem = LuCfg<NB, S>::SMEM;
    int grid = 0;
    const int rc = kernel_grid((const void *)k_lu_dag<NB, S>, NT, smem, &grid);
    if (rc)
        return rc;
    LuArgs F;
    F.tiles = (double *)(ws + L.off_tiles);
    F.L = (double *)(ws + L.off_L);
    F.piv = (int *)(ws + L.off_piv);
    F.p = L.p;
    F.G = make_graph(L.p, L.p, 0);
    Queues Q;
    lu_queues(L, ws, Q, watchdog_ns, trace, trace_cap);
    if (flags & TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK)
        Q.withheld = encode_task(L.p - 1, L.p - 1, L.p - 1);
    int g = grid;
    if ((unsigned)g > L.total)
        g = (int)L.total;
    k_lu_dag<NB, S><<<g, NT, smem, st>>>(F, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// The transformations of the factorization applied to right-hand sides in
// tile-row layout (Bt: p blocks of nb x ncp), chunk by chunk of APPLY_W
// columns: LB(k) = DGESSM on block k, SB(i, k) = DSSSSM on blocks (k, i);
// the apply graph of the flat tree (graph.cuh: ga_*).
struct LuApplyArgs {
    const double *tiles;
    const double *L;
    const int *piv;
    double *Bt;
    int p, nchunk;
    int64_t ncp;
    TGraph G;
};

template <int NB, int S>
__global__ void __launch_bounds__(NT, 1) k_lu_apply_dag(LuApplyArgs A, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    const TGraph &G = A.G;
    if (blockIdx.x == 0)
        for (int u = threadIdx.x; u < A.nchunk; u += NT)
            q_push(Q, 0, encode_task(0, 0, u));
    unsigned int ticket = NO_TICKET;   // thread 0's bulk-level claim
    for (;;) {
        if (threadIdx.x == 0)
            s_cmd = q_acquire(Q, s_code, ticket);
        __syncthreads();
        if (s_cmd != CMD_RUN)
            break;
        int k, i, cb;
        decode_task(s_code, k, i, cb);
        const int kind = ga_kind(G, 0, k, i);
        double *Bi = A.Bt + ((size_t)i * A.ncp + (size_t)cb * APPLY_W) * NB;
        const size_t tk = ((size_t)k * A.p + i);
        if (kind == K_LARFB) {
            lu_task_gessm<NB, S, APPLY_W>(sm, Bi, A.tiles + ((size_t)k * A.p + k) * (size_t)NB * NB,
                                          A.piv + tk * NB, APPLY_W);
        } else {
            double *Bk = A.Bt + ((size_t)k * A.ncp + (size_t)cb * APPLY_W) * NB;
            lu_task_ssssm<NB, S, APPLY_W>(sm, Bi, Bk, A.tiles + tk * (size_t)NB * NB, A.L + tk * (size_t)S * NB,
                                          A.piv + tk * NB, APPLY_W);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            GTask sp[2];
            const int ns = ga_specific(G, kind, k, i, sp);
            for (int s = 0; s < ns; s++) {
                const int sk = ga_kind(G, 0, sp[s].k, sp[s].i);
                q_signal(Q, ((size_t)sp[s].k * A.p + sp[s].i) * A.nchunk + cb, ga_ndeps(sk, sp[s].k),
                         sk == K_LARFB ? 0 : 1, encode_task(sp[s].k, sp[s].i, cb));
            }
            __threadfence();
            atomicAdd(&Q.ctrl->completed, 1u);
        }
    }
}

// Scheduler state of the apply: control block, counters, the LB queue and
// the SB queue.
struct LuApplySched {
    size_t cnt_bytes, q0_bytes, q1_bytes, total;
    unsigned long long n0, n1;
};
static LuApplySched lu_apply_sched(int p, int nchunk)
{
    LuApplySched a;
    a.n0 = (unsigned long long)p * nchunk;
    a.n1 = (unsigned long long)p * (p - 1) / 2 * nchunk;
    a.cnt_bytes = align256((size_t)p * p * nchunk * sizeof(unsigned int));
    a.q0_bytes = align256((a.n0 ? a.n0 : 1) * 8);
    a.q1_bytes = align256((a.n1 ? a.n1 : 1) * 8);
    a.total = 256 + a.cnt_bytes + a.q0_bytes + a.q1_bytes;
    return a;
}

template <int NB, int S>
static int launch_lu_apply_t(const LuLayout &L, const char *ws, double *Bt, int64_t ncp, char *sched,
                             cudaStream_t st, unsigned long long watchdog_ns)
{
    constexpr size_t smem = LuCfg<NB, S, APPLY_W>::SMEM;
    int grid_max = 0;
    const int rc = kernel_grid((const void *)k_lu_apply_dag<NB, S>, NT, smem, &grid_max);
    if (rc)
        return rc;
    LuApplyArgs A;
    A.tiles = (const double *)(ws + L.off_tiles);
    A.L = (const double *)(ws + L.off_L);
    A.piv = (const int *)(ws + L.off_piv);
    A.Bt = Bt;
    A.p = L.p;
    A.ncp = ncp;
    A.nchunk = (int)(ncp / APPLY_W);
    A.G = make_graph(L.p, L.p, 0);
    const LuApplySched a = lu_apply_sched(L.p, A.nchunk);
    Queues Q;
    Q.ctrl = (SchedCtrl *)sched;
    Q.cnt = (unsigned int *)(sched + 256);
    Q.slot[0] = (unsigned long long *)(sched + 256 + a.cnt_bytes);
    Q.slot[1] = (unsigned long long *)(sched + 256 + a.cnt_bytes + a.q0_bytes);
    Q.slot[2] = Q.slot[3] = nullptr;
    Q.cap[0] = (unsigned int)a.n0;
    Q.cap[1] = (unsigned int)a.n1;
    Q.cap[2] = Q.cap[3] = 0;
    Q.total = (unsigned int)(a.n0 + a.n1);
    Q.watchdog_ns = watchdog_ns;
    Q.withheld = ~0ull;
    Q.trace = nullptr;
    Q.trace_cap = 0;
    if (Q.total == 0)
        return 0;
    if (cudaMemsetAsync(sched, 0, a.total, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int grid = grid_max;
    if ((unsigned)grid > Q.total)
        grid = (int)Q.total;
    k_lu_apply_dag<NB, S><<<grid, NT, smem, st>>>(A, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

static int launch_lu_apply(const LuLayout &L, const char *ws, double *Bt, int64_t ncp, char *sched, cudaStream_t st,
                           unsigned long long watchdog_ns)
{
#define TQR_CASE(NB_, S_)                         \
    if (L.nb == NB_ && L.ib == S_)                \
        return launch_lu_apply_t<NB_, S_>(L, ws, Bt, ncp, sched, st, watchdog_ns);
    TQR_CASE(64, 16)
    TQR_CASE(64, 32)
    TQR_CASE(128, 16)
    TQR_CASE(128, 32)
#undef TQR_CASE
    return TILEQR_ERR_UNSUPPORTED;
}

static int64_t lu_ncp(int64_t nrhs) { return ((nrhs + APPLY_W - 1) / APPLY_W) * APPLY_W; }

static bool lu_desc_ok(const tileqr_desc *d)
{
    return d->T != nullptr && d->T2 == nullptr && d->m == d->n && lu_supported(d->nb, d->ib) &&
           d->workspace != nullptr;
}

}  // namespace tqr

using namespace tqr;

extern "C" int tileqr_lu_workspace_size(int64_t n, int nb, int ib, size_t *bytes)
{
    if (n < 0)
        return -1;
    if (nb < 1 || (n + nb - 1) / nb >= (1 << 21))
        return -2;
    if (ib < 1 || ib > nb || nb % ib != 0)
        return -3;
    if (bytes == nullptr)
        return -4;
    *bytes = lu_layout(n, nb, ib).end;
    return 0;
}

extern "C" int tileqr_lu(int64_t n, const double *A, int64_t lda, int nb, int ib, int flags, void *workspace,
                         size_t ws_bytes, tileqr_stream_t stream, tileqr_desc *out)
{
    if (n < 0)
        return -1;
    if (A == nullptr && n > 0)
        return -2;
    if (lda < (n > 1 ? n : 1))
        return -3;
    if (nb < 1 || (n + nb - 1) / nb >= (1 << 21))
        return -4;
    if (ib < 1 || ib > nb || nb % ib != 0)
        return -5;
    if (out == nullptr)
        return -10;
    if (!lu_supported(nb, ib))
        return TILEQR_ERR_UNSUPPORTED;
    const LuLayout L = lu_layout(n, nb, ib);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.end)
        return TILEQR_ERR_WORKSPACE;
    char *ws = (char *)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    std::memset(out, 0, sizeof(*out));
    out->m = n;
    out->n = n;
    out->nb = nb;
    out->ib = ib;
    out->p = L.p;
    out->q = L.p;
    out->precision = TILEQR_FP64;
    out->schedule = TILEQR_SCHED_DAG;
    out->tiles = (double *)(ws + L.off_tiles);
    out->T = (double *)(ws + L.off_L);
    out->sched = ws + L.off_ctrl;
    out->sched_bytes = L.end - L.off_ctrl;
    out->workspace = workspace;
    out->workspace_bytes = ws_bytes;
    out->domain = L.p;
    if (cudaMemsetAsync(ws + L.off_ctrl, 0, L.end - L.off_ctrl, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (n == 0)
        return 0;
    {
        int nsm = 1;
        if (device_sm_count(&nsm) != 0)
            return TILEQR_ERR_CUDA;
        const size_t warps = (size_t)L.p * L.p * nb;
        int ctas = (int)((warps + 7) / 8);
        if (ctas > nsm * 16)
            ctas = nsm * 16;
        k_cm2tile_eye<<<ctas > 0 ? ctas : 1, 256, 0, st>>>(A, lda, n, out->tiles, nb, L.p,
                                                          &((SchedCtrl *)(ws + L.off_ctrl))->nonfinite);
        count_launch();
        if (cudaGetLastError() != cudaSuccess)
            return TILEQR_ERR_CUDA;
    }
    const unsigned long long wd = (flags & TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK) ? 200ull * 1000000ull
                                                                               : watchdog_ns_default();
    unsigned long long *trace = nullptr;
    unsigned int tcap = 0;
    trace_target(&trace, &tcap);
#define TQR_CASE(NB_, S_)          \
    if (nb == NB_ && ib == S_)     \
        return launch_lu_t<NB_, S_>(L, ws, flags, st, wd, trace, tcap);
    TQR_CASE(64, 16)
    TQR_CASE(64, 32)
    TQR_CASE(128, 16)
    TQR_CASE(128, 32)
#undef TQR_CASE
    return TILEQR_ERR_UNSUPPORTED;
}

extern "C" int tileqr_lu_info(const tileqr_desc *d, tileqr_stream_t stream, int64_t *info)
{
    if (d == nullptr)
        return -1;
    if (info == nullptr)
        return -3;
    *info = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (d->n == 0)
        return 0;
    SchedCtrl c;
    if (cudaMemcpy(&c, d->sched, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    *info = c.info ? (int64_t)(~c.info) : 0;
    return 0;
}

extern "C" int tileqr_lu_get_factors(const tileqr_desc *d, double *F, int64_t ldf, double *Lx, int64_t ldlx,
                                     int *piv, int64_t ldpiv, tileqr_stream_t stream)
{
    if (d == nullptr || !lu_desc_ok(d))
        return -1;
    if (F == nullptr && d->n > 0)
        return -2;
    if (ldf < (d->n > 1 ? d->n : 1))
        return -3;
    if (Lx != nullptr && ldlx < (int64_t)d->p * d->ib)
        return -5;
    if (piv != nullptr && ldpiv < (d->p > 1 ? d->p : 1))
        return -7;
    if (d->n == 0)
        return 0;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_tile2cm(d->tiles, d->nb, d->p, d->p, d->n, d->n, F, ldf, 0, d->n, st);
    if (rc == 0 && Lx != nullptr)
        rc = launch_strips2cm(d->T, d->nb, d->ib, d->p, d->p, d->n, Lx, ldlx, st);
    if (rc == 0 && piv != nullptr) {
        const LuLayout L = lu_layout(d->n, d->nb, d->ib);
        const size_t total = (size_t)d->p * d->n;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096)
            blocks = 4096;
        k_piv2cm<<<blocks, 256, 0, st>>>((const int *)((const char *)d->workspace + L.off_piv), d->nb, d->p, d->n,
                                         piv, ldpiv);
        count_launch();
        rc = cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
    }
    return rc;
}

extern "C" int tileqr_lu_solve_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes)
{
    if (d == nullptr)
        return -1;
    if (nrhs < 0)
        return -2;
    if (bytes == nullptr)
        return -3;
    const int64_t ncp = lu_ncp(nrhs);
    *bytes = align256((size_t)d->p * d->nb * ncp * sizeof(double)) + lu_apply_sched(d->p, (int)(ncp / APPLY_W)).total +
             256;
    return 0;
}

extern "C" int tileqr_lu_solve(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                               size_t ws_bytes, tileqr_stream_t stream)
{
    if (d == nullptr || !lu_desc_ok(d))
        return -1;
    if (B == nullptr && nrhs > 0 && d->n > 0)
        return -2;
    if (ldb < (d->n > 1 ? d->n : 1))
        return -3;
    if (nrhs < 0)
        return -4;
    size_t need = 0;
    tileqr_lu_solve_workspace_size(d, nrhs, &need);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < need)
        return TILEQR_ERR_WORKSPACE;
    if (nrhs == 0 || d->n == 0)
        return 0;
    const LuLayout L = lu_layout(d->n, d->nb, d->ib);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ncp = lu_ncp(nrhs);
    double *Bt = (double *)workspace;
    char *sched = (char *)workspace + align256((size_t)d->p * d->nb * ncp * sizeof(double));
    int *flag = (int *)(sched + lu_apply_sched(d->p, (int)(ncp / APPLY_W)).total);
    if (cudaMemsetAsync(flag, 0, 256, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int rc = launch_cm2rows(B, ldb, d->n, nrhs, Bt, d->nb, d->p, ncp, st);
    if (rc)
        return rc;
    rc = launch_lu_apply(L, (const char *)d->workspace, Bt, ncp, sched, st, watchdog_ns_default());
    if (rc)
        return rc;
    const WsLayout W = make_layout(d->n, d->n, d->nb, d->ib, 0);
    rc = launch_trsm(W, d->tiles, Bt, ncp, flag, st, false, nrhs);
    if (rc)
        return rc;
    rc = launch_rows2cm(Bt, d->nb, d->p, ncp, d->n, nrhs, B, ldb, st);
    if (rc)
        return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int h_flag = 0;
    SchedCtrl c;
    if (cudaMemcpy(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (cudaMemcpy(&c, sched, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (c.error)
        return c.error;
    if (h_flag)
        return TILEQR_ERR_SINGULAR;
    return 0;
}
