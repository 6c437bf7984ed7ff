// cholesky.cu -- the tiled Cholesky factorization (Sec. 3.1, Algorithm 1) on
// the GPU: lower-triangle layout conversion, one persistent kernel running
// the task graph of DPOTF2 / DTRSM / DGSMM with the scheduler of the QR
// factorization (per-task counters, priority ready queues, bounded waits),
// and the C entry points.
#include <cstring>

#include "chol.cuh"
#include "factor.h"
#include "graph.cuh"
#include "sched.cuh"

namespace tqr {

struct CholArgs {
    double *tiles;
    int p;
};

// Lower triangle of the column-major n x n A into tiles (i >= j); the upper
// triangle is not read.  Padding beyond n is the identity on the diagonal
// (zero elsewhere), so the padded matrix is diag(A, I) and its Cholesky
// factor is diag(L, I).  Non-finite entries of the lower triangle are flagged.
__global__ void k_cm2tile_lower(const double *__restrict__ A, int64_t lda, int64_t n, double *__restrict__ tiles,
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
        if (i < j)
            continue;
        const int64_t col = (int64_t)j * nb + c, row0 = (int64_t)i * nb;
        double *dst = tiles + (t * nb + c) * nb;
        for (int r = lane; r < nb; r += 32) {
            const int64_t row = row0 + r;
            double v = 0.0;
            if (row >= col) {
                if (row < n && col < n) {
                    v = __ldg(A + col * lda + row);
                    bad |= !isfinite(v);
                } else if (row == col) {
                    v = 1.0;
                }
            }
            dst[r] = v;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0)
        atomicExch(nonfinite, 1);
}

// L (lower, zeros above the diagonal) from the tiles into column-major n x n.
__global__ void k_tile2cm_lower(const double *__restrict__ tiles, int nb, int p, int64_t n, double *__restrict__ L,
                                int64_t ldl)
{
    const int lane = threadIdx.x & 31;
    const size_t nseg = (size_t)p * n;
    const size_t wstride = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += wstride) {
        const int i = (int)(s % p);
        const int64_t col = (int64_t)(s / p);
        const int j = (int)(col / nb), c = (int)(col % nb);
        const int64_t row0 = (int64_t)i * nb;
        for (int r = lane; r < nb; r += 32) {
            const int64_t row = row0 + r;
            if (row >= n)
                break;
            L[col * ldl + row] = (row >= col && i >= j) ? tiles[(((size_t)j * p + i) * nb + c) * nb + r] : 0.0;
        }
    }
}

template <int NB>
__global__ void __launch_bounds__(NT, 2) k_chol_dag(CholArgs C, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    const int p = C.p;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (ld_relaxed_s32(&Q.ctrl->nonfinite) != 0)
            atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_NONFINITE);
        else
            q_push(Q, 0, encode_task(0, 0, 0));
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
        const unsigned long long t0 = Q.trace ? globaltimer_ns() : 0ull;
        double *Tij = C.tiles + ((size_t)j * p + i) * (size_t)NB * NB;
        const int kind = cg_kind(k, i, j);
        bool failed = false;
        if (kind == KC_POTF2) {
            const int f = task_potf2<NB>(sm, Tij);
            if (f != 0) {
                failed = true;
                if (threadIdx.x == 0) {
                    atomicCAS(&Q.ctrl->info, 0ull, (unsigned long long)k * NB + f);
                    atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_NOT_SPD);
                }
            }
        } else if (kind == KC_TRSM) {
            task_trsm<NB>(sm, Tij, C.tiles + ((size_t)k * p + k) * (size_t)NB * NB);
        } else {
            task_gsmm<NB>(sm, Tij, C.tiles + ((size_t)k * p + i) * (size_t)NB * NB,
                          C.tiles + ((size_t)k * p + j) * (size_t)NB * NB, i == j);
        }
        __syncthreads();
        if (!failed) {
            const int ns = cg_nsucc(p, k, i, j);
            for (int s = threadIdx.x; s < ns; s += NT) {
                const GTask t = cg_succ(p, k, i, j, s);
                const int tk = cg_kind(t.k, t.i, t.j);
                q_signal(Q, cg_cidx(p, t.k, t.i, t.j), cg_ndeps(t.k, t.i, t.j), cg_prio(tk, t.k, t.j),
                         encode_task(t.k, t.i, t.j));
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (Q.trace)
                trace_record(Q, s_code, t0, globaltimer_ns());
            __threadfence();
            atomicAdd(&Q.ctrl->completed, 1u);
        }
    }
}

// Workspace: tiles (p x p, only i >= j used), control block, counters, queues.
struct CholLayout {
    int64_t n;
    int nb, p;
    size_t off_tiles, off_ctrl, off_cnt, off_q[K_NKIND], end;
    unsigned int cap[K_NKIND], total;
};

static CholLayout chol_layout(int64_t n, int nb)
{
    CholLayout L{};
    L.n = n;
    L.nb = nb;
    L.p = (int)((n + nb - 1) / nb);
    L.off_tiles = 0;
    L.off_ctrl = align256((size_t)L.p * L.p * nb * nb * sizeof(double));
    L.off_cnt = L.off_ctrl + 256;
    size_t off = L.off_cnt + align256((size_t)L.p * L.p * L.p * sizeof(unsigned int));
    unsigned long long cnt[4];
    cg_count(L.p, cnt);
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

template <int NB>
static int launch_chol_t(const CholLayout &L, char *ws, cudaStream_t st, unsigned long long watchdog_ns,
                         unsigned long long *trace, unsigned int trace_cap)
{
    constexpr size_t smem = CholCfg<NB>::SMEM;
    int grid = 0;
    const int rc = kernel_grid((const void *)k_chol_dag<NB>, NT, smem, &grid);
    if (rc)
        return rc;
    CholArgs C;
    C.tiles = (double *)(ws + L.off_tiles);
    C.p = L.p;
    Queues Q;
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
    // two task CTAs per SM pay when the graph has the parallelism for them
    // (average about p^2 / 9 ready tasks); below 64 tile rows the critical
    // path rules, and a task alone on its SM finishes sooner
    int g = L.p >= 64 ? grid : grid / 2;
    if (g < 1)
        g = 1;
    if ((unsigned)g > L.total)
        g = (int)L.total;
    k_chol_dag<NB><<<g, NT, smem, st>>>(C, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

}  // namespace tqr

using namespace tqr;

extern "C" int tileqr_cholesky_workspace_size(int64_t n, int nb, size_t *bytes)
{
    if (n < 0)
        return -1;
    if (nb < 1 || (n + nb - 1) / nb >= (1 << 21))
        return -2;
    if (bytes == nullptr)
        return -3;
    *bytes = chol_layout(n, nb).end;
    return 0;
}

extern "C" int tileqr_cholesky(int64_t n, const double *A, int64_t lda, int nb, int flags, void *workspace,
                               size_t ws_bytes, tileqr_stream_t stream, tileqr_desc *out)
{
    (void)flags;
    if (n < 0)
        return -1;
    if (A == nullptr && n > 0)
        return -2;
    if (lda < (n > 1 ? n : 1))
        return -3;
    if (nb < 1 || (n + nb - 1) / nb >= (1 << 21))
        return -4;
    if (out == nullptr)
        return -9;
    if (nb != 64 && nb != 128)
        return TILEQR_ERR_UNSUPPORTED;
    const CholLayout L = chol_layout(n, nb);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.end)
        return TILEQR_ERR_WORKSPACE;
    char *ws = (char *)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    std::memset(out, 0, sizeof(*out));
    out->m = n;
    out->n = n;
    out->nb = nb;
    out->p = L.p;
    out->q = L.p;
    out->precision = TILEQR_FP64;
    out->schedule = TILEQR_SCHED_DAG;
    out->tiles = (double *)(ws + L.off_tiles);
    out->sched = ws + L.off_ctrl;
    out->sched_bytes = L.end - L.off_ctrl;
    out->workspace = workspace;
    out->workspace_bytes = ws_bytes;
    if (cudaMemsetAsync(ws + L.off_ctrl, 0, L.end - L.off_ctrl, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (n == 0)
        return 0;
    {
        int nsm = 1;
        if (device_sm_count(&nsm) != 0)
            return TILEQR_ERR_CUDA;
        size_t warps = (size_t)L.p * L.p * nb;
        int ctas = (int)((warps + 7) / 8);
        if (ctas > nsm * 16)
            ctas = nsm * 16;
        k_cm2tile_lower<<<ctas > 0 ? ctas : 1, 256, 0, st>>>(A, lda, n, out->tiles, nb, L.p,
                                                            &((SchedCtrl *)(ws + L.off_ctrl))->nonfinite);
        count_launch();
        if (cudaGetLastError() != cudaSuccess)
            return TILEQR_ERR_CUDA;
    }
    const unsigned long long wd = watchdog_ns_default();
    unsigned long long *trace = nullptr;
    unsigned int tcap = 0;
    trace_target(&trace, &tcap);
    int rc = TILEQR_ERR_UNSUPPORTED;
    if (nb == 64)
        rc = launch_chol_t<64>(L, ws, st, wd, trace, tcap);
    else
        rc = launch_chol_t<128>(L, ws, st, wd, trace, tcap);
    return rc;
}

extern "C" int tileqr_cholesky_get_L(const tileqr_desc *d, double *L, int64_t ldl, tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    if (L == nullptr && d->n > 0)
        return -2;
    if (ldl < (d->n > 1 ? d->n : 1))
        return -3;
    if (d->n == 0)
        return 0;
    int nsm = 1;
    if (device_sm_count(&nsm) != 0)
        return TILEQR_ERR_CUDA;
    size_t warps = (size_t)d->p * d->n;
    int ctas = (int)((warps + 7) / 8);
    if (ctas > nsm * 16)
        ctas = nsm * 16;
    k_tile2cm_lower<<<ctas > 0 ? ctas : 1, 256, 0, (cudaStream_t)stream>>>(d->tiles, d->nb, d->p, d->n, L, ldl);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

extern "C" int tileqr_cholesky_info(const tileqr_desc *d, tileqr_stream_t stream, int64_t *info)
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
    *info = (int64_t)c.info;
    return 0;
}
