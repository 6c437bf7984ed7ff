// apply.cu -- Q^T B and the triangular solve of the least-squares path.
//
// Q^T B replays the update transformations of the factorization on the
// columns of B, split into column chunks of APPLY_W.  For chunk c the tasks
// are the update kinds of the factorization's task graph restricted to one
// tile column (graph.cuh): LB = DLARFB with a domain head's V and T, SB =
// DSSRFB of a domain row into its head, TB = DTTMQR merging two heads (tree
// form).  In Algorithm 2's flat form: LB(k) <- SB(k,k-1); SB(i,k) <- (LB(k)
// if i = k+1 else SB(i-1,k)) and SB(i,k-1).  They run in one persistent
// kernel with the same counter / ready-queue scheduler, so consecutive
// steps k overlap as a wavefront.  Q B (NOTRANS) runs the same tasks in the
// reverse graph (graph.cuh: ga_predecessors), each with its inner blocks
// reversed and T_l in place of T_l^T.
#include "factor.h"
#include "graph.cuh"
#include "sched.cuh"
#include "tile_f64.cuh"

namespace tqr {

struct ApplyArgs {
    const double *tiles;
    const double *T;
    const double *T2;
    double *Bt;
    int p, q, steps, nchunk;
    int64_t ncp;
    TGraph G;
};

template <int NB, int S>
__device__ __forceinline__ double *chunk_ptr(const ApplyArgs &A, int i, int cb)
{
    return A.Bt + ((size_t)i * A.ncp + (size_t)cb * APPLY_W) * NB;
}

__device__ __forceinline__ size_t apply_cnt_idx(const ApplyArgs &A, int tt, int k, int i, int cb)
{
    return (((size_t)tt * A.steps + k) * A.p + i) * A.nchunk + cb;
}

template <int NB, int S, bool NOTRANS>
__global__ void __launch_bounds__(NT, 1) k_apply_dag(ApplyArgs A, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    const TGraph &G = A.G;
    if (blockIdx.x == 0) {
        if (!NOTRANS) {
            // step 0's DLARFBs (one per domain head and chunk) have no predecessors
            for (int u = threadIdx.x; u < A.nchunk * g_ndom(G, 0); u += NT)
                q_push(Q, 0, encode_task(0, g_head(G, 0, u / A.nchunk), u % A.nchunk));
        } else {
            // the reverse graph starts from the forward graph's sinks
            for (int u = threadIdx.x; u < 2 * A.steps * A.p; u += NT) {
                const int tt = u & 1, k = (u >> 1) / A.p, i = (u >> 1) % A.p;
                if (i < k || (tt == 1 && (((i - k) % G.H) != 0 || i == k)))
                    continue;
                GTask sp[2];
                const int kind = ga_kind(G, tt, k, i);
                if (ga_specific(G, kind, k, i, sp) == 0)
                    for (int cb = 0; cb < A.nchunk; cb++)
                        q_push(Q, kind == K_LARFB ? 0 : 1, encode_task(k, i, cb, tt));
            }
        }
    }
    unsigned int ticket = NO_TICKET;   // thread 0's bulk-level claim
    for (;;) {
        if (threadIdx.x == 0)
            s_cmd = q_acquire(Q, s_code, ticket);
        __syncthreads();
        if (s_cmd != CMD_RUN)
            break;
        int k, i, cb;
        decode_task(s_code, k, i, cb);
        const int kind = ga_kind(G, decode_tt(s_code), k, i);
        const double *Vt = A.tiles + ((size_t)k * A.p + i) * (size_t)NB * NB;
        const size_t strip = ((size_t)k * A.p + i) * (size_t)S * NB;
        if (kind == K_LARFB)
            task_larfb<NB, S, APPLY_W, NOTRANS>(sm, chunk_ptr<NB, S>(A, i, cb), Vt, A.T + strip, APPLY_W);
        else if (kind == K_SSRFB)
            task_ssrfb<NB, S, APPLY_W, false, NOTRANS>(sm, chunk_ptr<NB, S>(A, g_head(G, k, g_dom(G, k, i)), cb),
                                                       chunk_ptr<NB, S>(A, i, cb), Vt, A.T + strip, APPLY_W);
        else
            task_ssrfb<NB, S, APPLY_W, true, NOTRANS>(sm, chunk_ptr<NB, S>(A, g_partner(G, k, i), cb),
                                                      chunk_ptr<NB, S>(A, i, cb), Vt, A.T2 + strip, APPLY_W);
        __syncthreads();
        if (threadIdx.x == 0) {
            // successors: forward ones for Q^T; forward predecessors for Q, each
            // released by its own forward successors
            GTask sp[2], tmp[2];
            const int ns = NOTRANS ? ga_predecessors(G, kind, k, i, sp) : ga_specific(G, kind, k, i, sp);
            for (int s = 0; s < ns; s++) {
                const int tk = ga_kind(G, sp[s].tt, sp[s].k, sp[s].i);
                const int nd = NOTRANS ? ga_specific(G, tk, sp[s].k, sp[s].i, tmp) : ga_ndeps(tk, sp[s].k);
                q_signal(Q, apply_cnt_idx(A, sp[s].tt, sp[s].k, sp[s].i, cb), nd, tk == K_LARFB ? 0 : 1,
                         encode_task(sp[s].k, sp[s].i, cb, sp[s].tt));
            }
            __threadfence();
            atomicAdd(&Q.ctrl->completed, 1u);
        }
    }
}

// Scheduler state of the Q^T application: control block, counters (two
// banks for the tree form), the LB queue and the SB + TB queue.
struct ApplySched {
    size_t cnt_bytes, q0_bytes, q1_bytes;
    unsigned long long n0, n1;
};
static ApplySched apply_sched(const WsLayout &L, int nchunk)
{
    const TGraph G = make_graph(L.p, L.q, L.H);
    unsigned long long cnt[2];
    ga_count(G, cnt);
    ApplySched a;
    a.n0 = cnt[0] * (unsigned long long)nchunk;
    a.n1 = cnt[1] * (unsigned long long)nchunk;
    a.cnt_bytes = align256((size_t)(G.H < G.p ? 2 : 1) * L.steps * L.p * nchunk * sizeof(unsigned int));
    a.q0_bytes = align256((a.n0 ? a.n0 : 1) * 8);
    a.q1_bytes = align256((a.n1 ? a.n1 : 1) * 8);
    return a;
}

size_t apply_sched_bytes(const WsLayout &L, int nchunk)
{
    const ApplySched a = apply_sched(L, nchunk);
    return 256 + a.cnt_bytes + a.q0_bytes + a.q1_bytes;
}

template <int NB, int S, bool NOTRANS>
static int launch_apply_t(const WsLayout &L, const double *tiles, const double *T, const double *T2, double *Bt,
                          int64_t ncp, char *sched, cudaStream_t st, unsigned long long watchdog_ns)
{
    constexpr size_t smem = F64Cfg<NB, S, APPLY_W>::SMEM;
    int grid_max = 0;
    const int rc = kernel_grid((const void *)k_apply_dag<NB, S, NOTRANS>, NT, smem, &grid_max);
    if (rc)
        return rc;
    ApplyArgs A;
    A.tiles = tiles;
    A.T = T;
    A.T2 = T2;
    A.Bt = Bt;
    A.p = L.p;
    A.q = L.q;
    A.steps = L.steps;
    A.ncp = ncp;
    A.nchunk = (int)(ncp / APPLY_W);
    A.G = make_graph(L.p, L.q, L.H);
    const ApplySched a = apply_sched(L, A.nchunk);
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
    if (cudaMemsetAsync(sched, 0, apply_sched_bytes(L, A.nchunk), st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int grid = grid_max;
    if ((unsigned)grid > Q.total)
        grid = (int)Q.total;
    k_apply_dag<NB, S, NOTRANS><<<grid, NT, smem, st>>>(A, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_apply(const WsLayout &L, const double *tiles, const double *T, const double *T2, double *Bt,
                 int64_t ncp, char *sched, cudaStream_t st, unsigned long long watchdog_ns, bool notrans)
{
#define TQR_CASE(NB_, S_)                                                                        \
    if (L.nb == NB_ && L.ib == S_)                                                               \
        return notrans ? launch_apply_t<NB_, S_, true>(L, tiles, T, T2, Bt, ncp, sched, st, watchdog_ns)       \
                       : launch_apply_t<NB_, S_, false>(L, tiles, T, T2, Bt, ncp, sched, st, watchdog_ns);
    TQR_CASE(64, 16)
    TQR_CASE(64, 32)
    TQR_CASE(128, 16)
    TQR_CASE(128, 32)
    TQR_CASE(256, 16)
    TQR_CASE(256, 32)
#undef TQR_CASE
    return TILEQR_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------------------
// Tiled back substitution R X = Y, Y = the first q row blocks of Bt (m >= n).
// For j = q-1 .. 0: X_j = R_jj^{-1} Y_j (k_trsm_diag), then Y_i -= R_ij X_j
// for i < j (k_trsm_update).  One CTA per 32-column chunk (and row block).
__global__ void __launch_bounds__(NT) k_trsm_diag(const double *__restrict__ tiles, double *Bt, int nb,
                                                  int p, int64_t ncp, int j, int64_t n, int *flag)
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
    for (int c = last; c >= 0; c--) {
        const double d = ldcg(R + (size_t)c * nb + c);
        double x = 0.0;
        if (d != 0.0)
            x = ys[c * 33 + lane] / d;
        else if (threadIdx.x == 0)
            atomicCAS(flag, 0, (int)(col0 + c + 1));
        __syncthreads();
        if (warp == 0)
            ys[c * 33 + lane] = x;
        for (int r = warp; r < c; r += NWARP)
            ys[r * 33 + lane] = fma(-ldcg(R + (size_t)c * nb + r), x, ys[r * 33 + lane]);
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * 32; idx += NT) {
        const int c = idx / nb, r = idx - c * nb;
        Y[(size_t)c * nb + r] = (r <= last) ? ys[r * 33 + c] : 0.0;
    }
}

__global__ void __launch_bounds__(NT) k_trsm_update(const double *__restrict__ tiles, double *Bt, int nb,
                                                    int p, int64_t ncp, int j)
{
    extern __shared__ double xs[];  // nb x 32, [r][c] ld 33
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x, cb = blockIdx.y;
    const double *R = tiles + ((size_t)j * p + i) * (size_t)nb * nb;
    const double *X = Bt + ((size_t)j * ncp + (size_t)cb * 32) * nb;
    double *Y = Bt + ((size_t)i * ncp + (size_t)cb * 32) * nb;
    for (int idx = threadIdx.x; idx < nb * 32; idx += NT) {
        const int c = idx / nb, r = idx - c * nb;
        xs[r * 33 + c] = X[(size_t)c * nb + r];
    }
    __syncthreads();
    for (int r = warp; r < nb; r += NWARP) {
        double acc0 = Y[(size_t)lane * nb + r], acc1 = 0.0;
        int c = 0;
        for (; c + 1 < nb; c += 2) {
            acc0 = fma(-ldcg(R + (size_t)c * nb + r), xs[c * 33 + lane], acc0);
            acc1 = fma(-ldcg(R + (size_t)(c + 1) * nb + r), xs[(c + 1) * 33 + lane], acc1);
        }
        if (c < nb)
            acc0 = fma(-ldcg(R + (size_t)c * nb + r), xs[c * 33 + lane], acc0);
        Y[(size_t)lane * nb + r] = acc0 + acc1;
    }
}

int launch_trsm(const WsLayout &L, const double *tiles, double *Bt, int64_t ncp, int *flag, cudaStream_t st)
{
    const int nchunk = (int)(ncp / 32);
    const size_t smem = (size_t)L.nb * 33 * sizeof(double);
    if (kernel_smem_optin((const void *)k_trsm_diag, 256 * 33 * 8) != 0 ||
        kernel_smem_optin((const void *)k_trsm_update, 256 * 33 * 8) != 0)
        return TILEQR_ERR_CUDA;
    for (int j = L.q - 1; j >= 0; j--) {
        k_trsm_diag<<<nchunk, NT, smem, st>>>(tiles, Bt, L.nb, L.p, ncp, j, L.n, flag);
        count_launch();
        if (j > 0) {
            k_trsm_update<<<dim3(j, nchunk), NT, smem, st>>>(tiles, Bt, L.nb, L.p, ncp, j);
            count_launch();
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

}  // namespace tqr
