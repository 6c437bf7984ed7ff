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
#include "tile_mixed.cuh"

namespace tqr {

struct ApplyArgs {
    const double *tiles;
    const double *T;
    const double *T2;
    double *Bt;
    int p, q, steps, nchunk;
    int64_t ncp;
    TGraph G;
    // mixed form (tensor-core updates, chunks of nb = 128 columns): the
    // factorization's pre-split operands per tile pair (TF; TF2 of the tree
    // merges), the A operand of W for each pair at TW + pair * tw_stride +
    // tw_off (T^T inside the TF block for Q^T, the transposed copy for Q),
    // and the column exponents of Bt for the column scaling
    const unsigned char *TF, *TF2, *TW, *TW2;
    size_t tw_stride, tw_off;
    const int *cexp;
    int lm;
    int64_t ncols;   // live columns of Bt (the rest of its ncp are zero)
};

template <int NB, int S, int CW = APPLY_W>
__device__ __forceinline__ double *chunk_ptr(const ApplyArgs &A, int i, int cb)
{
    return A.Bt + ((size_t)i * A.ncp + (size_t)cb * CW) * NB;
}

__device__ __forceinline__ size_t apply_cnt_idx(const ApplyArgs &A, int tt, int k, int i, int cb)
{
    return (((size_t)tt * A.steps + k) * A.p + i) * A.nchunk + cb;
}

// MIXED: the updates on the tensor cores (task_update_mixed_tf, 3xTF32 with
// FP32 accumulation) on column chunks of nb = 128, for a TILEQR_TF32
// factorization; one CTA per SM, holding tensor memory for the whole launch.
template <int NB, int S, bool NOTRANS, bool MIXED = false>
__global__ void __launch_bounds__(NT, 1) k_apply_dag(ApplyArgs A, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[4];
    const TGraph &G = A.G;
    constexpr int CW = MIXED ? NB : APPLY_W;
    uint32_t tmem = 0, mphase = 0;
    if constexpr (MIXED) {
        if ((threadIdx.x >> 5) == 0)
            tc::tmem_alloc(&s_tmem, MIX_TMEM_COLS);
        if (threadIdx.x == 0)
            for (int b = 0; b < 4; b++)
                tc::mbar_init(&s_mbar[b], 1);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tmem = s_tmem;
    }
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
        if constexpr (MIXED) {
            unsigned char *smb = (unsigned char *)sm;
            const size_t pi = tf_index(A.p, i, k);
            const bool tt = kind != K_LARFB && kind != K_SSRFB;
            const unsigned char *pair = (tt ? A.TF2 : A.TF) + pi * TF_PAIR_BYTES;
            const unsigned char *tw = (tt ? A.TW2 : A.TW) + pi * A.tw_stride + A.tw_off;
            const int *cx = A.cexp + (size_t)cb * NB;
            int *err = &Q.ctrl->error;
            const int64_t left = A.ncols - (int64_t)cb * NB;
            const int nl = left < NB ? (int)left : NB;
            if (kind == K_LARFB)
                task_update_mixed_tf<S, VK_UNIT, true>(smb, nullptr, chunk_ptr<NB, S, CW>(A, i, cb), pair, tw, cx, A.lm,
                                                 tmem, s_mbar, mphase, err, nl);
            else if (kind == K_SSRFB)
                task_update_mixed_tf<S, VK_FULL, true>(smb, chunk_ptr<NB, S, CW>(A, g_head(G, k, g_dom(G, k, i)), cb),
                                                 chunk_ptr<NB, S, CW>(A, i, cb), pair, tw, cx, A.lm, tmem, s_mbar,
                                                 mphase, err, nl);
            else
                task_update_mixed_tf<S, VK_UPPER, true>(smb, chunk_ptr<NB, S, CW>(A, g_partner(G, k, i), cb),
                                                  chunk_ptr<NB, S, CW>(A, i, cb), pair, tw, cx, A.lm, tmem, s_mbar,
                                                  mphase, err, nl);
        } else {
            const double *Vt = A.tiles + ((size_t)k * A.p + i) * (size_t)NB * NB;
            const size_t strip = ((size_t)k * A.p + i) * (size_t)S * NB;
            if (kind == K_LARFB)
                task_larfb<NB, S, APPLY_W, NOTRANS>(sm, chunk_ptr<NB, S>(A, i, cb), Vt, A.T + strip, APPLY_W);
            else if (kind == K_SSRFB)
                task_ssrfb<NB, S, APPLY_W, false, NOTRANS>(sm,
                                                           chunk_ptr<NB, S>(A, g_head(G, k, g_dom(G, k, i)), cb),
                                                           chunk_ptr<NB, S>(A, i, cb), Vt, A.T + strip, APPLY_W);
            else
                task_ssrfb<NB, S, APPLY_W, true, NOTRANS>(sm, chunk_ptr<NB, S>(A, g_partner(G, k, i), cb),
                                                          chunk_ptr<NB, S>(A, i, cb), Vt, A.T2 + strip, APPLY_W);
        }
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
    if constexpr (MIXED) {
        tc::fence_before_sync();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0)
            tc::tmem_dealloc(tmem, MIX_TMEM_COLS);
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

// Queues of one application over nchunk column chunks (state at sched,
// zeroed here); returns the task count (0: nothing to run).
static unsigned int apply_queues(const WsLayout &L, int nchunk, char *sched, unsigned long long watchdog_ns,
                                 Queues &Q)
{
    const ApplySched a = apply_sched(L, nchunk);
    Q = Queues{};
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
    return Q.total;
}

static ApplyArgs apply_args(const WsLayout &L, const double *tiles, const double *T, const double *T2, double *Bt,
                            int64_t ncp, int chunk)
{
    ApplyArgs A{};
    A.tiles = tiles;
    A.T = T;
    A.T2 = T2;
    A.Bt = Bt;
    A.p = L.p;
    A.q = L.q;
    A.steps = L.steps;
    A.ncp = ncp;
    A.nchunk = (int)(ncp / chunk);
    A.G = make_graph(L.p, L.q, L.H);
    return A;
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
    const ApplyArgs A = apply_args(L, tiles, T, T2, Bt, ncp, APPLY_W);
    Queues Q;
    if (apply_queues(L, A.nchunk, sched, watchdog_ns, Q) == 0)
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

template <int S, bool NOTRANS>
static int launch_apply_mixed_t(const WsLayout &L, const MixedOperands &M, double *Bt, int64_t ncp, int64_t ncols,
                                const int *cexp, char *sched, cudaStream_t st, unsigned long long watchdog_ns)
{
    constexpr size_t smem = TF_UPDATE_SMEM_TOTAL;
    int grid_max = 0;
    int rc = kernel_grid((const void *)k_apply_dag<128, S, NOTRANS, true>, NT, smem, &grid_max);
    if (rc)
        return rc;
    // one CTA per SM: each holds MIX_TMEM_COLS of the SM's tensor memory
    int nsm = 0;
    if ((rc = device_sm_count(&nsm)) != 0)
        return rc;
    if (grid_max > nsm)
        grid_max = nsm;
    ApplyArgs A = apply_args(L, nullptr, nullptr, nullptr, Bt, ncp, 128);
    A.TF = M.TF;
    A.TF2 = M.TF2;
    if (NOTRANS) {
        A.TW = M.TN;
        A.TW2 = M.TN2;
        A.tw_stride = TF_BYTES;
        A.tw_off = 0;
    } else {
        A.TW = M.TF;
        A.TW2 = M.TF2;
        A.tw_stride = TF_PAIR_BYTES;
        A.tw_off = TF_OFF_T;
    }
    A.cexp = cexp;
    A.lm = ceil_log2_sqrt((int64_t)L.p * L.nb);
    A.ncols = ncols;
    Queues Q;
    if (apply_queues(L, A.nchunk, sched, watchdog_ns, Q) == 0)
        return 0;
    if (cudaMemsetAsync(sched, 0, apply_sched_bytes(L, A.nchunk), st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int grid = grid_max;
    if ((unsigned)grid > Q.total)
        grid = (int)Q.total;
    k_apply_dag<128, S, NOTRANS, true><<<grid, NT, smem, st>>>(A, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_apply_mixed(const WsLayout &L, const MixedOperands &M, double *Bt, int64_t ncp, int64_t ncols,
                       const int *cexp, char *sched, cudaStream_t st, unsigned long long watchdog_ns, bool notrans)
{
    if (L.nb != 128 || ncp % 128 != 0 || ncols < 0 || ncols > ncp || M.TF == nullptr || (L.H < L.p && M.TF2 == nullptr) ||
        (notrans && (M.TN == nullptr || (L.H < L.p && M.TN2 == nullptr))))
        return TILEQR_ERR_UNSUPPORTED;
    if (kernel_smem_optin((const void *)k_apply_dag<128, 16, false, true>, TF_UPDATE_SMEM_TOTAL) ||
        kernel_smem_optin((const void *)k_apply_dag<128, 16, true, true>, TF_UPDATE_SMEM_TOTAL) ||
        kernel_smem_optin((const void *)k_apply_dag<128, 32, false, true>, TF_UPDATE_SMEM_TOTAL) ||
        kernel_smem_optin((const void *)k_apply_dag<128, 32, true, true>, TF_UPDATE_SMEM_TOTAL))
        return TILEQR_ERR_CUDA;
    if (L.ib == 16)
        return notrans ? launch_apply_mixed_t<16, true>(L, M, Bt, ncp, ncols, cexp, sched, st, watchdog_ns)
                       : launch_apply_mixed_t<16, false>(L, M, Bt, ncp, ncols, cexp, sched, st, watchdog_ns);
    if (L.ib == 32)
        return notrans ? launch_apply_mixed_t<32, true>(L, M, Bt, ncp, ncols, cexp, sched, st, watchdog_ns)
                       : launch_apply_mixed_t<32, false>(L, M, Bt, ncp, ncols, cexp, sched, st, watchdog_ns);
    return TILEQR_ERR_UNSUPPORTED;
}

// T (not transposed) of every tile pair, pre-split like the T^T operand:
// TN(r, K = c) = TT(c, r), hi and lo parts transposed separately (exact).
// One CTA per pair (grid-stride); src pairs are src_stride bytes apart with
// T^T at offset TF_OFF_T, dst pairs TF_BYTES apart.
__global__ void __launch_bounds__(256) k_tf_transpose(const unsigned char *__restrict__ src, size_t src_stride,
                                                      unsigned char *dst, size_t npairs)
{
    extern __shared__ float ts[];   // [c][r], ld 129
    constexpr int LD = 129, HALF = TF_CHUNK_BYTES / 2;
    for (size_t pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const unsigned char *tt = src + pr * src_stride + TF_OFF_T;
        unsigned char *tn = dst + pr * TF_BYTES;
        for (int part = 0; part < 2; part++) {
            __syncthreads();
            // element (row a, K = k) of chunk ch, part: 4-byte word w of the
            // chunk's part in core-matrix order (tc::kmajor_off with K extent 32)
            for (int e = threadIdx.x; e < 128 * 128; e += 256) {
                const int ch = e >> 12, w = e & 4095;
                const int a = ((w >> 8) << 3) | ((w >> 2) & 7), k = (((w >> 5) & 7) << 2) | (w & 3);
                ts[(ch * 32 + k) * LD + a] = *(const float *)(tt + ch * TF_CHUNK_BYTES + part * HALF + 4 * w);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < 128 * 128; e += 256) {
                const int ch = e >> 12, w = e & 4095;
                const int r = ((w >> 8) << 3) | ((w >> 2) & 7), c = ch * 32 + ((((w >> 5) & 7) << 2) | (w & 3));
                *(float *)(tn + ch * TF_CHUNK_BYTES + part * HALF + 4 * w) = ts[r * LD + c];
            }
        }
    }
}

int launch_tf_transpose(const unsigned char *src, size_t src_stride, unsigned char *dst, size_t npairs,
                        cudaStream_t st)
{
    if (npairs == 0)
        return 0;
    constexpr size_t smem = (size_t)128 * 129 * sizeof(float);
    if (kernel_smem_optin((const void *)k_tf_transpose, smem))
        return TILEQR_ERR_CUDA;
    int nsm = 0;
    const int rc = device_sm_count(&nsm);
    if (rc)
        return rc;
    const size_t grid = npairs < (size_t)nsm * 2 ? npairs : (size_t)nsm * 2;
    k_tf_transpose<<<(unsigned)grid, 256, smem, st>>>(src, src_stride, dst, npairs);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

// cexp[c] = the largest biased FP64 exponent of column c of the tile-row
// buffer Bt (p blocks of nb x ncp), for the column scaling of the mixed
// application: block (x, y) takes column x over the tile rows y, y +
// gridDim.y, ..., cexp cleared beforehand.
__global__ void __launch_bounds__(256) k_rows_cexp(const double *__restrict__ Bt, int nb, int p, int64_t ncp,
                                                   int *cexp)
{
    __shared__ unsigned int red[8];
    const int64_t c = blockIdx.x;
    unsigned int e = 0;
    for (int64_t i = blockIdx.y; i < p; i += gridDim.y)
        for (int r = threadIdx.x; r < nb; r += 256)
            e = max(e, (unsigned int)(__double2hiint(Bt[(i * ncp + c) * nb + r]) >> 20) & 0x7FFu);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++)
            e = max(e, red[w]);
        if (e)
            atomicMax(cexp + c, (int)e);
    }
}

int launch_rows_cexp(const double *Bt, int nb, int p, int64_t ncp, int *cexp, cudaStream_t st)
{
    if (ncp == 0)
        return 0;
    if (cudaMemsetAsync(cexp, 0, (size_t)ncp * sizeof(int), st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    const int ysplit = p < 64 ? (p > 0 ? p : 1) : 64;
    k_rows_cexp<<<dim3((unsigned)ncp, (unsigned)ysplit), 256, 0, st>>>(Bt, nb, p, ncp, cexp);
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

}  // namespace tqr
