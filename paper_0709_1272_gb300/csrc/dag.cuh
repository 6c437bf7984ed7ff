// dag.cuh -- the persistent task-graph kernel of the tiled QR (Algorithm 2
// executed as the DAG of Sec. 4), shared by the FP64 and mixed-precision
// builds.  With MIXED, the DLARFB/DSSRFB tasks run on the tcgen05 tensor
// cores (tile_mixed.cuh) while DGEQRT/DTSQRT stay in FP64.
#pragma once
#include "graph.cuh"
#include "release.cuh"
#include "sched.cuh"
#include "tile_f64.cuh"
#include "tile_mixed.cuh"

namespace tqr {

struct FactorArgs {
    double *tiles;
    double *T;
    double *T2;   // DTTQRT T strips (tree form only)
    // mixed precision: the panels' full T^T as pre-split tf32 operands
    // (TF_PAIR_BYTES per tile pair; TF2 for DTTQRT); unused in FP64
    unsigned char *TF, *TF2;
    // mixed precision: the largest biased exponent of every matrix column
    // and ceil(log2 sqrt(m)), for the column scaling of the FP32 operands
    // (common.cuh); unused in FP64
    const int *cexp;
    int lm;
    int p, q, steps;
    // the matrix's columns in the last tile column and rows in the last tile
    // row (1..nb); the FP64 updates skip the zero padding past them
    int ncl, nrl;
    TGraph G;
};

template <int NB, int S>
__device__ __forceinline__ double *tile_ptr(const FactorArgs &F, int i, int j)
{
    return F.tiles + ((size_t)j * F.p + i) * (size_t)NB * NB;
}
template <int NB, int S>
__device__ __forceinline__ double *strip_ptr(const FactorArgs &F, int i, int k)
{
    return F.T + ((size_t)k * F.p + i) * (size_t)S * NB;
}
template <int NB, int S>
__device__ __forceinline__ double *strip2_ptr(const FactorArgs &F, int i, int k)
{
    return F.T2 + ((size_t)k * F.p + i) * (size_t)S * NB;
}

// The column exponents of tile column j (nullptr in FP64).
template <int NB>
__device__ __forceinline__ const int *cexp_ptr(const FactorArgs &F, int j)
{
    return F.cexp ? F.cexp + (size_t)j * NB : nullptr;
}

__device__ __forceinline__ unsigned char *tf_ptr(unsigned char *base, int p, int i, int k)
{
    return base + tf_index(p, i, k) * TF_PAIR_BYTES;
}

// Run the tile kernel of one task.  DTSQRT / DSSRFB eliminate row i into the
// head of its domain (row k in Algorithm 2); DTTQRT / DTTMQR merge domain
// head i into its partner head, reading only the upper triangle of tile
// (i, k).  With MIXED, the three update kinds run on the tensor cores.
template <int NB, int S, bool MIXED>
__device__ __forceinline__ void run_task(double *sm, const FactorArgs &F, int kind, int k, int i, int j,
                                         uint32_t tmem, uint64_t *mbar, uint32_t &mphase, int *err)
{
    const TGraph &G = F.G;
    unsigned char *smb = (unsigned char *)sm;
    switch (kind) {
    case K_GEQRT:
        if (!MIXED && k == F.q - 1 && F.ncl < NB)
            task_geqrt<NB, S, false, true>(sm, tile_ptr<NB, S>(F, i, k), strip_ptr<NB, S>(F, i, k), nullptr, 0,
                                           F.ncl);
        else
            task_geqrt<NB, S, MIXED>(sm, tile_ptr<NB, S>(F, i, k), strip_ptr<NB, S>(F, i, k), cexp_ptr<NB>(F, k),
                                     F.lm);
        if constexpr (MIXED)
            {
                __syncthreads();
                mixed_build_tfull<S, VK_UNIT>(smb, tile_ptr<NB, S>(F, i, k), strip_ptr<NB, S>(F, i, k),
                                              tf_ptr(F.TF, F.p, i, k));
            }
        break;
    case K_TSQRT:
        if (!MIXED && ((i == F.p - 1 && F.nrl < NB) || (k == F.q - 1 && F.ncl < NB)))
            task_tsqrt<NB, S, false, false, true>(sm, tile_ptr<NB, S>(F, g_head(G, k, g_dom(G, k, i)), k),
                                                  tile_ptr<NB, S>(F, i, k), strip_ptr<NB, S>(F, i, k), nullptr, 0,
                                                  i == F.p - 1 ? F.nrl : NB, k == F.q - 1 ? F.ncl : NB);
        else
            task_tsqrt<NB, S, MIXED, false>(sm, tile_ptr<NB, S>(F, g_head(G, k, g_dom(G, k, i)), k),
                                            tile_ptr<NB, S>(F, i, k), strip_ptr<NB, S>(F, i, k), cexp_ptr<NB>(F, k),
                                            F.lm);
        if constexpr (MIXED)
            {
                __syncthreads();
                mixed_build_tfull<S, VK_FULL>(smb, tile_ptr<NB, S>(F, i, k), strip_ptr<NB, S>(F, i, k),
                                              tf_ptr(F.TF, F.p, i, k));
            }
        break;
    case K_TTQRT:
        task_tsqrt<NB, S, MIXED, true>(sm, tile_ptr<NB, S>(F, g_partner(G, k, i), k), tile_ptr<NB, S>(F, i, k),
                                       strip2_ptr<NB, S>(F, i, k), cexp_ptr<NB>(F, k), F.lm);
        if constexpr (MIXED)
            {
                __syncthreads();
                mixed_build_tfull<S, VK_UPPER>(smb, tile_ptr<NB, S>(F, i, k), strip2_ptr<NB, S>(F, i, k),
                                               tf_ptr(F.TF2, F.p, i, k));
            }
        break;
    case K_LARFB:
        if constexpr (MIXED) {
            task_update_mixed_tf<S, VK_UNIT>(smb, nullptr, tile_ptr<NB, S>(F, i, j), tf_ptr(F.TF, F.p, i, k),
                                             tf_ptr(F.TF, F.p, i, k) + TF_OFF_T, cexp_ptr<NB>(F, j), F.lm, tmem,
                                             mbar, mphase, err);
        } else {
            if (j == F.q - 1 && F.ncl < NB)
                task_larfb<NB, S, FactorW<NB>::value, false, true>(sm, tile_ptr<NB, S>(F, i, j),
                                                                   tile_ptr<NB, S>(F, i, k),
                                                                   strip_ptr<NB, S>(F, i, k), F.ncl);
            else
                task_larfb<NB, S>(sm, tile_ptr<NB, S>(F, i, j), tile_ptr<NB, S>(F, i, k), strip_ptr<NB, S>(F, i, k));
        }
        break;
    case K_SSRFB: {
        double *top = tile_ptr<NB, S>(F, g_head(G, k, g_dom(G, k, i)), j);
        if constexpr (MIXED) {
            task_update_mixed_tf<S, VK_FULL>(smb, top, tile_ptr<NB, S>(F, i, j), tf_ptr(F.TF, F.p, i, k),
                                             tf_ptr(F.TF, F.p, i, k) + TF_OFF_T, cexp_ptr<NB>(F, j), F.lm, tmem,
                                             mbar, mphase, err);
        } else {
            if ((j == F.q - 1 && F.ncl < NB) || (i == F.p - 1 && F.nrl < NB))
                task_ssrfb_edge<NB, S>(sm, top, tile_ptr<NB, S>(F, i, j), tile_ptr<NB, S>(F, i, k),
                                       strip_ptr<NB, S>(F, i, k), j == F.q - 1 ? F.ncl : NB,
                                       i == F.p - 1 ? F.nrl : NB);
            else
                task_ssrfb<NB, S>(sm, top, tile_ptr<NB, S>(F, i, j), tile_ptr<NB, S>(F, i, k),
                                  strip_ptr<NB, S>(F, i, k));
        }
        break;
    }
    default: {   // K_TTMQR
        double *top = tile_ptr<NB, S>(F, g_partner(G, k, i), j);
        if constexpr (MIXED) {
            task_update_mixed_tf<S, VK_UPPER>(smb, top, tile_ptr<NB, S>(F, i, j), tf_ptr(F.TF2, F.p, i, k),
                                              tf_ptr(F.TF2, F.p, i, k) + TF_OFF_T, cexp_ptr<NB>(F, j), F.lm, tmem,
                                              mbar, mphase, err);
        } else
            task_ssrfb<NB, S, FactorW<NB>::value, true>(sm, top, tile_ptr<NB, S>(F, i, j), tile_ptr<NB, S>(F, i, k),
                                                        strip2_ptr<NB, S>(F, i, k));
        break;
    }
    }
}

// Dynamic shared memory and CTAs per SM of the persistent kernel.
template <int NB, int S, bool MIXED>
struct DagCfg {
    static constexpr size_t MIX = TF_BUILD_SMEM > TF_UPDATE_SMEM_TOTAL ? TF_BUILD_SMEM : TF_UPDATE_SMEM_TOTAL;
    static constexpr size_t SMEM = MIXED ? (F64Cfg<NB, S>::SMEM > MIX ? F64Cfg<NB, S>::SMEM : MIX)
                                         : F64Cfg<NB, S>::SMEM;
    static_assert(SMEM <= 232448, "shared memory budget");
    static constexpr int CTAS_PER_SM = MIXED ? 1 : F64Cfg<NB, S>::CTAS_PER_SM;
};

template <int NB, int S, bool MIXED>
__global__ void __launch_bounds__(NT, (DagCfg<NB, S, MIXED>::CTAS_PER_SM)) k_factor_dag(FactorArgs F, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[4];   // MMA commits (0, 1), operand copies (2, 3)
    uint32_t tmem = 0, mphase = 0;
    if (MIXED) {
        // one tensor-memory allocation and one mbarrier per persistent CTA
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
        // the step-0 DGEQRTs (one per domain head) have no predecessors
        if (ld_relaxed_s32(&Q.ctrl->nonfinite) != 0) {
            if (threadIdx.x == 0)
                atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_NONFINITE);
        } else {
            for (int d = threadIdx.x; d < g_ndom(F.G, 0); d += NT)
                q_push(Q, kind_prio(K_GEQRT), encode_task(0, g_head(F.G, 0, d), 0));
        }
    }
    // Thread ACQ claims the tasks; after each task it claims the next one
    // while warp 0 signals the finished task's successors, so the claim's
    // round trips to L2 overlap the release.
    constexpr int ACQ = 32;
    unsigned int ticket = NO_TICKET;   // thread ACQ's bulk-level claim
    if (threadIdx.x == ACQ)
        s_cmd = q_acquire(Q, s_code, ticket);
    for (;;) {
        __syncthreads();
        if (s_cmd != CMD_RUN)
            break;
        const unsigned long long code = s_code;
        int k, i, j;
        decode_task(code, k, i, j);
        const int kind = g_kind(F.G, decode_tt(code), k, i, j);
        if (Q.delay_seed) {   // schedule stress test (off by default)
            if (threadIdx.x == 0)
                stress_sleep(stress_delay_ns(code, Q.delay_seed, 0));
            __syncthreads();
        }
        const unsigned long long t0 = Q.trace ? globaltimer_ns() : 0ull;
        run_task<NB, S, MIXED>(sm, F, kind, k, i, j, tmem, s_mbar, mphase, &Q.ctrl->error);
        __syncthreads();
        if (threadIdx.x < 32) {
            if (Q.delay_seed && threadIdx.x == 0)
                stress_sleep(stress_delay_ns(code, Q.delay_seed, 1));
            __syncwarp();
            release_graph(Q, F.G, kind, k, i, j, threadIdx.x, 32);
            __syncwarp();
            if (threadIdx.x == 0) {
                if (Q.trace)
                    trace_record(Q, code, t0, globaltimer_ns());
                __threadfence();
                atomicAdd(&Q.ctrl->completed, 1u);
            }
        } else if (threadIdx.x == ACQ) {
            s_cmd = q_acquire(Q, s_code, ticket);
        }
    }
    if (MIXED) {
        tc::fence_before_sync();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0)
            tc::tmem_dealloc(tmem, MIX_TMEM_COLS);
    }
}

}  // namespace tqr

// ---------------------------------------------------------------------------
// Batched form: many independent matrices factored by one persistent launch.
// Every matrix has its own tiles, T strips and task counters; the four
// priority queues are shared, so tasks of all matrices interleave and the
// GPU stays full while small matrices finish.
namespace tqr {

struct MatInfo {
    double *tiles;
    double *T;
    unsigned char *TF;   // mixed precision: the panels' pre-split T^T operands (else nullptr)
    int *cexp;           // mixed precision: largest biased exponent per column (else nullptr)
    const double *A;
    int64_t m, n, lda;
    int p, q, steps, lm;  // lm = ceil(log2 sqrt(m)) (column scaling)
    size_t cnt_off;   // first task counter of this matrix
};

// batch task code: matrix (20 bits) | k (14) | i (15) | j (15)
__host__ __device__ inline unsigned long long encode_btask(int mat, int k, int i, int j)
{
    return ((unsigned long long)mat << 44) | ((unsigned long long)k << 30) | ((unsigned long long)i << 15) |
           (unsigned long long)j;
}
__host__ __device__ inline void decode_btask(unsigned long long c, int &mat, int &k, int &i, int &j)
{
    mat = (int)(c >> 44);
    k = (int)((c >> 30) & 0x3FFF);
    i = (int)((c >> 15) & 0x7FFF);
    j = (int)(c & 0x7FFF);
}

// Successors of task (k, i, j) of matrix `mat` in the graph of Algorithm 2
// (the flat tree: release_graph with one domain per step).
__device__ static void release_batched(const Queues &Q, const FactorArgs &F, size_t cnt_off, int mat, int k, int i,
                                       int j, int first, int stride)
{
    const int p = F.p, q = F.q;
    const int kind = task_kind(i, j, k);
    int nsucc = 0;
    switch (kind) {
    case K_GEQRT: nsucc = (q - k - 1) + (k + 1 < p ? 1 : 0); break;
    case K_LARFB: nsucc = (k + 1 < p) ? 1 : 0; break;
    case K_TSQRT: nsucc = (q - k - 1) + (i + 1 < p ? 1 : 0); break;
    default: nsucc = (i + 1 < p ? 1 : 0) + 1; break;
    }
    for (int s = first; s < nsucc; s += stride) {
        int ks, is, js;
        switch (kind) {
        case K_GEQRT:
            if (s < q - k - 1) { ks = k; is = k; js = k + 1 + s; }
            else { ks = k; is = k + 1; js = k; }
            break;
        case K_LARFB:
            ks = k; is = k + 1; js = j;
            break;
        case K_TSQRT:
            if (s < q - k - 1) { ks = k; is = i; js = k + 1 + s; }
            else { ks = k; is = i + 1; js = k; }
            break;
        default:
            if (s == 0 && i + 1 < p) { ks = k; is = i + 1; js = j; }
            else { ks = k + 1; is = i; js = j; }
            break;
        }
        const size_t idx = cnt_off + ((size_t)ks * p + is) * q + js;
        q_signal(Q, idx, task_ndeps(is, js, ks), kind_prio(task_kind(is, js, ks), ks, js),
                 encode_btask(mat, ks, is, js));
    }
}

template <int NB, int S, bool MIXED>
__global__ void __launch_bounds__(NT, (DagCfg<NB, S, MIXED>::CTAS_PER_SM))
    k_factor_dag_batched(const MatInfo *__restrict__ mats, int count, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[4];   // MMA commits (0, 1), operand copies (2, 3)
    __shared__ FactorArgs s_F;
    __shared__ size_t s_cnt;
    uint32_t tmem = 0, mphase = 0;
    if (MIXED) {
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
        if (ld_relaxed_s32(&Q.ctrl->nonfinite) != 0) {
            if (threadIdx.x == 0)
                atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_NONFINITE);
        } else {
            // the matrices' first panels in the order the host stored after
            // the table (largest first), so the longest chains start first
            const int *order = (const int *)(mats + count);
            for (int u = threadIdx.x; u < count; u += NT) {
                const int b = order[u];
                if (mats[b].steps > 0)
                    q_push(Q, K_GEQRT, encode_btask(b, 0, 0, 0));
            }
        }
    }
    // as in k_factor_dag: thread ACQ claims the next task (and loads its
    // matrix's descriptor) while warp 0 releases the finished one
    constexpr int ACQ = 32;
    unsigned int ticket = NO_TICKET;   // thread ACQ's bulk-level claim
    auto claim = [&]() {
        s_cmd = q_acquire(Q, s_code, ticket);
        if (s_cmd == CMD_RUN) {
            int mat, k, i, j;
            decode_btask(s_code, mat, k, i, j);
            const MatInfo &mi = mats[mat];
            s_F.tiles = mi.tiles;
            s_F.T = mi.T;
            s_F.T2 = nullptr;
            s_F.TF = mi.TF;
            s_F.TF2 = nullptr;
            s_F.cexp = mi.cexp;
            s_F.lm = mi.lm;
            s_F.p = mi.p;
            s_F.q = mi.q;
            s_F.steps = mi.steps;
            s_F.ncl = (int)(mi.n - (int64_t)(mi.q - 1) * NB);
            s_F.nrl = (int)(mi.m - (int64_t)(mi.p - 1) * NB);
            s_F.G = make_graph(mi.p, mi.q, 0);
            s_cnt = mi.cnt_off;
        }
    };
    if (threadIdx.x == ACQ)
        claim();
    for (;;) {
        __syncthreads();
        if (s_cmd != CMD_RUN)
            break;
        const unsigned long long code = s_code;
        int mat, k, i, j;
        decode_btask(code, mat, k, i, j);
        const FactorArgs F = s_F;
        const size_t cnt_off = s_cnt;
        const unsigned long long t0 = Q.trace ? globaltimer_ns() : 0ull;
        run_task<NB, S, MIXED>(sm, F, task_kind(i, j, k), k, i, j, tmem, s_mbar, mphase, &Q.ctrl->error);
        __syncthreads();
        if (threadIdx.x < 32) {
            release_batched(Q, F, cnt_off, mat, k, i, j, threadIdx.x, 32);
            __syncwarp();
            if (threadIdx.x == 0) {
                if (Q.trace)
                    trace_record(Q, code, t0, globaltimer_ns());
                __threadfence();
                atomicAdd(&Q.ctrl->completed, 1u);
            }
        } else if (threadIdx.x == ACQ) {
            claim();
        }
    }
    if (MIXED) {
        tc::fence_before_sync();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0)
            tc::tmem_dealloc(tmem, MIX_TMEM_COLS);
    }
}

}  // namespace tqr
