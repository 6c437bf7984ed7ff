// factor.cu -- the tiled QR factorization (Algorithm 2) on the GPU: one
// persistent kernel executing the task graph of Sec. 4, and the fork-join
// comparator (one launch per task kind per step).
#include <cstdio>

#include "dag.cuh"
#include "factor.h"

namespace tqr {

// ---------------------------------------------------------------------------
// Fork-join comparator: per step k the host launches GEQRT, then the LARFB
// row, then the TSQRT chain (one CTA, serial in i), then one CTA per column j
// running its SSRFB chain over i.  Each launch waits for the previous one.
// The tasks run through run_task, the same tile kernels (and ragged-edge
// instances) as the task graph, so both schedules give the same bits.
template <int NB, int S>
__device__ __forceinline__ void bulk_task(double *sm, const FactorArgs &F, int kind, int k, int i, int j)
{
    uint32_t mphase = 0;
    run_task<NB, S, false>(sm, F, kind, k, i, j, 0u, nullptr, mphase, nullptr);
}
template <int NB, int S>
__global__ void __launch_bounds__(NT, 1) k_bulk_geqrt(FactorArgs F, int k)
{
    extern __shared__ double sm[];
    bulk_task<NB, S>(sm, F, K_GEQRT, k, k, k);
}
template <int NB, int S>
__global__ void __launch_bounds__(NT, 1) k_bulk_larfb(FactorArgs F, int k)
{
    extern __shared__ double sm[];
    bulk_task<NB, S>(sm, F, K_LARFB, k, k, k + 1 + (int)blockIdx.x);
}
template <int NB, int S>
__global__ void __launch_bounds__(NT, 1) k_bulk_tsqrt(FactorArgs F, int k)
{
    extern __shared__ double sm[];
    for (int i = k + 1; i < F.p; i++) {
        bulk_task<NB, S>(sm, F, K_TSQRT, k, i, k);
        __syncthreads();
    }
}
template <int NB, int S>
__global__ void __launch_bounds__(NT, 1) k_bulk_ssrfb(FactorArgs F, int k)
{
    extern __shared__ double sm[];
    const int j = k + 1 + blockIdx.x;
    for (int i = k + 1; i < F.p; i++) {
        bulk_task<NB, S>(sm, F, K_SSRFB, k, i, j);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side.
template <int NB, int S>
static int launch_factor_t(const WsLayout &L, char *ws, int schedule, int flags, cudaStream_t st,
                           unsigned long long watchdog_ns, unsigned long long *trace,
                           unsigned int trace_cap)
{
    constexpr size_t smem = F64Cfg<NB, S>::SMEM;
    int grid_dag = 0;
    int rc = kernel_grid((const void *)k_factor_dag<NB, S, false>, NT, smem, &grid_dag);
    if (rc)
        return rc;
    if (schedule != TILEQR_SCHED_DAG) {
        const void *bulk[4] = {(const void *)k_bulk_geqrt<NB, S>, (const void *)k_bulk_larfb<NB, S>,
                               (const void *)k_bulk_tsqrt<NB, S>, (const void *)k_bulk_ssrfb<NB, S>};
        for (const void *fn : bulk)
            if ((rc = kernel_smem_optin(fn, smem)) != 0)
                return rc;
    }
    FactorArgs F;
    F.tiles = (double *)(ws + L.off_tiles);
    F.T = (double *)(ws + L.off_T);
    F.T2 = (L.H < L.p) ? (double *)(ws + L.off_T2) : nullptr;
    F.TF = F.TF2 = nullptr;
    F.cexp = nullptr;
    F.lm = 0;
    F.p = L.p;
    F.q = L.q;
    F.steps = L.steps;
    F.ncl = (int)(L.n - (int64_t)(L.q - 1) * L.nb);
    F.nrl = (int)(L.m - (int64_t)(L.p - 1) * L.nb);
    F.G = make_graph(L.p, L.q, L.H);
    if (schedule == TILEQR_SCHED_DAG) {
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
        if (flags & TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK)
            Q.withheld = encode_task(L.steps - 1, L.steps - 1, L.steps - 1);
        if (flags & TILEQR_FLAG_TEST_RANDOM_DELAYS)
            Q.delay_seed = ((unsigned long long)(((unsigned int)flags) >> 8) << 1) | 1ull;
        Q.trace = trace;
        Q.trace_cap = trace_cap;
        int grid = grid_dag;
        if ((unsigned)grid > L.total)
            grid = (int)L.total;
        k_factor_dag<NB, S, false><<<grid, NT, smem, st>>>(F, Q);
        count_launch();
    } else {
        for (int k = 0; k < L.steps; k++) {
            k_bulk_geqrt<NB, S><<<1, NT, smem, st>>>(F, k);
            count_launch();
            if (L.q - k - 1 > 0) {
                k_bulk_larfb<NB, S><<<L.q - k - 1, NT, smem, st>>>(F, k);
                count_launch();
            }
            if (L.p - k - 1 > 0) {
                k_bulk_tsqrt<NB, S><<<1, NT, smem, st>>>(F, k);
                count_launch();
                if (L.q - k - 1 > 0) {
                    k_bulk_ssrfb<NB, S><<<L.q - k - 1, NT, smem, st>>>(F, k);
                    count_launch();
                }
            }
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

bool factor_supported(int nb, int ib)
{
    return (nb == 64 || nb == 128 || nb == 256) && (ib == 16 || ib == 32);
}

int launch_factor(const WsLayout &L, char *ws, int schedule, int flags, cudaStream_t st,
                  unsigned long long watchdog_ns, unsigned long long *trace, unsigned int trace_cap)
{
#define TQR_CASE(NB_, S_)                                                                        \
    if (L.nb == NB_ && L.ib == S_)                                                               \
        return launch_factor_t<NB_, S_>(L, ws, schedule, flags, st, watchdog_ns, trace, trace_cap);
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

namespace tqr {

template <int NB, int S>
static int launch_factor_dag_at_t(const WsLayout &L, double *tiles, double *T, char *sched,
                                  cudaStream_t st, unsigned long long watchdog_ns)
{
    constexpr size_t smem = F64Cfg<NB, S>::SMEM;
    int grid_dag = 0;
    const int rc = kernel_grid((const void *)k_factor_dag<NB, S, false>, NT, smem, &grid_dag);
    if (rc)
        return rc;
    FactorArgs F;
    F.tiles = tiles;
    F.T = T;
    F.T2 = nullptr;
    F.TF = F.TF2 = nullptr;
    F.cexp = nullptr;
    F.lm = 0;
    F.p = L.p;
    F.q = L.q;
    F.steps = L.steps;
    F.ncl = (int)(L.n - (int64_t)(L.q - 1) * L.nb);
    F.nrl = (int)(L.m - (int64_t)(L.p - 1) * L.nb);
    F.G = make_graph(L.p, L.q, 0);
    Queues Q;
    Q.ctrl = (SchedCtrl *)sched;
    Q.cnt = (unsigned int *)(sched + (L.off_cnt - L.off_ctrl));
    for (int t = 0; t < K_NKIND; t++) {
        Q.slot[t] = (unsigned long long *)(sched + (L.off_q[t] - L.off_ctrl));
        Q.cap[t] = L.cap[t];
    }
    Q.total = L.total;
    Q.watchdog_ns = watchdog_ns;
    Q.withheld = ~0ull;
    Q.trace = nullptr;
    Q.trace_cap = 0;
    int grid = grid_dag;
    if ((unsigned)grid > L.total)
        grid = (int)L.total;
    k_factor_dag<NB, S, false><<<grid, NT, smem, st>>>(F, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_factor_dag_at(const WsLayout &L, double *tiles, double *T, char *sched, cudaStream_t st,
                         unsigned long long watchdog_ns)
{
#define TQR_CASE(NB_, S_)                                                                        \
    if (L.nb == NB_ && L.ib == S_)                                                               \
        return launch_factor_dag_at_t<NB_, S_>(L, tiles, T, sched, st, watchdog_ns);
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
