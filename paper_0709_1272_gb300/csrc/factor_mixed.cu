// factor_mixed.cu -- the mixed-precision build of the persistent task-graph
// kernel (TILEQR_TF32): DLARFB / DSSRFB / DTTMQR as 3xTF32 products on the
// tcgen05 tensor cores with FP32 accumulation, with the panels' full T formed
// once per panel; DGEQRT / DTSQRT / DTTQRT in FP64 (nb = 128).
#include "dag.cuh"
#include "factor.h"

namespace tqr {

template <int S>
static int launch_factor_mixed_t(const WsLayout &L, char *ws, int flags, cudaStream_t st,
                                 unsigned long long watchdog_ns, unsigned long long *trace, unsigned int trace_cap)
{
    constexpr int NB = 128;
    constexpr size_t smem = DagCfg<NB, S, true>::SMEM;
    int grid_dag = 0;
    int rc = kernel_grid((const void *)k_factor_dag<NB, S, true>, NT, smem, &grid_dag);
    if (rc)
        return rc;
    // one CTA per SM: each holds 256 of the SM's 512 tensor-memory columns
    if ((rc = device_sm_count(&grid_dag)) != 0)
        return rc;
    FactorArgs F;
    F.tiles = (double *)(ws + L.off_tiles);
    F.T = (double *)(ws + L.off_T);
    F.T2 = (L.H < L.p) ? (double *)(ws + L.off_T2) : nullptr;
    F.TF = L.off_TF2 > L.off_TF ? (unsigned char *)(ws + L.off_TF) : nullptr;
    F.TF2 = (F.T2 != nullptr && L.off_ctrl > L.off_TF2) ? (unsigned char *)(ws + L.off_TF2) : nullptr;
    // the tensor-core updates need the panels' T^T operands (a TILEQR_TF32 layout)
    if (F.TF == nullptr || (F.T2 != nullptr && F.TF2 == nullptr))
        return TILEQR_ERR_WORKSPACE;
    if (L.off_cexp == 0)
        return TILEQR_ERR_WORKSPACE;
    F.cexp = (const int *)(ws + L.off_cexp);
    F.lm = ceil_log2_sqrt(L.m);
    F.p = L.p;
    F.q = L.q;
    F.steps = L.steps;
    F.ncl = (int)(L.n - (int64_t)(L.q - 1) * L.nb);
    F.nrl = (int)(L.m - (int64_t)(L.p - 1) * L.nb);
    F.G = make_graph(L.p, L.q, L.H);
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
    k_factor_dag<NB, S, true><<<grid, NT, smem, st>>>(F, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

bool factor_mixed_supported(int nb, int ib) { return nb == 128 && (ib == 16 || ib == 32); }

int launch_factor_mixed(const WsLayout &L, char *ws, int flags, cudaStream_t st, unsigned long long watchdog_ns,
                        unsigned long long *trace, unsigned int trace_cap)
{
    if (L.nb != 128)
        return TILEQR_ERR_UNSUPPORTED;
    if (L.ib == 16)
        return launch_factor_mixed_t<16>(L, ws, flags, st, watchdog_ns, trace, trace_cap);
    if (L.ib == 32)
        return launch_factor_mixed_t<32>(L, ws, flags, st, watchdog_ns, trace, trace_cap);
    return TILEQR_ERR_UNSUPPORTED;
}

}  // namespace tqr
