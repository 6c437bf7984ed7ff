// batched.cu -- many independent tiled QR factorizations in one persistent
// launch (the batched form): a per-matrix table in the workspace, one layout
// kernel over all matrices, one task-graph kernel over all tasks.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dag.cuh"
#include "factor.h"

namespace tqr {

// Column-major -> tiles for every matrix of the batch; blockIdx.y walks the
// matrices, each CTA's warps copy tile columns (nb contiguous doubles).
__global__ void k_cm2tile_batched(const MatInfo *__restrict__ mats, int count, int nb, int *nonfinite)
{
    const int lane = threadIdx.x & 31;
    bool bad = false;
    for (int b = blockIdx.y; b < count; b += gridDim.y) {
        const MatInfo mi = mats[b];
        if (mi.steps == 0)
            continue;
        const size_t nseg = (size_t)mi.p * mi.q * nb;
        const size_t wstride = (size_t)gridDim.x * (blockDim.x >> 5);
        for (size_t s = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += wstride) {
            const int c = (int)(s % nb);
            const size_t t = s / nb;
            const int i = (int)(t % mi.p), j = (int)(t / mi.p);
            const int64_t col = (int64_t)j * nb + c, row0 = (int64_t)i * nb;
            int valid = 0;
            if (col < mi.n) {
                const int64_t rem = mi.m - row0;
                valid = rem < nb ? (int)rem : nb;
            }
            const double *src = mi.A + col * mi.lda + row0;
            double *dst = mi.tiles + (t * nb + c) * nb;
            unsigned int emax = 0;
            for (int r = lane; r < nb; r += 32) {
                double v = 0.0;
                if (r < valid) {
                    v = __ldg(src + r);
                    bad |= !isfinite(v);
                    emax = max(emax, (unsigned int)(__double2hiint(v) >> 20) & 0x7FFu);
                }
                dst[r] = v;
            }
            // mixed precision: the column's largest exponent (column scaling)
            if (mi.cexp != nullptr) {
                emax = __reduce_max_sync(0xffffffffu, emax);
                if (lane == 0 && emax > 0 && col < mi.n)
                    atomicMax(mi.cexp + col, (int)emax);
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0)
        atomicExch(nonfinite, 1);
}

namespace {

struct BatchLayout {
    size_t off_ctrl, off_mats, off_cnt, off_q[K_NKIND], off_cexp, off_data, end;
    unsigned long long cap[K_NKIND], total, counters;
    double flops;
};

BatchLayout batch_layout(int count, const int64_t *m, const int64_t *n, int nb, int ib, int precision,
                         std::vector<MatInfo> *infos_out)
{
    BatchLayout B{};
    unsigned long long cnt = 0;
    size_t data = 0, ncols = 0;
    std::vector<MatInfo> infos(count);
    for (int b = 0; b < count; b++) {
        MatInfo &mi = infos[b];
        std::memset(&mi, 0, sizeof(mi));
        mi.m = m[b];
        mi.n = n[b];
        mi.p = (int)((m[b] + nb - 1) / nb);
        mi.q = (int)((n[b] + nb - 1) / nb);
        mi.steps = (m[b] > 0 && n[b] > 0) ? (mi.p < mi.q ? mi.p : mi.q) : 0;
        mi.cnt_off = cnt;
        cnt += (unsigned long long)mi.steps * mi.p * mi.q;
        if (mi.steps > 0) {
            unsigned long long lv[K_NKIND];
            g_level_counts(make_graph(mi.p, mi.q, 0), lv);
            for (int t = 0; t < K_NKIND; t++)
                B.cap[t] += lv[t];
        }
        // data offsets relative to the data section: tiles then T strips
        mi.tiles = (double *)(uintptr_t)data;
        data += align256((size_t)mi.p * mi.q * nb * nb * sizeof(double));
        mi.T = (double *)(uintptr_t)data;
        data += align256((size_t)mi.p * mi.q * ib * nb * sizeof(double));
        if (precision == TILEQR_TF32 && mi.steps > 0) {
            mi.TF = (unsigned char *)(uintptr_t)data;
            data += align256(tf_pairs(mi.p, mi.steps) * TF_PAIR_BYTES);
            // column exponents: offset (in ints) into the cleared cexp region
            mi.cexp = (int *)(uintptr_t)ncols;
            ncols += (size_t)n[b];
            mi.lm = ceil_log2_sqrt(m[b]);
        }
        const double mm = (double)m[b], nn = (double)n[b];
        if (m[b] >= n[b])
            B.flops += 2.0 * nn * nn * (mm - nn / 3.0);
        else
            B.flops += 2.0 * mm * mm * (nn - mm / 3.0);
    }
    B.counters = cnt;
    B.total = 0;
    for (int t = 0; t < K_NKIND; t++)
        B.total += B.cap[t];
    size_t off = 0;
    B.off_ctrl = off;
    off += 256;
    B.off_cnt = off;
    off += align256((size_t)(cnt ? cnt : 1) * 4);
    for (int t = 0; t < K_NKIND; t++) {
        B.off_q[t] = off;
        off += align256((size_t)(B.cap[t] ? B.cap[t] : 1) * 8);
    }
    // mixed precision: the column exponents of every matrix, cleared with
    // the scheduler state before each factorization
    B.off_cexp = off;
    off += ncols ? align256(ncols * sizeof(int)) : 0;
    B.off_mats = off;
    // the per-matrix table, then the order of the first pushes (count ints)
    off += align256((size_t)(count ? count : 1) * sizeof(MatInfo) + (size_t)(count ? count : 1) * sizeof(int));
    B.off_data = off;
    off += data;
    B.end = off;
    if (infos_out)
        *infos_out = infos;
    return B;
}

template <int NB, int S, bool MIXED>
int launch_batched_t(const tileqr_batch *bt, cudaStream_t st)
{
    constexpr size_t smem = DagCfg<NB, S, MIXED>::SMEM;
    int grid_dag = 0;
    int rc = kernel_grid((const void *)k_factor_dag_batched<NB, S, MIXED>, NT, smem, &grid_dag);
    if (rc)
        return rc;
    // the mixed kernel runs one CTA per SM (256 of the 512 tensor-memory columns each)
    if (MIXED && (rc = device_sm_count(&grid_dag)) != 0)
        return rc;
    char *ws = (char *)bt->workspace;
    Queues Q;
    Q.ctrl = (SchedCtrl *)(ws + bt->off_ctrl);
    Q.cnt = (unsigned int *)(ws + bt->off_cnt);
    for (int t = 0; t < K_NKIND; t++) {
        Q.slot[t] = (unsigned long long *)(ws + bt->off_q[t]);
        Q.cap[t] = bt->cap[t];
    }
    Q.total = (unsigned int)bt->total_tasks;
    Q.watchdog_ns = watchdog_ns_default();
    Q.withheld = ~0ull;
    Q.trace = nullptr;
    Q.trace_cap = 0;
    int grid = grid_dag;
    if ((unsigned long long)grid > bt->total_tasks)
        grid = (int)bt->total_tasks;
    k_factor_dag_batched<NB, S, MIXED><<<grid, NT, smem, st>>>((const MatInfo *)(ws + bt->off_mats), bt->count, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

}  // namespace
}  // namespace tqr

using namespace tqr;

static int check_batch_args(int count, const int64_t *m, const int64_t *n, int nb, int ib, int precision)
{
    if (count < 0 || count >= (1 << 20))
        return -1;
    if (count > 0 && (m == nullptr || n == nullptr))
        return -2;
    for (int b = 0; b < count; b++) {
        if (m[b] < 0 || n[b] < 0)
            return -2;
        if ((m[b] + nb - 1) / nb >= (1 << 14) || (n[b] + nb - 1) / nb >= (1 << 14))
            return -2;
    }
    if (precision == TILEQR_FP64 && !factor_supported(nb, ib))
        return TILEQR_ERR_UNSUPPORTED;
    if (precision == TILEQR_TF32 && !factor_mixed_supported(nb, ib))
        return TILEQR_ERR_UNSUPPORTED;
    if (precision != TILEQR_FP64 && precision != TILEQR_TF32)
        return TILEQR_ERR_UNSUPPORTED;
    return 0;
}

extern "C" int tileqr_batched_workspace_size(int count, const int64_t *m, const int64_t *n, int nb, int ib,
                                             int precision, size_t *bytes)
{
    int rc = check_batch_args(count, m, n, nb, ib, precision);
    if (rc)
        return rc;
    if (bytes == nullptr)
        return -7;
    *bytes = batch_layout(count, m, n, nb, ib, precision, nullptr).end;
    return 0;
}

extern "C" int tileqr_batched_prepare(int count, const int64_t *m, const int64_t *n, const double *const *A,
                                      const int64_t *lda, int nb, int ib, int precision, void *workspace,
                                      size_t ws_bytes, tileqr_stream_t stream, tileqr_batch *out)
{
    int rc = check_batch_args(count, m, n, nb, ib, precision);
    if (rc)
        return rc;
    if (count > 0 && (A == nullptr || lda == nullptr))
        return -4;
    if (out == nullptr)
        return -12;
    std::vector<MatInfo> infos;
    const BatchLayout B = batch_layout(count, m, n, nb, ib, precision, &infos);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < B.end)
        return TILEQR_ERR_WORKSPACE;
    char *ws = (char *)workspace;
    for (int b = 0; b < count; b++) {
        if (lda[b] < (m[b] > 1 ? m[b] : 1))
            return -5;
        if (A[b] == nullptr && m[b] > 0 && n[b] > 0)
            return -4;
        infos[b].A = A[b];
        infos[b].lda = lda[b];
        infos[b].tiles = (double *)(ws + B.off_data + (uintptr_t)infos[b].tiles);
        infos[b].T = (double *)(ws + B.off_data + (uintptr_t)infos[b].T);
        if (precision == TILEQR_TF32 && infos[b].steps > 0) {
            infos[b].TF = (unsigned char *)(ws + B.off_data + (uintptr_t)infos[b].TF);
            infos[b].cexp = (int *)(ws + B.off_cexp) + (uintptr_t)infos[b].cexp;
        }
    }
    std::memset(out, 0, sizeof(*out));
    out->count = count;
    out->nb = nb;
    out->ib = ib;
    out->precision = precision;
    out->total_tasks = B.total;
    for (int t = 0; t < K_NKIND; t++) {
        out->cap[t] = (uint32_t)B.cap[t];
        out->off_q[t] = B.off_q[t];
    }
    out->off_ctrl = B.off_ctrl;
    out->off_cnt = B.off_cnt;
    out->off_mats = B.off_mats;
    out->sched_bytes = B.off_mats - B.off_ctrl;
    out->workspace = workspace;
    out->workspace_bytes = ws_bytes;
    out->flops = B.flops;
    if (count == 0)
        return 0;
    cudaStream_t st = (cudaStream_t)stream;
    // largest matrices (by flop count) start first: their chains are the longest
    std::vector<int> order(count);
    for (int b = 0; b < count; b++)
        order[b] = b;
    auto work = [&](int b) {
        const double mm = (double)m[b], nn = (double)n[b];
        return m[b] >= n[b] ? nn * nn * (mm - nn / 3.0) : mm * mm * (nn - mm / 3.0);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    std::vector<char> table((size_t)count * sizeof(MatInfo) + (size_t)count * sizeof(int));
    std::memcpy(table.data(), infos.data(), (size_t)count * sizeof(MatInfo));
    std::memcpy(table.data() + (size_t)count * sizeof(MatInfo), order.data(), (size_t)count * sizeof(int));
    if (cudaMemcpyAsync(ws + B.off_mats, table.data(), table.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    return 0;
}

extern "C" int tileqr_factor_batched(const tileqr_batch *bt, tileqr_stream_t stream)
{
    if (bt == nullptr)
        return -1;
    if (bt->count == 0 || bt->total_tasks == 0)
        return 0;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)bt->workspace;
    if (cudaMemsetAsync(ws + bt->off_ctrl, 0, bt->sched_bytes, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    const int gy = bt->count < 65535 ? bt->count : 65535;
    k_cm2tile_batched<<<dim3(8, gy), 256, 0, st>>>((const MatInfo *)(ws + bt->off_mats), bt->count, bt->nb,
                                                   &((SchedCtrl *)(ws + bt->off_ctrl))->nonfinite);
    count_launch();
    if (cudaGetLastError() != cudaSuccess)
        return TILEQR_ERR_CUDA;
    const bool mixed = bt->precision == TILEQR_TF32;
#define TQR_CASE(NB_, S_, MX_)                                                                   \
    if (bt->nb == NB_ && bt->ib == S_ && mixed == MX_)                                           \
        return launch_batched_t<NB_, S_, MX_>(bt, st);
    TQR_CASE(64, 16, false)
    TQR_CASE(64, 32, false)
    TQR_CASE(128, 16, false)
    TQR_CASE(128, 32, false)
    TQR_CASE(256, 16, false)
    TQR_CASE(256, 32, false)
    TQR_CASE(128, 16, true)
    TQR_CASE(128, 32, true)
#undef TQR_CASE
    return TILEQR_ERR_UNSUPPORTED;
}

extern "C" int tileqr_batched_status(const tileqr_batch *bt, tileqr_stream_t stream)
{
    if (bt == nullptr)
        return -1;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (bt->count == 0)
        return 0;
    SchedCtrl c;
    if (cudaMemcpy(&c, (char *)bt->workspace + bt->off_ctrl, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (c.nonfinite)
        return TILEQR_ERR_NONFINITE;
    return c.error;
}

extern "C" int tileqr_batched_get(const tileqr_batch *bt, int index, tileqr_desc *out)
{
    if (bt == nullptr)
        return -1;
    if (index < 0 || index >= bt->count)
        return -2;
    if (out == nullptr)
        return -3;
    MatInfo mi;
    if (cudaMemcpy(&mi, (char *)bt->workspace + bt->off_mats + (size_t)index * sizeof(MatInfo), sizeof(mi),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    std::memset(out, 0, sizeof(*out));
    out->m = mi.m;
    out->n = mi.n;
    out->nb = bt->nb;
    out->ib = bt->ib;
    out->p = mi.p;
    out->q = mi.q;
    out->precision = bt->precision;
    out->schedule = TILEQR_SCHED_DAG;
    out->tiles = mi.tiles;
    out->T = mi.T;
    out->sched = (char *)bt->workspace + bt->off_ctrl;
    out->sched_bytes = bt->sched_bytes;
    out->workspace = bt->workspace;
    out->workspace_bytes = bt->workspace_bytes;
    return 0;
}
