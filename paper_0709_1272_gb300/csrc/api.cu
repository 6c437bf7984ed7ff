// api.cu -- the C ABI of libtileqr (declared in include/tileqr.h): argument
// checking, workspace layout, and the launch sequences of the factorization,
// Q^T application and least-squares solve.  All device memory comes from the
// caller's workspace.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "factor.h"
#include "graph.cuh"
#include "tile_mixed.cuh"

namespace tqr {
static std::atomic<unsigned long long> g_launches{0};
static cudaEvent_t g_ev_before = nullptr, g_ev_after = nullptr;
static unsigned long long *g_trace = nullptr;
static unsigned long long g_trace_cap = 0;
void count_launch(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void trace_target(unsigned long long **records, unsigned int *capacity)
{
    *records = g_trace;
    *capacity = (unsigned int)(g_trace_cap > 0xffffffffull ? 0xffffffffull : g_trace_cap);
}

unsigned long long watchdog_ns_default()
{
    const char *e = std::getenv("TILEQR_WATCHDOG_MS");
    long ms = e ? std::atol(e) : 0;
    if (ms <= 0)
        ms = 10000;
    return (unsigned long long)ms * 1000000ull;
}
}  // namespace tqr

namespace tqr {
WsLayout make_layout(int64_t m, int64_t n, int nb, int ib, int h, int precision)
{
    WsLayout L{};
    L.m = m;
    L.n = n;
    L.nb = nb;
    L.ib = ib;
    L.p = (int)((m + nb - 1) / nb);
    L.q = (int)((n + nb - 1) / nb);
    L.steps = L.p < L.q ? L.p : L.q;
    const TGraph G = make_graph(L.p, L.q, h);
    L.H = G.H;
    const bool tree = G.H < G.p;
    const size_t tiles = (size_t)L.p * L.q * nb * nb * sizeof(double);
    const size_t tst = (size_t)L.p * L.q * ib * nb * sizeof(double);
    L.off_tiles = 0;
    L.off_T = align256(tiles);
    L.off_T2 = L.off_T + align256(tst);
    // pre-split T^T, V^T and V operands: 3 x 128 x 128 tf32 hi + lo per tile pair (384 KB)
    const size_t tfb = (precision == TILEQR_TF32 && nb == 128) ? tf_pairs(L.p, L.steps) * TF_PAIR_BYTES : 0;
    L.off_TF = L.off_T2 + (tree ? align256(tst) : 0);
    L.off_TF2 = L.off_TF + align256(tfb);
    L.off_ctrl = L.off_TF2 + (tree ? align256(tfb) : 0);
    L.off_cnt = L.off_ctrl + 256;
    size_t off = L.off_cnt + align256(g_ncounters(G) * sizeof(unsigned int));
    unsigned long long caps[K_NKIND];
    g_level_counts(G, caps);
    unsigned long long tot = 0;
    for (int t = 0; t < K_NKIND; t++) {
        L.cap[t] = (unsigned int)caps[t];
        tot += caps[t];
        L.off_q[t] = off;
        off += align256((size_t)(caps[t] ? caps[t] : 1) * sizeof(unsigned long long));
    }
    L.total = (unsigned int)tot;
    // per-column exponents of the mixed-precision path, in the range that is
    // cleared with the scheduler state before every factorization
    L.off_cexp = 0;
    if (tfb > 0) {
        L.off_cexp = off;
        off += align256((size_t)(n > 0 ? n : 1) * sizeof(int));
    }
    L.end = off;
    return L;
}
}  // namespace tqr

using namespace tqr;

static int check_geom(int64_t m, int64_t n, int nb, int ib)
{
    if (m < 0)
        return -1;
    if (n < 0)
        return -2;
    if (nb < 1)
        return -5;
    if (ib < 1 || ib > nb || nb % ib != 0)
        return -6;
    // task codes hold 21-bit tile indices
    if ((m + nb - 1) / nb >= (1 << 21) || (n + nb - 1) / nb >= (1 << 21))
        return -1;
    return 0;
}

extern "C" int tileqr_workspace_size(int64_t m, int64_t n, int nb, int ib, int precision, size_t *bytes)
{
    int rc = check_geom(m, n, nb, ib);
    if (rc)
        return rc;
    if (precision != TILEQR_FP64 && precision != TILEQR_TF32 && precision != TILEQR_SPLIT_BF16)
        return -5;
    if (!bytes)
        return -6;
    *bytes = make_layout(m, n, nb, ib, 0, precision).end;
    return 0;
}

extern "C" int tileqr_workspace_size_tree(int64_t m, int64_t n, int nb, int ib, int precision, int domain,
                                          size_t *bytes)
{
    int rc = check_geom(m, n, nb, ib);
    if (rc)
        return rc;
    if (precision != TILEQR_FP64 && precision != TILEQR_TF32 && precision != TILEQR_SPLIT_BF16)
        return -5;
    if (domain < 0)
        return -6;
    if (!bytes)
        return -7;
    *bytes = make_layout(m, n, nb, ib, domain, precision).end;
    return 0;
}

// The factorization proper; `domain` 0 = Algorithm 2's flat tree.  Argument
// errors are reported with the positions of tileqr_factor; the caller remaps.
static int factor_impl(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib, int domain,
                       int precision, int schedule, int flags, void *workspace, size_t ws_bytes,
                       tileqr_stream_t stream, tileqr_desc *out)
{
    if (m < 0)
        return -1;
    if (n < 0)
        return -2;
    if (A == nullptr && m > 0 && n > 0)
        return -3;
    if (lda < (m > 1 ? m : 1))
        return -4;
    int rc = check_geom(m, n, nb, ib);
    if (rc == -5)
        return -5;
    if (rc == -6)
        return -6;
    if (rc)
        return rc;
    if (precision != TILEQR_FP64 && precision != TILEQR_TF32 && precision != TILEQR_SPLIT_BF16)
        return -7;
    if (schedule != TILEQR_SCHED_DAG && schedule != TILEQR_SCHED_BULK)
        return -8;
    if (out == nullptr)
        return -13;
    if (precision == TILEQR_SPLIT_BF16)
        return TILEQR_ERR_UNSUPPORTED;
    if (precision == TILEQR_FP64 && !factor_supported(nb, ib))
        return TILEQR_ERR_UNSUPPORTED;
    if (precision == TILEQR_TF32 && (schedule != TILEQR_SCHED_DAG || !factor_mixed_supported(nb, ib)))
        return TILEQR_ERR_UNSUPPORTED;
    const WsLayout L = make_layout(m, n, nb, ib, domain, precision);
    const bool tree = L.H < L.p;
    if (tree && schedule != TILEQR_SCHED_DAG)
        return TILEQR_ERR_UNSUPPORTED;
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.end)
        return TILEQR_ERR_WORKSPACE;
    char *ws = (char *)workspace;
    cudaStream_t st = (cudaStream_t)stream;

    std::memset(out, 0, sizeof(*out));
    out->m = m;
    out->n = n;
    out->nb = nb;
    out->ib = ib;
    out->p = L.p;
    out->q = L.q;
    out->precision = precision;
    out->schedule = schedule;
    out->tiles = (double *)(ws + L.off_tiles);
    out->T = (double *)(ws + L.off_T);
    out->sched = ws + L.off_ctrl;
    out->sched_bytes = L.end - L.off_ctrl;
    out->workspace = workspace;
    out->workspace_bytes = ws_bytes;
    out->domain = L.H;
    out->T2 = tree ? (double *)(ws + L.off_T2) : nullptr;

    // reset the scheduler state (control block, counters, queues)
    if (cudaMemsetAsync(ws + L.off_ctrl, 0, L.end - L.off_ctrl, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    // T2 strips of rows that are not merged stay zero (documented contents)
    if (tree && cudaMemsetAsync(ws + L.off_T2, 0, L.off_TF - L.off_T2, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (m == 0 || n == 0)
        return 0;
    rc = launch_cm2tile(A, lda, m, n, out->tiles, nb, L.p, L.q, (SchedCtrl *)(ws + L.off_ctrl),
                        L.off_cexp ? (int *)(ws + L.off_cexp) : nullptr, st);
    if (rc)
        return rc;
    unsigned long long wd = watchdog_ns_default();
    if (flags & TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK)
        wd = 300ull * 1000000ull;
    if (schedule == TILEQR_SCHED_BULK) {
        // the fork-join comparator has no device scheduler; a non-finite input
        // is still reported through the control block by tileqr_status
    }
    if (g_ev_before && g_ev_after && cudaEventRecord(g_ev_before, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    const unsigned int tcap = (unsigned int)(g_trace_cap > 0xffffffffull ? 0xffffffffull : g_trace_cap);
    if (precision == TILEQR_TF32)
        rc = launch_factor_mixed(L, ws, flags, st, wd, g_trace, tcap);
    else
        rc = launch_factor(L, ws, schedule, flags, st, wd, g_trace, tcap);
    if (rc == 0 && g_ev_before && g_ev_after && cudaEventRecord(g_ev_after, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    return rc;
}

extern "C" int tileqr_factor(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib,
                             int precision, int schedule, int flags, void *workspace, size_t ws_bytes,
                             tileqr_stream_t stream, tileqr_desc *out)
{
    return factor_impl(m, n, A, lda, nb, ib, 0, precision, schedule, flags, workspace, ws_bytes, stream, out);
}

extern "C" int tileqr_factor_tree(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib, int domain,
                                  int precision, int flags, void *workspace, size_t ws_bytes,
                                  tileqr_stream_t stream, tileqr_desc *out)
{
    if (domain < 0)
        return -7;
    const int rc = factor_impl(m, n, A, lda, nb, ib, domain, precision, TILEQR_SCHED_DAG, flags, workspace,
                               ws_bytes, stream, out);
    // positions of tileqr_factor_tree: precision 8, out 13
    if (rc == -7)
        return -8;
    return rc;
}

extern "C" int tileqr_status(const tileqr_desc *d, tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (d->m == 0 || d->n == 0)
        return 0;
    SchedCtrl c;
    if (cudaMemcpy(&c, d->sched, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (c.nonfinite)
        return TILEQR_ERR_NONFINITE;
    return c.error;
}

extern "C" int tileqr_get_R(const tileqr_desc *d, double *R, int64_t ldr, tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    const int64_t k = d->m < d->n ? d->m : d->n;
    if (R == nullptr && k > 0)
        return -2;
    if (ldr < (k > 1 ? k : 1))
        return -3;
    if (k == 0)
        return 0;
    return launch_tile2cm(d->tiles, d->nb, d->p, d->q, d->m, d->n, R, ldr, 1, k, (cudaStream_t)stream);
}

extern "C" int tileqr_get_tree_T(const tileqr_desc *d, double *T2, int64_t ldt, tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    if (d->T2 == nullptr)
        return TILEQR_ERR_UNSUPPORTED;
    if (T2 == nullptr && d->n > 0)
        return -2;
    if (ldt < (int64_t)d->p * d->ib || ldt < 1)
        return -3;
    if (d->m == 0 || d->n == 0)
        return 0;
    return launch_strips2cm(d->T2, d->nb, d->ib, d->p, d->q, d->n, T2, ldt, (cudaStream_t)stream);
}

extern "C" int tileqr_get_factors(const tileqr_desc *d, double *AV, int64_t ldav, double *T, int64_t ldt,
                                  tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    if (AV == nullptr && d->m > 0 && d->n > 0)
        return -2;
    if (ldav < (d->m > 1 ? d->m : 1))
        return -3;
    if (T != nullptr && ldt < (int64_t)d->p * d->ib)
        return -5;
    if (d->m == 0 || d->n == 0)
        return 0;
    int rc = launch_tile2cm(d->tiles, d->nb, d->p, d->q, d->m, d->n, AV, ldav, 0, d->m, (cudaStream_t)stream);
    if (rc == 0 && T != nullptr)
        rc = launch_strips2cm(d->T, d->nb, d->ib, d->p, d->q, d->n, T, ldt, (cudaStream_t)stream);
    return rc;
}

static int64_t apply_ncp(int64_t nrhs) { return ((nrhs + APPLY_W - 1) / APPLY_W) * APPLY_W; }

extern "C" int tileqr_apply_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes)
{
    if (d == nullptr)
        return -1;
    if (nrhs < 0)
        return -2;
    if (bytes == nullptr)
        return -3;
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain);
    const int64_t ncp = apply_ncp(nrhs);
    *bytes = align256((size_t)L.p * L.nb * ncp * sizeof(double)) + apply_sched_bytes(L, (int)(ncp / APPLY_W)) + 256;
    return 0;
}

// Q^T applied to Bt (tile-row layout) inside the apply workspace.
static int apply_core(const tileqr_desc *d, const WsLayout &L, double *B, int64_t ldb, int64_t nrhs,
                      char *aws, cudaStream_t st, double **Bt_out, int64_t *ncp_out, int **flag_out,
                      bool notrans = false)
{
    const int64_t ncp = apply_ncp(nrhs);
    double *Bt = (double *)aws;
    char *sched = aws + align256((size_t)L.p * L.nb * ncp * sizeof(double));
    int *flag = (int *)(sched + apply_sched_bytes(L, (int)(ncp / APPLY_W)));
    if (cudaMemsetAsync(flag, 0, 256, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int rc = launch_cm2rows(B, ldb, d->m, nrhs, Bt, d->nb, d->p, ncp, st);
    if (rc)
        return rc;
    rc = launch_apply(L, d->tiles, d->T, d->T2, Bt, ncp, sched, st, watchdog_ns_default(), notrans);
    *Bt_out = Bt;
    *ncp_out = ncp;
    *flag_out = flag;
    return rc;
}

static int apply_impl(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                      size_t ws_bytes, tileqr_stream_t stream, bool notrans)
{
    if (d == nullptr)
        return -1;
    if (B == nullptr && nrhs > 0 && d->m > 0)
        return -2;
    if (ldb < (d->m > 1 ? d->m : 1))
        return -3;
    if (nrhs < 0)
        return -4;
    size_t need = 0;
    tileqr_apply_workspace_size(d, nrhs, &need);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < need)
        return TILEQR_ERR_WORKSPACE;
    if (nrhs == 0 || d->m == 0 || d->n == 0)
        return 0;
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain);
    cudaStream_t st = (cudaStream_t)stream;
    double *Bt;
    int64_t ncp;
    int *flag;
    int rc = apply_core(d, L, B, ldb, nrhs, (char *)workspace, st, &Bt, &ncp, &flag, notrans);
    if (rc)
        return rc;
    return launch_rows2cm(Bt, d->nb, d->p, ncp, d->m, nrhs, B, ldb, st);
}

extern "C" int tileqr_apply_qt(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                               size_t ws_bytes, tileqr_stream_t stream)
{
    return apply_impl(d, B, ldb, nrhs, workspace, ws_bytes, stream, false);
}

extern "C" int tileqr_apply_q(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                              size_t ws_bytes, tileqr_stream_t stream)
{
    return apply_impl(d, B, ldb, nrhs, workspace, ws_bytes, stream, true);
}

// ---------------------------------------------------------------------------
// Mixed application (TILEQR_TF32 factorizations, nb 128): Q^T B or Q B on
// the tensor cores from the operands the factorization kept.
namespace tqr {

size_t mixed_tn_bytes(const WsLayout &L)
{
    return (L.H < L.p ? 2 : 1) * tf_pairs(L.p, L.steps) * TF_BYTES;
}

int mixed_operands(const tileqr_desc *d, const WsLayout &L, unsigned char *TN, cudaStream_t st, MixedOperands *M)
{
    if (d->precision != TILEQR_TF32 || d->nb != 128 || d->workspace == nullptr || L.off_TF2 <= L.off_TF)
        return TILEQR_ERR_UNSUPPORTED;
    const unsigned char *ws = (const unsigned char *)d->workspace;
    const size_t npairs = tf_pairs(L.p, L.steps);
    const bool tree = L.H < L.p;
    *M = MixedOperands{};
    M->TF = ws + L.off_TF;
    M->TF2 = tree ? ws + L.off_TF2 : nullptr;
    if (TN != nullptr) {
        int rc = launch_tf_transpose(M->TF, TF_PAIR_BYTES, TN, npairs, st);
        if (rc)
            return rc;
        M->TN = TN;
        if (tree) {
            if ((rc = launch_tf_transpose(M->TF2, TF_PAIR_BYTES, TN + npairs * TF_BYTES, npairs, st)) != 0)
                return rc;
            M->TN2 = TN + npairs * TF_BYTES;
        }
    }
    return 0;
}

}  // namespace tqr

static int64_t mixed_ncp(int64_t nrhs) { return ((nrhs + 127) / 128) * 128; }

extern "C" int tileqr_apply_mixed_workspace_size(const tileqr_desc *d, int64_t nrhs, size_t *bytes)
{
    if (d == nullptr)
        return -1;
    if (nrhs < 0)
        return -2;
    if (bytes == nullptr)
        return -3;
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain, d->precision);
    const int64_t ncp = mixed_ncp(nrhs);
    *bytes = align256((size_t)L.p * L.nb * ncp * sizeof(double)) + align256(mixed_tn_bytes(L)) +
             align256(apply_sched_bytes(L, (int)(ncp / 128))) + align256((size_t)(ncp ? ncp : 1) * sizeof(int));
    return 0;
}

extern "C" int tileqr_apply_mixed(const tileqr_desc *d, int trans, double *B, int64_t ldb, int64_t nrhs,
                                  void *workspace, size_t ws_bytes, tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    if (trans != 0 && trans != 1)
        return -2;
    if (B == nullptr && nrhs > 0 && d->m > 0)
        return -3;
    if (ldb < (d->m > 1 ? d->m : 1))
        return -4;
    if (nrhs < 0)
        return -5;
    if (d->precision != TILEQR_TF32 || d->nb != 128)
        return TILEQR_ERR_UNSUPPORTED;
    size_t need = 0;
    tileqr_apply_mixed_workspace_size(d, nrhs, &need);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < need)
        return TILEQR_ERR_WORKSPACE;
    if (nrhs == 0 || d->m == 0 || d->n == 0)
        return 0;
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain, d->precision);
    const int64_t ncp = mixed_ncp(nrhs);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    double *Bt = (double *)ws;
    size_t off = align256((size_t)L.p * L.nb * ncp * sizeof(double));
    unsigned char *TN = (unsigned char *)ws + off;
    off += align256(mixed_tn_bytes(L));
    char *sched = ws + off;
    off += align256(apply_sched_bytes(L, (int)(ncp / 128)));
    int *cexp = (int *)(ws + off);
    if (cudaMemsetAsync(sched, 0, 256, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    MixedOperands M;
    int rc = mixed_operands(d, L, trans ? nullptr : TN, st, &M);
    if (rc == 0)
        rc = launch_cm2rows(B, ldb, d->m, nrhs, Bt, d->nb, d->p, ncp, st);
    if (rc == 0)
        rc = launch_rows_cexp(Bt, d->nb, d->p, ncp, cexp, st);
    if (rc == 0)
        rc = launch_apply_mixed(L, M, Bt, ncp, nrhs, cexp, sched, st, watchdog_ns_default(), trans == 0);
    if (rc == 0)
        rc = launch_rows2cm(Bt, d->nb, d->p, ncp, d->m, nrhs, B, ldb, st);
    if (rc)
        return rc;
    SchedCtrl c;
    if (cudaMemcpyAsync(&c, sched, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    return c.error;
}

extern "C" int tileqr_form_q(const tileqr_desc *d, double *Q, int64_t ldq, int64_t ncols, void *workspace,
                             size_t ws_bytes, tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    if (Q == nullptr && ncols > 0 && d->m > 0)
        return -2;
    if (ldq < (d->m > 1 ? d->m : 1))
        return -3;
    if (ncols < 0 || ncols > d->m)
        return -4;
    size_t need = 0;
    tileqr_apply_workspace_size(d, ncols, &need);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < need)
        return TILEQR_ERR_WORKSPACE;
    int rc = launch_eye(Q, ldq, d->m, ncols, (cudaStream_t)stream);
    if (rc)
        return rc;
    if (d->n == 0)
        return 0;
    return apply_impl(d, Q, ldq, ncols, workspace, ws_bytes, stream, true);
}

extern "C" int tileqr_solve_ls(const tileqr_desc *d, double *B, int64_t ldb, int64_t nrhs, void *workspace,
                               size_t ws_bytes, tileqr_stream_t stream)
{
    if (d == nullptr)
        return -1;
    if (d->m < d->n)
        return -1;
    if (B == nullptr && nrhs > 0 && d->m > 0)
        return -2;
    if (ldb < (d->m > 1 ? d->m : 1))
        return -3;
    if (nrhs < 0)
        return -4;
    size_t need = 0;
    tileqr_apply_workspace_size(d, nrhs, &need);
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < need)
        return TILEQR_ERR_WORKSPACE;
    if (nrhs == 0 || d->n == 0)
        return 0;
    const WsLayout L = make_layout(d->m, d->n, d->nb, d->ib, d->domain);
    cudaStream_t st = (cudaStream_t)stream;
    double *Bt;
    int64_t ncp;
    int *flag;
    int rc = apply_core(d, L, B, ldb, nrhs, (char *)workspace, st, &Bt, &ncp, &flag);
    if (rc)
        return rc;
    rc = launch_trsm(L, d->tiles, Bt, ncp, flag, st, false, nrhs);
    if (rc)
        return rc;
    rc = launch_rows2cm(Bt, d->nb, d->p, ncp, d->m, nrhs, B, ldb, st);
    if (rc)
        return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int h_flag = 0;
    SchedCtrl c;
    if (cudaMemcpy(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    char *sched = (char *)workspace + align256((size_t)L.p * L.nb * ncp * sizeof(double));
    if (cudaMemcpy(&c, sched, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (c.error)
        return c.error;
    if (h_flag)
        return TILEQR_ERR_SINGULAR;
    return 0;
}

extern "C" const char *tileqr_strerror(int code)
{
    if (code == 0)
        return "success";
    if (code < 0)
        return "illegal argument";
    switch (code) {
    case TILEQR_ERR_CUDA: return "CUDA runtime error";
    case TILEQR_ERR_TIMEOUT: return "scheduler watchdog: no progress";
    case TILEQR_ERR_NONFINITE: return "input holds NaN or Inf";
    case TILEQR_ERR_WORKSPACE: return "workspace too small or misaligned";
    case TILEQR_ERR_SINGULAR: return "R has an exact zero on its diagonal";
    case TILEQR_ERR_UNSUPPORTED: return "unsupported (nb, ib, precision)";
    case TILEQR_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed scratch of tileqr_factor_noalloc";
    case TILEQR_ERR_NOT_SPD: return "matrix is not positive definite";
    default: return "unknown error";
    }
}

extern "C" uint64_t tileqr_launch_count(void) { return g_launches.load(); }
extern "C" void tileqr_reset_launch_count(void) { g_launches.store(0); }
extern "C" void tileqr_set_trace(void *records, uint64_t capacity)
{
    g_trace = (unsigned long long *)records;
    g_trace_cap = records ? capacity : 0;
}

extern "C" int tileqr_trace_count(const tileqr_desc *d, tileqr_stream_t stream, uint64_t *count)
{
    if (d == nullptr)
        return -1;
    if (count == nullptr)
        return -3;
    *count = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (d->m == 0 || d->n == 0)
        return 0;
    SchedCtrl c;
    if (cudaMemcpy(&c, d->sched, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    *count = c.trace_cursor;
    return 0;
}

extern "C" void tileqr_set_profile_events(void *before, void *after)
{
    g_ev_before = (cudaEvent_t)before;
    g_ev_after = (cudaEvent_t)after;
}

// ---------------------------------------------------------------------------
// Task-graph introspection (host only): enumerate the tasks of the graph the
// kernels execute and their successors, from the same functions.

extern "C" int tileqr_task_graph(int64_t m, int64_t n, int nb, int domain, int what, int32_t *tasks,
                                 int32_t *ndeps, int64_t *succ_ptr, int64_t *succ, int64_t *ntasks,
                                 int64_t *nedges)
{
    if (m < 0)
        return -1;
    if (n < 0)
        return -2;
    if (nb < 1)
        return -3;
    if (domain < 0)
        return -4;
    if (what < 0 || what > 4)
        return -5;
    if (ntasks == nullptr)
        return -10;
    if (nedges == nullptr)
        return -11;
    if (what == 3) {
        // tiled Cholesky graph of an m x m matrix
        const int p = (int)((m + nb - 1) / nb);
        std::vector<GTask> list;
        std::map<size_t, int64_t> index;
        // every (k, i, j) with k <= j <= i is one task
        for (int k = 0; k < p; k++)
            for (int i = k; i < p; i++)
                for (int j = k; j <= i; j++) {
                    index[cg_cidx(p, k, i, j)] = (int64_t)list.size();
                    list.push_back(GTask{0, k, i, j});
                }
        std::vector<std::vector<int64_t>> out(list.size());
        int64_t ne = 0;
        for (size_t t = 0; t < list.size(); t++) {
            const GTask a = list[t];
            const int ns = cg_nsucc(p, a.k, a.i, a.j);
            for (int s2 = 0; s2 < ns; s2++) {
                const GTask b = cg_succ(p, a.k, a.i, a.j, s2);
                auto it = index.find(cg_cidx(p, b.k, b.i, b.j));
                if (it == index.end())
                    return -99;
                out[t].push_back(it->second);
                ne++;
            }
        }
        *ntasks = (int64_t)list.size();
        *nedges = ne;
        if (tasks == nullptr)
            return 0;
        if (ndeps == nullptr)
            return -7;
        if (succ_ptr == nullptr)
            return -8;
        if (succ == nullptr && ne > 0)
            return -9;
        int64_t pos = 0;
        for (size_t t = 0; t < list.size(); t++) {
            const GTask a = list[t];
            tasks[4 * t + 0] = cg_kind(a.k, a.i, a.j);
            tasks[4 * t + 1] = a.i;
            tasks[4 * t + 2] = a.j;
            tasks[4 * t + 3] = a.k;
            ndeps[t] = cg_ndeps(a.k, a.i, a.j);
            succ_ptr[t] = pos;
            for (int64_t v : out[t])
                succ[pos++] = v;
        }
        succ_ptr[list.size()] = pos;
        return 0;
    }
    const bool lu = what == 4;   // the LU graph is the flat factorization graph, LU kind names
    if (lu) {
        n = m;
        domain = 0;
        what = 0;
    }
    const int p = (int)((m + nb - 1) / nb), q = (int)((n + nb - 1) / nb);
    const TGraph G = make_graph(p, q, domain);
    // tasks in (tt, k, i, j) order; the key is the counter index
    std::vector<GTask> list;
    std::map<size_t, int64_t> index;
    for (int k = 0; k < G.steps; k++)
        for (int i = k; i < p; i++) {
            const bool head = ((i - k) % G.H) == 0;
            for (int tt = 0; tt < 2; tt++) {
                if (tt == 1 && !(head && i > k))
                    continue;
                if (what >= 1) {
                    index[g_cidx(G, tt, k, i, 0)] = (int64_t)list.size();
                    list.push_back(GTask{tt, k, i, -1});
                } else {
                    for (int j = k; j < q; j++) {
                        index[g_cidx(G, tt, k, i, j)] = (int64_t)list.size();
                        list.push_back(GTask{tt, k, i, j});
                    }
                }
            }
        }
    std::vector<std::vector<int64_t>> out(list.size());
    int64_t ne = 0;
    for (size_t t = 0; t < list.size(); t++) {
        const GTask a = list[t];
        GTask sp[2];
        std::vector<GTask> ss;
        if (what >= 1) {
            const int kind = ga_kind(G, a.tt, a.k, a.i);
            const int ns = what == 1 ? ga_specific(G, kind, a.k, a.i, sp) : ga_predecessors(G, kind, a.k, a.i, sp);
            for (int s2 = 0; s2 < ns; s2++)
                ss.push_back(GTask{sp[s2].tt, sp[s2].k, sp[s2].i, 0});
        } else {
            const int kind = g_kind(G, a.tt, a.k, a.i, a.j);
            const int fan = g_fanout(G, kind, a.k);
            for (int s2 = 0; s2 < fan; s2++)
                ss.push_back(g_fan_task(kind, a.k, a.i, s2));
            const int ns = g_specific(G, kind, a.k, a.i, a.j, sp);
            for (int s2 = 0; s2 < ns; s2++)
                ss.push_back(sp[s2]);
        }
        for (const GTask &b : ss) {
            auto it = index.find(g_cidx(G, b.tt, b.k, b.i, b.j));
            if (it == index.end())
                return -99;   // a successor outside the graph: an internal error
            out[t].push_back(it->second);
            ne++;
        }
    }
    *ntasks = (int64_t)list.size();
    *nedges = ne;
    if (tasks == nullptr)
        return 0;
    if (ndeps == nullptr)
        return -7;
    if (succ_ptr == nullptr)
        return -8;
    if (succ == nullptr && ne > 0)
        return -9;
    int64_t pos = 0;
    for (size_t t = 0; t < list.size(); t++) {
        const GTask a = list[t];
        const int kind = what >= 1 ? ga_kind(G, a.tt, a.k, a.i) : g_kind(G, a.tt, a.k, a.i, a.j);
        tasks[4 * t + 0] = lu ? lu_kind_of(kind) : kind;
        tasks[4 * t + 1] = a.i;
        tasks[4 * t + 2] = a.j;
        tasks[4 * t + 3] = a.k;
        GTask tmp[2];
        ndeps[t] = what == 1 ? ga_ndeps(kind, a.k)
                             : (what == 2 ? ga_specific(G, kind, a.k, a.i, tmp) : g_ndeps(kind, a.k));
        succ_ptr[t] = pos;
        for (int64_t v : out[t])
            succ[pos++] = v;
    }
    succ_ptr[list.size()] = pos;
    return 0;
}
