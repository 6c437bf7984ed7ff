// noalloc.cu -- tileqr_factor_noalloc: the factorization for callers that
// cannot allocate device memory at all.
//
// Who needs it: services that reserve their whole device-memory budget at
// start-up and forbid any allocation afterwards (cudaMalloc can synchronise
// the device and can fail long after start-up), and code embedded in a host
// framework that owns every device allocation through its own allocator and
// gives plug-ins only the buffers they read and write.  Such a caller owns
// the input matrix and the output tiles, but has nothing to hand over for the
// scheduler's scratch (dependency counters and ready queues).
//
// Here that scratch lives in one file-scope device array of a fixed size,
// created when the library's module is loaded on a device and held by every
// device that loads the library until the process exits.  Host code cannot
// use the array's name as a device address (it is a host-side stand-in), so
// the device address is looked up once per device with cudaGetSymbolAddress.
#include <cstring>
#include <mutex>

#include "factor.h"

namespace tqr {

// Upper bound of the scheduler scratch of one call: the control block, one
// counter per task and the four ready queues.  4 MiB covers tile grids up to
// about 80 x 80 (e.g. 10240 x 10240 at nb 128, 20480 x 20480 at nb 256).
constexpr size_t NOALLOC_SCRATCH_BYTES = 4u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[NOALLOC_MAX_DEVICES];

// Device address of the scratch on the current device (looked up on the
// first call per device, with that device current).
static int noalloc_scratch(char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return TILEQR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_addr[dev] == nullptr) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr)
            return TILEQR_ERR_CUDA;
        g_noalloc_addr[dev] = ptr;
    }
    *out = (char *)g_noalloc_addr[dev];
    return 0;
}

}  // namespace tqr

using namespace tqr;

extern "C" int tileqr_factor_noalloc(int64_t m, int64_t n, const double *A, int64_t lda, int nb, int ib,
                                     double *tiles, size_t tiles_bytes, double *T, size_t T_bytes,
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
    if (nb < 1)
        return -5;
    if (ib < 1 || ib > nb || nb % ib != 0)
        return -6;
    if (out == nullptr)
        return -12;
    if ((m + nb - 1) / nb >= (1 << 21) || (n + nb - 1) / nb >= (1 << 21))
        return -1;
    if (!factor_supported(nb, ib))
        return TILEQR_ERR_UNSUPPORTED;
    const WsLayout L = make_layout(m, n, nb, ib);
    // the size limit is decided from the shape alone, before any device work
    const size_t sched_bytes = L.end - L.off_ctrl;
    if (sched_bytes > NOALLOC_SCRATCH_BYTES)
        return TILEQR_ERR_SCRATCH_LIMIT;
    const size_t need_tiles = (size_t)L.p * L.q * nb * nb * sizeof(double);
    const size_t need_T = (size_t)L.p * L.q * ib * nb * sizeof(double);
    if (m > 0 && n > 0) {
        if (tiles == nullptr || tiles_bytes < need_tiles)
            return -7;
        if (T == nullptr || T_bytes < need_T)
            return -9;
    }
    char *sched = nullptr;
    int rc = noalloc_scratch(&sched);
    if (rc)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;

    std::memset(out, 0, sizeof(*out));
    out->m = m;
    out->n = n;
    out->nb = nb;
    out->ib = ib;
    out->p = L.p;
    out->q = L.q;
    out->precision = TILEQR_FP64;
    out->schedule = TILEQR_SCHED_DAG;
    out->tiles = tiles;
    out->T = T;
    out->sched = sched;
    out->sched_bytes = sched_bytes;
    out->workspace = nullptr;
    out->workspace_bytes = 0;

    // every call shares the scratch: clear the counters, queues and status
    // left behind by the previous call before this one starts
    if (cudaMemsetAsync(sched, 0, sched_bytes, st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    if (m == 0 || n == 0)
        return 0;
    rc = launch_cm2tile(A, lda, m, n, tiles, nb, L.p, L.q, (SchedCtrl *)sched, nullptr, st);
    if (rc)
        return rc;
    return launch_factor_dag_at(L, tiles, T, sched, st, watchdog_ns_default());
}
