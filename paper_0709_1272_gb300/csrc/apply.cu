// apply.cu -- Q^T B and the triangular solve of the least-squares path.
//
// Q^T B replays the transformations of Algorithm 2 on the columns of B, split
// into column chunks of APPLY_W.  For chunk c the tasks are LB(k) (DLARFB
// with V_kk, T_kk on row block k) and SB(i,k) (DSSRFB with V_ik, T_ik on row
// blocks k and i).  Their dependencies are those of the factorization
// restricted to one tile column: LB(k) <- SB(k,k-1); SB(i,k) <- (LB(k) if
// i = k+1 else SB(i-1,k)) and SB(i,k-1).  They run in one persistent kernel
// with the same counter / ready-queue scheduler, so consecutive steps k
// overlap as a wavefront.
#include "factor.h"
#include "sched.cuh"
#include "tile_f64.cuh"

namespace tqr {

struct ApplyArgs {
    const double *tiles;
    const double *T;
    double *Bt;
    int p, q, steps, nchunk;
    int64_t ncp;
};

template <int NB, int S>
__device__ __forceinline__ double *chunk_ptr(const ApplyArgs &A, int i, int cb)
{
    return A.Bt + ((size_t)i * A.ncp + (size_t)cb * APPLY_W) * NB;
}

__device__ __forceinline__ size_t apply_cnt_idx(const ApplyArgs &A, int k, int i, int cb)
{
    return ((size_t)k * A.p + i) * A.nchunk + cb;
}

template <int NB, int S>
__global__ void __launch_bounds__(NT, 1) k_apply_dag(ApplyArgs A, Queues Q)
{
    extern __shared__ double sm[];
    __shared__ unsigned long long s_code;
    __shared__ int s_cmd;
    if (blockIdx.x == 0)
        for (int cb = threadIdx.x; cb < A.nchunk; cb += NT)
            q_push(Q, 0, encode_task(0, 0, cb));
    for (;;) {
        if (threadIdx.x == 0)
            s_cmd = q_acquire(Q, s_code);
        __syncthreads();
        if (s_cmd != CMD_RUN)
            break;
        int k, i, cb;
        decode_task(s_code, k, i, cb);
        const double *Vt = A.tiles + ((size_t)k * A.p + i) * (size_t)NB * NB;
        const double *Tt = A.T + ((size_t)k * A.p + i) * (size_t)S * NB;
        if (i == k)
            task_larfb<NB, S, APPLY_W>(sm, chunk_ptr<NB, S>(A, k, cb), Vt, Tt, APPLY_W);
        else
            task_ssrfb<NB, S, APPLY_W>(sm, chunk_ptr<NB, S>(A, k, cb), chunk_ptr<NB, S>(A, i, cb), Vt, Tt,
                                       APPLY_W);
        __syncthreads();
        if (threadIdx.x == 0) {
            // successors
            if (i == k) {
                if (k + 1 < A.p)
                    q_signal(Q, apply_cnt_idx(A, k, k + 1, cb), 1 + (k > 0 ? 1 : 0), 1,
                             encode_task(k, k + 1, cb));
            } else {
                if (i + 1 < A.p)
                    q_signal(Q, apply_cnt_idx(A, k, i + 1, cb), 1 + (k > 0 ? 1 : 0), 1,
                             encode_task(k, i + 1, cb));
                if (k + 1 < A.steps) {
                    if (i == k + 1)
                        q_signal(Q, apply_cnt_idx(A, k + 1, i, cb), 1, 0, encode_task(k + 1, i, cb));
                    else
                        q_signal(Q, apply_cnt_idx(A, k + 1, i, cb), 2, 1, encode_task(k + 1, i, cb));
                }
            }
            __threadfence();
            atomicAdd(&Q.ctrl->completed, 1u);
        }
    }
}

size_t apply_sched_bytes(const WsLayout &L, int nchunk)
{
    size_t cnt = (size_t)L.steps * L.p * nchunk * sizeof(unsigned int);
    unsigned long long nlb = (unsigned long long)L.steps * nchunk, nsb = 0;
    for (int k = 0; k < L.steps; k++)
        nsb += (unsigned long long)(L.p - k - 1) * nchunk;
    return 256 + align256(cnt) + align256((nlb ? nlb : 1) * 8) + align256((nsb ? nsb : 1) * 8);
}

template <int NB, int S>
static int launch_apply_t(const WsLayout &L, const double *tiles, const double *T, double *Bt,
                          int64_t ncp, char *sched, cudaStream_t st, unsigned long long watchdog_ns)
{
    constexpr size_t smem = F64Cfg<NB, S, APPLY_W>::SMEM;
    static int grid_max = 0;
    if (grid_max == 0) {
        cudaFuncSetAttribute(k_apply_dag<NB, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_dag<NB, S>, NT, smem);
        if (per_sm < 1)
            return TILEQR_ERR_CUDA;
        grid_max = nsm * per_sm;
    }
    ApplyArgs A;
    A.tiles = tiles;
    A.T = T;
    A.Bt = Bt;
    A.p = L.p;
    A.q = L.q;
    A.steps = L.steps;
    A.ncp = ncp;
    A.nchunk = (int)(ncp / APPLY_W);
    const size_t cnt_bytes = align256((size_t)L.steps * L.p * A.nchunk * sizeof(unsigned int));
    unsigned long long nlb = (unsigned long long)L.steps * A.nchunk, nsb = 0;
    for (int k = 0; k < L.steps; k++)
        nsb += (unsigned long long)(L.p - k - 1) * A.nchunk;
    Queues Q;
    Q.ctrl = (SchedCtrl *)sched;
    Q.cnt = (unsigned int *)(sched + 256);
    Q.slot[0] = (unsigned long long *)(sched + 256 + cnt_bytes);
    Q.slot[1] = (unsigned long long *)(sched + 256 + cnt_bytes + align256((nlb ? nlb : 1) * 8));
    Q.slot[2] = Q.slot[3] = nullptr;
    Q.cap[0] = (unsigned int)nlb;
    Q.cap[1] = (unsigned int)nsb;
    Q.cap[2] = Q.cap[3] = 0;
    Q.total = (unsigned int)(nlb + nsb);
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
    k_apply_dag<NB, S><<<grid, NT, smem, st>>>(A, Q);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : TILEQR_ERR_CUDA;
}

int launch_apply(const WsLayout &L, const double *tiles, const double *T, double *Bt, int64_t ncp,
                 char *sched, cudaStream_t st, unsigned long long watchdog_ns)
{
#define TQR_CASE(NB_, S_)                                                                        \
    if (L.nb == NB_ && L.ib == S_)                                                               \
        return launch_apply_t<NB_, S_>(L, tiles, T, Bt, ncp, sched, st, watchdog_ns);
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
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_trsm_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 33 * 8);
        cudaFuncSetAttribute(k_trsm_update, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 33 * 8);
        attr = true;
    }
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
