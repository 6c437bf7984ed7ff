// mixed_tile.cu -- one update task of the mixed-precision (TILEQR_TF32)
// factorization on caller tiles: the panel's full T built from its
// reflectors and T strip (mixed_build_tfull), then DLARFB or DSSRFB as three
// 3xTF32 tcgen05 products (task_update_mixed_tf), exactly the code the
// persistent kernel runs for those tasks.  It exists so that the accuracy of
// a single task can be checked against FP64 tile kernels (Sec. 3.2.1).
#include <cstring>

#include "dag.cuh"
#include "factor.h"

namespace tqr {

// Largest biased exponent of every column of the stacked pair [B; C] (the
// column scaling the factorization takes from A's columns), B optional.
__global__ void k_pair_cexp(const double *__restrict__ B, const double *__restrict__ C, int *cexp)
{
    const int c = threadIdx.x;
    unsigned int e = 0;
    for (int r = 0; r < 128; r++) {
        e = max(e, (unsigned int)(__double2hiint(C[(size_t)c * 128 + r]) >> 20) & 0x7FFu);
        if (B)
            e = max(e, (unsigned int)(__double2hiint(B[(size_t)c * 128 + r]) >> 20) & 0x7FFu);
    }
    cexp[c] = (int)e;
}

template <int S, int VK>
__global__ void __launch_bounds__(NT, 1) k_mixed_update_one(const double *V, const double *Tstrip, double *B,
                                                            double *C, unsigned char *TF, const int *cexp, int lm,
                                                            int *err)
{
    extern __shared__ double sm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[4];
    unsigned char *smb = (unsigned char *)sm;
    if ((threadIdx.x >> 5) == 0)
        tc::tmem_alloc(&s_tmem, MIX_TMEM_COLS);
    if (threadIdx.x == 0)
        for (int b = 0; b < 4; b++)
            tc::mbar_init(&s_mbar[b], 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    mixed_build_tfull<S, VK>(smb, V, Tstrip, TF);
    __syncthreads();
    uint32_t phase = 0;
    task_update_mixed_tf<S, VK>(smb, B, C, TF, TF + TF_OFF_T, cexp, lm, tmem, s_mbar, phase, err);
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        tc::tmem_dealloc(tmem, MIX_TMEM_COLS);
}

template <int S, int VK>
static int launch_mixed_update_one(const double *V, const double *T, double *B, double *C, char *ws,
                                   cudaStream_t st)
{
    constexpr size_t smem = DagCfg<128, S, true>::SMEM;
    const int rc = kernel_smem_optin((const void *)k_mixed_update_one<S, VK>, smem);
    if (rc)
        return rc;
    unsigned char *TF = (unsigned char *)ws;
    int *cexp = (int *)(ws + TF_PAIR_BYTES);
    int *err = cexp + 128;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    k_pair_cexp<<<1, 128, 0, st>>>(VK == VK_FULL ? B : nullptr, C, cexp);
    k_mixed_update_one<S, VK><<<1, NT, smem, st>>>(V, T, VK == VK_FULL ? B : nullptr, C, TF, cexp,
                                                   ceil_log2_sqrt(VK == VK_FULL ? 256 : 128), err);
    count_launch(2);
    if (cudaGetLastError() != cudaSuccess)
        return TILEQR_ERR_CUDA;
    int h_err = 0;
    if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TILEQR_ERR_CUDA;
    return h_err;
}

}  // namespace tqr

using namespace tqr;

extern "C" int tileqr_mixed_update_tile(int kind, int ib, const double *V, const double *T, double *B, double *C,
                                        void *workspace, size_t ws_bytes, tileqr_stream_t stream)
{
    if (kind != TILEQR_UPDATE_LARFB && kind != TILEQR_UPDATE_SSRFB)
        return -1;
    if (ib != 16 && ib != 32)
        return TILEQR_ERR_UNSUPPORTED;
    if (V == nullptr)
        return -3;
    if (T == nullptr)
        return -4;
    if (kind == TILEQR_UPDATE_SSRFB && (B == nullptr || ((uintptr_t)B & 15) != 0))
        return -5;
    if (C == nullptr || ((uintptr_t)C & 15) != 0)
        return -6;
    if (workspace == nullptr || ((uintptr_t)workspace & 255) != 0 || ws_bytes < TILEQR_MIXED_UPDATE_WS_BYTES)
        return TILEQR_ERR_WORKSPACE;
    static_assert(TF_PAIR_BYTES + 129 * sizeof(int) <= TILEQR_MIXED_UPDATE_WS_BYTES, "workspace of one update");
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    if (kind == TILEQR_UPDATE_LARFB)
        return ib == 16 ? launch_mixed_update_one<16, VK_UNIT>(V, T, nullptr, C, ws, st)
                        : launch_mixed_update_one<32, VK_UNIT>(V, T, nullptr, C, ws, st);
    return ib == 16 ? launch_mixed_update_one<16, VK_FULL>(V, T, B, C, ws, st)
                    : launch_mixed_update_one<32, VK_FULL>(V, T, B, C, ws, st);
}
