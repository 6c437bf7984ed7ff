// launch_cfg.cu -- per-device launch set-up shared by every launch site of
// the library: the dynamic shared-memory opt-in of a kernel and the size of
// its persistent grid (SMs x resident CTAs), made once per (device, kernel)
// under a mutex.  The library may be driven from several host threads and on
// several devices of one process; each device gets its own opt-in (an
// attribute set while another device was current does not carry over).
#include "factor.h"
#include "launch_cache.h"

namespace tqr {

static int current_device(int *dev)
{
    if (cudaGetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return TILEQR_ERR_CUDA;
    }
    return 0;
}

int kernel_grid(const void *func, int threads, size_t smem, int *grid)
{
    static LaunchCache<int> cache;
    int dev = 0;
    int rc = current_device(&dev);
    if (rc)
        return rc;
    return cache.get(
        dev, func, smem, threads,
        [&](int &g) {
            int nsm = 0, per_sm = 0;
            if (smem > 0 &&
                cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                return (int)TILEQR_ERR_CUDA;
            }
            if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess ||
                nsm < 1 || per_sm < 1) {
                cudaGetLastError();
                return (int)TILEQR_ERR_CUDA;
            }
            g = nsm * per_sm;
            return 0;
        },
        grid);
}

int kernel_smem_optin(const void *func, size_t smem)
{
    static LaunchCache<char> cache;
    int dev = 0;
    int rc = current_device(&dev);
    if (rc)
        return rc;
    char done = 0;
    return cache.get(
        dev, func, smem, 0,
        [&](char &v) {
            if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                return (int)TILEQR_ERR_CUDA;
            }
            v = 1;
            return 0;
        },
        &done);
}

int device_sm_count(int *nsm)
{
    static LaunchCache<int> cache;
    int dev = 0;
    int rc = current_device(&dev);
    if (rc)
        return rc;
    return cache.get(
        dev, nullptr, 0, 0,
        [&](int &v) {
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
                cudaGetLastError();
                return (int)TILEQR_ERR_CUDA;
            }
            return 0;
        },
        nsm);
}

}  // namespace tqr
