// launch_cfg.cu -- per-device launch set-up shared by every launch site of
// the library: the dynamic shared-memory opt-in of a kernel and the size of
// its persistent grid (SMs x resident CTAs), made once per (device, kernel)
// under a mutex.  The library may be driven from several host threads and on
// several devices of one process; each device gets its own opt-in (an
// attribute set while another device was current does not carry over).
#include "factor.h"
#include "launch_cache.h"

#include <map>
#include <mutex>
#include <utility>

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
    if ((rc = kernel_smem_optin(func, smem)) != 0)
        return rc;
    return cache.get(
        dev, func, smem, threads,
        [&](int &g) {
            int nsm = 0, per_sm = 0;
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

// The opt-in only ever raises a kernel's dynamic shared-memory limit: sizes
// within the default 48 KB need none, and a kernel launched with several
// sizes (a tile size per call) keeps the largest opt-in made on the device,
// so a later call with a smaller size cannot lower the limit under an
// earlier one.
int kernel_smem_optin(const void *func, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> raised;   // largest opt-in per (device, kernel)
    if (smem <= 48 * 1024)
        return 0;
    int dev = 0;
    const int rc = current_device(&dev);
    if (rc)
        return rc;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = raised[std::make_pair(dev, func)];
    if (smem <= cur)
        return 0;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return TILEQR_ERR_CUDA;
    }
    cur = smem;
    return 0;
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
