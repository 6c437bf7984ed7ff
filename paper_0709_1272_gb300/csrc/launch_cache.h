// launch_cache.h -- a per-device, thread-safe memo for the one-time set-up of
// a kernel launch (the dynamic shared-memory opt-in and the persistent grid
// size).  Both are properties of a (device, kernel) pair: the opt-in applies
// to the device that is current when it is made, and the grid depends on that
// device's SM count.  Plain C++ (no CUDA types), so it is unit-tested on the
// host with a fake set-up function.
#pragma once
#include <cstddef>
#include <map>
#include <mutex>
#include <tuple>

namespace tqr {

template <typename V>
class LaunchCache {
  public:
    // Returns the cached value of (dev, key, smem, threads) in *out, running
    // setup(V &) to produce it on the first call for that key.  A set-up that
    // fails (non-zero return) caches nothing and is tried again on the next
    // call.  The mutex is held during set-up, so each key is set up once even
    // when several host threads ask at the same time.
    template <typename F>
    int get(int dev, const void *key, size_t smem, int threads, F &&setup, V *out)
    {
        std::lock_guard<std::mutex> lock(mu_);
        const Key k{dev, key, smem, threads};
        auto it = map_.find(k);
        if (it != map_.end()) {
            *out = it->second;
            return 0;
        }
        V v{};
        const int rc = setup(v);
        if (rc != 0)
            return rc;
        map_.emplace(k, v);
        *out = v;
        return 0;
    }
    size_t size()
    {
        std::lock_guard<std::mutex> lock(mu_);
        return map_.size();
    }

  private:
    using Key = std::tuple<int, const void *, size_t, int>;
    std::mutex mu_;
    std::map<Key, V> map_;
};

}  // namespace tqr
