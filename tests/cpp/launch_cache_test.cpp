// Host-only test of the per-device launch memo (launch_cache.h) with a fake
// set-up function: several host threads ask for several (device, kernel)
// pairs at once; every pair must be set up exactly once, each caller must get
// its own pair's value, and a failed set-up must not be cached.
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "launch_cache.h"

int main()
{
    constexpr int NDEV = 3, NKER = 4, NTHREAD = 8, REPS = 200;
    static char kernels[NKER];
    tqr::LaunchCache<int> cache;
    std::atomic<int> setups[NDEV][NKER];
    for (auto &row : setups)
        for (auto &c : row)
            c = 0;
    std::atomic<int> bad{0};
    std::vector<std::thread> th;
    for (int t = 0; t < NTHREAD; t++)
        th.emplace_back([&, t]() {
            for (int r = 0; r < REPS; r++) {
                const int dev = (t + r) % NDEV, ker = (t * 7 + r) % NKER;
                int v = -1;
                const int rc = cache.get(dev, &kernels[ker], 1024, 256,
                                         [&](int &out) {
                                             setups[dev][ker]++;
                                             std::this_thread::yield();
                                             out = 100 * dev + ker;
                                             return 0;
                                         },
                                         &v);
                if (rc != 0 || v != 100 * dev + ker)
                    bad++;
            }
        });
    for (auto &x : th)
        x.join();
    int fails = bad.load();
    for (int d = 0; d < NDEV; d++)
        for (int k = 0; k < NKER; k++)
            if (setups[d][k].load() != 1) {
                std::printf("device %d kernel %d set up %d times\n", d, k, setups[d][k].load());
                fails++;
            }
    if (cache.size() != (size_t)NDEV * NKER)
        fails++;
    // a failing set-up returns its code, caches nothing, and is retried
    int calls = 0, v = 0;
    int rc = cache.get(7, &kernels[0], 1024, 256, [&](int &) { calls++; return 1001; }, &v);
    if (rc != 1001)
        fails++;
    rc = cache.get(7, &kernels[0], 1024, 256, [&](int &o) { calls++; o = 5; return 0; }, &v);
    if (rc != 0 || v != 5 || calls != 2)
        fails++;
    // the shared-memory size is part of the key
    rc = cache.get(7, &kernels[0], 2048, 256, [&](int &o) { calls++; o = 6; return 0; }, &v);
    if (rc != 0 || v != 6 || calls != 3)
        fails++;
    std::printf("%s\n", fails ? "FAIL" : "OK");
    return fails ? 1 : 0;
}
