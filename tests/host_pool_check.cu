// Host-only check of the context's worker pool (HostPool, no GPU): every
// index of every run() is handled exactly once, by the workers and the
// calling thread together, over many runs of sizes from 0 to 100000 in a
// row; run() returns only when all of them are done.  Prints "ok".
#include <atomic>
#include <cstdio>
#include <vector>

#include "gace_host.h"

int main() {
    HostPool pool;
    const uint32_t sizes[] = {0, 1, 2, 3, 7, 63, 64, 65, 1000, 4096, 100000};
    uint64_t handled = 0;
    for (int round = 0; round < 300; ++round) {
        const uint32_t n = sizes[round % (sizeof(sizes) / sizeof(sizes[0]))];
        std::vector<std::atomic<uint32_t>> seen(n);
        for (auto& s : seen) s.store(0);
        pool.run(n, [&](uint32_t i) { seen[i].fetch_add(1, std::memory_order_relaxed); });
        for (uint32_t i = 0; i < n; ++i) {
            if (seen[i].load() != 1) {
                printf("round %d, n %u: index %u handled %u times\n", round, n, i, seen[i].load());
                return 1;
            }
        }
        handled += n;
    }
    printf("ok %llu\n", (unsigned long long)handled);
    return 0;
}
