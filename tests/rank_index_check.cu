// Host-only check of a rank-coded column's search structures (no GPU): for
// random endpoint sets of 32- and 64-bit keys (spread, crowded, spanning the
// whole domain, with the smallest and largest keys), the planner's level-order
// search tree and its bucket index are built (build_rank_tree,
// build_rank_buckets under each rank_search setting) and searched the way the
// rank pass reads them (RankArgs), and every probe key's rank must be the
// number of endpoints <= the key.  Prints "ok" or the first mismatch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <set>
#include <vector>

#include "gace_host.h"

namespace {

// The rank pass's tree descent: one compare per level from node 1.
uint32_t tree_rank(const RankCode& rc, uint64_t k) {
    const bool is64 = rc.dtype == GACE_I64;
    uint32_t n = 1;
    for (uint32_t d = 0; d < rc.levels; ++d) {
        const uint64_t e = is64 ? (static_cast<uint64_t>(rc.tree[2 * (n - 1) + 1]) << 32) | rc.tree[2 * (n - 1)]
                                : rc.tree[n - 1];
        n = 2 * n + (k >= e ? 1u : 0u);
    }
    const uint32_t r = n - (1u << rc.levels);
    const uint32_t m = static_cast<uint32_t>(rc.keys.size());
    return r < m ? r : m;
}

// The rank pass's bucket-index search: the key's bucket gives the first
// candidate endpoint, `steps` halvings over the sorted endpoints the rank.
uint32_t bucket_rank(const RankCode& rc, uint64_t k) {
    const bool is64 = rc.dtype == GACE_I64;
    const uint64_t d = k >= rc.bbase ? k - rc.bbase : 0;
    const int top = d ? 63 - __builtin_clzll(d) : -1;  // index of d's highest set bit
    const int s = std::max(static_cast<int>(rc.bsmin), top - static_cast<int>(rc.bmbits));
    const uint64_t b = (static_cast<uint64_t>(s - static_cast<int>(rc.bsmin)) << rc.bmbits) + (s < 64 ? d >> s : 0);
    const uint16_t* start = reinterpret_cast<const uint16_t*>(rc.tree.data());
    const uint32_t* ends = rc.tree.data() + rank_start_words(rc.bnb);
    uint32_t n = start[b < rc.bnb ? b : rc.bnb - 1];
    for (uint32_t h = (1u << rc.bsteps) >> 1; h; h >>= 1) {
        const uint32_t i = n + h - 1;
        const uint64_t e = is64 ? (static_cast<uint64_t>(ends[2 * i + 1]) << 32) | ends[2 * i] : ends[i];
        n += k >= e ? h : 0u;
    }
    const uint32_t m = static_cast<uint32_t>(rc.keys.size());
    return n < m ? n : m;
}

}  // namespace

int main() {
    std::mt19937_64 rng(12345);
    int checked = 0;
    for (int trial = 0; trial < 240; ++trial) {
        const bool is64 = trial % 2 == 1;
        const uint64_t kmax = is64 ? ~0ull : 0xFFFFFFFFull;
        const int shape = (trial / 2) % 4;
        const uint32_t sizes[] = {1, 2, 3, 7, 100, 700, 2047};
        const uint32_t m = sizes[(trial / 8) % 7];
        std::set<uint64_t> ks;
        const uint64_t mid = is64 ? (1ull << 63) : (1ull << 31);
        while (ks.size() < m) {
            uint64_t k;
            if (shape == 0) {
                k = rng() & kmax;  // spread over the domain
            } else if (shape == 1) {
                // Zipf-like: crowded just above the order-preserving zero
                const double u = (static_cast<double>(rng() >> 11) + 0.5) / 9007199254740992.0;
                k = mid + static_cast<uint64_t>(std::min(1e15, std::pow(u, -5.0)));
            } else if (shape == 2) {
                k = mid - 64 + rng() % (2 * m + 128);  // a narrow range
            } else {
                k = ks.empty() ? 0 : (ks.size() == 1 ? kmax : (rng() & kmax));  // both ends of the domain
            }
            if (k <= kmax) ks.insert(k);
        }
        std::vector<uint64_t> keys(ks.begin(), ks.end());
        std::vector<uint64_t> probes = {0, kmax, keys.front(), keys.back()};
        for (uint64_t k : keys) {
            if (k) probes.push_back(k - 1);
            if (k < kmax) probes.push_back(k + 1);
            probes.push_back(k);
        }
        for (int i = 0; i < 300; ++i) probes.push_back(rng() & kmax);
        for (int i = 0; i < 300; ++i)
            probes.push_back(keys.front() + (keys.back() > keys.front() ? rng() % (keys.back() - keys.front()) : 0));
        for (uint32_t search = 0; search <= 2; ++search) {
            RankCode rc;
            rc.keys = keys;
            rc.dtype = is64 ? GACE_I64 : GACE_I32;
            build_rank_tree(rc);
            build_rank_buckets(rc, search);
            if (search == 2 && rc.levels != 0) {
                printf("trial %d: rank_search 2 kept the search tree\n", trial);
                return 1;
            }
            for (uint64_t k : probes) {
                const uint32_t want = static_cast<uint32_t>(std::upper_bound(keys.begin(), keys.end(), k) - keys.begin());
                const uint32_t got = rc.levels ? tree_rank(rc, k) : bucket_rank(rc, k);
                if (got != want) {
                    printf("trial %d search %u (%s, m %u): key %llu rank %u, expected %u\n", trial, search,
                           rc.levels ? "tree" : "buckets", m, (unsigned long long)k, got, want);
                    return 1;
                }
                ++checked;
            }
            // the int64 endpoint pairs of a bucket index start 8-byte aligned
            if (!rc.levels && (rank_start_words(rc.bnb) % 2) != 0) {
                printf("trial %d: endpoints not 8-byte aligned\n", trial);
                return 1;
            }
        }
    }
    printf("ok %d\n", checked);
    return 0;
}
