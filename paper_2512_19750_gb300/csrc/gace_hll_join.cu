// gace_hll_join.cu -- K4 HyperLogLog registers and K5/K6 join-cardinality
// kernels.
//
// NDV is the statistic behind the drift signal D of the paper (Section III-C,
// Eq. 1); the sketch is HyperLogLog (Flajolet, Fusy, Gandouet & Meunier,
// AofA 2007) with a 64-bit splitmix64-based hash.  Each CTA keeps a private
// copy of the 2^p registers in shared memory, 32-bit up to p = 14 (raised by
// one atomicMax) and one byte each above (raised by a compare-and-swap on the
// containing word), updated only when a row's rank would raise its register;
// the copy is then merged into 32-bit global registers with atomicMax, again
// only where it would raise them.
//
// Join cardinality (the join-correlation failures the method targets,
// Section IV-F) is the dot product of filtered key-frequency histograms.
// Filtered rows are histogrammed with global atomics (warp-aggregated with
// __match_any_sync on skewed fact keys); the gather form sums h_D[fact.key]
// over filtered fact rows, reaching the same integer without a fact
// histogram: the dimension histogram (tens of MB) stays resident in the
// 129 MB L2 while the fact table streams from HBM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"
#include "gace_launch.cuh"
#include "gace_side_dev.cuh"

namespace gace {
namespace {

using namespace dev;
using namespace side_dev;

constexpr int kHllThreads = 1024;
constexpr int kJoinThreads = 256;

// Groups of four rows a thread takes per iteration (their loads issued together).
#ifndef GACE_HLL_UNROLL
#define GACE_HLL_UNROLL 1
#endif

template <int REGS, int DT>
__global__ void __launch_bounds__(kHllThreads, 2) k_hll(const __grid_constant__ HllArgs A) {
    extern __shared__ uint32_t sregs[];
    const uint32_t m = 1u << A.p;
    if (REGS != kHllGlobal) {
        hll_clear<REGS>(sregs, m, threadIdx.x, kHllThreads);
        __syncthreads();
    }
    hll_groups<REGS, DT, GACE_HLL_UNROLL>(A, sregs, static_cast<uint64_t>(blockIdx.x) * kHllThreads + threadIdx.x,
                                          (A.nrows + 3) / 4, static_cast<uint64_t>(gridDim.x) * kHllThreads);
    if (REGS != kHllGlobal) {
        __syncthreads();
        hll_merge<REGS>(A, sregs, m, threadIdx.x, kHllThreads);
    }
}

// h[key] += 1 over a small key domain: a shared-memory histogram per CTA
// (equal keys of a warp combined first), then its nonzero bins into h.
__global__ void __launch_bounds__(kHistThreads, 1)
    k_hist_smem(const __grid_constant__ SideArgs A, uint32_t* hist, int strict) {
    extern __shared__ __align__(16) uint32_t shist[];
    __shared__ unsigned long long scratch[kHistThreads / 32];
    const uint32_t K = static_cast<uint32_t>(A.domain);
    const int lane = threadIdx.x & 31;
    for (uint32_t i = threadIdx.x; i < K; i += kHistThreads) shist[i] = 0;
    __syncthreads();
    unsigned long long npass = 0, acc = 0;
    side_groups<0, kSmemHistAgg>(A, shist, strict, nullptr, 0, 0, nullptr,
                         static_cast<uint64_t>(blockIdx.x) * kHistThreads + (threadIdx.x - lane), (A.nrows + 3) / 4,
                         static_cast<uint64_t>(gridDim.x) * kHistThreads, npass, acc);
    __syncthreads();
    hist_merge(shist, hist, K, threadIdx.x, kHistThreads);
    const unsigned long long tp = block_sum_u64<kHistThreads / 32>(npass, scratch);
    if (threadIdx.x == 0 && tp) atomicAdd(A.pass_count, tp);
}

// The same over tiles staged in shared memory: the stage buffers, then the
// histogram; 32 warps take a tile 128 rows each.
template <bool KEY64>
__global__ void __launch_bounds__(kHistThreads, 1)
    k_hist_smem_staged(const __grid_constant__ SideArgs A, uint32_t* hist, int strict) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long scratch[kHistThreads / 32];
    uint32_t* shist = reinterpret_cast<uint32_t*>(smem + A.smem_bytes);
    const uint32_t K = static_cast<uint32_t>(A.domain);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t i = tid; i < K; i += kHistThreads) shist[i] = 0;
    __syncthreads();
    unsigned long long npass = 0, acc = 0;
    if (!side_tiles<0, kSmemHistAgg, KEY64, 1, kHistThreads / 32>(A, reinterpret_cast<uint64_t*>(smem),
                                                                  smem + kSideStageOff, tid, lane, warp, blockIdx.x,
                                                                  A.ntiles, gridDim.x, shist, strict, nullptr, 0, 0,
                                                                  nullptr, npass, acc))
        return;  // a pipeline wait gave up: the status says so
    __syncthreads();
    hist_merge(shist, hist, K, tid, kHistThreads);
    const unsigned long long tp = block_sum_u64<kHistThreads / 32>(npass, scratch);
    if (tid == 0 && tp) atomicAdd(A.pass_count, tp);
}

#ifndef GACE_GATHER_GROUPS
#define GACE_GATHER_GROUPS 1
#endif
// Groups of four rows per thread and iteration: gathers (a weight load that
// waits on its key) run best one group at a time with more threads resident;
// histogram updates two at a time.
template <int MODE>
__host__ __device__ constexpr int side_unroll() { return (MODE == 1 || MODE == 2) ? GACE_GATHER_GROUPS : 2; }

#ifndef GACE_GATHER_CTAS
#define GACE_GATHER_CTAS 4
#endif
template <int MODE, bool AGG>
__global__ void __launch_bounds__(kJoinThreads, (MODE == 1 || MODE == 2) ? GACE_GATHER_CTAS : 4)
    k_side(const __grid_constant__ SideArgs A, uint32_t* hist, int strict, const void* weight,
           unsigned long long* out_sum, uint32_t fk2_slot, uint64_t domain2,
           unsigned long long* w64) {
    __shared__ unsigned long long scratch[kJoinThreads / 32];
    const int lane = threadIdx.x & 31;
    unsigned long long npass = 0, acc = 0;
    // warp-uniform trip count so that every lane reaches the warp collectives
    side_groups<MODE, AGG, side_unroll<MODE>()>(A, hist, strict, weight, fk2_slot, domain2, w64,
                           static_cast<uint64_t>(blockIdx.x) * kJoinThreads + (threadIdx.x - lane),
                           (A.nrows + 3) / 4, static_cast<uint64_t>(gridDim.x) * kJoinThreads, npass, acc);
    const unsigned long long tp = block_sum_u64<kJoinThreads / 32>(npass, scratch);
    if (threadIdx.x == 0 && tp) atomicAdd(A.pass_count, tp);
    if (MODE == 1 || MODE == 2) {
        const unsigned long long ta = block_sum_u64<kJoinThreads / 32>(acc, scratch);
        if (threadIdx.x == 0 && ta) atomicAdd(out_sum, ta);
    }
}

// The side modes over tiles staged in shared memory by the bulk-copy pipeline
// (tables whose referenced columns are 16-byte aligned and narrow enough for
// two stages); three CTAs per SM.
template <int MODE, bool AGG, bool KEY64, int NQ>
__global__ void __launch_bounds__(kJoinThreads, 3)
    k_side_staged(const __grid_constant__ SideArgs A, uint32_t* hist, int strict, const void* weight,
                  unsigned long long* out_sum, uint32_t fk2_slot, uint64_t domain2, unsigned long long* w64) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long scratch[kJoinThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long npass = 0, acc = 0;
    // skewed keys into a global histogram: a hot-key cache after the stages
    uint32_t* hot = nullptr;
    if (MODE == 0 && AGG && kHotCache && A.domain <= 0xFFFFFFFFull) {
        hot = reinterpret_cast<uint32_t*>(smem + A.smem_bytes);
        hot_init(hot, kHotLog, tid, kJoinThreads);
    }
    if (!side_tiles<MODE, AGG, KEY64, NQ>(A, reinterpret_cast<uint64_t*>(smem), smem + kSideStageOff, tid, lane, warp,
                               blockIdx.x, A.ntiles, gridDim.x, hist, strict, weight, fk2_slot, domain2, w64, npass,
                               acc, hot, kHotLog))
        return;  // a pipeline wait gave up: the status says so
    if (hot) {
        __syncthreads();
        hot_flush(hot, kHotLog, hist, tid, kJoinThreads);
    }
    const unsigned long long tp = block_sum_u64<kJoinThreads / 32>(npass, scratch);
    if (threadIdx.x == 0 && tp) atomicAdd(A.pass_count, tp);
    if (MODE == 1 || MODE == 2) {
        const unsigned long long ta = block_sum_u64<kJoinThreads / 32>(acc, scratch);
        if (threadIdx.x == 0 && ta) atomicAdd(out_sum, ta);
    }
}

template <bool B64>
__global__ void __launch_bounds__(kJoinThreads)
    k_dot(const uint32_t* a, const void* b, uint64_t n, unsigned long long* sum) {
    __shared__ unsigned long long scratch[kJoinThreads / 32];
    const unsigned long long acc = dot_range<B64>(a, b, static_cast<uint64_t>(blockIdx.x) * kJoinThreads + threadIdx.x,
                                                  n, static_cast<uint64_t>(gridDim.x) * kJoinThreads);
    const unsigned long long t = block_sum_u64<kJoinThreads / 32>(acc, scratch);
    if (threadIdx.x == 0 && t) atomicAdd(sum, t);
}

template <bool B64>
__global__ void __launch_bounds__(kJoinThreads)
    k_max(const void* a, uint64_t n, unsigned long long* mx) {
    const unsigned long long best = warp_max_u64(max_range<B64>(
        a, static_cast<uint64_t>(blockIdx.x) * kJoinThreads + threadIdx.x, n,
        static_cast<uint64_t>(gridDim.x) * kJoinThreads));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(mx, best);
}

int grid_for(uint64_t units, int per_cta, int sms, int ctas_per_sm) {
    const uint64_t need = (units + per_cta - 1) / per_cta;
    const uint64_t cap = static_cast<uint64_t>(sms) * ctas_per_sm;
    return static_cast<int>(need < 1 ? 1 : (need < cap ? need : cap));
}

}  // namespace

template <int REGS, int DT>
static cudaError_t hll_launch_t(const HllArgs& a, int sms, cudaStream_t s) {
    const uint64_t groups = (a.nrows + 3) / 4;
    const uint32_t smem = REGS == kHllWords ? (4u << a.p) : REGS == kHllBytes ? (1u << a.p) : 0u;
    cudaError_t e = smem_allow_max<k_hll<REGS, DT>>();
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hll<REGS, DT>, kHllThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    k_hll<REGS, DT><<<grid_for(groups, kHllThreads, sms, occ), kHllThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t hll_launch_dt(const HllArgs& a, int sms, cudaStream_t s) {
    // 32-bit registers in shared memory up to p = 14 (64 KB: two CTAs per
    // SM), one-byte registers up to p = 17 (128 KB), else straight to global
    if (a.p <= kHllWordsMaxP) return hll_launch_t<kHllWords, DT>(a, sms, s);
    if (a.p <= 17) return hll_launch_t<kHllBytes, DT>(a, sms, s);
    return hll_launch_t<kHllGlobal, DT>(a, sms, s);
}

cudaError_t hll_launch(const HllArgs& a, int sms, cudaStream_t s) {
    switch (a.dtype) {
        case 0: return hll_launch_dt<0>(a, sms, s);
        case 1: return hll_launch_dt<1>(a, sms, s);
        default: return hll_launch_dt<2>(a, sms, s);
    }
}

// A staged side launch: grid = min(tiles, SMs x resident CTAs).
template <int MODE, bool AGG, bool KEY64, int NQ>
static cudaError_t staged_launch_t(const SideArgs& a, int sms, cudaStream_t s, uint32_t* hist, int strict,
                                 const void* weight, unsigned long long* out_sum, uint32_t fk2_slot, uint64_t domain2,
                                 unsigned long long* w64) {
    const uint32_t smem = a.smem_bytes + (MODE == 0 && AGG && kHotCache ? 8u << kHotLog : 0u);
    cudaError_t e = smem_allow_max<k_side_staged<MODE, AGG, KEY64, NQ>>();
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_side_staged<MODE, AGG, KEY64, NQ>, kJoinThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const uint64_t cap = static_cast<uint64_t>(sms) * occ;
    const int grid = static_cast<int>(a.ntiles < cap ? (a.ntiles ? a.ntiles : 1) : cap);
    k_side_staged<MODE, AGG, KEY64, NQ><<<grid, kJoinThreads, smem, s>>>(a, hist, strict, weight, out_sum, fk2_slot,
                                                                       domain2, w64);
    return cudaGetLastError();
}

template <int MODE, bool AGG>
static cudaError_t staged_launch(const SideArgs& a, int sms, cudaStream_t s, uint32_t* hist, int strict,
                                 const void* weight, unsigned long long* out_sum, uint32_t fk2_slot, uint64_t domain2,
                                 unsigned long long* w64) {
    // gathers take 16 rows per lane when a tile holds such a step for every warp
    constexpr int NQ = side_nq<MODE>();
    if (NQ > 2 && a.tile_rows % (128u * NQ * kSideWarps) != 0) {
        if (a.slot_dtype[a.key_slot] == 1)
            return staged_launch_t<MODE, AGG, true, 2>(a, sms, s, hist, strict, weight, out_sum, fk2_slot, domain2, w64);
        return staged_launch_t<MODE, AGG, false, 2>(a, sms, s, hist, strict, weight, out_sum, fk2_slot, domain2, w64);
    }
    if (a.slot_dtype[a.key_slot] == 1)
        return staged_launch_t<MODE, AGG, true, NQ>(a, sms, s, hist, strict, weight, out_sum, fk2_slot, domain2, w64);
    return staged_launch_t<MODE, AGG, false, NQ>(a, sms, s, hist, strict, weight, out_sum, fk2_slot, domain2, w64);
}

cudaError_t hist_launch(const SideArgs& a, uint32_t* hist, int strict, int aggregate, int sms,
                        cudaStream_t s) {
    // small domains over enough rows (each CTA at least 4 rows per bin, so
    // that its merge stays a small part of its work): shared-memory histograms
#ifndef GACE_HIST_STAGED
#define GACE_HIST_STAGED 1
#endif
    if (GACE_HIST_STAGED && aggregate && a.domain <= kSmemHistMax && a.nrows >= 4 * a.domain * 16 &&
        a.stage_bytes && a.tile_rows % (128u * (kHistThreads / 32)) == 0) {
        const uint32_t smem = a.smem_bytes + static_cast<uint32_t>(a.domain) * 4u;
        const bool key64 = a.slot_dtype[a.key_slot] == 1;
        auto kern = key64 ? k_hist_smem_staged<true> : k_hist_smem_staged<false>;
        cudaError_t e = key64 ? smem_allow_max<k_hist_smem_staged<true>>() : smem_allow_max<k_hist_smem_staged<false>>();
        if (e != cudaSuccess) return e;
        uint64_t want = a.nrows / (4 * a.domain);
        if (want > a.ntiles) want = a.ntiles;
        const int grid = static_cast<int>(want < static_cast<uint64_t>(sms) ? (want ? want : 1) : sms);
        kern<<<grid, kHistThreads, smem, s>>>(a, hist, strict);
        return cudaGetLastError();
    }
    if (aggregate && a.domain <= kSmemHistMax && a.nrows >= 4 * a.domain * 16) {
        const uint32_t smem = static_cast<uint32_t>(a.domain) * 4u;
        cudaError_t e = smem_allow_max<k_hist_smem>();
        if (e != cudaSuccess) return e;
        const uint64_t want = a.nrows / (4 * a.domain);
        const int grid = static_cast<int>(want < static_cast<uint64_t>(sms) ? want : sms);
        k_hist_smem<<<grid, kHistThreads, smem, s>>>(a, hist, strict);
        return cudaGetLastError();
    }
    if (a.stage_bytes)
        return aggregate ? staged_launch<0, true>(a, sms, s, hist, strict, nullptr, nullptr, 0, 0, nullptr)
                         : staged_launch<0, false>(a, sms, s, hist, strict, nullptr, nullptr, 0, 0, nullptr);
    const int grid = grid_for((a.nrows + 3) / 4, kJoinThreads, sms, 8);
    if (aggregate)
        k_side<0, true><<<grid, kJoinThreads, 0, s>>>(a, hist, strict, nullptr, nullptr, 0, 0, nullptr);
    else
        k_side<0, false><<<grid, kJoinThreads, 0, s>>>(a, hist, strict, nullptr, nullptr, 0, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t chain_weight_launch(const SideArgs& a, uint32_t fk2_slot, uint64_t domain2,
                                const uint32_t* h2, unsigned long long* w, int sms,
                                cudaStream_t s) {
    if (a.stage_bytes) return staged_launch<3, false>(a, sms, s, nullptr, 1, h2, nullptr, fk2_slot, domain2, w);
    const int grid = grid_for((a.nrows + 3) / 4, kJoinThreads, sms, 8);
    k_side<3, false><<<grid, kJoinThreads, 0, s>>>(a, nullptr, 1, h2, nullptr, fk2_slot, domain2, w);
    return cudaGetLastError();
}

cudaError_t gather_launch(const SideArgs& a, const void* weight, int weight64,
                          unsigned long long* sum, int sms, cudaStream_t s) {
    if (a.stage_bytes)
        return weight64 ? staged_launch<2, false>(a, sms, s, nullptr, 0, weight, sum, 0, 0, nullptr)
                        : staged_launch<1, false>(a, sms, s, nullptr, 0, weight, sum, 0, 0, nullptr);
    const int grid = grid_for((a.nrows + 3) / 4, kJoinThreads, sms, 8);
    if (weight64)
        k_side<2, false><<<grid, kJoinThreads, 0, s>>>(a, nullptr, 0, weight, sum, 0, 0, nullptr);
    else
        k_side<1, false><<<grid, kJoinThreads, 0, s>>>(a, nullptr, 0, weight, sum, 0, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t dot_launch(const uint32_t* a, const void* b, int b64, uint64_t n,
                       unsigned long long* sum, int sms, cudaStream_t s) {
    const int grid = grid_for(n, kJoinThreads, sms, 8);
    if (b64)
        k_dot<true><<<grid, kJoinThreads, 0, s>>>(a, b, n, sum);
    else
        k_dot<false><<<grid, kJoinThreads, 0, s>>>(a, b, n, sum);
    return cudaGetLastError();
}

cudaError_t max_launch(const void* a, int a64, uint64_t n, unsigned long long* mx, int sms,
                       cudaStream_t s) {
    const int grid = grid_for(n, kJoinThreads, sms, 8);
    if (a64)
        k_max<true><<<grid, kJoinThreads, 0, s>>>(a, n, mx);
    else
        k_max<false><<<grid, kJoinThreads, 0, s>>>(a, n, mx);
    return cudaGetLastError();
}

}  // namespace gace
