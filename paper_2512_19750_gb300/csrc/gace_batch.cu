// gace_batch.cu -- the batched form: one persistent kernel drains a device
// work queue of (job, row-range) items.
//
// A batch mixes predicate probes, HyperLogLog sketches and join phases over
// many tables.  Every CTA repeatedly takes the next item index with one
// atomicAdd on the phase's queue head and runs that item with all its warps:
//   probe      wide passes: the wide-pass code over the item's 128-row
//              slices, counters in shared memory, added to the job's 64-bit
//              totals at item end (narrow passes are drained by
//              k_batch_probe, the staged pipeline over whole tiles);
//   HLL        a CTA copy of the registers in shared memory for the item's
//              rows, merged into the job's global registers where larger;
//   join side  filtered histogram, gather or chain-weight update over the
//              item's rows, pass counts and sums reduced per CTA;
//   max / dot  over a range of histogram entries.
// Items of one job are independent, so CTAs never wait on each other; jobs
// that read what other jobs write (a join's sum reads its histogram) are put
// in a later phase, i.e. a later launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"

#include "gace_probe_dev.cuh"
#include "gace_probe_narrow.cuh"
#include "gace_side_dev.cuh"

namespace gace {
namespace {

using namespace dev;
using namespace probe_dev;
using namespace side_dev;

// A wide probe item (narrow ones go to k_batch_probe): the wide-pass code
// over the item's 128-row slices, then the CTA counters into the pass's totals.
__device__ __forceinline__ void probe_item(const BatchJob& J, const BatchItem& it, unsigned char* smem, int tid,
                                           int lane, int warp) {
    const ProbeArgs& A = *J.probe;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid);
    __syncthreads();
    const uint64_t first = it.begin / kSliceRows + warp;
    const uint64_t end = (it.end + kSliceRows - 1) / kSliceRows;
    const uint32_t nsr = wide_slices(A, S, lane, first, end, kProbeWarps);
    if (lane < static_cast<int>(A.nsets) && nsr) atomicAdd(&S.ns[lane], nsr);
    __syncthreads();
    flush(A, S, tid);
}

template <int DT>
__device__ __forceinline__ void hll_item_t(const HllArgs& H, const BatchItem& it, uint32_t* sregs, int tid) {
    const uint64_t first = it.begin / 4 + tid, end = (it.end + 3) / 4;
    const uint32_t m = 1u << H.p;
    // the host sizes shared memory for 2^p 32-bit registers up to p = 14,
    // one-byte registers for p = 15, 16
    if (H.p <= kHllWordsMaxP) {
        hll_clear<kHllWords>(sregs, m, tid, kThreads);
        __syncthreads();
        hll_groups<kHllWords, DT, 2>(H, sregs, first, end, kThreads);
        __syncthreads();
        hll_merge<kHllWords>(H, sregs, m, tid, kThreads);
    } else if (H.p <= 16) {
        hll_clear<kHllBytes>(sregs, m, tid, kThreads);
        __syncthreads();
        hll_groups<kHllBytes, DT, 2>(H, sregs, first, end, kThreads);
        __syncthreads();
        hll_merge<kHllBytes>(H, sregs, m, tid, kThreads);
    } else {
        hll_groups<kHllGlobal, DT, 2>(H, sregs, first, end, kThreads);
    }
}

__device__ __forceinline__ void side_item(const BatchJob& J, const BatchItem& it, unsigned long long* scratch,
                                          int tid, int lane) {
    const SideArgs& SA = *J.side;
    unsigned long long npass = 0, acc = 0;
    const uint64_t first = it.begin / 4 + static_cast<uint64_t>(tid - lane);
    const uint64_t end = (it.end + 3) / 4;
    switch (J.kind) {
        case kJobHist:
        case kJobHistAgg:  // equal keys of a warp combined: skewed keys do not serialise on one address
            side_groups<0, true>(SA, J.hist, J.strict, nullptr, 0, 0, nullptr, first, end, kThreads, npass, acc);
            break;
        case kJobGather32:
            side_groups<1, false>(SA, nullptr, 0, J.weight, 0, 0, nullptr, first, end, kThreads, npass, acc);
            break;
        case kJobGather64:
            side_groups<2, false>(SA, nullptr, 0, J.weight, 0, 0, nullptr, first, end, kThreads, npass, acc);
            break;
        default:  // kJobChain
            side_groups<3, false>(SA, nullptr, 1, J.weight, J.fk2_slot, J.domain2, J.w64, first, end, kThreads,
                                  npass, acc);
            break;
    }
    const unsigned long long tp = block_sum_u64<kProbeWarps>(npass, scratch);
    if (tid == 0 && tp) atomicAdd(SA.pass_count, tp);
    if (J.kind == kJobGather32 || J.kind == kJobGather64) {
        const unsigned long long ta = block_sum_u64<kProbeWarps>(acc, scratch);
        if (tid == 0 && ta) atomicAdd(J.out, ta);
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_batch(const BatchItem* __restrict__ items, uint32_t nitems,
                                                    const BatchJob* __restrict__ jobs, unsigned int* head) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ unsigned long long scratch[kProbeWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(head, 1u);
        __syncthreads();
        const uint32_t k = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (k >= nitems) return;
        const BatchItem it = items[k];
        const BatchJob& J = jobs[it.job];
        const uint32_t kind = J.kind;
        if (kind == kJobProbe) {
            probe_item(J, it, smem, tid, lane, warp);
        } else if (kind == kJobHll) {
            uint32_t* sregs = reinterpret_cast<uint32_t*>(smem);
            if (J.hll.dtype == 0)
                hll_item_t<0>(J.hll, it, sregs, tid);
            else if (J.hll.dtype == 1)
                hll_item_t<1>(J.hll, it, sregs, tid);
            else
                hll_item_t<2>(J.hll, it, sregs, tid);
        } else if (kind <= kJobChain) {
            side_item(J, it, scratch, tid, lane);
        } else if (kind == kJobMax32 || kind == kJobMax64) {
            const unsigned long long best = warp_max_u64(
                kind == kJobMax64 ? max_range<true>(J.weight, it.begin + tid, it.end, kThreads)
                                  : max_range<false>(J.weight, it.begin + tid, it.end, kThreads));
            if (lane == 0 && best) atomicMax(J.out, best);
        } else {
            const unsigned long long acc =
                kind == kJobDot64 ? dot_range<true>(J.hist, J.weight, it.begin + tid, it.end, kThreads)
                                  : dot_range<false>(J.hist, J.weight, it.begin + tid, it.end, kThreads);
            const unsigned long long t = block_sum_u64<kProbeWarps>(acc, scratch);
            if (tid == 0 && t) atomicAdd(J.out, t);
        }
        __syncthreads();  // shared memory is reused by the next item
    }
}

// Narrow and single-predicate probe items only: the gate's small probes, which
// are HBM-bound and want the register budget and occupancy of the plain
// narrow kernels rather than the general kernel's.  The pass arguments are
// copied into shared memory once per item.
// Three CTAs per SM: the class launch is sized by its largest pass's shared
// memory (three CTAs' worth in practice), and the registers of the fourth
// would only add spills.
#ifndef GACE_BATCH_PROBE_CTAS
#define GACE_BATCH_PROBE_CTAS 3
#endif
__global__ void __launch_bounds__(kThreads, GACE_BATCH_PROBE_CTAS) k_batch_probe(const BatchItem* __restrict__ items, uint32_t nitems,
                                                             const BatchJob* __restrict__ jobs, unsigned int* head) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ __align__(16) ProbeArgs sA;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(head, 1u);
        __syncthreads();
        const uint32_t k = s_item;
        if (k >= nitems) return;
        const BatchItem it = items[k];
        {
            const uint4* src = reinterpret_cast<const uint4*>(jobs[it.job].probe);
            uint4* dst = reinterpret_cast<uint4*>(&sA);
            for (uint32_t i = tid; i < sizeof(ProbeArgs) / 16; i += kThreads) dst[i] = src[i];
        }
        __syncthreads();  // sA and s_item are read below; both are rewritten only after the next barrier
        const ProbeArgs& A = sA;
        const Smem S = carve(A, smem, warp);
        load_tables(A, S, tid);
        __syncthreads();
        const uint64_t first = it.begin / A.tile_rows;
        uint64_t end = (it.end + A.tile_rows - 1) / A.tile_rows;
        if (end > A.ntiles) end = A.ntiles;
        bool ok;
        switch (probe_variant(A)) {
            case 1: ok = narrow_run<false, 1>(A, S, tid, lane, warp, first, end, 1); break;
            case 2: ok = narrow_run<true, 1>(A, S, tid, lane, warp, first, end, 1); break;
            case 3: ok = narrow_run<true, kMaxSets>(A, S, tid, lane, warp, first, end, 1); break;
            case 4: {
                // one predicate on all rows of narrow rows (at most 8 bytes):
                // 16 rows per lane, as the plain single-predicate kernel
                uint32_t rowbytes = 0;
                for (uint32_t s = 0; s < A.nslots; ++s) rowbytes += A.slots[s].width;
                ok = rowbytes <= 8 ? single_run<false, 4>(A, S, tid, lane, warp, first, end, 1)
                                   : single_run<false>(A, S, tid, lane, warp, first, end, 1);
                break;
            }
            default: ok = single_run<true>(A, S, tid, lane, warp, first, end, 1); break;
        }
        if (!ok) return;  // uniform over the CTA; the status word says why
        __syncthreads();
        flush(A, S, tid);
        __syncthreads();  // shared memory is reused by the next item
    }
}

// Join sides of tables staged through shared memory (gathers, chain weights,
// histograms over large key domains): per item, the staged tile pipeline over
// the item's tiles.  The side arguments are copied into shared memory once per
// item.
template <int MODE, bool AGG>
__device__ __forceinline__ bool side_item_staged(const SideArgs& A, const BatchJob& J, const BatchItem& it,
                                                 unsigned char* smem, int tid, int lane, int warp,
                                                 unsigned long long& npass, unsigned long long& acc) {
    const uint64_t first = it.begin / A.tile_rows;
    uint64_t end = (it.end + A.tile_rows - 1) / A.tile_rows;
    if (end > A.ntiles) end = A.ntiles;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* stages = smem + kSideStageOff;
    // gathers take 16 rows per lane when a tile holds such a step for every warp
    constexpr int NQ = side_nq<MODE>();
    if (NQ > 2 && A.tile_rows % (128u * NQ * kSideWarps) != 0) {
        if (A.slot_dtype[A.key_slot] == 1)
            return side_tiles<MODE, AGG, true, 2>(A, bars, stages, tid, lane, warp, first, end, 1, J.hist, J.strict,
                                                  J.weight, J.fk2_slot, J.domain2, J.w64, npass, acc);
        return side_tiles<MODE, AGG, false, 2>(A, bars, stages, tid, lane, warp, first, end, 1, J.hist, J.strict,
                                               J.weight, J.fk2_slot, J.domain2, J.w64, npass, acc);
    }
    // skewed keys into a global histogram: a hot-key cache after the stages
    uint32_t* hot = nullptr;
    if (MODE == 0 && AGG && kHotCache && A.domain <= 0xFFFFFFFFull) {
        hot = reinterpret_cast<uint32_t*>(smem + A.smem_bytes);
        hot_init(hot, kHotLog, tid, kThreads);
    }
    const bool ok = A.slot_dtype[A.key_slot] == 1
                        ? side_tiles<MODE, AGG, true, NQ>(A, bars, stages, tid, lane, warp, first, end, 1, J.hist,
                                                          J.strict, J.weight, J.fk2_slot, J.domain2, J.w64, npass,
                                                          acc, hot, kHotLog)
                        : side_tiles<MODE, AGG, false, NQ>(A, bars, stages, tid, lane, warp, first, end, 1, J.hist,
                                                           J.strict, J.weight, J.fk2_slot, J.domain2, J.w64, npass,
                                                           acc, hot, kHotLog);
    if (ok && hot) {
        __syncthreads();
        hot_flush(hot, kHotLog, J.hist, tid, kThreads);
    }
    return ok;
}

#ifndef GACE_BATCH_SIDE_CTAS
#define GACE_BATCH_SIDE_CTAS 2
#endif
__global__ void __launch_bounds__(kThreads, GACE_BATCH_SIDE_CTAS) k_batch_side(const BatchItem* __restrict__ items, uint32_t nitems,
                                                            const BatchJob* __restrict__ jobs, unsigned int* head) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ __align__(16) SideArgs sA;
    __shared__ unsigned long long scratch[kProbeWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(head, 1u);
        __syncthreads();
        const uint32_t k = s_item;
        if (k >= nitems) return;
        const BatchItem it = items[k];
        const BatchJob& J = jobs[it.job];
        {
            const uint4* src = reinterpret_cast<const uint4*>(J.side);
            uint4* dst = reinterpret_cast<uint4*>(&sA);
            for (uint32_t i = tid; i < sizeof(SideArgs) / 16; i += kThreads) dst[i] = src[i];
        }
        __syncthreads();  // sA and s_item are read below; both are rewritten only after the next barrier
        unsigned long long npass = 0, acc = 0;
        bool ok;
        switch (J.kind) {
            case kJobHist:
            case kJobHistAgg: ok = side_item_staged<0, true>(sA, J, it, smem, tid, lane, warp, npass, acc); break;
            case kJobGather32: ok = side_item_staged<1, false>(sA, J, it, smem, tid, lane, warp, npass, acc); break;
            case kJobGather64: ok = side_item_staged<2, false>(sA, J, it, smem, tid, lane, warp, npass, acc); break;
            default: ok = side_item_staged<3, false>(sA, J, it, smem, tid, lane, warp, npass, acc); break;
        }
        if (!ok) return;  // uniform over the CTA; the status word says why
        const unsigned long long tp = block_sum_u64<kProbeWarps>(npass, scratch);
        if (tid == 0 && tp) atomicAdd(sA.pass_count, tp);
        if (J.kind == kJobGather32 || J.kind == kJobGather64) {
            const unsigned long long ta = block_sum_u64<kProbeWarps>(acc, scratch);
            if (tid == 0 && ta) atomicAdd(J.out, ta);
        }
        __syncthreads();  // shared memory is reused by the next item
    }
}

// Join histograms over small key domains: per item, a shared-memory
// histogram of the item's rows (after the staging buffers when the side's
// columns stream through the tile pipeline), then its nonzero bins into the
// job's global histogram.
__global__ void __launch_bounds__(kHistThreads, 1) k_batch_hist(const BatchItem* __restrict__ items, uint32_t nitems,
                                                                const BatchJob* __restrict__ jobs,
                                                                unsigned int* head) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ __align__(16) SideArgs sA;
    __shared__ unsigned long long scratch[kHistThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(head, 1u);
        __syncthreads();
        const uint32_t k = s_item;
        if (k >= nitems) return;
        const BatchItem it = items[k];
        const BatchJob& J = jobs[it.job];
        {
            const uint4* src = reinterpret_cast<const uint4*>(J.side);
            uint4* dst = reinterpret_cast<uint4*>(&sA);
            for (uint32_t i = tid; i < sizeof(SideArgs) / 16; i += kHistThreads) dst[i] = src[i];
        }
        __syncthreads();  // sA and s_item are read below; both are rewritten only after the next barrier
        const SideArgs& SA = sA;
        const bool staged = SA.stage_bytes && SA.tile_rows % (128u * (kHistThreads / 32)) == 0;
        uint32_t* shist = reinterpret_cast<uint32_t*>(smem + (staged ? SA.smem_bytes : 0u));
        const uint32_t K = static_cast<uint32_t>(SA.domain);
        for (uint32_t i = tid; i < K; i += kHistThreads) shist[i] = 0;
        __syncthreads();
        unsigned long long npass = 0, acc = 0;
        if (staged) {
            const uint64_t first = it.begin / SA.tile_rows;
            uint64_t end = (it.end + SA.tile_rows - 1) / SA.tile_rows;
            if (end > SA.ntiles) end = SA.ntiles;
            uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
            const bool ok = SA.slot_dtype[SA.key_slot] == 1
                                ? side_tiles<0, kSmemHistAgg, true, 1, kHistThreads / 32>(
                                      SA, bars, smem + kSideStageOff, tid, lane, warp, first, end, 1, shist, J.strict,
                                      nullptr, 0, 0, nullptr, npass, acc)
                                : side_tiles<0, kSmemHistAgg, false, 1, kHistThreads / 32>(
                                      SA, bars, smem + kSideStageOff, tid, lane, warp, first, end, 1, shist, J.strict,
                                      nullptr, 0, 0, nullptr, npass, acc);
            if (!ok) return;  // uniform over the CTA; the status word says why
        } else {
            side_groups<0, kSmemHistAgg>(SA, shist, J.strict, nullptr, 0, 0, nullptr, it.begin / 4 + (tid - lane),
                                         (it.end + 3) / 4, kHistThreads, npass, acc);
        }
        __syncthreads();
        hist_merge(shist, J.hist, K, tid, kHistThreads);
        const unsigned long long tp = block_sum_u64<kHistThreads / 32>(npass, scratch);  // synchronises
        if (tid == 0 && tp) atomicAdd(SA.pass_count, tp);
    }
}

// Scatter / gather of the served form: CTA b takes descriptors b, b + grid, ...
__global__ void __launch_bounds__(256) k_copy(const CopyDesc* __restrict__ d, uint32_t n) {
    for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
        const CopyDesc c = d[k];
        uint4* dst = reinterpret_cast<uint4*>(c.dst);
        const uint64_t nw = c.bytes / 16;
        if (c.src) {
            const uint4* src = reinterpret_cast<const uint4*>(c.src);
            for (uint64_t i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
        } else {
            for (uint64_t i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

}  // namespace

// One thread waits, with the context's limit, on an mbarrier phase that
// nothing completes: the bounded wait every pipeline uses gives up, sets the
// timeout status and returns (the failure path, exercised without a fault).
__global__ void __launch_bounds__(32) k_wait_check(unsigned int* status, uint64_t timeout_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(b, 0, timeout_ns)) atomicOr(status, kStatusTimeout);
}

// Roofline calibration of the integer pipes.  kind 0: eight independent chains
// per thread of alternating 32-bit xor and add with run-time constants (no
// single instruction does both, and neither folds across the other), two
// operations per step; kind 1: 32-bit range tests (x - lo) <= span, 16
// constants against eight values, each test's outcome added to a per-value
// count (one operation per test: the unit in which a range evaluated by
// compare is counted), the values perturbed once per iteration so that no
// test is loop-invariant.  The results feed one conditional store so that
// nothing is dead.
template <int KIND>
__global__ void __launch_bounds__(256, 8) k_int_peak(uint32_t iters, uint32_t k1, uint32_t k2, uint32_t* sink) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * (2u * i + 1u) + blockIdx.x * 7919u + i;
    if (KIND == 0) {
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    x[i] ^= k1;
                    x[i] += k2;
                }
            }
        }
    } else {
        uint32_t c[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = 0;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint32_t lo = k1 + static_cast<uint32_t>(u) * k2;
#pragma unroll
                for (int i = 0; i < 8; ++i) c[i] += (x[i] - lo) <= k2 ? 1u : 0u;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] ^= c[i];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] += c[i];
    }
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) r ^= x[i];
    if (r == 0x9E3779B9u) sink[0] = r;
}

cudaError_t int_peak_launch(int kind, uint32_t iters, int grid, uint32_t* sink, cudaStream_t s) {
    if (kind == 0)
        k_int_peak<0><<<grid, 256, 0, s>>>(iters, 0x5bd1e995u, 0x68e31da4u, sink);
    else
        k_int_peak<1><<<grid, 256, 0, s>>>(iters, 0x1000u, 0x40000u, sink);
    return cudaGetLastError();
}

// Operations one thread of k_int_peak performs per iteration.
uint64_t int_peak_ops_per_iter(int kind) { return kind == 0 ? 16u * 8u * 2u : 16u * 8u; }

int int_peak_occupancy(int kind) {
    int n = 0;
    cudaError_t e = kind == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_int_peak<0>, 256, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_int_peak<1>, 256, 0);
    return e == cudaSuccess ? n : 0;
}

cudaError_t copy_launch(const CopyDesc* descs, uint32_t n, int grid, cudaStream_t s) {
    k_copy<<<grid, 256, 0, s>>>(descs, n);
    return cudaGetLastError();
}

namespace host {
cudaError_t wait_check_launch(unsigned int* status, uint64_t timeout_ns, cudaStream_t s) {
    k_wait_check<<<1, 32, 0, s>>>(status, timeout_ns);
    return cudaGetLastError();
}
}  // namespace host

template <typename K>
static cudaError_t configure_one(K kernel, int smem_optin) {
    // the kernel's own static shared memory counts against the opt-in limit
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_optin - static_cast<int>(fa.sharedSizeBytes));
}

cudaError_t batch_configure(int smem_optin) {
    cudaError_t e = configure_one(k_batch, smem_optin);
    if (e == cudaSuccess) e = configure_one(k_batch_probe, smem_optin);
    if (e == cudaSuccess) e = configure_one(k_batch_hist, smem_optin);
    if (e == cudaSuccess) e = configure_one(k_batch_side, smem_optin);
    return e;
}

int batch_occupancy(uint32_t smem_bytes, int cls) {
    int n = 0;
    cudaError_t e;
    if (cls == kClassProbe)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_probe, kThreads, smem_bytes);
    else if (cls == kClassHist)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_hist, kHistThreads, smem_bytes);
    else if (cls == kClassSide)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_side, kThreads, smem_bytes);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch, kThreads, smem_bytes);
    return e == cudaSuccess ? n : 0;
}

cudaError_t batch_launch(const BatchItem* items, uint32_t nitems, const BatchJob* jobs, unsigned int* head,
                         int grid, uint32_t smem_bytes, int cls, cudaStream_t s) {
    if (cls == kClassProbe)
        k_batch_probe<<<grid, kThreads, smem_bytes, s>>>(items, nitems, jobs, head);
    else if (cls == kClassHist)
        k_batch_hist<<<grid, kHistThreads, smem_bytes, s>>>(items, nitems, jobs, head);
    else if (cls == kClassSide)
        k_batch_side<<<grid, kThreads, smem_bytes, s>>>(items, nitems, jobs, head);
    else
        k_batch<<<grid, kThreads, smem_bytes, s>>>(items, nitems, jobs, head);
    return cudaGetLastError();
}

}  // namespace gace
