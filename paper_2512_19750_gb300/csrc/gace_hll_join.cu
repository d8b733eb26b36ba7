// gace_hll_join.cu -- K4 HyperLogLog registers and K5/K6 join-cardinality
// kernels.
//
// NDV is the statistic behind the drift signal D of the paper (Section III-C,
// Eq. 1); the sketch is HyperLogLog (Flajolet, Fusy, Gandouet & Meunier,
// AofA 2007) with a 64-bit splitmix64-based hash.  Each CTA keeps a private
// copy of the 2^p one-byte registers in shared memory (max-updated with a
// compare-and-swap on the containing word, skipped whenever the register is
// already large enough, which is the common case on skewed data), then merges
// it into 32-bit global registers with atomicMax, again only where it would
// raise them.
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

namespace gace {
namespace {

using namespace dev;

constexpr int kHllThreads = 1024;
constexpr int kJoinThreads = 256;
constexpr uint32_t kCasLimit = 1u << 20;

// Canonical 64-bit key of an element: int32 sign-extended, int64 as is,
// float32 bits zero-extended with -0 -> +0 and every NaN -> 0x7FC00000.
__device__ __forceinline__ uint64_t canonical_key(uint32_t dtype, uint32_t lo, uint32_t hi) {
    if (dtype == 0) return static_cast<uint64_t>(static_cast<int64_t>(static_cast<int32_t>(lo)));
    if (dtype == 1) return join64(lo, hi);
    if ((lo & 0x7FFFFFFFu) == 0) return 0;
    if ((lo & 0x7F800000u) == 0x7F800000u && (lo & 0x007FFFFFu) != 0) return 0x7FC00000ull;
    return lo;
}

__device__ __forceinline__ void hll_rank(uint64_t key, uint64_t seedhash, uint32_t p,
                                         uint32_t& j, uint32_t& rho) {
    const uint64_t h = splitmix64(key ^ seedhash);
    j = static_cast<uint32_t>(h >> (64 - p));
    const uint64_t w = h << p;
    rho = w ? static_cast<uint32_t>(__clzll(static_cast<long long>(w))) + 1u : 65u - p;
}

// byte-wise max in shared memory via CAS on the containing word (bounded)
__device__ __forceinline__ void smem_byte_max(uint32_t* words, uint32_t j, uint32_t rho,
                                              unsigned int* status) {
    uint32_t* w = &words[j >> 2];
    const uint32_t sh = (j & 3u) * 8u;
    uint32_t old = *reinterpret_cast<volatile uint32_t*>(w);
    for (uint32_t n = 0; ((old >> sh) & 0xFFu) < rho; ++n) {
        if (n >= kCasLimit) {
            atomicOr(status, kStatusCasLimit);
            return;
        }
        const uint32_t nw = (old & ~(0xFFu << sh)) | (rho << sh);
        const uint32_t prev = atomicCAS(w, old, nw);
        if (prev == old) return;
        old = prev;
    }
}

template <bool SMEM, int DT>
__global__ void __launch_bounds__(kHllThreads, 2) k_hll(const __grid_constant__ HllArgs A) {
    extern __shared__ uint32_t sregs[];
    const uint32_t m = 1u << A.p;
    if (SMEM) {
        for (uint32_t i = threadIdx.x; i < m / 4; i += kHllThreads) sregs[i] = 0;
        __syncthreads();
    }
    const unsigned char* sbytes = reinterpret_cast<const unsigned char*>(sregs);
    constexpr uint32_t width = DT == 1 ? 8 : 4;
    const uint64_t ngroups = (A.nrows + 3) / 4;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kHllThreads;
    for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * kHllThreads + threadIdx.x; g < ngroups;
         g += stride) {
        const uint64_t row0 = g * 4;
        Quad v;
        load_quad_global(A.col, width, row0, A.nrows, v);
        // ranks of the four values first (independent), then the register checks
        uint32_t j[4], rho[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            hll_rank(canonical_key(DT, v.lo[r], v.hi[r]), A.seedhash, A.p, j[r], rho[r]);
            if (row0 + r >= A.nrows) rho[r] = 0;  // past the end: never raises a register
        }
        if (SMEM) {
            uint32_t cur[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) cur[r] = *reinterpret_cast<const volatile unsigned char*>(&sbytes[j[r]]);
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (rho[r] > cur[r]) smem_byte_max(sregs, j[r], rho[r], A.status);
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (rho[r] > *reinterpret_cast<volatile uint32_t*>(&A.regs[j[r]])) atomicMax(&A.regs[j[r]], rho[r]);
        }
    }
    if (SMEM) {
        __syncthreads();
        for (uint32_t jj = threadIdx.x; jj < m; jj += kHllThreads) {
            const uint32_t r = sbytes[jj];
            if (r && r > __ldcg(&A.regs[jj])) atomicMax(&A.regs[jj], r);
        }
    }
}

// ---------------------------------------------------------------- join sides

__device__ __forceinline__ void side_pass(const SideArgs& A, uint64_t row0, bool pass[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) pass[r] = row0 + r < A.nrows;
    for (uint32_t t = 0; t < A.nterms; ++t) {
        const FilterTerm& ft = A.terms[t];
        Quad v;
        load_quad_global(A.slot_ptr[ft.slot], A.slot_dtype[ft.slot] == 1 ? 8 : 4, row0, A.nrows, v);
#pragma unroll
        for (int r = 0; r < 4; ++r)
            pass[r] = pass[r] && term_holds(ft.kind, ft.c, v.lo[r], v.hi[r], A.pool);
    }
}

__device__ __forceinline__ void side_keys(const SideArgs& A, uint32_t slot, uint64_t row0,
                                          int64_t key[4]) {
    Quad v;
    const uint32_t dt = A.slot_dtype[slot];
    load_quad_global(A.slot_ptr[slot], dt == 1 ? 8 : 4, row0, A.nrows, v);
#pragma unroll
    for (int r = 0; r < 4; ++r)
        key[r] = dt == 1 ? static_cast<int64_t>(join64(v.lo[r], v.hi[r]))
                         : static_cast<int64_t>(static_cast<int32_t>(v.lo[r]));
}

// MODE 0: histogram; 1: gather uint32 weights; 2: gather uint64 weights;
// 3: chain weights w[key] += h2[fk2].
template <int MODE, bool AGG>
__global__ void __launch_bounds__(kJoinThreads)
    k_side(const __grid_constant__ SideArgs A, uint32_t* hist, int strict, const void* weight,
           unsigned long long* out_sum, uint32_t fk2_slot, uint64_t domain2,
           unsigned long long* w64) {
    __shared__ unsigned long long scratch[kJoinThreads / 32];
    const uint64_t ngroups = (A.nrows + 3) / 4;
    const int lane = threadIdx.x & 31;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kJoinThreads;
    unsigned long long npass = 0, acc = 0;
    // warp-uniform trip count so that every lane reaches the warp collectives
    for (uint64_t gb = static_cast<uint64_t>(blockIdx.x) * kJoinThreads + (threadIdx.x - lane);
         gb < ngroups; gb += stride) {
        const uint64_t g = gb + lane;
        const uint64_t row0 = g * 4;
        int64_t key[4];
        side_keys(A, A.key_slot, row0, key);
        int64_t fk2[4] = {0, 0, 0, 0};
        if (MODE == 3) side_keys(A, fk2_slot, row0, fk2);
        bool pass[4];
        side_pass(A, row0, pass);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const bool in_dom = key[r] >= 0 && static_cast<uint64_t>(key[r]) < A.domain;
            npass += pass[r] ? 1 : 0;
            if (pass[r] && !in_dom && strict) atomicOr(A.status, kStatusKeyDomain);
            const bool use = pass[r] && in_dom;
            if (MODE == 0) {
                if (AGG) {
                    const unsigned long long k = use ? static_cast<unsigned long long>(key[r]) : ~0ull;
                    const unsigned grp = __match_any_sync(kFullMask, k);
                    if (use && (__ffs(grp) - 1) == lane) atomicAdd(&hist[k], __popc(grp));
                } else if (use) {
                    atomicAdd(&hist[key[r]], 1u);
                }
            } else if (MODE == 1) {
                if (use) acc += static_cast<const uint32_t*>(weight)[key[r]];
            } else if (MODE == 2) {
                if (use) acc += static_cast<const unsigned long long*>(weight)[key[r]];
            } else {
                if (use && fk2[r] >= 0 && static_cast<uint64_t>(fk2[r]) < domain2) {
                    const uint32_t h = static_cast<const uint32_t*>(weight)[fk2[r]];
                    if (h) atomicAdd(&w64[key[r]], static_cast<unsigned long long>(h));
                }
            }
        }
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
    unsigned long long acc = 0;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kJoinThreads;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kJoinThreads + threadIdx.x; i < n;
         i += stride) {
        const unsigned long long x = a[i];
        if (x) {
            if (B64)
                acc += x * static_cast<const unsigned long long*>(b)[i];
            else
                acc += x * static_cast<unsigned long long>(static_cast<const uint32_t*>(b)[i]);
        }
    }
    const unsigned long long t = block_sum_u64<kJoinThreads / 32>(acc, scratch);
    if (threadIdx.x == 0 && t) atomicAdd(sum, t);
}

template <bool B64>
__global__ void __launch_bounds__(kJoinThreads)
    k_max(const void* a, uint64_t n, unsigned long long* mx) {
    unsigned long long best = 0;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kJoinThreads;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kJoinThreads + threadIdx.x; i < n;
         i += stride) {
        const unsigned long long x = B64 ? static_cast<const unsigned long long*>(a)[i]
                                         : static_cast<const uint32_t*>(a)[i];
        best = x > best ? x : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(kFullMask, best, o);
        best = y > best ? y : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(mx, best);
}

int grid_for(uint64_t units, int per_cta, int sms, int ctas_per_sm) {
    const uint64_t need = (units + per_cta - 1) / per_cta;
    const uint64_t cap = static_cast<uint64_t>(sms) * ctas_per_sm;
    return static_cast<int>(need < 1 ? 1 : (need < cap ? need : cap));
}

}  // namespace

template <bool SMEM, int DT>
static cudaError_t hll_launch_t(const HllArgs& a, int sms, cudaStream_t s) {
    const uint64_t groups = (a.nrows + 3) / 4;
    const uint32_t smem = SMEM ? (1u << a.p) : 0u;
    cudaError_t e = cudaFuncSetAttribute(k_hll<SMEM, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hll<SMEM, DT>, kHllThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    k_hll<SMEM, DT><<<grid_for(groups, kHllThreads, sms, occ), kHllThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t hll_launch(const HllArgs& a, int sms, cudaStream_t s) {
    // registers in shared memory up to p = 17 (128 KB), else straight to global
    const bool sm = a.p <= 17;
    switch (a.dtype) {
        case 0: return sm ? hll_launch_t<true, 0>(a, sms, s) : hll_launch_t<false, 0>(a, sms, s);
        case 1: return sm ? hll_launch_t<true, 1>(a, sms, s) : hll_launch_t<false, 1>(a, sms, s);
        default: return sm ? hll_launch_t<true, 2>(a, sms, s) : hll_launch_t<false, 2>(a, sms, s);
    }
}

cudaError_t hist_launch(const SideArgs& a, uint32_t* hist, int strict, int aggregate, int sms,
                        cudaStream_t s) {
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
    const int grid = grid_for((a.nrows + 3) / 4, kJoinThreads, sms, 8);
    k_side<3, false><<<grid, kJoinThreads, 0, s>>>(a, nullptr, 1, h2, nullptr, fk2_slot, domain2, w);
    return cudaGetLastError();
}

cudaError_t gather_launch(const SideArgs& a, const void* weight, int weight64,
                          unsigned long long* sum, int sms, cudaStream_t s) {
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
