// gace_device.cuh -- device helpers shared by the libgace kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_internal.h"

namespace gace {
namespace dev {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014): add the
// golden-ratio increment, two xor-shift-multiply rounds, a final xor-shift.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Invalidates an mbarrier whose phases are all complete, so that its shared
// memory can be re-initialised or used for something else.
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait that lets the hardware suspend the thread for up to `hint_ns`
// while the phase is incomplete, instead of returning at once.
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of an mbarrier, giving up after timeout_ns (and
// after a hard cap on polls) so that no wait can spin forever.  Each poll
// lets the hardware suspend the thread (up to 1 ms) until the phase completes.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t polls = 0; polls < (1u << 26); ++polls) {
        if (mbar_try_wait_hint(bar, parity, 1000000u)) return true;
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// One bulk (non-tensor) async copy global -> this CTA's shared memory,
// completing `bytes` of transaction count on mbarrier `bar`.  Both addresses
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ uint32_t popc4(uint4 a, uint4 b) {
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

__device__ __forceinline__ uint4 and4(uint4 a, uint4 b) {
    return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

__device__ __forceinline__ uint4 ldg4(const void* p) {
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// Four consecutive elements (rows row0 .. row0+3) of a column as raw words:
// lo[r] holds the element (or its low word), hi[r] the high word of int64.
// Rows at or past nrows read as zero.
struct Quad {
    uint32_t lo[4];
    uint32_t hi[4];
};

__device__ __forceinline__ void load_quad_global(const void* base, uint32_t width, uint64_t row0,
                                                 uint64_t nrows, Quad& q) {
    const bool aligned = (reinterpret_cast<uintptr_t>(base) & 15u) == 0;
    if (width == 4) {
        const uint32_t* p = static_cast<const uint32_t*>(base);
        if (aligned && row0 + 3 < nrows) {
            uint4 v = ldg4(p + row0);
            q.lo[0] = v.x; q.lo[1] = v.y; q.lo[2] = v.z; q.lo[3] = v.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) q.lo[r] = (row0 + r < nrows) ? __ldg(p + row0 + r) : 0u;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) q.hi[r] = 0;
    } else {
        const unsigned long long* p = static_cast<const unsigned long long*>(base);
        if (aligned && row0 + 3 < nrows) {
            uint4 a = ldg4(p + row0);
            uint4 b = ldg4(p + row0 + 2);
            q.lo[0] = a.x; q.hi[0] = a.y; q.lo[1] = a.z; q.hi[1] = a.w;
            q.lo[2] = b.x; q.hi[2] = b.y; q.lo[3] = b.z; q.hi[3] = b.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                unsigned long long v = (row0 + r < nrows) ? __ldg(p + row0 + r) : 0ull;
                q.lo[r] = static_cast<uint32_t>(v);
                q.hi[r] = static_cast<uint32_t>(v >> 32);
            }
        }
    }
}

__device__ __forceinline__ void load_quad_smem(const unsigned char* p, uint32_t width, Quad& q) {
    if (width == 4) {
        uint4 v = *reinterpret_cast<const uint4*>(p);
        q.lo[0] = v.x; q.lo[1] = v.y; q.lo[2] = v.z; q.lo[3] = v.w;
#pragma unroll
        for (int r = 0; r < 4; ++r) q.hi[r] = 0;
    } else {
        uint4 a = reinterpret_cast<const uint4*>(p)[0];
        uint4 b = reinterpret_cast<const uint4*>(p)[1];
        q.lo[0] = a.x; q.hi[0] = a.y; q.lo[1] = a.z; q.hi[1] = a.w;
        q.lo[2] = b.x; q.hi[2] = b.y; q.lo[3] = b.z; q.hi[3] = b.w;
    }
}

__device__ __forceinline__ uint64_t join64(uint32_t lo, uint32_t hi) {
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// Evaluates one normalised term on a raw element (lo, hi words).
__device__ __forceinline__ bool term_holds(uint32_t kind, const DevTerm& c, uint32_t lo,
                                           uint32_t hi, const uint32_t* pool) {
    switch (kind) {
        case kRangeI32:
            return (lo - c.a_lo) <= c.b_lo;
        case kRangeI64:
            return (join64(lo, hi) - join64(c.a_lo, c.a_hi)) <= join64(c.b_lo, c.b_hi);
        case kRangeF32: {
            const float x = __uint_as_float(lo);
            return x >= __uint_as_float(c.a_lo) && x <= __uint_as_float(c.b_lo);
        }
        case kInI32: {
            bool h = false;
            for (uint32_t k = 0; k < c.b_lo; ++k) h |= (lo == pool[c.a_lo + k]);
            return h;
        }
        case kInI64: {
            bool h = false;
            for (uint32_t k = 0; k < c.b_lo; ++k)
                h |= (lo == pool[c.a_lo + 2 * k]) & (hi == pool[c.a_lo + 2 * k + 1]);
            return h;
        }
        case kInF32: {
            const float x = __uint_as_float(lo);
            bool h = false;
            for (uint32_t k = 0; k < c.b_lo; ++k) h |= (x == __uint_as_float(pool[c.a_lo + k]));
            return h;
        }
        default:
            return false;
    }
}

// Sum of a 64-bit value over a CTA; returns the total in thread 0.
template <int NWARPS>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long* scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NWARPS; ++w) t += scratch[w];
    __syncthreads();
    return t;
}

}  // namespace dev
}  // namespace gace
