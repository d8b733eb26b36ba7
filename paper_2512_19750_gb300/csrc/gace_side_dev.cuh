// gace_side_dev.cuh -- device code of HyperLogLog and of the join sides,
// written over ranges of rows so that the dedicated kernels and the batched
// work-queue kernel run the same code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "gace_device.cuh"
#include "gace_hot.h"
#include "gace_internal.h"
#include "gace_stage.cuh"

namespace gace {
namespace side_dev {

using namespace dev;

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

// x ^= x >> s (0 < s < 32) and x *= c on a 64-bit value held as two words.
__device__ __forceinline__ void xs_words(uint32_t& lo, uint32_t& hi, int s) {
    lo ^= __funnelshift_r(lo, hi, s);
    hi ^= hi >> s;
}
__device__ __forceinline__ void mul_words(uint32_t& lo, uint32_t& hi, uint64_t c) {
    const uint32_t cl = static_cast<uint32_t>(c), ch = static_cast<uint32_t>(c >> 32);
    const uint32_t nh = __umulhi(lo, cl) + lo * ch + hi * cl;
    lo *= cl;
    hi = nh;
}

// Register index j = the top p bits of the hash (p <= 18: within its high
// word) and rho = the leading zeros of the remaining 64 - p bits, + 1 (65 - p
// when they are all zero).  The hash, splitmix64 of key ^ seedhash, is taken
// word by word; the remaining bits are the high word's low 32 - p bits, then
// the low word, so rho is the leading zeros of the first, plus those of the
// second when the first is zero (a zero word has 32), less p, plus 1.
__device__ __forceinline__ void hll_rank(uint64_t key, uint64_t seedhash, uint32_t p,
                                         uint32_t& j, uint32_t& rho) {
    const uint64_t x = (key ^ seedhash) + 0x9E3779B97F4A7C15ull;
    uint32_t lo = static_cast<uint32_t>(x), hi = static_cast<uint32_t>(x >> 32);
    xs_words(lo, hi, 30);
    mul_words(lo, hi, 0xBF58476D1CE4E5B9ull);
    xs_words(lo, hi, 27);
    mul_words(lo, hi, 0x94D049BB133111EBull);
    xs_words(lo, hi, 31);
    j = hi >> (32 - p);
    const uint32_t rh = hi & ((1u << (32 - p)) - 1u);
    rho = static_cast<uint32_t>(__clz(rh)) + (rh ? 0u : static_cast<uint32_t>(__clz(lo))) + 1u - p;
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

// Where a CTA keeps the registers it updates: the job's global 32-bit
// registers, a shared-memory copy of one-byte registers (raised by a CAS on
// the containing word), or a shared-memory copy of 32-bit registers (raised
// by one atomicMax, no retry loop: a CTA's copy starts at zero and is raised
// a few times per register as its rows arrive, which on data with many
// distinct values makes the CAS loop the kernel's bottleneck).
enum HllRegs : int { kHllGlobal = 0, kHllBytes = 1, kHllWords = 2 };
// The largest p whose 32-bit registers a CTA keeps in shared memory (64 KB).
constexpr uint32_t kHllWordsMaxP = 14;

// HLL of one group of four rows starting at row0 (values in v): rank of each
// value, then a max-update of its register where the rank would raise it.
template <int REGS, int DT>
__device__ __forceinline__ void hll_quad(const HllArgs& A, uint32_t* sregs, const Quad& v, uint64_t row0) {
    // ranks of the four values first (independent), then the register checks
    uint32_t j[4], rho[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) hll_rank(canonical_key(DT, v.lo[r], v.hi[r]), A.seedhash, A.p, j[r], rho[r]);
    if (row0 + 3 >= A.nrows) {  // only the table's last quad runs past its end
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (row0 + r >= A.nrows) rho[r] = 0;  // never raises a register
    }
    if (REGS == kHllWords) {
        uint32_t cur[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) cur[r] = reinterpret_cast<const volatile uint32_t*>(sregs)[j[r]];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (rho[r] > cur[r]) atomicMax(&sregs[j[r]], rho[r]);
    } else if (REGS == kHllBytes) {
        const unsigned char* sbytes = reinterpret_cast<const unsigned char*>(sregs);
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

// HLL over groups of four rows g = first, first + stride, ... < end; U = 2
// takes two groups per iteration with both loads issued before either is
// hashed (the second load may fall past `end`; it is bounded by the table and
// ignored), for kernels with few warps per SM.
template <int REGS, int DT, int U = 1>
__device__ __forceinline__ void hll_groups(const HllArgs& A, uint32_t* sregs, uint64_t first, uint64_t end,
                                           uint64_t stride) {
    constexpr uint32_t width = DT == 1 ? 8 : 4;
    if constexpr (U == 1) {
        for (uint64_t g = first; g < end; g += stride) {
            Quad v;
            load_quad_global(A.col, width, g * 4, A.nrows, v);
            hll_quad<REGS, DT>(A, sregs, v, g * 4);
        }
    } else {
        for (uint64_t g = first; g < end; g += 2 * stride) {
            const uint64_t g2 = g + stride;
            Quad v0, v1;
            load_quad_global(A.col, width, g * 4, A.nrows, v0);
            load_quad_global(A.col, width, g2 * 4, A.nrows, v1);
            hll_quad<REGS, DT>(A, sregs, v0, g * 4);
            if (g2 < end) hll_quad<REGS, DT>(A, sregs, v1, g2 * 4);
        }
    }
}

// Clears a CTA's shared-memory registers (m of them, REGS kHllBytes or kHllWords).
template <int REGS>
__device__ __forceinline__ void hll_clear(uint32_t* sregs, uint32_t m, uint32_t tid, uint32_t nthreads) {
    const uint32_t words = REGS == kHllWords ? m : m / 4;
    for (uint32_t i = tid; i < words; i += nthreads) sregs[i] = 0;
}

// A CTA's shared-memory registers into the global ones, only where larger.
template <int REGS>
__device__ __forceinline__ void hll_merge(const HllArgs& A, const uint32_t* sregs, uint32_t m, uint32_t tid,
                                          uint32_t nthreads) {
    const unsigned char* sbytes = reinterpret_cast<const unsigned char*>(sregs);
    for (uint32_t jj = tid; jj < m; jj += nthreads) {
        const uint32_t r = REGS == kHllWords ? sregs[jj] : sbytes[jj];
        if (r && r > __ldcg(&A.regs[jj])) atomicMax(&A.regs[jj], r);
    }
}

// ---------------------------------------------------------------- join sides

// Filter of U groups of four rows (starting rows row0[u]): each term's U
// loads are issued before any is tested.
template <int U>
__device__ __forceinline__ void side_pass_u(const SideArgs& A, const uint64_t (&row0)[U], bool (&p)[U][4]) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < 4; ++r) p[u][r] = row0[u] + r < A.nrows;
    for (uint32_t t = 0; t < A.nterms; ++t) {
        const FilterTerm& ft = A.terms[t];
        const uint32_t w = A.slot_dtype[ft.slot] == 1 ? 8 : 4;
        Quad v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) load_quad_global(A.slot_ptr[ft.slot], w, row0[u], A.nrows, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int r = 0; r < 4; ++r)
                p[u][r] = p[u][r] && term_holds(ft.kind, ft.c, v[u].lo[r], v[u].hi[r], A.pool);
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


// One side of a join over warp-uniform groups of four rows: gb = first (the
// warp's first group), first + stride, ... < end, lane l taking group gb + l;
// U such sweeps per iteration (side_groups), their loads issued together.
// MODE 0: h[key] += 1 (AGG: equal keys of a warp combined with match_any);
// 1: acc += weight32[key]; 2: acc += weight64[key]; 3: w64[key] += h2[fk2].
// npass counts the rows that pass the filter; a passing row with a key outside
// [0, domain) sets kStatusKeyDomain when strict.
template <int MODE, bool AGG>
__device__ __forceinline__ void side_rows(const SideArgs& A, uint32_t* hist, int strict, const void* weight,
                                          uint64_t domain2, unsigned long long* w64, const int64_t key[4],
                                          const int64_t fk2[4], const bool pass_in[4], bool mine,
                                          unsigned long long& npass, unsigned long long& acc) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const bool pass = pass_in[r] && mine;
        const bool in_dom = key[r] >= 0 && static_cast<uint64_t>(key[r]) < A.domain;
        npass += pass ? 1 : 0;
        if (pass && !in_dom && strict) atomicOr(A.status, kStatusKeyDomain);
        const bool use = pass && in_dom;
        if (MODE == 0) {
            if (AGG) {
                // a domain below 2^32 keeps every key below 0xFFFFFFFF, free to
                // mark the lanes without a row: a 32-bit match suffices
                unsigned grp;
                if (A.domain <= 0xFFFFFFFFull)
                    grp = __match_any_sync(kFullMask, use ? static_cast<uint32_t>(key[r]) : 0xFFFFFFFFu);
                else
                    grp = __match_any_sync(kFullMask, use ? static_cast<unsigned long long>(key[r]) : ~0ull);
                if (use && (__ffs(grp) - 1) == lane) atomicAdd(&hist[key[r]], __popc(grp));
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

template <int MODE, bool AGG, int U = 2>
__device__ __forceinline__ void side_groups(const SideArgs& A, uint32_t* hist, int strict, const void* weight,
                                            uint32_t fk2_slot, uint64_t domain2, unsigned long long* w64,
                                            uint64_t first, uint64_t end, uint64_t stride,
                                            unsigned long long& npass, unsigned long long& acc) {
    const int lane = threadIdx.x & 31;
    for (uint64_t gb = first; gb < end; gb += U * stride) {
        uint64_t row0[U];
        bool mine[U];
        int64_t key[U][4], fk2[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t gu = gb + u * stride + lane;
            row0[u] = gu * 4;
            mine[u] = gu < end;  // groups past the range read as rows past the table (or are ignored)
            side_keys(A, A.key_slot, row0[u], key[u]);
#pragma unroll
            for (int r = 0; r < 4; ++r) fk2[u][r] = 0;
            if (MODE == 3) side_keys(A, fk2_slot, row0[u], fk2[u]);
        }
        bool p[U][4];
        side_pass_u<U>(A, row0, p);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (gb + u * stride < end)  // warp-uniform: every lane reaches the match_any of each sweep
                side_rows<MODE, AGG>(A, hist, strict, weight, domain2, w64, key[u], fk2[u], p[u], mine[u], npass,
                                     acc);
    }
}

// ------------------------------------------------------- staged side scans
//
// The same side modes over tiles that a bulk-copy pipeline stages in shared
// memory (tile_pipeline): no warp waits on a column load, so a gather's only
// latency is its weight load from L2.  A lane takes eight rows of each 256-row
// slice (quad h = rows slice0 + 128 h + 4 lane + r, bit 4 h + r of its masks).

template <int NQ>
__device__ __forceinline__ void side_vals(const SideArgs& A, uint32_t slot, bool staged, const unsigned char* sbuf,
                                          uint32_t j, uint64_t slice0, int lane, Vals<NQ>& v) {
    if (staged)
        load_vals_smem<NQ>(sbuf + A.slot_soff[slot], j * 128u * NQ, A.slot_width[slot], lane, v);
    else
        load_vals_global<NQ>(A.slot_ptr[slot], A.slot_width[slot], slice0, A.nrows, lane, v);
}

// Rows (bits) of the lane's values on which one filter term holds; the kind
// is tested once for all rows.
template <int NQ>
__device__ __forceinline__ uint32_t filter_bits(const FilterTerm& ft, const Vals<NQ>& v, const uint32_t* pool) {
    constexpr int R = 4 * NQ;
    const DevTerm& c = ft.c;
    uint32_t b = 0u;
    switch (ft.kind) {
        case kRangeI32: {
#define PR(i) ((v.lo[i] - c.a_lo) <= c.b_lo)
            GACE_ROWBITS(R, PR, b);
#undef PR
            break;
        }
        case kRangeI64: {
            const uint64_t lo = join64(c.a_lo, c.a_hi), span = join64(c.b_lo, c.b_hi);
#define PR(i) ((join64(v.lo[i], v.hi[i]) - lo) <= span)
            GACE_ROWBITS(R, PR, b);
#undef PR
            break;
        }
        case kRangeF32: {
            const float lo = __uint_as_float(c.a_lo), hi = __uint_as_float(c.b_lo);
#define PR(i) (__uint_as_float(v.lo[i]) >= lo && __uint_as_float(v.lo[i]) <= hi)
            GACE_ROWBITS(R, PR, b);
#undef PR
            break;
        }
        default: {  // IN lists
#define PT(i) term_holds(ft.kind, c, v.lo[i], v.hi[i], pool)
            GACE_ROWBITS(R, PT, b);
#undef PT
            break;
        }
    }
    return b;
}

__device__ __forceinline__ int64_t key_of(uint32_t dtype, uint32_t lo, uint32_t hi) {
    return dtype == 1 ? static_cast<int64_t>(join64(lo, hi)) : static_cast<int64_t>(static_cast<int32_t>(lo));
}

// Key of row i of the lane's values as an index, and whether it lies in
// [0, domain).  An int32 key is in the domain iff its bits, read unsigned, are
// below min(domain, 2^31) (negative keys read as 2^31 or more).
template <bool KEY64, int NQ>
__device__ __forceinline__ uint64_t key_index(const Vals<NQ>& v, int i, uint64_t domain, uint32_t dom32,
                                              bool& in_dom) {
    if (KEY64) {
        const uint64_t k = join64(v.lo[i], v.hi[i]);
        in_dom = k < domain;  // a negative key reads as 2^63 or more
        return k;
    }
    in_dom = v.lo[i] < dom32;
    return v.lo[i];
}

// Rows of one staged side scan step per lane: gathers take 16 (sixteen
// weight loads in flight before any is added), the atomic modes 8.
template <int MODE>
__host__ __device__ constexpr int side_nq() { return (MODE == 1 || MODE == 2) ? 4 : 2; }

// A CTA's cache of hot histogram keys in shared memory (global histograms
// of skewed keys: every CTA adding to a Zipf-hot key's one L2 address
// serialises): 2^hot_log slots of (key, count), keys first.  A key takes the
// slot its hash selects if the slot is free; a key that finds its slot taken
// by another goes to the global histogram.  Every count lands in exactly one
// place; hot_flush adds the slots into the global histogram.  Keys are below
// 0xFFFFFFFF (the empty mark), so the domain must be below 2^32.
constexpr uint32_t kHotEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ void hot_init(uint32_t* hot, uint32_t hot_log, int tid, int nthreads) {
    for (uint32_t i = tid; i < (1u << hot_log); i += nthreads) {
        hot[i] = kHotEmpty;
        hot[(1u << hot_log) + i] = 0;
    }
}

__device__ __forceinline__ void hot_add(uint32_t* hot, uint32_t hot_log, uint32_t* hist, uint32_t k, uint32_t c) {
    const uint32_t slot = (k * 0x9E3779B1u) >> (32 - hot_log);
    uint32_t cur = hot[slot];
    if (cur == kHotEmpty) {
        cur = atomicCAS(&hot[slot], kHotEmpty, k);
        if (cur == kHotEmpty) cur = k;  // claimed
    }
    if (cur == k)
        atomicAdd(&hot[(1u << hot_log) + slot], c);
    else
        atomicAdd(&hist[k], c);
}

__device__ __forceinline__ void hot_flush(const uint32_t* hot, uint32_t hot_log, uint32_t* hist, int tid,
                                          int nthreads) {
    for (uint32_t i = tid; i < (1u << hot_log); i += nthreads) {
        const uint32_t k = hot[i], c = hot[(1u << hot_log) + i];
        if (k != kHotEmpty && c) atomicAdd(&hist[k], c);
    }
}

// One side mode over tiles [first, end) of the staged scan (stride: the grid's
// CTAs); npass and acc are per thread.  MODE as in side_rows; KEY64: the key
// column is int64 (else int32); NQ quads of rows per lane and step, WARPS warps
// per CTA (a tile holds a multiple of 128 NQ WARPS rows).  False when a
// pipeline wait gave up (kStatusTimeout set).
template <int MODE, bool AGG, bool KEY64, int NQ = side_nq<MODE>(), int WARPS = kSideWarps>
__device__ __forceinline__ bool side_tiles(const SideArgs& A, uint64_t* bars, unsigned char* stages, int tid,
                                           int lane, int warp, uint64_t first, uint64_t end, uint64_t stride,
                                           uint32_t* hist, int strict, const void* weight, uint32_t fk2_slot,
                                           uint64_t domain2, unsigned long long* w64, unsigned long long& npass,
                                           unsigned long long& acc, uint32_t* hot = nullptr, uint32_t hot_log = 0) {
    constexpr int R = 4 * NQ;
    constexpr uint32_t kSlice = 128u * NQ;
    constexpr uint32_t kAll = R == 32 ? 0xFFFFFFFFu : (1u << R) - 1u;
    bool bad_key = false;
    const uint32_t dom32 = A.domain < 0x80000000ull ? static_cast<uint32_t>(A.domain) : 0x80000000u;
    // 32-bit gathers: the weights loaded in one step are added in the lane's
    // next step, so that their latency overlaps the next tile's wait and filter
    using W = typename std::conditional<MODE == 2, unsigned long long, uint32_t>::type;
    W wp[R];
#pragma unroll
    for (int i = 0; i < R; ++i) wp[i] = 0;
    const uint32_t fk2_dt = MODE == 3 ? A.slot_dtype[fk2_slot] : 0u;
    const bool ok = tile_pipeline<kSlice, WARPS>(
        A, bars, stages, tid, warp, first, end, stride,
        [&](unsigned char* stage, uint64_t* bar, uint64_t tile) {
            const uint32_t b = smem_u32(bar);
            mbar_arrive_expect_tx(b, A.stage_bytes);
            const uint64_t row0 = tile * A.tile_rows;
            for (uint32_t s = 0; s < A.nslots; ++s) {
                const unsigned char* src = static_cast<const unsigned char*>(A.slot_ptr[s]) + row0 * A.slot_width[s];
                bulk_g2s(smem_u32(stage + A.slot_soff[s]), src, A.tile_rows * A.slot_width[s], b);
            }
        },
        [&](bool staged, const unsigned char* sbuf, uint32_t j, uint64_t slice0, bool tile_full) {
            uint32_t pass = kAll;
            if (!tile_full) {
#define PV(i) (slice0 + 128u * ((i) / 4) + 4u * lane + ((i) % 4) < A.nrows)
                GACE_ROWBITS(R, PV, pass);
#undef PV
            }
            for (uint32_t t = 0; t < A.nterms; ++t) {
                const FilterTerm& ft = A.terms[t];
                Vals<NQ> v;
                side_vals<NQ>(A, ft.slot, staged, sbuf, j, slice0, lane, v);
                pass &= filter_bits<NQ>(ft, v, A.pool);
            }
            npass += __popc(pass);
            if (MODE == 1) {
#pragma unroll
                for (int i = 0; i < R; ++i) acc += wp[i];
#pragma unroll
                for (int i = 0; i < R; ++i) wp[i] = 0;
            }
            if (!__any_sync(kFullMask, pass != 0u)) return;  // warp-uniform
            Vals<NQ> kv;
            side_vals<NQ>(A, A.key_slot, staged, sbuf, j, slice0, lane, kv);
            uint32_t use = 0u;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                bool in_dom;
                key_index<KEY64>(kv, i, A.domain, dom32, in_dom);
                if (in_dom) use |= 1u << i;
            }
            bad_key |= (pass & ~use) != 0u;
            use &= pass;
            if (MODE == 1 || MODE == 2) {
                // every weight load of the step issued at once; added next step
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    bool d;
                    const uint64_t k = key_index<KEY64>(kv, i, A.domain, dom32, d);
                    if ((use >> i) & 1u) wp[i] = __ldg(static_cast<const W*>(weight) + k);
                }
                if (MODE == 2) {  // 64-bit weights: no registers to carry them over, added at once
#pragma unroll
                    for (int i = 0; i < R; ++i) acc += wp[i];
#pragma unroll
                    for (int i = 0; i < R; ++i) wp[i] = 0;
                }
            } else if (MODE == 0) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const bool u = (use >> i) & 1u;
                    bool d;
                    const uint64_t k = key_index<KEY64>(kv, i, A.domain, dom32, d);
                    if (AGG) {
                        unsigned grp;
                        if (!KEY64 || A.domain <= 0xFFFFFFFFull)  // keys below 0xFFFFFFFF: a 32-bit match
                            grp = __match_any_sync(kFullMask, u ? static_cast<uint32_t>(k) : 0xFFFFFFFFu);
                        else
                            grp = __match_any_sync(kFullMask, u ? static_cast<unsigned long long>(k) : ~0ull);
                        if (u && (__ffs(grp) - 1) == lane) {
                            if (hot)
                                hot_add(hot, hot_log, hist, static_cast<uint32_t>(k), __popc(grp));
                            else
                                atomicAdd(&hist[k], __popc(grp));
                        }
                    } else if (u) {
                        atomicAdd(&hist[k], 1u);
                    }
                }
            } else {
                Vals<NQ> fv;
                side_vals<NQ>(A, fk2_slot, staged, sbuf, j, slice0, lane, fv);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int64_t f2 = key_of(fk2_dt, fv.lo[i], fv.hi[i]);
                    if (((use >> i) & 1u) && f2 >= 0 && static_cast<uint64_t>(f2) < domain2) {
                        const uint32_t h = static_cast<const uint32_t*>(weight)[f2];
                        bool d;
                        if (h)
                            atomicAdd(&w64[key_index<KEY64>(kv, i, A.domain, dom32, d)],
                                      static_cast<unsigned long long>(h));
                    }
                }
            }
        },
        false, AllTiles());
    if (MODE == 1)
#pragma unroll
        for (int i = 0; i < R; ++i) acc += wp[i];
    if (bad_key && strict) atomicOr(A.status, kStatusKeyDomain);
    return ok;
}

// Shared-memory histograms add each row with its own atomic: combining a
// warp's equal keys first (__match_any_sync, which global histograms need)
// costs more there than the same-address conflicts it saves, even on
// Zipf-hot keys.
#ifndef GACE_SMEM_HIST_AGG
#define GACE_SMEM_HIST_AGG 0
#endif
constexpr bool kSmemHistAgg = GACE_SMEM_HIST_AGG != 0;

// A CTA's shared-memory histogram of K bins into the global one (nonzero bins).
__device__ __forceinline__ void hist_merge(const uint32_t* shist, uint32_t* ghist, uint32_t K, uint32_t tid,
                                           uint32_t nthreads) {
    for (uint32_t i = tid; i < K; i += nthreads) {
        const uint32_t v = shist[i];
        if (v) atomicAdd(&ghist[i], v);
    }
}

// Largest element of a[first], a[first + stride], ... < end (per thread).
template <bool B64>
__device__ __forceinline__ unsigned long long max_range(const void* a, uint64_t first, uint64_t end,
                                                        uint64_t stride) {
    unsigned long long best = 0;
    for (uint64_t i = first; i < end; i += stride) {
        const unsigned long long x = B64 ? static_cast<const unsigned long long*>(a)[i]
                                         : static_cast<const uint32_t*>(a)[i];
        best = x > best ? x : best;
    }
    return best;
}

// sum of a[i] * b[i] over i = first, first + stride, ... < end (per thread).
template <bool B64>
__device__ __forceinline__ unsigned long long dot_range(const uint32_t* a, const void* b, uint64_t first,
                                                        uint64_t end, uint64_t stride) {
    unsigned long long acc = 0;
    for (uint64_t i = first; i < end; i += stride) {
        const unsigned long long x = a[i];
        if (x) {
            if (B64)
                acc += x * static_cast<const unsigned long long*>(b)[i];
            else
                acc += x * static_cast<unsigned long long>(static_cast<const uint32_t*>(b)[i]);
        }
    }
    return acc;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(kFullMask, v, o);
        v = y > v ? y : v;
    }
    return v;
}

}  // namespace side_dev
}  // namespace gace
