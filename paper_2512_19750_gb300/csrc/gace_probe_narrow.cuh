// gace_probe_narrow.cuh -- the narrow evaluations of a probe pass (at most 32
// predicates and 32 distinct terms: the single probes the gate issues) over a
// range of tiles, shared by the probe kernels (a grid striding over the whole
// table) and the batched work-queue kernel (one CTA over a work item's tiles).
//
// One thread streams tiles of the referenced columns into shared memory with
// bulk async copies (cp.async.bulk + mbarrier transaction counts) a few tiles
// ahead; the warps evaluate 256-row slices, eight rows per lane:
//   narrow_run  per-term 32-row ballot masks in shared memory, lane p ANDs
//               predicate p's terms and keeps its counts in registers;
//   single_run  one predicate on one row set: every lane ANDs the terms of its
//               eight rows in registers and counts the rows that pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"
#include "gace_probe_dev.cuh"
#include "gace_stage.cuh"

namespace gace {
namespace probe_dev {

__device__ __forceinline__ void issue_tile(const ProbeArgs& A, unsigned char* stage_base,
                                           uint64_t* bar, uint64_t tile) {
    const uint32_t b = smem_u32(bar);
    mbar_arrive_expect_tx(b, A.stage_bytes);
    const uint64_t row0 = tile * A.tile_rows;
    for (uint32_t s = 0; s < A.nslots; ++s) {
        const SlotDesc& sd = A.slots[s];
        const unsigned char* src = static_cast<const unsigned char*>(sd.ptr) + row0 * sd.width;
        bulk_g2s(smem_u32(stage_base + sd.soff), src, A.tile_rows * sd.width, b);
    }
}

// Whether any row of a tile lies in a sampled block of some row set (every
// set of a pass that skips tiles is a block sample): the tile's blocks are
// hashed as the per-row membership test hashes them.
__device__ __forceinline__ bool probe_tile_live(const ProbeArgs& A, uint64_t tile) {
    const uint64_t l0 = tile * A.tile_rows;
    const uint64_t r0 = A.row0 + l0;  // table-global ids of the tile's first and last rows
    const uint64_t r1 = A.row0 + (l0 + A.tile_rows < A.nrows ? l0 + A.tile_rows : A.nrows) - 1;
    for (uint32_t q = 0; q < A.nsets; ++q) {
        const SetDesc& sd = A.sets[q];
        if (sd.kind != 2 || sd.mode != 2) return true;
        const uint64_t b0 = sd.block_shift >= 0 ? r0 >> sd.block_shift : r0 / sd.block_rows;
        const uint64_t b1 = sd.block_shift >= 0 ? r1 >> sd.block_shift : r1 / sd.block_rows;
        for (uint64_t b = b0; b <= b1; ++b)
            if (splitmix64(b ^ sd.seedhash) < sd.thresh) return true;
    }
    return false;
}

// The staged tile pipeline of the narrow evaluations over the pass's column
// slots: each warp runs `body(staged, sbuf, j, slice0, tile_full)` on its
// slices of every tile that can hold a counted row (tile_pipeline gives the
// contract).
// HASH: the pass has hashed row sets, so it may skip tiles.
template <uint32_t kSlice, bool HASH, class Body>
__device__ __forceinline__ bool run_tiles(const ProbeArgs& A, const Smem& S, int tid, int warp, uint64_t first,
                                          uint64_t end, uint64_t stride, Body&& body) {
    return tile_pipeline<kSlice, kProbeWarps>(
        A, S.bars, S.stages, tid, warp, first, end, stride,
        [&](unsigned char* stage, uint64_t* bar, uint64_t tile) { issue_tile(A, stage, bar, tile); }, body,
        HASH && A.skip_tiles != 0, [&](uint64_t tile) { return probe_tile_live(A, tile); });
}

// HASH: some row set is a hashed sample (else the only device set is "all rows",
// whose mask is the validity mask, all ones on full tiles).  MAXS: sets held
// in registers per lane.
// Over tiles [first, end) with the given stride, the counters end in the
// CTA's shared counters (the caller has loaded the tables, synchronised, and
// flushes afterwards).  False when a wait gave up.
template <bool HASH, int MAXS>
__device__ __forceinline__ bool narrow_run(const ProbeArgs& A, const Smem& S, int tid, int lane, int warp,
                                           uint64_t first, uint64_t end, uint64_t stride) {
    constexpr int NQ = 2;
    constexpr uint32_t kSlice = 128 * NQ;

    // lane-owned counters: predicate `lane`, term `lane`, row set `lane`
    uint32_t cnt[MAXS], mc[MAXS];
#pragma unroll
    for (int q = 0; q < MAXS; ++q) cnt[q] = mc[q] = 0;
    uint32_t nsr = 0;
    const bool has_pred = lane < static_cast<int>(A.npreds);
    const bool has_term = A.want_marg && lane < static_cast<int>(A.nterms);
    const uint32_t pb = has_pred ? S.poff[lane] : 0, pe = has_pred ? S.poff[lane + 1] : 0;
    const uint32_t nsets = HASH ? A.nsets : 1;

    const bool ok = run_tiles<kSlice, HASH>(A, S, tid, warp, first, end, stride,
                                      [&](bool staged, const unsigned char* sbuf, uint32_t j, uint64_t slice0,
                                          bool tile_full) {
        uint4 vm[NQ];
        if (HASH) {
            set_masks<NQ>(A, slice0, S.keep, lane);
            __syncwarp();
            // a slice with no row in any set adds nothing: skip its evaluation
            uint32_t any = 0;
            for (uint32_t q = 0; q < nsets; ++q)
#pragma unroll
                for (int h = 0; h < NQ; ++h) {
                    const uint4 k = S.keep[q * NQ + h];
                    any |= k.x | k.y | k.z | k.w;
                }
            if (!any) {
                __syncwarp();  // every lane has read S.keep before lane 0 rewrites it
                return;
            }
        } else if (!tile_full) {
#define PV(i) (slice0 + 128u * ((i) / 4) + 4u * lane + ((i) % 4) < A.nrows)
            GACE_BALLOTS(NQ, PV, vm);
#undef PV
        }
        for (uint32_t s = 0; s < A.nslots; ++s) {
            const SlotDesc& sd = A.slots[s];
            Vals<NQ> v;
            if (staged)
                load_vals_smem<NQ>(sbuf + sd.soff, j * kSlice, sd.width, lane, v);
            else
                load_vals_global<NQ>(sd.ptr, sd.width, slice0, A.nrows, lane, v);
            eval_slot<NQ>(sd, v, S.st, S.pool, S.tm, lane);
        }
        __syncwarp();
        if (has_pred) {
            uint4 acc[NQ];
#pragma unroll
            for (int h = 0; h < NQ; ++h) acc[h] = S.tm[S.pterm[pb] * NQ + h];
            for (uint32_t k = pb + 1; k < pe; ++k) {
                const uint32_t t = S.pterm[k];
#pragma unroll
                for (int h = 0; h < NQ; ++h) acc[h] = and4(acc[h], S.tm[t * NQ + h]);
            }
            if (HASH) {
#pragma unroll
                for (int q = 0; q < MAXS; ++q)
                    if (q < static_cast<int>(nsets))
#pragma unroll
                        for (int h = 0; h < NQ; ++h) cnt[q] += popc4(acc[h], S.keep[q * NQ + h]);
            } else if (tile_full) {
#pragma unroll
                for (int h = 0; h < NQ; ++h)
                    cnt[0] += __popc(acc[h].x) + __popc(acc[h].y) + __popc(acc[h].z) + __popc(acc[h].w);
            } else {
#pragma unroll
                for (int h = 0; h < NQ; ++h) cnt[0] += popc4(acc[h], vm[h]);
            }
        }
        if (has_term) {
#pragma unroll
            for (int h = 0; h < NQ; ++h) {
                const uint4 m = S.tm[lane * NQ + h];
                if (HASH) {
#pragma unroll
                    for (int q = 0; q < MAXS; ++q)
                        if (q < static_cast<int>(nsets)) mc[q] += popc4(m, S.keep[q * NQ + h]);
                } else if (tile_full) {
                    mc[0] += __popc(m.x) + __popc(m.y) + __popc(m.z) + __popc(m.w);
                } else {
                    mc[0] += popc4(m, vm[h]);
                }
            }
        }
        if (HASH && lane < static_cast<int>(nsets)) {
#pragma unroll
            for (int h = 0; h < NQ; ++h) {
                const uint4 k = S.keep[lane * NQ + h];
                nsr += __popc(k.x) + __popc(k.y) + __popc(k.z) + __popc(k.w);
            }
        }
        __syncwarp();
    });
    if (!ok) return false;
    // warps -> CTA counters
#pragma unroll
    for (int q = 0; q < MAXS; ++q) {
        if (q < static_cast<int>(nsets)) {
            if (has_pred && cnt[q]) atomicAdd(&S.cnt[q * A.npreds + lane], cnt[q]);
            if (has_term && mc[q]) atomicAdd(&S.marg[q * A.nterms + lane], mc[q]);
        }
    }
    if (HASH && lane < static_cast<int>(nsets) && nsr) atomicAdd(&S.ns[lane], nsr);
    return true;
}

// Single-predicate evaluation of one column slot: for every term of the slot,
// the lane's row results as a bit mask; ok &= mask; with marginals, the warp
// total of (mask & base) goes to lane t.
template <int NQ>
__device__ __forceinline__ void single_slot(const SlotDesc& sd, const Vals<NQ>& v, const DevTerm* st,
                                            const uint32_t* pool, uint32_t& ok, uint32_t base, bool marg,
                                            int lane, uint32_t& tc) {
    constexpr int R = 4 * NQ;
    const uint32_t rb = sd.rbeg, re = sd.rend, ie = sd.iend;
    for (uint32_t t = rb; t < ie; ++t) {
        uint32_t cb;
        if (sd.dtype == 0) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            if (t < re) {
#define PR(i) ((v.lo[i] - c.x) <= c.y)
                GACE_ROWBITS(R, PR, cb);
#undef PR
            } else {
                cb = 0u;
                for (uint32_t k = 0; k < c.y; ++k) {
                    const uint32_t x = pool[c.x + k];
                    uint32_t e;
#define PE(i) (v.lo[i] == x)
                    GACE_ROWBITS(R, PE, e);
#undef PE
                    cb |= e;
                }
            }
        } else if (sd.dtype == 1) {
            if (t < re) {
                const DevTerm c = st[t];
                const uint64_t lo = join64(c.a_lo, c.a_hi), span = join64(c.b_lo, c.b_hi);
#define PR(i) ((join64(v.lo[i], v.hi[i]) - lo) <= span)
                GACE_ROWBITS(R, PR, cb);
#undef PR
            } else {
                const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
                cb = 0u;
                for (uint32_t k = 0; k < c.y; ++k) {
                    const uint32_t xl = pool[c.x + 2 * k], xh = pool[c.x + 2 * k + 1];
                    uint32_t e;
#define PE(i) (v.lo[i] == xl && v.hi[i] == xh)
                    GACE_ROWBITS(R, PE, e);
#undef PE
                    cb |= e;
                }
            }
        } else {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            if (t < re) {
                const float lo = __uint_as_float(c.x), hi = __uint_as_float(c.y);
#define PR(i) (__uint_as_float(v.lo[i]) >= lo && __uint_as_float(v.lo[i]) <= hi)
                GACE_ROWBITS(R, PR, cb);
#undef PR
            } else {
                cb = 0u;
                for (uint32_t k = 0; k < c.y; ++k) {
                    const float y = __uint_as_float(pool[c.x + k]);
                    uint32_t e;
#define PE(i) (__uint_as_float(v.lo[i]) == y)
                    GACE_ROWBITS(R, PE, e);
#undef PE
                    cb |= e;
                }
            }
        }
        ok &= cb;
        if (marg) {
            const uint32_t c = __reduce_add_sync(kFullMask, __popc(cb & base));
            if (lane == static_cast<int>(t)) tc += c;
        }
    }
}

// One predicate on one row set (the gate's single probe): every lane ANDs the
// terms of its 4 NQ rows in predicate registers and counts the rows that
// pass; no per-term masks go through shared memory.  HASH: the set is a hashed
// sample.  NQ: 2, or 4 for passes of narrow rows (half the per-slice work per
// row; the hashed form keeps 2 to stay within the registers of four CTAs per
// SM).
template <bool HASH, int NQ = 2>
__device__ __forceinline__ bool single_run(const ProbeArgs& A, const Smem& S, int tid, int lane, int warp,
                                           uint64_t first, uint64_t end, uint64_t stride) {
    constexpr int R = 4 * NQ;
    constexpr uint32_t kSlice = 128 * NQ;
    constexpr uint32_t kAll = (1u << R) - 1u;
    uint32_t cnt = 0, nsr = 0, tc = 0;
    const bool marg = A.want_marg != 0;

    const bool ok_run = run_tiles<kSlice, HASH>(A, S, tid, warp, first, end, stride,
                                          [&](bool staged, const unsigned char* sbuf, uint32_t j, uint64_t slice0,
                                              bool tile_full) {
        // bit i: row slice0 + 128 (i / 4) + 4 lane + i % 4 is in the row set
        uint32_t base = kAll;
        if (HASH) {
            const SetDesc& sd = A.sets[0];
            base = 0u;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const uint64_t row = slice0 + 128u * (i / 4) + 4u * lane + (i % 4);
                uint64_t x = A.row0 + row;  // hashed by table-global id
                if (sd.kind == 2) x = sd.block_shift >= 0 ? (x >> sd.block_shift) : (x / sd.block_rows);
                if (row < A.nrows && splitmix64(x ^ sd.seedhash) < sd.thresh) base |= 1u << i;
            }
        } else if (!tile_full) {
#define PV(i) (slice0 + 128u * ((i) / 4) + 4u * lane + ((i) % 4) < A.nrows)
            GACE_ROWBITS(R, PV, base);
#undef PV
        }
        if (HASH && !__any_sync(kFullMask, base != 0u)) return;  // no row of the slice is in the set
        uint32_t ok = base;
        for (uint32_t s = 0; s < A.nslots; ++s) {
            const SlotDesc& sd = A.slots[s];
            Vals<NQ> v;
            if (staged)
                load_vals_smem<NQ>(sbuf + sd.soff, j * kSlice, sd.width, lane, v);
            else
                load_vals_global<NQ>(sd.ptr, sd.width, slice0, A.nrows, lane, v);
            single_slot<NQ>(sd, v, S.st, S.pool, ok, base, marg, lane, tc);
        }
        cnt += __popc(ok);
        if (HASH) nsr += __popc(base);
    });
    if (!ok_run) return false;
    cnt = __reduce_add_sync(kFullMask, cnt);
    nsr = __reduce_add_sync(kFullMask, nsr);
    if (lane == 0 && cnt) atomicAdd(&S.cnt[0], cnt);
    if (HASH && lane == 0 && nsr) atomicAdd(&S.ns[0], nsr);
    if (marg && lane < static_cast<int>(A.nterms) && tc) atomicAdd(&S.marg[lane], tc);
    return true;
}

}  // namespace probe_dev
}  // namespace gace
