// gace_stage.cuh -- the staged tile pipeline shared by the scans that stream
// columns through shared memory (the narrow probe evaluations and the join
// sides), and the per-lane row layout they read the staged tiles in.
//
// One thread keeps up to `nstages` tiles of the referenced columns in flight
// with bulk async copies (cp.async.bulk, completion by mbarrier transaction
// count); the CTA's warps evaluate slices of each tile as it lands.  A lane
// holds 4 NQ rows of a slice: quad h covers rows slice0 + 128 h + 4 lane + r.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"

namespace gace {
namespace dev {

// Values of NQ quads per lane: quad h covers rows slice0 + 128 h + 4 lane + r.
template <int NQ>
struct Vals {
    uint32_t lo[4 * NQ];
    uint32_t hi[4 * NQ];
};

template <int NQ>
__device__ __forceinline__ void load_vals_smem(const unsigned char* slot_tile, uint32_t slice_local,
                                               uint32_t width, int lane, Vals<NQ>& v) {
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
        Quad q;
        load_quad_smem(slot_tile + (slice_local + 128u * h + 4u * lane) * width, width, q);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            v.lo[4 * h + r] = q.lo[r];
            v.hi[4 * h + r] = q.hi[r];
        }
    }
}

template <int NQ>
__device__ __forceinline__ void load_vals_global(const void* ptr, uint32_t width, uint64_t slice0,
                                                 uint64_t nrows, int lane, Vals<NQ>& v) {
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
        Quad q;
        load_quad_global(ptr, width, slice0 + 128u * h + 4u * lane, nrows, q);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            v.lo[4 * h + r] = q.lo[r];
            v.hi[4 * h + r] = q.hi[r];
        }
    }
}

// Bit i of the result: per-row predicate `pred_expr(i)` for the lane's 4 NQ rows.
#define GACE_ROWBITS(R_, pred_expr, out)               \
    do {                                               \
        out = 0u;                                      \
        _Pragma("unroll") for (int i_ = 0; i_ < R_; ++i_) \
            if (pred_expr(i_)) out |= 1u << i_;        \
    } while (0)

// The staged tile pipeline.  `A` carries the scan's geometry (fields nrows,
// nstaged, tile_rows, stage_bytes, nstages, timeout_ns, status); `bars` holds
// nstages mbarriers and `stages` nstages buffers of stage_bytes.  The CTA takes
// tiles first, first + stride, ... below end (a whole grid striding over the
// table, or one CTA over the tiles of a work item); when `skip` is set, only
// the tiles for which live(tile) holds (a tile that is not live has no row the
// scan counts: it is neither copied nor evaluated).  Warp 0 finds the tiles
// to copy and its lane 0 issues them with issue(stage buffer, mbarrier, tile);
// each of the kWarps warps runs body(staged, stage buffer, j, slice0,
// tile_full) on slices j = warp, warp + kWarps, ... of kSlice rows.  Tiles
// from nstaged on (the partial last tile, and every tile of a scan that is not
// staged) are not copied: the body reads them with plain loads.  Returns true
// with the mbarriers invalidated (their shared memory free for reuse), or false
// when a wait gave up: the status bit is set and the CTA's copies in flight
// have been waited for (with the same limit).
template <uint32_t kSlice, int kWarps, class Args, class Issue, class Body, class Live>
__device__ __forceinline__ bool tile_pipeline(const Args& A, uint64_t* bars, unsigned char* stages, int tid,
                                              int warp, uint64_t first, uint64_t end, uint64_t stride,
                                              Issue&& issue, Body&& body, bool skip, Live&& live) {
    const int lane = tid & 31;
    const uint64_t staged_end = end < A.nstaged ? end : A.nstaged;
    // The first tile at or after t on the CTA's progression that is live (end
    // if none); with `skip`, a warp-collective search 32 candidates at a time.
    auto next = [&](uint64_t t) -> uint64_t {
        if (!skip) return t;
        for (; t < end; t += 32 * stride) {
            const uint64_t c = t + static_cast<uint64_t>(lane) * stride;
            const unsigned m = __ballot_sync(kFullMask, c < end && live(c));
            if (m) return t + static_cast<uint64_t>(__ffs(m) - 1) * stride;
        }
        return end;
    };
    if (tid == 0) {
        for (uint32_t s = 0; s < A.nstages; ++s) mbar_init(smem_u32(&bars[s]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    // warp 0 copies the tile nstages tiles ahead of the one evaluated: without
    // skipping, tile + nstages * stride; with it, the cursor ptile
    uint64_t ptile = end;
    if (warp == 0) {
        ptile = next(first);
        for (uint32_t s = 0; s < A.nstages; ++s) {
            const uint64_t pt = skip ? ptile : first + s * stride;
            if (pt < staged_end && lane == 0) issue(stages + s * A.stage_bytes, &bars[s], pt);
            if (skip && ptile < end) ptile = next(ptile + stride);
        }
    }
    const uint32_t nslices = A.tile_rows / kSlice;
    uint64_t tile = next(first);
    uint64_t it = 0;
    for (;; ++it) {
        if (tile >= end) {
            if (tid == 0)
                for (uint32_t s = 0; s < A.nstages; ++s) mbar_inval(smem_u32(&bars[s]));
            return true;
        }
        const bool staged = tile < A.nstaged;
        const uint32_t stage = static_cast<uint32_t>(it % A.nstages);
        bool fail = false;
        if (staged)
            fail = !mbar_wait_bounded(smem_u32(&bars[stage]), static_cast<uint32_t>((it / A.nstages) & 1),
                                      A.timeout_ns);
        if (!fail) {
            const unsigned char* sbuf = stages + stage * A.stage_bytes;
            const uint64_t tile_row0 = tile * A.tile_rows;
            const bool tile_full = tile_row0 + A.tile_rows <= A.nrows;
            for (uint32_t j = warp; j < nslices; j += kWarps) {
                const uint64_t slice0 = tile_row0 + static_cast<uint64_t>(j) * kSlice;
                if (slice0 >= A.nrows) break;
                body(staged, sbuf, j, slice0, tile_full);
            }
        }
        if (__syncthreads_or(fail)) break;
        if (warp == 0) {
            const uint64_t pt = skip ? ptile : tile + A.nstages * stride;
            if (pt < staged_end && lane == 0) issue(stages + stage * A.stage_bytes, &bars[stage], pt);
            if (skip && ptile < end) ptile = next(ptile + stride);
        }
        tile = next(tile + stride);
    }
    if (warp == 0) {
        if (lane == 0) atomicOr(A.status, kStatusTimeout);
        // let this CTA's copies in flight (the tiles from the failed one on)
        // land before its shared memory is left
        uint64_t t2 = tile;
        for (uint32_t k = 0; k < A.nstages; ++k) {
            const uint64_t it2 = it + k;
            if (t2 < staged_end && lane == 0)
                mbar_wait_bounded(smem_u32(&bars[it2 % A.nstages]), static_cast<uint32_t>((it2 / A.nstages) & 1),
                                  A.timeout_ns);
            if (t2 < end) t2 = next(t2 + stride);
        }
    }
    return false;
}

// Every tile live: the pipeline without tile skipping.
struct AllTiles {
    __device__ __forceinline__ bool operator()(uint64_t) const { return true; }
};

}  // namespace dev
}  // namespace gace
