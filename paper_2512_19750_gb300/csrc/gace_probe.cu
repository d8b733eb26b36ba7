// gace_probe.cu -- K1: fused predicate-batch scan over device-resident columns.
//
// The Measurement Engine probe (Section III-B of the paper) counts the rows of
// a full table, a seeded row sample or a seeded block sample on which each
// candidate conjunction holds; Section IV-I evaluates the candidates with a
// per-row bitmask ("Key-Only + Bitmask").  Here one pass evaluates a whole
// batch on up to eight row sets at once:
//
//   * each CTA owns a strided set of row tiles; one thread streams the tiles of
//     the referenced columns only into shared memory with bulk async copies
//     (cp.async.bulk + mbarrier transaction counts), `nstages` tiles ahead;
//   * a warp takes 128-row slices, four consecutive rows per lane; each term is
//     evaluated per row and turned into 32-row bit masks with __ballot_sync
//     (the bitmask of the paper), four masks per term per slice;
//   * lanes then take predicates (and terms, for marginals): a predicate's mask
//     is the AND of its terms' masks, counted with __popc against each row
//     set's membership mask, and added to 32-bit shared counters;
//   * counters go to the global 64-bit totals once per CTA at the end.
//
// Row-set membership is a counter-based hash of the global row (or block) id,
// so samples do not depend on tiling.  Nothing spins without a limit: every
// mbarrier wait gives up after the context's timeout and reports it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"

namespace gace {
namespace {

using namespace dev;

constexpr int kThreads = kProbeWarps * 32;

__device__ __forceinline__ void issue_tile(const ProbeArgs& A, unsigned char* stage_base,
                                           uint64_t* bar, uint64_t tile) {
    const uint32_t b = smem_u32(bar);
    mbar_arrive_expect_tx(b, A.stage_bytes);
    const uint64_t row0 = tile * A.tile_rows;
    for (uint32_t s = 0; s < A.nslots; ++s) {
        const SlotDesc& sd = A.slots[s];
        const unsigned char* src =
            static_cast<const unsigned char*>(sd.ptr) + row0 * sd.width;
        bulk_g2s(smem_u32(stage_base + sd.soff), src, A.tile_rows * sd.width, b);
    }
}

// Membership masks of the slice's 128 rows in every row set.
__device__ __forceinline__ void set_masks(const ProbeArgs& A, uint64_t row0, uint4* keep,
                                          int lane) {
    bool valid[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) valid[r] = row0 + r < A.nrows;
    uint64_t h[4] = {0, 0, 0, 0};
    for (uint32_t q = 0; q < A.nsets; ++q) {
        const SetDesc& sd = A.sets[q];
        bool k[4];
        if (sd.kind == 0 || sd.mode == 1) {
#pragma unroll
            for (int r = 0; r < 4; ++r) k[r] = valid[r];
        } else if (sd.mode == 0) {
#pragma unroll
            for (int r = 0; r < 4; ++r) k[r] = false;
        } else {
            if (!sd.share_prev) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    uint64_t x = row0 + r;
                    if (sd.kind == 2)
                        x = sd.block_shift >= 0 ? (x >> sd.block_shift) : (x / sd.block_rows);
                    h[r] = splitmix64(x ^ sd.seedhash);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) k[r] = valid[r] && (h[r] < sd.thresh);
        }
        uint4 m;
        m.x = __ballot_sync(kFullMask, k[0]);
        m.y = __ballot_sync(kFullMask, k[1]);
        m.z = __ballot_sync(kFullMask, k[2]);
        m.w = __ballot_sync(kFullMask, k[3]);
        if (lane == 0) keep[q] = m;
    }
}

// Evaluates the terms of one column slot on the lane's four rows and stores
// the warp's four 32-row masks per term.
__device__ __forceinline__ void eval_slot(const SlotDesc& sd, const Quad& v, const DevTerm* st,
                                          const uint32_t* pool, uint4* tm, int lane) {
    if (sd.dtype == 0) {
        for (uint32_t t = sd.rbeg; t < sd.rend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            uint4 m;
            m.x = __ballot_sync(kFullMask, (v.lo[0] - c.x) <= c.y);
            m.y = __ballot_sync(kFullMask, (v.lo[1] - c.x) <= c.y);
            m.z = __ballot_sync(kFullMask, (v.lo[2] - c.x) <= c.y);
            m.w = __ballot_sync(kFullMask, (v.lo[3] - c.x) <= c.y);
            if (lane == 0) tm[t] = m;
        }
        for (uint32_t t = sd.rend; t < sd.iend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            bool h0 = false, h1 = false, h2 = false, h3 = false;
            for (uint32_t k = 0; k < c.y; ++k) {
                const uint32_t x = pool[c.x + k];
                h0 |= v.lo[0] == x;
                h1 |= v.lo[1] == x;
                h2 |= v.lo[2] == x;
                h3 |= v.lo[3] == x;
            }
            uint4 m;
            m.x = __ballot_sync(kFullMask, h0);
            m.y = __ballot_sync(kFullMask, h1);
            m.z = __ballot_sync(kFullMask, h2);
            m.w = __ballot_sync(kFullMask, h3);
            if (lane == 0) tm[t] = m;
        }
    } else if (sd.dtype == 1) {
        uint64_t x[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) x[r] = join64(v.lo[r], v.hi[r]);
        for (uint32_t t = sd.rbeg; t < sd.rend; ++t) {
            const DevTerm c = st[t];
            const uint64_t lo = join64(c.a_lo, c.a_hi), span = join64(c.b_lo, c.b_hi);
            uint4 m;
            m.x = __ballot_sync(kFullMask, (x[0] - lo) <= span);
            m.y = __ballot_sync(kFullMask, (x[1] - lo) <= span);
            m.z = __ballot_sync(kFullMask, (x[2] - lo) <= span);
            m.w = __ballot_sync(kFullMask, (x[3] - lo) <= span);
            if (lane == 0) tm[t] = m;
        }
        for (uint32_t t = sd.rend; t < sd.iend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            bool h0 = false, h1 = false, h2 = false, h3 = false;
            for (uint32_t k = 0; k < c.y; ++k) {
                const uint64_t y = join64(pool[c.x + 2 * k], pool[c.x + 2 * k + 1]);
                h0 |= x[0] == y;
                h1 |= x[1] == y;
                h2 |= x[2] == y;
                h3 |= x[3] == y;
            }
            uint4 m;
            m.x = __ballot_sync(kFullMask, h0);
            m.y = __ballot_sync(kFullMask, h1);
            m.z = __ballot_sync(kFullMask, h2);
            m.w = __ballot_sync(kFullMask, h3);
            if (lane == 0) tm[t] = m;
        }
    } else {
        float x[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) x[r] = __uint_as_float(v.lo[r]);
        for (uint32_t t = sd.rbeg; t < sd.rend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            const float lo = __uint_as_float(c.x), hi = __uint_as_float(c.y);
            uint4 m;
            m.x = __ballot_sync(kFullMask, x[0] >= lo && x[0] <= hi);
            m.y = __ballot_sync(kFullMask, x[1] >= lo && x[1] <= hi);
            m.z = __ballot_sync(kFullMask, x[2] >= lo && x[2] <= hi);
            m.w = __ballot_sync(kFullMask, x[3] >= lo && x[3] <= hi);
            if (lane == 0) tm[t] = m;
        }
        for (uint32_t t = sd.rend; t < sd.iend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            bool h0 = false, h1 = false, h2 = false, h3 = false;
            for (uint32_t k = 0; k < c.y; ++k) {
                const float y = __uint_as_float(pool[c.x + k]);
                h0 |= x[0] == y;
                h1 |= x[1] == y;
                h2 |= x[2] == y;
                h3 |= x[3] == y;
            }
            uint4 m;
            m.x = __ballot_sync(kFullMask, h0);
            m.y = __ballot_sync(kFullMask, h1);
            m.z = __ballot_sync(kFullMask, h2);
            m.w = __ballot_sync(kFullMask, h3);
            if (lane == 0) tm[t] = m;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_probe(const __grid_constant__ ProbeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* stages = smem + A.off_stage;
    DevTerm* st = reinterpret_cast<DevTerm*>(smem + A.off_terms);
    uint32_t* spool = reinterpret_cast<uint32_t*>(smem + A.off_pool);
    uint32_t* spoff = reinterpret_cast<uint32_t*>(smem + A.off_poff);
    uint32_t* spterm = reinterpret_cast<uint32_t*>(smem + A.off_pterm);
    uint4* tm = reinterpret_cast<uint4*>(smem + A.off_tm) + warp * A.nterms;
    uint4* keep = reinterpret_cast<uint4*>(smem + A.off_keep) + warp * A.nsets;
    uint32_t* scnt = reinterpret_cast<uint32_t*>(smem + A.off_cnt);
    uint32_t* smarg = reinterpret_cast<uint32_t*>(smem + A.off_marg);
    uint32_t* sns = reinterpret_cast<uint32_t*>(smem + A.off_ns);

    for (uint32_t i = tid; i < A.nterms; i += kThreads) st[i] = A.terms[i];
    for (uint32_t i = tid; i < A.npool; i += kThreads) spool[i] = A.pool[i];
    for (uint32_t i = tid; i <= A.npreds; i += kThreads) spoff[i] = A.pred_off[i];
    for (uint32_t i = tid; i < A.npredterms; i += kThreads) spterm[i] = A.pred_terms[i];
    for (uint32_t i = tid; i < A.nsets * A.npreds; i += kThreads) scnt[i] = 0;
    if (A.want_marg)
        for (uint32_t i = tid; i < A.nsets * A.nterms; i += kThreads) smarg[i] = 0;
    for (uint32_t i = tid; i < A.nsets; i += kThreads) sns[i] = 0;
    if (tid == 0) {
        for (uint32_t s = 0; s < A.nstages; ++s) mbar_init(smem_u32(&bars[s]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint64_t stride = gridDim.x;
    if (tid == 0) {
        for (uint32_t s = 0; s < A.nstages; ++s) {
            const uint64_t tile = blockIdx.x + s * stride;
            if (tile < A.nstaged) issue_tile(A, stages + s * A.stage_bytes, &bars[s], tile);
        }
    }

    const uint32_t nslices = A.tile_rows / kSliceRows;
    uint64_t it = 0;
    bool aborted = false;
    for (;; ++it) {
        const uint64_t tile = blockIdx.x + it * stride;
        if (tile >= A.ntiles) break;
        const bool staged = tile < A.nstaged;
        const uint32_t stage = static_cast<uint32_t>(it % A.nstages);
        bool fail = false;
        if (staged)
            fail = !mbar_wait_bounded(smem_u32(&bars[stage]),
                                      static_cast<uint32_t>((it / A.nstages) & 1), A.timeout_ns);
        if (!fail) {
            const unsigned char* sbuf = stages + stage * A.stage_bytes;
            const uint64_t tile_row0 = tile * A.tile_rows;
            for (uint32_t j = warp; j < nslices; j += kProbeWarps) {
                const uint64_t slice0 = tile_row0 + static_cast<uint64_t>(j) * kSliceRows;
                if (slice0 >= A.nrows) break;
                const uint64_t row0 = slice0 + 4u * lane;
                set_masks(A, row0, keep, lane);
                for (uint32_t s = 0; s < A.nslots; ++s) {
                    const SlotDesc& sd = A.slots[s];
                    Quad v;
                    if (staged)
                        load_quad_smem(sbuf + sd.soff + (j * kSliceRows + 4u * lane) * sd.width,
                                       sd.width, v);
                    else
                        load_quad_global(sd.ptr, sd.width, row0, A.nrows, v);
                    eval_slot(sd, v, st, spool, tm, lane);
                }
                __syncwarp();
                for (uint32_t p = lane; p < A.npreds; p += 32) {
                    const uint32_t b = spoff[p], e = spoff[p + 1];
                    uint4 acc = tm[spterm[b]];
                    for (uint32_t k = b + 1; k < e; ++k) acc = and4(acc, tm[spterm[k]]);
                    for (uint32_t q = 0; q < A.nsets; ++q) {
                        const uint32_t c = popc4(acc, keep[q]);
                        if (c) atomicAdd(&scnt[q * A.npreds + p], c);
                    }
                }
                if (A.want_marg) {
                    for (uint32_t t = lane; t < A.nterms; t += 32) {
                        const uint4 m = tm[t];
                        for (uint32_t q = 0; q < A.nsets; ++q) {
                            const uint32_t c = popc4(m, keep[q]);
                            if (c) atomicAdd(&smarg[q * A.nterms + t], c);
                        }
                    }
                }
                if (lane < A.nsets) {
                    const uint4 k = keep[lane];
                    atomicAdd(&sns[lane], __popc(k.x) + __popc(k.y) + __popc(k.z) + __popc(k.w));
                }
                __syncwarp();
            }
        }
        if (__syncthreads_or(fail)) {
            aborted = true;
            break;
        }
        if (tid == 0) {
            const uint64_t next = tile + A.nstages * stride;
            if (next < A.nstaged) issue_tile(A, stages + stage * A.stage_bytes, &bars[stage], next);
        }
    }

    if (aborted) {
        if (tid == 0) {
            atomicOr(A.status, kStatusTimeout);
            // let this CTA's copies in flight land before its shared memory goes away
            for (uint32_t k = 0; k < A.nstages; ++k) {
                const uint64_t it2 = it + k;
                const uint64_t tile2 = blockIdx.x + it2 * stride;
                if (tile2 < A.nstaged)
                    mbar_wait_bounded(smem_u32(&bars[it2 % A.nstages]),
                                      static_cast<uint32_t>((it2 / A.nstages) & 1), A.timeout_ns);
            }
        }
        return;
    }

    __syncthreads();
    for (uint32_t i = tid; i < A.nsets * A.npreds; i += kThreads) {
        const uint32_t v = scnt[i];
        if (v) atomicAdd(&A.counts[i], static_cast<unsigned long long>(v));
    }
    if (A.want_marg) {
        for (uint32_t i = tid; i < A.nsets * A.nterms; i += kThreads) {
            const uint32_t v = smarg[i];
            if (v) atomicAdd(&A.marg[i], static_cast<unsigned long long>(v));
        }
    }
    for (uint32_t i = tid; i < A.nsets; i += kThreads)
        if (sns[i]) atomicAdd(&A.nsamp[i], static_cast<unsigned long long>(sns[i]));
}

uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

}  // namespace

uint32_t probe_layout(ProbeArgs& a) {
    uint32_t off = align_up(kMaxStages * 8, 128);
    a.off_stage = off;
    off += a.nstages * a.stage_bytes;
    off = align_up(off, 16);
    a.off_terms = off;
    off += a.nterms * 16;
    a.off_pool = off;
    off = align_up(off + a.npool * 4, 16);
    a.off_poff = off;
    off += (a.npreds + 1) * 4;
    a.off_pterm = off;
    off = align_up(off + a.npredterms * 4, 16);
    a.off_tm = off;
    off += kProbeWarps * a.nterms * 16;
    a.off_keep = off;
    off += kProbeWarps * a.nsets * 16;
    a.off_cnt = off;
    off += a.nsets * a.npreds * 4;
    a.off_marg = off;
    off += a.want_marg ? a.nsets * a.nterms * 4 : 0;
    a.off_ns = off;
    off = align_up(off + a.nsets * 4, 16);
    a.smem_bytes = off;
    return off;
}

cudaError_t probe_configure() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

int probe_occupancy(const ProbeArgs& a) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe, kThreads, a.smem_bytes) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t probe_launch(const ProbeArgs& a, int grid, cudaStream_t s) {
    k_probe<<<grid, kThreads, a.smem_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gace
