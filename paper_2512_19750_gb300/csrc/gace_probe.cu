// gace_probe.cu -- K1: fused predicate-batch scan over device-resident columns.
//
// The Measurement Engine probe (Section III-B of the paper) counts the rows of
// a full table, a seeded row sample or a seeded block sample on which each
// candidate conjunction holds; Section IV-H evaluates the candidates with a
// per-row bitmask ("Key-Only + Bitmask").  One pass evaluates a whole batch on
// up to eight row sets at once.  A warp takes 128-row slices, four
// consecutive rows per lane; each term becomes four 32-row bit masks through
// __ballot_sync, and a predicate's mask is the AND of its terms' masks,
// counted with __popc against each row set's membership mask.  Row-set
// membership is a counter-based hash of the global row (or block) id, so
// samples do not depend on tiling.
//
// Two kernels share that core:
//   k_probe_narrow  a batch of at most 32 predicates and 32 distinct terms (the
//                   single probes the gate issues): one thread streams tiles of
//                   the referenced columns into shared memory with bulk async
//                   copies (cp.async.bulk + mbarrier transaction counts) a few
//                   tiles ahead; lane p keeps predicate p's counts in registers.
//                   Small stages keep many CTAs per SM so the scan is HBM-bound.
//   k_probe_wide    larger batches, split on the host into passes of at most
//                   256 predicates / 256 terms: direct vectorised loads (the
//                   pass is ALU-bound), unrolled term evaluation, lanes take
//                   predicates and add to 32-bit shared counters.
// Counters reach the global 64-bit totals once per CTA.  No wait spins without
// a limit: every mbarrier wait gives up after the context's timeout.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"
#include "gace_probe_dev.cuh"

namespace gace {
namespace {

using namespace dev;
using namespace probe_dev;

// ---------------------------------------------------------------- narrow

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

// The staged tile pipeline shared by the narrow kernels: one thread keeps
// `nstages` bulk copies of the referenced columns in flight; each warp runs
// `body(staged, sbuf, j, slice0, tile_full)` on its slices of every tile.  The
// last (partial) tile, and every tile when a column is not 16-byte aligned, is
// read with plain loads by the body.  Returns false when a wait gave up (the
// status bit is set and the CTA's copies in flight have been waited for).
template <uint32_t kSlice, class Body>
__device__ __forceinline__ bool run_tiles(const ProbeArgs& A, const Smem& S, int tid, int warp,
                                          Body&& body) {
    if (tid == 0) {
        for (uint32_t s = 0; s < A.nstages; ++s) mbar_init(smem_u32(&S.bars[s]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t stride = gridDim.x;
    if (tid == 0) {
        for (uint32_t s = 0; s < A.nstages; ++s) {
            const uint64_t tile = blockIdx.x + s * stride;
            if (tile < A.nstaged) issue_tile(A, S.stages + s * A.stage_bytes, &S.bars[s], tile);
        }
    }
    const uint32_t nslices = A.tile_rows / kSlice;
    uint64_t it = 0;
    for (;; ++it) {
        const uint64_t tile = blockIdx.x + it * stride;
        if (tile >= A.ntiles) return true;
        const bool staged = tile < A.nstaged;
        const uint32_t stage = static_cast<uint32_t>(it % A.nstages);
        bool fail = false;
        if (staged)
            fail = !mbar_wait_bounded(smem_u32(&S.bars[stage]),
                                      static_cast<uint32_t>((it / A.nstages) & 1), A.timeout_ns);
        if (!fail) {
            const unsigned char* sbuf = S.stages + stage * A.stage_bytes;
            const uint64_t tile_row0 = tile * A.tile_rows;
            const bool tile_full = tile_row0 + A.tile_rows <= A.nrows;
            for (uint32_t j = warp; j < nslices; j += kProbeWarps) {
                const uint64_t slice0 = tile_row0 + static_cast<uint64_t>(j) * kSlice;
                if (slice0 >= A.nrows) break;
                body(staged, sbuf, j, slice0, tile_full);
            }
        }
        if (__syncthreads_or(fail)) break;
        if (tid == 0) {
            const uint64_t next = tile + A.nstages * stride;
            if (next < A.nstaged) issue_tile(A, S.stages + stage * A.stage_bytes, &S.bars[stage], next);
        }
    }
    if (tid == 0) {
        atomicOr(A.status, kStatusTimeout);
        // let this CTA's copies in flight land before its shared memory goes away
        for (uint32_t k = 0; k < A.nstages; ++k) {
            const uint64_t it2 = it + k;
            const uint64_t tile2 = blockIdx.x + it2 * stride;
            if (tile2 < A.nstaged)
                mbar_wait_bounded(smem_u32(&S.bars[it2 % A.nstages]),
                                  static_cast<uint32_t>((it2 / A.nstages) & 1), A.timeout_ns);
        }
    }
    return false;
}

// HASH: some row set is a hashed sample (else the only device set is "all rows",
// whose mask is the validity mask, all ones on full tiles).  MAXS: sets held
// in registers per lane.
template <bool HASH, int MAXS>
__global__ void __launch_bounds__(kThreads, 4) k_probe_narrow(const __grid_constant__ ProbeArgs A) {
    constexpr int NQ = 2;
    constexpr uint32_t kSlice = 128 * NQ;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid);
    __syncthreads();  // the tables are read below, before the pipeline's own barrier

    // lane-owned counters: predicate `lane`, term `lane`, row set `lane`
    uint32_t cnt[MAXS], mc[MAXS];
#pragma unroll
    for (int q = 0; q < MAXS; ++q) cnt[q] = mc[q] = 0;
    uint32_t nsr = 0;
    const bool has_pred = lane < static_cast<int>(A.npreds);
    const bool has_term = A.want_marg && lane < static_cast<int>(A.nterms);
    const uint32_t pb = has_pred ? S.poff[lane] : 0, pe = has_pred ? S.poff[lane + 1] : 0;
    const uint32_t nsets = HASH ? A.nsets : 1;

    const bool ok = run_tiles<kSlice>(A, S, tid, warp, [&](bool staged, const unsigned char* sbuf, uint32_t j,
                                                           uint64_t slice0, bool tile_full) {
        uint4 vm[NQ];
        if (HASH) {
            set_masks<NQ>(A, slice0, S.keep, lane);
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
    if (!ok) return;
    // warps -> CTA counters -> global
#pragma unroll
    for (int q = 0; q < MAXS; ++q) {
        if (q < static_cast<int>(nsets)) {
            if (has_pred && cnt[q]) atomicAdd(&S.cnt[q * A.npreds + lane], cnt[q]);
            if (has_term && mc[q]) atomicAdd(&S.marg[q * A.nterms + lane], mc[q]);
        }
    }
    if (HASH && lane < static_cast<int>(nsets) && nsr) atomicAdd(&S.ns[lane], nsr);
    __syncthreads();
    flush(A, S, tid);
}

// Bit i of the result: per-row predicate `pred_expr(i)` for the lane's 4 NQ rows.
#define GACE_ROWBITS(R_, pred_expr, out)               \
    do {                                               \
        out = 0u;                                      \
        _Pragma("unroll") for (int i_ = 0; i_ < R_; ++i_) \
            if (pred_expr(i_)) out |= 1u << i_;        \
    } while (0)

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
// terms of its eight rows in predicate registers and counts the rows that pass;
// no per-term masks go through shared memory.  HASH: the set is a hashed sample.
template <bool HASH>
__global__ void __launch_bounds__(kThreads, 4) k_probe_single(const __grid_constant__ ProbeArgs A) {
    constexpr int NQ = 2, R = 4 * NQ;
    constexpr uint32_t kSlice = 128 * NQ;
    constexpr uint32_t kAll = (1u << R) - 1u;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid);
    __syncthreads();
    uint32_t cnt = 0, nsr = 0, tc = 0;
    const bool marg = A.want_marg != 0;

    const bool ok_run = run_tiles<kSlice>(A, S, tid, warp, [&](bool staged, const unsigned char* sbuf, uint32_t j,
                                                               uint64_t slice0, bool tile_full) {
        // bit i: row slice0 + 128 (i / 4) + 4 lane + i % 4 is in the row set
        uint32_t base = kAll;
        if (HASH) {
            const SetDesc& sd = A.sets[0];
            base = 0u;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const uint64_t row = slice0 + 128u * (i / 4) + 4u * lane + (i % 4);
                uint64_t x = row;
                if (sd.kind == 2) x = sd.block_shift >= 0 ? (row >> sd.block_shift) : (row / sd.block_rows);
                if (row < A.nrows && splitmix64(x ^ sd.seedhash) < sd.thresh) base |= 1u << i;
            }
        } else if (!tile_full) {
#define PV(i) (slice0 + 128u * ((i) / 4) + 4u * lane + ((i) % 4) < A.nrows)
            GACE_ROWBITS(R, PV, base);
#undef PV
        }
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
    if (!ok_run) return;
    cnt = __reduce_add_sync(kFullMask, cnt);
    nsr = __reduce_add_sync(kFullMask, nsr);
    if (lane == 0 && cnt) atomicAdd(&S.cnt[0], cnt);
    if (HASH && lane == 0 && nsr) atomicAdd(&S.ns[0], nsr);
    if (marg && lane < static_cast<int>(A.nterms) && tc) atomicAdd(&S.marg[lane], tc);
    __syncthreads();
    flush(A, S, tid);
}

__global__ void __launch_bounds__(kThreads) k_probe_wide(const __grid_constant__ ProbeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid);
    __syncthreads();
    const uint64_t nslices = (A.nrows + kSliceRows - 1) / kSliceRows;
    const uint32_t nsr = wide_slices(A, S, lane, static_cast<uint64_t>(blockIdx.x) * kProbeWarps + warp, nslices,
                                     static_cast<uint64_t>(gridDim.x) * kProbeWarps);
    if (lane < static_cast<int>(A.nsets) && nsr) atomicAdd(&S.ns[lane], nsr);
    __syncthreads();
    flush(A, S, tid);
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
    const uint32_t nq = a.narrow ? 2 : 1;  // quads per lane
    a.off_tm = off;
    off += kProbeWarps * a.nterms * 16 * nq;
    a.off_keep = off;
    off += kProbeWarps * a.nsets * 16 * nq;
    a.off_cnt = off;
    off += a.nsets * a.npreds * 4;
    a.off_marg = off;
    off += a.want_marg ? a.nsets * a.nterms * 4 : 0;
    a.off_ns = off;
    off = align_up(off + a.nsets * 4, 16);
    a.smem_bytes = off;
    return off;
}

template <typename K>
static cudaError_t set_smem(K kernel, int optin) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

// 0: wide, 1: narrow all rows, 2: narrow hashed single set, 3: narrow hashed
// sets, 4: single predicate on all rows, 5: single predicate on one hashed set
static int variant(const ProbeArgs& a) {
    if (!a.narrow) return 0;
    bool hash = false;
    for (uint32_t q = 0; q < a.nsets; ++q)
        if (a.sets[q].mode == 2) hash = true;
    // the single kernel ANDs every term of the pass: only when the one predicate uses them all
    if (a.npreds == 1 && a.nsets == 1 && a.npredterms == a.nterms) return hash ? 5 : 4;
    if (!hash) return 1;
    return a.nsets == 1 ? 2 : 3;
}

cudaError_t probe_configure() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((e = set_smem(k_probe_narrow<false, 1>, optin))) return e;
    if ((e = set_smem(k_probe_narrow<true, 1>, optin))) return e;
    if ((e = set_smem(k_probe_narrow<true, kMaxSets>, optin))) return e;
    if ((e = set_smem(k_probe_single<false>, optin))) return e;
    if ((e = set_smem(k_probe_single<true>, optin))) return e;
    return set_smem(k_probe_wide, optin);
}

int probe_occupancy(const ProbeArgs& a) {
    int n = 0;
    cudaError_t e = cudaSuccess;
    switch (variant(a)) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_wide, kThreads, a.smem_bytes); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_narrow<false, 1>, kThreads, a.smem_bytes); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_narrow<true, 1>, kThreads, a.smem_bytes); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_narrow<true, kMaxSets>, kThreads, a.smem_bytes); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_single<false>, kThreads, a.smem_bytes); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_single<true>, kThreads, a.smem_bytes); break;
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t probe_launch(const ProbeArgs& a, int grid, cudaStream_t s) {
    switch (variant(a)) {
        case 0: k_probe_wide<<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 1: k_probe_narrow<false, 1><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 2: k_probe_narrow<true, 1><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 3: k_probe_narrow<true, kMaxSets><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 4: k_probe_single<false><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        default: k_probe_single<true><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace gace
