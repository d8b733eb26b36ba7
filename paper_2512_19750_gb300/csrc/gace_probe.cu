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

namespace gace {
namespace {

using namespace dev;

constexpr int kThreads = kProbeWarps * 32;

struct Smem {
    uint64_t* bars;
    unsigned char* stages;
    DevTerm* st;
    uint32_t* pool;
    uint32_t* poff;
    uint32_t* pterm;
    uint4* tm;    // this warp's term masks
    uint4* keep;  // this warp's row-set masks
    uint32_t* cnt;
    uint32_t* marg;
    uint32_t* ns;
};

__device__ __forceinline__ Smem carve(const ProbeArgs& A, unsigned char* smem, int warp) {
    Smem s;
    s.bars = reinterpret_cast<uint64_t*>(smem);
    s.stages = smem + A.off_stage;
    s.st = reinterpret_cast<DevTerm*>(smem + A.off_terms);
    s.pool = reinterpret_cast<uint32_t*>(smem + A.off_pool);
    s.poff = reinterpret_cast<uint32_t*>(smem + A.off_poff);
    s.pterm = reinterpret_cast<uint32_t*>(smem + A.off_pterm);
    const uint32_t nq = A.narrow ? 2 : 1;
    s.tm = reinterpret_cast<uint4*>(smem + A.off_tm) + warp * A.nterms * nq;
    s.keep = reinterpret_cast<uint4*>(smem + A.off_keep) + warp * A.nsets * nq;
    s.cnt = reinterpret_cast<uint32_t*>(smem + A.off_cnt);
    s.marg = reinterpret_cast<uint32_t*>(smem + A.off_marg);
    s.ns = reinterpret_cast<uint32_t*>(smem + A.off_ns);
    return s;
}

// Copies the pass tables into shared memory and zeroes the CTA counters.
__device__ __forceinline__ void load_tables(const ProbeArgs& A, const Smem& s, int tid) {
    for (uint32_t i = tid; i < A.nterms; i += kThreads) s.st[i] = A.terms[i];
    for (uint32_t i = tid; i < A.npool; i += kThreads) s.pool[i] = A.pool[i];
    for (uint32_t i = tid; i <= A.npreds; i += kThreads) s.poff[i] = A.pred_off[i];
    for (uint32_t i = tid; i < A.npredterms; i += kThreads) s.pterm[i] = A.pred_terms[i];
    for (uint32_t i = tid; i < A.nsets * A.npreds; i += kThreads) s.cnt[i] = 0;
    if (A.want_marg)
        for (uint32_t i = tid; i < A.nsets * A.nterms; i += kThreads) s.marg[i] = 0;
    for (uint32_t i = tid; i < A.nsets; i += kThreads) s.ns[i] = 0;
}

// CTA counters -> global 64-bit totals (zeros skipped).
__device__ __forceinline__ void flush(const ProbeArgs& A, const Smem& s, int tid) {
    for (uint32_t i = tid; i < A.nsets * A.npreds; i += kThreads) {
        const uint32_t v = s.cnt[i];
        if (v) atomicAdd(&A.counts[i], static_cast<unsigned long long>(v));
    }
    if (A.want_marg) {
        for (uint32_t i = tid; i < A.nsets * A.nterms; i += kThreads) {
            const uint32_t v = s.marg[i];
            if (v) atomicAdd(&A.marg[i], static_cast<unsigned long long>(v));
        }
    }
    for (uint32_t i = tid; i < A.nsets; i += kThreads)
        if (s.ns[i]) atomicAdd(&A.nsamp[i], static_cast<unsigned long long>(s.ns[i]));
}

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

// Ballots of a per-row predicate over the lane's 4 NQ rows: NQ masks of 4 x 32 rows.
#define GACE_BALLOTS(NQ_, pred_expr, out)                               \
    _Pragma("unroll") for (int h_ = 0; h_ < NQ_; ++h_) {               \
        out[h_].x = __ballot_sync(kFullMask, pred_expr(4 * h_ + 0));    \
        out[h_].y = __ballot_sync(kFullMask, pred_expr(4 * h_ + 1));    \
        out[h_].z = __ballot_sync(kFullMask, pred_expr(4 * h_ + 2));    \
        out[h_].w = __ballot_sync(kFullMask, pred_expr(4 * h_ + 3));    \
    }

// Membership masks of a slice's rows in every row set: keep[q * NQ + h].
template <int NQ>
__device__ __forceinline__ void set_masks(const ProbeArgs& A, uint64_t slice0, uint4* keep,
                                          int lane) {
    constexpr int R = 4 * NQ;
    bool valid[R];
    uint64_t row[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        row[i] = slice0 + 128u * (i / 4) + 4u * lane + (i % 4);
        valid[i] = row[i] < A.nrows;
    }
    uint64_t hsh[R];
#pragma unroll
    for (int i = 0; i < R; ++i) hsh[i] = 0;
    for (uint32_t q = 0; q < A.nsets; ++q) {
        const SetDesc& sd = A.sets[q];
        bool k[R];
        if (sd.kind == 0 || sd.mode == 1) {
#pragma unroll
            for (int i = 0; i < R; ++i) k[i] = valid[i];
        } else if (sd.mode == 0) {
#pragma unroll
            for (int i = 0; i < R; ++i) k[i] = false;
        } else {
            if (!sd.share_prev) {
                if (sd.kind == 1) {
#pragma unroll
                    for (int i = 0; i < R; ++i) hsh[i] = splitmix64(row[i] ^ sd.seedhash);
                } else if (sd.block_shift >= 2) {
                    // the four rows of a quad (a multiple of 4 apart from 0) share one block
#pragma unroll
                    for (int h = 0; h < NQ; ++h) {
                        const uint64_t hb = splitmix64((row[4 * h] >> sd.block_shift) ^ sd.seedhash);
#pragma unroll
                        for (int r = 0; r < 4; ++r) hsh[4 * h + r] = hb;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        const uint64_t b = sd.block_shift >= 0 ? (row[i] >> sd.block_shift) : (row[i] / sd.block_rows);
                        hsh[i] = splitmix64(b ^ sd.seedhash);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < R; ++i) k[i] = valid[i] && (hsh[i] < sd.thresh);
        }
        uint4 m[NQ];
#define PK(i) (k[i])
        GACE_BALLOTS(NQ, PK, m);
#undef PK
        if (lane == 0) {
#pragma unroll
            for (int h = 0; h < NQ; ++h) keep[q * NQ + h] = m[h];
        }
    }
}

template <int NQ>
__device__ __forceinline__ void store_masks(uint4* tm, uint32_t t, const uint4 (&m)[NQ], int lane) {
    if (lane == 0) {
#pragma unroll
        for (int h = 0; h < NQ; ++h) tm[t * NQ + h] = m[h];
    }
}

// Evaluates the terms of one column slot on the lane's 4 NQ rows and stores the
// warp's NQ x 4 masks of 32 rows per term at tm[t * NQ + h].
template <int NQ>
__device__ __forceinline__ void eval_slot(const SlotDesc& sd, const Vals<NQ>& v, const DevTerm* st,
                                          const uint32_t* pool, uint4* tm, int lane) {
    constexpr int R = 4 * NQ;
    if (sd.dtype == 0) {
        for (uint32_t t = sd.rbeg; t < sd.rend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            uint4 m[NQ];
#define PR(i) ((v.lo[i] - c.x) <= c.y)
            GACE_BALLOTS(NQ, PR, m);
#undef PR
            store_masks<NQ>(tm, t, m, lane);
        }
        for (uint32_t t = sd.rend; t < sd.iend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            bool hit[R];
#pragma unroll
            for (int i = 0; i < R; ++i) hit[i] = false;
            for (uint32_t k = 0; k < c.y; ++k) {
                const uint32_t x = pool[c.x + k];
#pragma unroll
                for (int i = 0; i < R; ++i) hit[i] |= v.lo[i] == x;
            }
            uint4 m[NQ];
#define PH(i) (hit[i])
            GACE_BALLOTS(NQ, PH, m);
#undef PH
            store_masks<NQ>(tm, t, m, lane);
        }
    } else if (sd.dtype == 1) {
        uint64_t x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = join64(v.lo[i], v.hi[i]);
        for (uint32_t t = sd.rbeg; t < sd.rend; ++t) {
            const DevTerm c = st[t];
            const uint64_t lo = join64(c.a_lo, c.a_hi), span = join64(c.b_lo, c.b_hi);
            uint4 m[NQ];
#define PR(i) ((x[i] - lo) <= span)
            GACE_BALLOTS(NQ, PR, m);
#undef PR
            store_masks<NQ>(tm, t, m, lane);
        }
        for (uint32_t t = sd.rend; t < sd.iend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            bool hit[R];
#pragma unroll
            for (int i = 0; i < R; ++i) hit[i] = false;
            for (uint32_t k = 0; k < c.y; ++k) {
                const uint64_t y = join64(pool[c.x + 2 * k], pool[c.x + 2 * k + 1]);
#pragma unroll
                for (int i = 0; i < R; ++i) hit[i] |= x[i] == y;
            }
            uint4 m[NQ];
#define PH(i) (hit[i])
            GACE_BALLOTS(NQ, PH, m);
#undef PH
            store_masks<NQ>(tm, t, m, lane);
        }
    } else {
        float x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = __uint_as_float(v.lo[i]);
        for (uint32_t t = sd.rbeg; t < sd.rend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            const float lo = __uint_as_float(c.x), hi = __uint_as_float(c.y);
            uint4 m[NQ];
#define PR(i) (x[i] >= lo && x[i] <= hi)
            GACE_BALLOTS(NQ, PR, m);
#undef PR
            store_masks<NQ>(tm, t, m, lane);
        }
        for (uint32_t t = sd.rend; t < sd.iend; ++t) {
            const uint2 c = *reinterpret_cast<const uint2*>(&st[t]);
            bool hit[R];
#pragma unroll
            for (int i = 0; i < R; ++i) hit[i] = false;
            for (uint32_t k = 0; k < c.y; ++k) {
                const float y = __uint_as_float(pool[c.x + k]);
#pragma unroll
                for (int i = 0; i < R; ++i) hit[i] |= x[i] == y;
            }
            uint4 m[NQ];
#define PH(i) (hit[i])
            GACE_BALLOTS(NQ, PH, m);
#undef PH
            store_masks<NQ>(tm, t, m, lane);
        }
    }
}

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

// ---------------------------------------------------------------- wide

// 32 x 32 bit transpose across a warp: lane i holds row i (bit j = M[i][j]);
// afterwards lane j holds column j (bit i = M[i][j]).  Five butterfly stages
// swap the off-diagonal blocks of halving size.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu
                         : s == 8  ? 0x00FF00FFu
                         : s == 4  ? 0x0F0F0F0Fu
                         : s == 2  ? 0x33333333u
                                   : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(kFullMask, x, s);
        x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
    }
    return x;
}

// Mask of the group's EQ/IN terms that hold for key (lo, hi): open addressing,
// linear probing; an entry with an empty mask ends the search.
__device__ __forceinline__ uint32_t vs_lookup(const uint32_t* tab, uint32_t cap, bool is64, uint32_t h,
                                              uint32_t lo, uint32_t hi) {
    for (uint32_t p = 0; p < cap; ++p) {
        const uint32_t at = (h + p) & (cap - 1);
        if (is64) {
            const uint4 e = reinterpret_cast<const uint4*>(tab)[at];
            if (e.z == 0) return 0;
            if (e.x == lo && e.y == hi) return e.z;
        } else {
            const uint2 e = reinterpret_cast<const uint2*>(tab)[at];
            if (e.y == 0) return 0;
            if (e.x == lo) return e.y;
        }
    }
    return 0;
}

// EQ and IN terms of one column slot in a wide pass: one table lookup per row
// gives the 32-bit mask of the group's terms that hold; a warp transpose of
// each row-group's masks hands lane t the 32-row mask of term t.
template <int NQ>
__device__ __forceinline__ void eval_valueset(const SlotDesc& sd, const Vals<NQ>& v, const uint32_t* pool,
                                              uint4* tm, int lane) {
    constexpr int R = 4 * NQ;
    const bool is64 = sd.dtype == 1;
    const uint32_t cap = 1u << sd.tlog;
    const uint32_t ew = is64 ? 4u : 2u;
    uint32_t klo[R], khi[R], hb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        klo[i] = v.lo[i];
        khi[i] = is64 ? v.hi[i] : 0u;
        if (sd.dtype == 2 && (klo[i] << 1) == 0) klo[i] = 0;  // -0 equals +0
        hb[i] = vs_hash(klo[i], khi[i], is64, sd.tlog);
    }
    const uint32_t nvs = sd.iend - sd.rend;
    for (uint32_t g = 0; g < sd.ngroups; ++g) {
        const uint32_t* tab = pool + sd.toff + g * cap * ew;
        uint32_t w[R];
#pragma unroll
        for (int i = 0; i < R; ++i) w[i] = vs_lookup(tab, cap, is64, hb[i], klo[i], khi[i]);
        uint4 out[NQ];
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            out[h].x = transpose32(w[4 * h + 0], lane);
            out[h].y = transpose32(w[4 * h + 1], lane);
            out[h].z = transpose32(w[4 * h + 2], lane);
            out[h].w = transpose32(w[4 * h + 3], lane);
        }
        const uint32_t k = 32u * g + lane;
        if (k < nvs) {
#pragma unroll
            for (int h = 0; h < NQ; ++h) tm[(sd.rend + k) * NQ + h] = out[h];
        }
    }
}


__global__ void __launch_bounds__(kThreads) k_probe_wide(const __grid_constant__ ProbeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid);
    __syncthreads();

    const uint64_t nslices = (A.nrows + kSliceRows - 1) / kSliceRows;
    const uint64_t wstride = static_cast<uint64_t>(gridDim.x) * kProbeWarps;
    uint32_t nsr = 0;
    for (uint64_t sl = static_cast<uint64_t>(blockIdx.x) * kProbeWarps + warp; sl < nslices; sl += wstride) {
        const uint64_t slice0 = sl * kSliceRows;
        set_masks<1>(A, slice0, S.keep, lane);
        for (uint32_t s = 0; s < A.nslots; ++s) {
            const SlotDesc& sd = A.slots[s];
            Vals<1> v;
            load_vals_global<1>(sd.ptr, sd.width, slice0, A.nrows, lane, v);
            SlotDesc ranges = sd;  // ranges by compare; EQ and IN terms by table
            ranges.iend = sd.rend;
            eval_slot<1>(ranges, v, S.st, S.pool, S.tm, lane);
            if (sd.iend > sd.rend) eval_valueset<1>(sd, v, S.pool, S.tm, lane);
        }
        __syncwarp();
        for (uint32_t p = lane; p < A.npreds; p += 32) {
            const uint32_t b = S.poff[p], e = S.poff[p + 1];
            uint4 acc = S.tm[S.pterm[b]];
            for (uint32_t k = b + 1; k < e; ++k) acc = and4(acc, S.tm[S.pterm[k]]);
            for (uint32_t q = 0; q < A.nsets; ++q) {
                const uint32_t c = popc4(acc, S.keep[q]);
                if (c) atomicAdd(&S.cnt[q * A.npreds + p], c);
            }
        }
        if (A.want_marg) {
            for (uint32_t t = lane; t < A.nterms; t += 32) {
                const uint4 m = S.tm[t];
                for (uint32_t q = 0; q < A.nsets; ++q) {
                    const uint32_t c = popc4(m, S.keep[q]);
                    if (c) atomicAdd(&S.marg[q * A.nterms + t], c);
                }
            }
        }
        if (lane < static_cast<int>(A.nsets)) {
            const uint4 k = S.keep[lane];
            nsr += __popc(k.x) + __popc(k.y) + __popc(k.z) + __popc(k.w);
        }
        __syncwarp();
    }
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
