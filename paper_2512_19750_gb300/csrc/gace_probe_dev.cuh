// gace_probe_dev.cuh -- device code of the predicate-batch probe shared by the
// probe kernels and the batched work-queue kernel (one definition, included by
// each translation unit that launches it).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"
#include "gace_stage.cuh"

namespace gace {
namespace probe_dev {

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

// Copies the pass tables into shared memory and zeroes the CTA counters
// (nthreads: the CTA's threads).
__device__ __forceinline__ void load_tables(const ProbeArgs& A, const Smem& s, int tid, int nthreads = kThreads) {
    for (uint32_t i = tid; i < A.nterms; i += nthreads) s.st[i] = A.terms[i];
    for (uint32_t i = tid; i < A.npool; i += nthreads) s.pool[i] = A.pool[i];
    for (uint32_t i = tid; i <= A.npreds; i += nthreads) s.poff[i] = A.pred_off[i];
    for (uint32_t i = tid; i < A.npredterms; i += nthreads) s.pterm[i] = A.pred_terms[i];
    for (uint32_t i = tid; i < A.nsets * A.npreds; i += nthreads) s.cnt[i] = 0;
    if (A.want_marg)
        for (uint32_t i = tid; i < A.nsets * A.nterms; i += nthreads) s.marg[i] = 0;
    for (uint32_t i = tid; i < A.nsets; i += nthreads) s.ns[i] = 0;
}

// CTA counters -> global 64-bit totals (zeros skipped).
__device__ __forceinline__ void flush(const ProbeArgs& A, const Smem& s, int tid, int nthreads = kThreads) {
    for (uint32_t i = tid; i < A.nsets * A.npreds; i += nthreads) {
        const uint32_t v = s.cnt[i];
        if (v) atomicAdd(&A.counts[i], static_cast<unsigned long long>(v));
    }
    if (A.want_marg) {
        for (uint32_t i = tid; i < A.nsets * A.nterms; i += nthreads) {
            const uint32_t v = s.marg[i];
            if (v) atomicAdd(&A.marg[i], static_cast<unsigned long long>(v));
        }
    }
    for (uint32_t i = tid; i < A.nsets; i += nthreads)
        if (s.ns[i]) atomicAdd(&A.nsamp[i], static_cast<unsigned long long>(s.ns[i]));
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
                // membership hashes the table-global row (or block) id
                if (sd.kind == 1) {
#pragma unroll
                    for (int i = 0; i < R; ++i) hsh[i] = splitmix64((A.row0 + row[i]) ^ sd.seedhash);
                } else if (sd.block_shift >= 2) {
                    // the four rows of a quad (a multiple of 4 apart from 0, and row0 a
                    // multiple of 4) share one block
#pragma unroll
                    for (int h = 0; h < NQ; ++h) {
                        const uint64_t hb = splitmix64(((A.row0 + row[4 * h]) >> sd.block_shift) ^ sd.seedhash);
#pragma unroll
                        for (int r = 0; r < 4; ++r) hsh[4 * h + r] = hb;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        const uint64_t g = A.row0 + row[i];
                        const uint64_t b = sd.block_shift >= 0 ? (g >> sd.block_shift) : (g / sd.block_rows);
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

// ---------------------------------------------------------------- wide

// 32 x 32 bit transpose across a warp: lane i holds row i (bit j = M[i][j]);
// afterwards lane j holds column j (bit i = M[i][j]).  Five butterfly stages
// swap the off-diagonal blocks of halving size s: a lane keeps the bits of its
// own half (mask M) and takes the partner's other half, rotated into place by
// s (lower lanes) or 32 - s (upper lanes); the bits a rotation wraps around
// land where M keeps the lane's own bits, so one funnel shift and one
// three-input logic operation do the stage.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu
                         : s == 8  ? 0x00FF00FFu
                         : s == 4  ? 0x0F0F0F0Fu
                         : s == 2  ? 0x33333333u
                                   : 0x55555555u;
        const bool up = (lane & s) != 0;
        const uint32_t y = __shfl_xor_sync(kFullMask, x, s);
        const uint32_t t = __funnelshift_l(y, y, up ? 32 - s : s);
        const uint32_t keep = up ? ~m : m;
        x = (x & keep) | (t & ~keep);
    }
    return x;
}

// The 128-row masks of a group of nt <= 32 terms from each lane's four row
// words (bit t of lane l's word i: term t holds for row 4 l + i): lane t gets
// term t's.  A group of at most 16 (8) terms packs two (four) row words into
// one word before the transpose, then fetches the other words of its term from
// the lanes 16 (8, 16, 24) above.  Bits of w above the group's terms are 0.
__device__ __forceinline__ uint4 transpose_group(const uint32_t (&w)[4], uint32_t nt, int lane) {
    uint4 o;
    if (nt <= 8) {
        const uint32_t x = transpose32(w[0] | (w[1] << 8) | (w[2] << 16) | (w[3] << 24), lane);
        o.x = x;
        o.y = __shfl_down_sync(kFullMask, x, 8);
        o.z = __shfl_down_sync(kFullMask, x, 16);
        o.w = __shfl_down_sync(kFullMask, x, 24);
    } else if (nt <= 16) {
        const uint32_t a = transpose32(w[0] | (w[1] << 16), lane);
        const uint32_t b = transpose32(w[2] | (w[3] << 16), lane);
        o.x = a;
        o.y = __shfl_down_sync(kFullMask, a, 16);
        o.z = b;
        o.w = __shfl_down_sync(kFullMask, b, 16);
    } else {
        o.x = transpose32(w[0], lane);
        o.y = transpose32(w[1], lane);
        o.z = transpose32(w[2], lane);
        o.w = transpose32(w[3], lane);
    }
    return o;
}

// Mask of the group's EQ/IN terms that hold for key (lo, hi): the masks of
// its two candidate slots whose key matches (an empty slot's mask is 0).
__device__ __forceinline__ uint32_t vs_lookup(const uint32_t* tab, bool is64, uint32_t s1, uint32_t s2, uint32_t lo,
                                              uint32_t hi) {
    if (is64) {
        const uint4 a = reinterpret_cast<const uint4*>(tab)[s1];
        const uint4 b = reinterpret_cast<const uint4*>(tab)[s2];
        return ((a.x == lo && a.y == hi) ? a.z : 0u) | ((b.x == lo && b.y == hi) ? b.z : 0u);
    }
    const uint2 a = reinterpret_cast<const uint2*>(tab)[s1];
    const uint2 b = reinterpret_cast<const uint2*>(tab)[s2];
    return (a.x == lo ? a.y : 0u) | (b.x == lo ? b.y : 0u);
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
    uint32_t klo[R], khi[R], s1[R], s2[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        klo[i] = v.lo[i];
        khi[i] = is64 ? v.hi[i] : 0u;
        if (sd.dtype == 2 && (klo[i] << 1) == 0) klo[i] = 0;  // -0 equals +0
        if (is64) {
            s1[i] = vs_slot(klo[i], khi[i], sd.vm1, sd.tlog);
            s2[i] = vs_slot(klo[i], khi[i], sd.vm2, sd.tlog);
        } else {  // vs_slot with a zero high word
            s1[i] = (klo[i] * sd.vm1) >> (32 - sd.tlog);
            s2[i] = (klo[i] * sd.vm2) >> (32 - sd.tlog);
        }
    }
    const uint32_t nvs = sd.iend - sd.rend;
    for (uint32_t g = 0; g < sd.ngroups; ++g) {
        const uint32_t* tab = pool + sd.toff + g * cap * ew;
        uint32_t w[R];
#pragma unroll
        for (int i = 0; i < R; ++i) w[i] = vs_lookup(tab, is64, s1[i], s2[i], klo[i], khi[i]);
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


// Order-preserving unsigned key of one value (the host's value_key): low word
// in lo, high word in hi (0 unless 64-bit).
__device__ __forceinline__ void value_key(uint32_t dtype, uint32_t vlo, uint32_t vhi, uint32_t& lo,
                                          uint32_t& hi) {
    if (dtype == 0) {
        lo = vlo ^ 0x80000000u;
        hi = 0;
    } else if (dtype == 1) {
        lo = vlo;
        hi = vhi ^ 0x80000000u;
    } else {
        uint32_t f = (vlo << 1) == 0 ? 0u : vlo;  // -0 is +0
        if ((f & 0x7FFFFFFFu) > 0x7F800000u)
            lo = 0;  // NaN: below every range
        else
            lo = (f & 0x80000000u) ? ~f : (f | 0x80000000u);
        hi = 0;
    }
}

// Range terms of one column slot in a wide pass: per group of 32, every row
// descends the group's interval tree (7 levels, level-order keys in shared
// memory, so a level's lanes read distinct banks) to the number of endpoints
// <= its key, which indexes the 32-bit mask of the group's terms that contain
// it; a warp transpose of each row-group's masks hands lane t the 32-row mask
// of term t.
template <int NQ>
__device__ __forceinline__ void eval_range_trees(const SlotDesc& sd, const Vals<NQ>& v, const uint32_t* pool,
                                                 uint4* tm, int lane) {
    constexpr int R = 4 * NQ;
    const bool is64 = sd.dtype == 1;
    uint32_t klo[R], khi[R];
#pragma unroll
    for (int i = 0; i < R; ++i) value_key(sd.dtype, v.lo[i], v.hi[i], klo[i], khi[i]);
    const uint32_t nr = sd.rtree;
    const uint32_t gw = is64 ? kTreeWords64 : kTreeWords32;
    for (uint32_t g = 0; g < sd.rgroups; ++g) {
        const uint32_t* tree = pool + sd.roff + g * gw;
        const uint32_t* masks = tree + (is64 ? 2 * kTreeNodes + 2 : kTreeNodes + 1);
        uint32_t w[R];
        if (is64) {
            const uint2* node = reinterpret_cast<const uint2*>(tree);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                uint32_t n = 1;
#pragma unroll
                for (int d = 0; d < kTreeLevels; ++d) {
                    const uint2 e = node[n - 1];
                    const bool ge = khi[i] > e.y || (khi[i] == e.y && klo[i] >= e.x);
                    n = 2 * n + (ge ? 1u : 0u);
                }
                w[i] = masks[n - (1u << kTreeLevels)];
            }
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                uint32_t n = 1;
#pragma unroll
                for (int d = 0; d < kTreeLevels; ++d) n = 2 * n + (klo[i] >= tree[n - 1] ? 1u : 0u);
                w[i] = masks[n - (1u << kTreeLevels)];
            }
        }
        uint4 out[NQ];
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            out[h].x = transpose32(w[4 * h + 0], lane);
            out[h].y = transpose32(w[4 * h + 1], lane);
            out[h].z = transpose32(w[4 * h + 2], lane);
            out[h].w = transpose32(w[4 * h + 3], lane);
        }
        const uint32_t k = 32u * g + lane;
        if (k < nr) {
#pragma unroll
            for (int h = 0; h < NQ; ++h) tm[(sd.rbeg + k) * NQ + h] = out[h];
        }
    }
}

// Range terms of a rank-coded column slot in a wide pass: each row's rank
// among the column's endpoints (rk, computed once per call) indexes the 32-bit
// mask of each group's terms that contain the row's value; a warp transpose of
// each row-group's masks hands lane t the 32-row mask of term t.
template <int NQ>
__device__ __forceinline__ void eval_rank_groups(const SlotDesc& sd, const uint32_t (&rk)[4 * NQ],
                                                 const uint32_t* pool, uint4* tm, int lane) {
    constexpr int R = 4 * NQ;
    const uint32_t nr = sd.rend - sd.rbeg;
    uint32_t lr[R];  // local ranks
    if (sd.rmap & kRankMap16) {
        const uint16_t* map = reinterpret_cast<const uint16_t*>(pool + (sd.rmap & ~kRankMap16) - 1);
#pragma unroll
        for (int i = 0; i < R; ++i) lr[i] = map[rk[i]];
    } else if (sd.rmap) {
        const unsigned char* map = reinterpret_cast<const unsigned char*>(pool + sd.rmap - 1);
#pragma unroll
        for (int i = 0; i < R; ++i) lr[i] = map[rk[i]];
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i) lr[i] = rk[i];
    }
    for (uint32_t g = 0; g < sd.rgroups; ++g) {
        const uint32_t* tab = pool + sd.roff + g * sd.rstride;
        uint32_t w[R];
#pragma unroll
        for (int i = 0; i < R; ++i) w[i] = tab[lr[i]];
        uint4 out[NQ];
        if constexpr (NQ == 1) {
            out[0] = transpose_group(w, nr - 32u * g, lane);
        } else {
#pragma unroll
            for (int h = 0; h < NQ; ++h) {
                out[h].x = transpose32(w[4 * h + 0], lane);
                out[h].y = transpose32(w[4 * h + 1], lane);
                out[h].z = transpose32(w[4 * h + 2], lane);
                out[h].w = transpose32(w[4 * h + 3], lane);
            }
        }
        const uint32_t k = 32u * g + lane;
        if (k < nr) {
#pragma unroll
            for (int h = 0; h < NQ; ++h) tm[(sd.rbeg + k) * NQ + h] = out[h];
        }
    }
}

// The four ranks of the lane's rows of a slice, packed in v.lo[0] and v.lo[1]
// (rank arrays are padded to whole slices, so the load never passes their end).
__device__ __forceinline__ void load_ranks(const uint16_t* rank, uint64_t slice0, int lane, Vals<1>& v) {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(rank + slice0 + 4u * lane));
    v.lo[0] = r.x;
    v.lo[1] = r.y;
}

// One slot's values of the lane's rows of a slice, or their ranks.
__device__ __forceinline__ void load_slot(const SlotDesc& d, uint64_t slice0, uint64_t nrows, int lane, Vals<1>& v) {
    if (d.rank)
        load_ranks(d.rank, slice0, lane, v);
    else
        load_vals_global<1>(d.ptr, d.width, slice0, nrows, lane, v);
}

// The wide pass over warp slices sl = first, first + stride, ... < end of
// 128 rows each: row-set masks, range terms by interval tree, EQ and IN terms
// by table, then lanes take predicates (and terms, for marginals) and add
// popcounts into the CTA's 32-bit counters.  Returns the warp's count of
// rows in each row set `lane` (lanes < nsets).
// RANKS_ONLY: every slot's range terms are rank-coded (no trees, no compares).
template <bool RANKS_ONLY = false>
__device__ __forceinline__ uint32_t wide_slices(const ProbeArgs& A, const Smem& S, int lane, uint64_t first,
                                                uint64_t end, uint64_t stride) {
    uint32_t nsr = 0;
    // Column loads run one column ahead of the evaluation (and the next
    // slice's first column is loaded before the counting), so that a warp does
    // not wait out the memory latency once per column.
    Vals<1> cur;        // the current slot's values, or its rows' ranks (rank-coded slots)
    bool have = false;  // cur holds the current slice's first slot
    uint4 km = make_uint4(0u, 0u, 0u, 0u);  // this lane's row-set mask of the current slice (lanes < nsets)
    if (A.setmask && lane < static_cast<int>(A.nsets) && first < end) km = A.setmask[first * A.nsets + lane];
    for (uint64_t sl = first; sl < end; sl += stride) {
        const uint64_t slice0 = sl * kSliceRows;
        if (!have && A.nslots) load_slot(A.slots[0], slice0, A.nrows, lane, cur);
        have = false;
        if (A.setmask) {  // computed once for every pass of the call; the next slice's loaded a slice ahead
            if (lane < static_cast<int>(A.nsets)) {
                S.keep[lane] = km;
                if (sl + stride < end) km = A.setmask[(sl + stride) * A.nsets + lane];
            }
        } else {
            set_masks<1>(A, slice0, S.keep, lane);
        }
        __syncwarp();
        // the row sets with a row in this slice (warp-uniform): sparse samples
        // are empty in most slices, and a slice in no set needs no evaluation
        uint32_t active = 0, whole = 0;  // sets with a row / with every row of the slice
        for (uint32_t q = 0; q < A.nsets; ++q) {
            const uint4 k = S.keep[q];
            if (k.x | k.y | k.z | k.w) active |= 1u << q;
            if ((k.x & k.y & k.z & k.w) == kFullMask) whole |= 1u << q;
        }
        if (!active) {
            __syncwarp();  // every lane has read S.keep before lane 0 rewrites it
            continue;
        }
        const uint64_t next = sl + stride;
        for (uint32_t s = 0; s < A.nslots; ++s) {
            const SlotDesc& sd = A.slots[s];
            const Vals<1> v = cur;
            if (s + 1 < A.nslots) {
                load_slot(A.slots[s + 1], slice0, A.nrows, lane, cur);
            } else if (next < end) {
                load_slot(A.slots[0], next * kSliceRows, A.nrows, lane, cur);
                have = true;
            }
            if (sd.rank) {  // ranges by the rows' ranks (the slot has no EQ/IN terms)
                const uint32_t rk[4] = {v.lo[0] & 0xFFFFu, v.lo[0] >> 16, v.lo[1] & 0xFFFFu, v.lo[1] >> 16};
                eval_rank_groups<1>(sd, rk, S.pool, S.tm, lane);
                continue;
            }
            if (!RANKS_ONLY) {
                if (sd.rgroups) eval_range_trees<1>(sd, v, S.pool, S.tm, lane);  // ranges by tree
                if (sd.rbeg + sd.rtree < sd.rend) {  // the remaining ranges by compare
                    SlotDesc ranges = sd;
                    ranges.rbeg = sd.rbeg + sd.rtree;
                    ranges.iend = sd.rend;
                    eval_slot<1>(ranges, v, S.st, S.pool, S.tm, lane);
                }
            }
            if (sd.iend > sd.rend) eval_valueset<1>(sd, v, S.pool, S.tm, lane);  // EQ and IN by table
        }
        __syncwarp();
        // a set holding every row of the slice counts the mask's bits alone
        for (uint32_t p = lane; p < A.npreds; p += 32) {
            const uint32_t b = S.poff[p], e = S.poff[p + 1];
            uint4 acc = S.tm[S.pterm[b]];
            for (uint32_t k = b + 1; k < e; ++k) acc = and4(acc, S.tm[S.pterm[k]]);
            const uint32_t all = __popc(acc.x) + __popc(acc.y) + __popc(acc.z) + __popc(acc.w);
            if (!all) continue;
            for (uint32_t a = active; a; a &= a - 1) {
                const uint32_t q = __ffs(a) - 1;
                const uint32_t c = (whole >> q) & 1u ? all : popc4(acc, S.keep[q]);
                if (c) atomicAdd(&S.cnt[q * A.npreds + p], c);
            }
        }
        if (A.want_marg) {
            for (uint32_t t = lane; t < A.nterms; t += 32) {
                const uint4 m = S.tm[t];
                const uint32_t all = __popc(m.x) + __popc(m.y) + __popc(m.z) + __popc(m.w);
                if (!all) continue;
                for (uint32_t a = active; a; a &= a - 1) {
                    const uint32_t q = __ffs(a) - 1;
                    const uint32_t c = (whole >> q) & 1u ? all : popc4(m, S.keep[q]);
                    if (c) atomicAdd(&S.marg[q * A.nterms + t], c);
                }
            }
        }
        if (lane < static_cast<int>(A.nsets)) {
            const uint4 k = S.keep[lane];
            nsr += __popc(k.x) + __popc(k.y) + __popc(k.z) + __popc(k.w);
        }
        __syncwarp();  // S.keep and S.tm are rewritten by the next slice
    }
    return nsr;
}

}  // namespace probe_dev
}  // namespace gace
