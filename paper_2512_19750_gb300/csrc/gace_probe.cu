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
#include <algorithm>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"
#include "gace_launch.cuh"
#include "gace_probe_dev.cuh"
#include "gace_probe_narrow.cuh"

namespace gace {
namespace {

using namespace dev;
using namespace probe_dev;

// ---------------------------------------------------------------- narrow

// Grid-striding kernels over the whole table (HASH: some row set is a hashed
// sample; MAXS: row sets held in registers per lane).
template <bool HASH, int MAXS>
__global__ void __launch_bounds__(kThreads, 4) k_probe_narrow(const __grid_constant__ ProbeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid);
    __syncthreads();  // the tables are read below, before the pipeline's own barrier
    if (!narrow_run<HASH, MAXS>(A, S, tid, lane, warp, blockIdx.x, A.ntiles, gridDim.x)) return;
    __syncthreads();
    flush(A, S, tid);
}

template <bool HASH, int NQ = 2>
__global__ void __launch_bounds__(kThreads, 4) k_probe_single(const __grid_constant__ ProbeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid);
    __syncthreads();
    if (!single_run<HASH, NQ>(A, S, tid, lane, warp, blockIdx.x, A.ntiles, gridDim.x)) return;
    __syncthreads();
    flush(A, S, tid);
}

constexpr int kWideThreads = kWideWarps * 32;

#if GACE_WIDE_MINCTAS > 0
#define GACE_WIDE_BOUNDS __launch_bounds__(kWideThreads, GACE_WIDE_MINCTAS)
#else
#define GACE_WIDE_BOUNDS __launch_bounds__(kWideThreads)
#endif

template <bool RANKS_ONLY>
__global__ void GACE_WIDE_BOUNDS k_probe_wide(const __grid_constant__ ProbeArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Smem S = carve(A, smem, warp);
    load_tables(A, S, tid, kWideThreads);
    __syncthreads();
    const uint64_t nslices = (A.nrows + kSliceRows - 1) / kSliceRows;
    const uint32_t nsr = wide_slices<RANKS_ONLY>(A, S, lane, static_cast<uint64_t>(blockIdx.x) * kWideWarps + warp,
                                                 nslices, static_cast<uint64_t>(gridDim.x) * kWideWarps);
    if (lane < static_cast<int>(A.nsets) && nsr) atomicAdd(&S.ns[lane], nsr);
    __syncthreads();
    flush(A, S, tid, kWideThreads);
}

// Row-set masks of 128-row slices (one warp per slice, grid-striding), the
// same masks the wide pass would compute, into out[slice * nsets + set]; with
// qmask, also each quad's membership word, qmask[slice * 32 + lane]: bit
// 4 q + i set when row 4 lane + i of the slice is in set q.
__global__ void __launch_bounds__(256) k_probe_setmask(const __grid_constant__ ProbeArgs A, uint4* out,
                                                       uint32_t* qmask) {
    __shared__ uint4 keep[8][kMaxSets];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nslices = (A.nrows + kSliceRows - 1) / kSliceRows;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
    for (uint64_t sl = static_cast<uint64_t>(blockIdx.x) * (blockDim.x / 32) + warp; sl < nslices; sl += stride) {
        set_masks<1>(A, sl * kSliceRows, keep[warp], lane);
        __syncwarp();
        if (lane < static_cast<int>(A.nsets)) out[sl * A.nsets + lane] = keep[warp][lane];
        if (qmask) {
            uint32_t w = 0;
            for (uint32_t q = 0; q < A.nsets; ++q) {
                const uint4 k = keep[warp][q];
                w |= (((k.x >> lane) & 1u) | (((k.y >> lane) & 1u) << 1) | (((k.z >> lane) & 1u) << 2) |
                      (((k.w >> lane) & 1u) << 3)) << (4 * q);
            }
            qmask[sl * 32 + lane] = w;
        }
        __syncwarp();  // keep[warp] is rewritten for the next slice
    }
}

// Rank coding of one column (RankArgs): the endpoints' search tree (or their
// bucket index) staged in shared memory, then four rows per thread per step:
// with the tree, their descents interleaved level by level (one compare
// each), to the number of endpoints <= each key; with the bucket index, each
// key's bucket gives the index of the first endpoint at or after the bucket's
// lower bound, and `steps` halvings over the sorted endpoints from there count
// those <= the key (the bucket holds fewer than 2^steps, and endpoints of
// later buckets are larger than the key).  With histograms, each row's rank
// is counted in a shared-memory histogram of every set that holds it, added
// to the global one at the end.
template <bool BUCKET>
__global__ void __launch_bounds__(256) k_probe_rank(const __grid_constant__ RankArgs A) {
    extern __shared__ __align__(16) uint32_t tree[];
    const bool is64 = A.dtype == 1;
    uint32_t* hist = tree + A.words;  // [set][rank], when A.hist
    const uint32_t bins = A.hist ? A.nsets * (A.m + 1) : 0u;
    for (uint32_t i = threadIdx.x; i < A.words; i += blockDim.x) tree[i] = A.tree[i];
    for (uint32_t i = threadIdx.x; i < bins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint16_t* start = reinterpret_cast<const uint16_t*>(tree);
    const uint32_t* ends = tree + rank_start_words(A.nb);  // 8-byte aligned
    const uint32_t width = is64 ? 8u : 4u;
    const uint64_t step = static_cast<uint64_t>(gridDim.x) * blockDim.x * 4u;
    for (uint64_t r0 = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4u; r0 < A.nout; r0 += step) {
        Quad q;
        load_quad_global(A.col, width, r0, A.nrows, q);
        uint32_t klo[4], khi[4], n[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) value_key(A.dtype, q.lo[i], q.hi[i], klo[i], khi[i]);
        uint32_t rk[4];
        if (BUCKET) {
            if (is64) {
                const uint2* e2 = reinterpret_cast<const uint2*>(ends);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint64_t k = (static_cast<uint64_t>(khi[i]) << 32) | klo[i];
                    const uint64_t d = k >= A.base ? k - A.base : 0ull;
                    const int s = max(static_cast<int>(A.smin), 63 - __clzll(static_cast<long long>(d)) -
                                                                     static_cast<int>(A.mbits));
                    const uint64_t b = (static_cast<uint64_t>(s - static_cast<int>(A.smin)) << A.mbits) + (d >> s);
                    n[i] = start[b < A.nb ? b : A.nb - 1];
                }
                for (uint32_t h = (1u << A.steps) >> 1; h; h >>= 1) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint2 e = e2[n[i] + h - 1];
                        n[i] += (khi[i] > e.y || (khi[i] == e.y && klo[i] >= e.x)) ? h : 0u;
                    }
                }
            } else {
                const uint32_t base = static_cast<uint32_t>(A.base);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t d = klo[i] >= base ? klo[i] - base : 0u;
                    const int s = max(static_cast<int>(A.smin), 31 - __clz(d) - static_cast<int>(A.mbits));
                    const uint32_t b = (static_cast<uint32_t>(s - static_cast<int>(A.smin)) << A.mbits) + (d >> s);
                    n[i] = start[b < A.nb ? b : A.nb - 1];
                }
                for (uint32_t h = (1u << A.steps) >> 1; h; h >>= 1) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) n[i] += klo[i] >= ends[n[i] + h - 1] ? h : 0u;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) rk[i] = r0 + i < A.nrows ? (n[i] < A.m ? n[i] : A.m) : 0u;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) n[i] = 1;
            if (is64) {
                const uint2* node = reinterpret_cast<const uint2*>(tree);
                for (uint32_t d = 0; d < A.levels; ++d) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint2 e = node[n[i] - 1];
                        n[i] = 2 * n[i] + ((khi[i] > e.y || (khi[i] == e.y && klo[i] >= e.x)) ? 1u : 0u);
                    }
                }
            } else {
                for (uint32_t d = 0; d < A.levels; ++d) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) n[i] = 2 * n[i] + (klo[i] >= tree[n[i] - 1] ? 1u : 0u);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t r = n[i] - (1u << A.levels);
                rk[i] = r0 + i < A.nrows ? (r < A.m ? r : A.m) : 0u;
            }
        }
        if (A.out) *reinterpret_cast<uint2*>(A.out + r0) = make_uint2(rk[0] | (rk[1] << 16), rk[2] | (rk[3] << 16));
        if (A.hist) {
            // bit 4 s + i: row r0 + i is in set s
            const uint32_t valid = r0 + 4 <= A.nrows ? 0xFu : (r0 < A.nrows ? (1u << (A.nrows - r0)) - 1u : 0u);
            uint32_t member = A.qmask ? A.qmask[r0 >> 2] : 0u;
            for (uint32_t s = 0; s < A.nsets; ++s) {
                const uint32_t bits = ((A.full_sets >> s) & 1u) ? valid : ((member >> (4 * s)) & valid);
                if (!bits) continue;
                uint32_t* hs = hist + s * (A.m + 1);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if ((bits >> i) & 1u) atomicAdd(hs + rk[i], 1u);
            }
        }
    }
    if (A.hist) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < bins; i += blockDim.x)
            if (hist[i]) atomicAdd(A.hist + i, static_cast<unsigned long long>(hist[i]));
    }
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
    const uint32_t warps = a.nwarps ? a.nwarps : kProbeWarps;
    a.off_tm = off;
    off += warps * a.nterms * 16 * nq;
    a.off_keep = off;
    off += warps * a.nsets * 16 * nq;
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

// probe_variant's cases; 6: a wide pass whose range terms are all
// rank-coded; 7: one predicate on all rows of columns of at most 8 bytes per
// row, 16 rows per lane
static int variant(const ProbeArgs& a) {
    const int v = probe_variant(a);
    if (v == 0 && a.ranks_only) return 6;
    if (v == 4) {
        uint32_t rowbytes = 0;
        for (uint32_t s = 0; s < a.nslots; ++s) rowbytes += a.slots[s].width;
        if (rowbytes <= 8) return 7;
    }
    return v;
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
    if ((e = set_smem(k_probe_single<false, 4>, optin))) return e;
    if ((e = set_smem(k_probe_single<true>, optin))) return e;
    if ((e = set_smem(k_probe_wide<true>, optin))) return e;
    return set_smem(k_probe_wide<false>, optin);
}

int probe_occupancy(const ProbeArgs& a) {
    int n = 0;
    cudaError_t e = cudaSuccess;
    switch (variant(a)) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_wide<false>, kWideThreads, a.smem_bytes); break;
        case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_wide<true>, kWideThreads, a.smem_bytes); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_narrow<false, 1>, kThreads, a.smem_bytes); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_narrow<true, 1>, kThreads, a.smem_bytes); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_narrow<true, kMaxSets>, kThreads, a.smem_bytes); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_single<false>, kThreads, a.smem_bytes); break;
        case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_single<false, 4>, kThreads, a.smem_bytes); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_probe_single<true>, kThreads, a.smem_bytes); break;
    }
    return e == cudaSuccess ? n : 0;
}

uint32_t rank_smem(const RankArgs& a) {
    return a.words * 4u + (a.hist ? a.nsets * (a.m + 1) * 4u : 0u);
}

template <bool BUCKET>
static cudaError_t rank_launch_t(const RankArgs& a, int sms, cudaStream_t s) {
    const uint32_t smem = rank_smem(a);
    cudaError_t e = smem_allow_max<k_probe_rank<BUCKET>>();
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_rank<BUCKET>, 256, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // a full wave of resident CTAs (each histogram flush costs one global add per bin)
    const uint64_t quads = a.nout / 4;
    const uint64_t cap = static_cast<uint64_t>(sms) * static_cast<uint64_t>(per_sm) * 256;
    uint64_t threads = quads < cap ? quads : cap;
    uint64_t grid = threads ? (threads + 255) / 256 : 1;
    // each CTA keeps 32-bit counts of the rows it ranks
    while (a.hist && (quads + grid * 256 - 1) / (grid * 256) * 1024 >= (1ull << 31)) grid *= 2;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    k_probe_rank<BUCKET><<<static_cast<int>(grid), 256, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t rank_launch(const RankArgs& a, int sms, cudaStream_t s) {
    return a.levels ? rank_launch_t<false>(a, sms, s) : rank_launch_t<true>(a, sms, s);
}

cudaError_t setmask_launch(const ProbeArgs& a, uint4* out, uint32_t* qmask, int sms, cudaStream_t s) {
    const uint64_t nslices = (a.nrows + kSliceRows - 1) / kSliceRows;
    const uint64_t warps = static_cast<uint64_t>(sms) * 64;  // a full SM of warps each
    const uint64_t grid = (std::min<uint64_t>(nslices, warps) + 7) / 8;
    k_probe_setmask<<<static_cast<int>(grid ? grid : 1), 256, 0, s>>>(a, out, qmask);
    return cudaGetLastError();
}

cudaError_t probe_launch(const ProbeArgs& a, int grid, cudaStream_t s) {
    switch (variant(a)) {
        case 0: k_probe_wide<false><<<grid, kWideThreads, a.smem_bytes, s>>>(a); break;
        case 6: k_probe_wide<true><<<grid, kWideThreads, a.smem_bytes, s>>>(a); break;
        case 1: k_probe_narrow<false, 1><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 2: k_probe_narrow<true, 1><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 3: k_probe_narrow<true, kMaxSets><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 4: k_probe_single<false><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        case 7: k_probe_single<false, 4><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
        default: k_probe_single<true><<<grid, kThreads, a.smem_bytes, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace gace
