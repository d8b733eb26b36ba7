// gace_sample.cu -- K3b: materialised samples.
//
// The Measurement Engine samples rows or blocks of a table (Section III-B);
// the gate probes the same sample again and again while queries are planned
// (Section III-A).  Materialising a sample once turns every later probe of it
// from a scan of all N rows (with one hash per row or block) into a full scan
// of the r N kept rows.  Two passes over the table, both deciding membership
// exactly as the probe kernels do (H(row or block id, seed) < T(rate)):
//
//   k_sample_count    the kept rows of every tile of kTileRows rows (no column
//                     is read: one hash per row);
//   k_sample_scatter  every kept row's values, in row order, to position
//                     tile_off[tile] + (kept rows before it in its tile) of
//                     each destination column; only kept rows are loaded, so
//                     a 1 % row sample reads about the 32-byte sectors that
//                     hold a kept row, and a block sample reads its blocks.
//
// Row order is kept, so the sample table is the sample's rows in table order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gace_device.cuh"
#include "gace_internal.h"

namespace gace {
namespace {

using namespace dev;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ bool kept(const SampleArgs& A, uint64_t row) {
    const SetDesc& s = A.set;
    uint64_t x = row;
    if (s.kind == 2) x = s.block_shift >= 0 ? (row >> s.block_shift) : (row / s.block_rows);
    return splitmix64(x ^ s.seedhash) < s.thresh;
}

__global__ void __launch_bounds__(kThreads) k_sample_count(const __grid_constant__ SampleArgs A) {
    __shared__ uint32_t part[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const uint64_t r0 = tile * kSampleTileRows;
        uint32_t n = 0;
        for (uint32_t k = threadIdx.x; k < kSampleTileRows; k += kThreads) {
            const uint64_t row = r0 + k;
            n += (row < A.nrows && kept(A, row)) ? 1u : 0u;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(kFullMask, n, o);
        if (lane == 0) part[warp] = n;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) t += part[w];
            A.tile_count[tile] = t;
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void copy_value(const void* src, void* dst, uint64_t row, uint64_t at) {
    static_cast<T*>(dst)[at] = __ldg(static_cast<const T*>(src) + row);
}

__global__ void __launch_bounds__(kThreads) k_sample_scatter(const __grid_constant__ SampleArgs A) {
    __shared__ uint32_t part[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const uint64_t r0 = tile * kSampleTileRows;
        uint64_t base = A.tile_off[tile];
        if (A.tile_count[tile] == 0) continue;  // block-uniform: no barrier is skipped by part of the CTA
        for (uint32_t k = 0; k < kSampleTileRows; k += kThreads) {
            const uint64_t row = r0 + k + threadIdx.x;
            const bool keep = row < A.nrows && kept(A, row);
            const uint32_t mask = __ballot_sync(kFullMask, keep);
            if (lane == 0) part[warp] = __popc(mask);
            __syncthreads();
            uint32_t before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = part[w];
                before += w < warp ? c : 0u;
                total += c;
            }
            if (keep) {
                const uint64_t at = base + before + __popc(mask & ((1u << lane) - 1u));
                for (uint32_t c = 0; c < A.ncols; ++c) {
                    if (A.width[c] == 8)
                        copy_value<unsigned long long>(A.src[c], A.dst[c], row, at);
                    else
                        copy_value<uint32_t>(A.src[c], A.dst[c], row, at);
                }
            }
            base += total;
            __syncthreads();  // part is rewritten by the next step
        }
    }
}

}  // namespace

cudaError_t sample_count_launch(const SampleArgs& a, int grid, cudaStream_t s) {
    k_sample_count<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t sample_scatter_launch(const SampleArgs& a, int grid, cudaStream_t s) {
    k_sample_scatter<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gace
