// gace_launch.cuh -- host-side launch helper shared by the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace gace {

// Raises kernel K's dynamic shared-memory limit to the device's opt-in
// maximum (less K's static shared memory), once per device.  Every caller
// sets the same value, so launches of K from several contexts on several
// host threads never meet another caller's smaller limit, as they would if
// each launch set the limit to its own exact size between another thread's
// setting and launch.
template <auto K>
cudaError_t smem_allow_max() {
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, K)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - static_cast<int>(fa.sharedSizeBytes));
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
    return e;
}

}  // namespace gace
