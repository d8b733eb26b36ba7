// gace_noalloc.cu -- HyperLogLog for callers that cannot allocate device memory.
//
// gace_ndv needs a context, and a context allocates (its workspace, its status
// word, pinned staging).  Some callers cannot do that: an optimizer's planning
// hook must not trigger cudaMalloc's device-wide synchronisation and unbounded
// latency while a query is being planned, and a process whose device memory is
// owned by another allocator (a database buffer manager, a framework's caching
// allocator under a hard cap) cannot add raw allocations behind its back.
// gace_ndv_noalloc serves them: the same k_hll kernel, with its scratch (the
// 32-bit registers, the packed byte registers, the value histogram and the
// status word) in one fixed file-scope device array.
//
// That array lives in every GPU that loads the library until the process exits.
// Every call uses the whole of it, so calls that overlap on the GPU (other
// streams, other host threads) race: callers serialise them.  Each call clears
// what must start at zero.  Host code never hands the array's name to a kernel
// (in host code it is only a stand-in): every call looks up its device address
// with cudaGetSymbolAddress on the current device, which allocates nothing once
// the library's module is loaded on that device, and is never stale (a device
// reset or a new primary context gives a new address, and the next call sees
// it).  With lazy module loading (CUDA's default) the first call on a device
// loads the module, and that load may allocate and synchronise: callers warm
// the entry point up once per device before the code that must not allocate,
// or set CUDA_MODULE_LOADING=EAGER.  Every call waits for its stream and reads
// its results back into host memory, so no call may be made while a stream is
// being captured into a CUDA graph.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>

#include "../../include/gace.h"
#include "gace_internal.h"

namespace gace {
void set_last_error_message(const char* msg);
}

namespace {

constexpr uint32_t kMaxP = GACE_NOALLOC_MAX_P;
constexpr size_t kRegsOff = 0;                                // uint32[2^kMaxP]
constexpr size_t kPackedOff = (size_t(1) << kMaxP) * 4;       // uint8[2^kMaxP]
constexpr size_t kHistOff = kPackedOff + (size_t(1) << kMaxP);  // uint32[66], padded
constexpr size_t kStatusOff = kHistOff + 512;                 // uint32
constexpr size_t kScratchBytes = kStatusOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Register values as bytes, and how many registers hold each value 0..65.
__global__ void __launch_bounds__(256) k_pack_hist(const uint32_t* regs, uint32_t m,
                                                   unsigned char* packed, uint32_t* hist) {
    __shared__ uint32_t sh[66];
    for (int i = threadIdx.x; i < 66; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const uint32_t r = regs[j];
        packed[j] = static_cast<unsigned char>(r);
        atomicAdd(&sh[r < 65 ? r : 65], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 66; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

gace_status fail_msg(gace_status s, const char* msg) {
    gace::set_last_error_message(msg);
    return s;
}

gace_status cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return fail_msg(GACE_ECUDA, buf);
}

// Device address of the scratch array on the current device, looked up on
// every call (a cached address would outlive a device reset).
gace_status scratch_address(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    *out = static_cast<unsigned char*>(p);
    return GACE_OK;
}

uint64_t splitmix64_seed(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

}  // namespace

extern "C" gace_status gace_ndv_noalloc(const void* column, int32_t dtype, uint64_t nrows, uint32_t p,
                                        uint64_t hash_seed, void* stream, uint8_t* registers_out,
                                        double* estimate_out) {
    char buf[160];
    if (p < 4 || p > kMaxP) {
        snprintf(buf, sizeof(buf), "p = %u outside 4..%u, the most the no-allocation scratch holds", p, kMaxP);
        return fail_msg(GACE_EINVAL, buf);
    }
    if (dtype < GACE_I32 || dtype > GACE_F32) return fail_msg(GACE_EINVAL, "dtype is not int32/int64/float32");
    if (nrows > 0 && !column) return fail_msg(GACE_EINVAL, "column is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char* base = nullptr;
    if (gace_status st = scratch_address(&base)) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t m = 1u << p;
    uint32_t* regs = reinterpret_cast<uint32_t*>(base + kRegsOff);
    unsigned char* packed = base + kPackedOff;
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kHistOff);
    unsigned int* status = reinterpret_cast<unsigned int*>(base + kStatusOff);
    if ((e = cudaMemsetAsync(regs, 0, static_cast<size_t>(m) * 4, s)) != cudaSuccess) return cuda_fail(e, "clear registers");
    if ((e = cudaMemsetAsync(hist, 0, 66 * 4, s)) != cudaSuccess) return cuda_fail(e, "clear histogram");
    if ((e = cudaMemsetAsync(status, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "clear status");
    if (nrows > 0) {
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
        gace::HllArgs a{};
        a.col = column;
        a.nrows = nrows;
        a.dtype = static_cast<uint32_t>(dtype);
        a.p = p;
        a.seedhash = splitmix64_seed(hash_seed);
        a.aligned = (reinterpret_cast<uintptr_t>(column) & 15u) == 0;
        a.regs = regs;
        a.status = status;
        if ((e = gace::hll_launch(a, sms, s)) != cudaSuccess) return cuda_fail(e, "HLL launch");
    }
    k_pack_hist<<<(m + 255) / 256 < 64 ? (m + 255) / 256 : 64, 256, 0, s>>>(regs, m, packed, hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pack launch");
    uint32_t counts[66];
    unsigned int st = 0;
    if (registers_out && (e = cudaMemcpyAsync(registers_out, packed, m, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "copy registers");
    if ((e = cudaMemcpyAsync(counts, hist, sizeof(counts), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "copy histogram");
    if ((e = cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "copy status");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (st) return fail_msg(GACE_ETIMEDOUT, "a bounded device CAS loop gave up");
    if (estimate_out) {
        uint64_t c[66];
        for (int k = 0; k < 66; ++k) c[k] = counts[k];
        *estimate_out = gace::hll_estimate_from_hist(c, p);
    }
    return GACE_OK;
}
