// resample_noalloc.cu -- systematic resampling that allocates nothing.
//
// smc_k_resample needs a caller-allocated device scratch block for the scan
// tile descriptors.  Some callers cannot allocate device memory at the point
// where they resample: a host framework that has reserved the whole device
// budget for its own pool, or a latency-critical loop that must not pay the
// implicit device synchronisation of cudaMalloc/cudaFree.  This variant keeps
// its scratch in a fixed, statically sized device array instead, so a call
// only launches kernels and a memset on the caller's stream.
#include <cstdio>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/smc.h"
#include "smc_kernels.cuh"

namespace {

// Fixed scratch, 64 KiB on every device that loads the library (held until
// the process exits).  It covers the look-back descriptors of up to
// SMC_NOALLOC_MAX_N particles (checked below against the layout in use).
constexpr size_t NOALLOC_SCRATCH_BYTES = 64 * 1024;
static __device__ __align__(256) unsigned char g_resample_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
cudaError_t scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_resample_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

smc_status smc_k_resample_noalloc(const double* W, int64_t N, uint64_t r64, uint64_t* q,
                                  int32_t* ancestors, int32_t* status_out, void* stream) {
    if (N < 1 || !W || !q || !ancestors || !status_out) return SMC_E_INVAL;
    if (N > SMC_NOALLOC_MAX_N || (size_t)smc::resample_scratch_bytes(N) > NOALLOC_SCRATCH_BYTES) {
        fprintf(stderr,
                "smc_k_resample_noalloc: N = %lld exceeds the fixed scratch limit of %lld particles; "
                "use smc_k_resample with caller-allocated scratch\n",
                (long long)N, (long long)SMC_NOALLOC_MAX_N);
        return SMC_E_INVAL;
    }
    void* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        fprintf(stderr, "smc_k_resample_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
        return SMC_E_CUDA;
    }
    // launch_resample_flat clears the tile descriptors and writes the header
    // before the scan reads them, so leftovers of an earlier call are harmless.
    e = smc::launch_resample_flat(W, N, r64, reinterpret_cast<unsigned long long*>(q), ancestors, status_out,
                                  scratch, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        fprintf(stderr, "smc_k_resample_noalloc: %s\n", cudaGetErrorString(e));
        return e == cudaErrorInvalidValue ? SMC_E_INVAL : SMC_E_CUDA;
    }
    return SMC_OK;
}

}  // extern "C"
