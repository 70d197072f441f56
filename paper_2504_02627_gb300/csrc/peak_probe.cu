// peak_probe.cu -- the issue-rate ceiling of the warp-level BF16 tensor-core
// path (mma.sync m16n8k16, FP32 accumulation) on the running GPU, the
// denominator the benchmark gives the warp-MMA trajectory kernels beside the
// dense tcgen05 peak.  Independent accumulators per warp, operands in
// registers, no memory traffic: 2 CTAs of 256 threads per SM, each warp
// issuing eight independent MMA chains.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/smc.h"

namespace {

__global__ void __launch_bounds__(256) k_mma_peak(float* out, int iters) {
    uint32_t a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = 0x3f803f80u ^ ((uint32_t)threadIdx.x << 3) ^ (uint32_t)i;
#pragma unroll
    for (int i = 0; i < 2; ++i) b[i] = 0x3c003c00u ^ ((uint32_t)threadIdx.x << 2) ^ (uint32_t)i;
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[j][i] = 0.0f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                "{%8, %9}, {%0, %1, %2, %3};"
                : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" smc_status smc_k_mma_peak(int64_t iters, double* tflops, void* stream) {
    if (iters < 1 || iters > (1 << 24) || !tflops) return SMC_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
        return SMC_E_CUDA;
    const int grid = 2 * nsm, bs = 256;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&out), sizeof(float) * grid * bs, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    if (e == cudaSuccess) {
        k_mma_peak<<<grid, bs, 0, s>>>(out, (int)std::min<int64_t>(iters, 1024));   // warm-up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) k_mma_peak<<<grid, bs, 0, s>>>(out, (int)iters);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (out) cudaFreeAsync(out, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.0f)) return SMC_E_CUDA;
    const double flops = 2.0 * 16 * 8 * 16 * 8.0 * (double)iters * grid * (bs / 32);
    *tflops = flops / (ms * 1e-3) / 1e12;
    return SMC_OK;
}
