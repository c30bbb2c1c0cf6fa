// Measurement entry points (no counterpart in the paper): per-kernel CUDA
// event timing of one generation, and an FP32 fused-multiply-add throughput
// probe used as the measured denominator of the rollout's roofline.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/empc.h"
#include "empc_internal.h"

namespace {

// Eight independent FMA chains per thread; each iteration issues 8 FFMAs.
__global__ void ffma_probe_kernel(float* out, int iters, float a, float b) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fmaf(v[j], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += v[j];
    if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" {

empc_status empc_measure_fp32_peak(double* tflops) {
    if (!tflops) return EMPC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EMPC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EMPC_ECUDA;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * 65536) != cudaSuccess) return EMPC_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8, iters = 1 << 15;
    ffma_probe_kernel<<<blocks, threads>>>(out, 256, 0.999f, 1e-3f);
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        ffma_probe_kernel<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return EMPC_ECUDA;
    const double flops = 2.0 * 8.0 * (double)iters * threads * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    return EMPC_OK;
}

}  // extern "C"
