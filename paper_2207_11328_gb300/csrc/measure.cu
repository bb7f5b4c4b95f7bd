// FP32 CUDA-core throughput of this device, measured: the ALU roof of the
// interaction kernels (their arithmetic is FP32 FMA/ADD/MUL on the CUDA
// cores; no part of the method is a dense contraction for the tensor cores).
#include <cuda_runtime.h>

#include "sph.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (covers the FMA latency)

__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0f) out[blockIdx.x] = s;  // never true: keeps the chains live
}

}  // namespace

extern "C" int sph_fp32_peak(void* stream, double* tflops) {
    if (!tflops) return SPH_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SPH_ERR_CUDA;
    const int threads = 256, blocks = sms * 8, iters = 512;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) return SPH_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_peak<<<blocks, threads, 0, st>>>(out, iters / 8, 0.9999999f, 1e-7f);  // warm-up
    float best = 3.4e38f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, st);
        k_fma_peak<<<blocks, threads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || !(best > 0.f)) return SPH_ERR_CUDA;
    const double flops = 2.0 * kChains * 16.0 * iters * (double)threads * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    return SPH_OK;
}
