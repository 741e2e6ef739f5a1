// Measured FP32 FMA throughput of the device (yk_fp32_fma_peak): the
// denominator of the far-field kernels' roofline. The far-field P2P
// evaluation (the quadrature sums of Eq. double-layer-def) runs on the CUDA
// cores and is bound by the FP32 FMA pipe, so its fraction of peak is taken
// against what plain chains of FMAs achieve on the same GPU at the same
// moment, rather than against a figure derived from unit counts and a
// nominal clock.
//
// Kernel: every thread runs FMA_CHAINS independent FMA chains for `iters`
// x 16 steps; grid = 8 blocks of 256 threads per SM (16 warps per
// scheduler, 8 independent FMAs in flight per warp: far more than the
// pipe latency needs). The result is kept live by a store that
// only happens when the sum is not finite, which never occurs for the
// inputs used, so the compiler cannot drop the chains.
#include <cuda_runtime.h>

#include <algorithm>

#include "yk_internal.cuh"

namespace yk {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_TPB = 256;

__global__ void __launch_bounds__(FMA_TPB) k_fma_chains(float a, float b, int iters,
                                                       float* __restrict__ sink) {
    float v[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) v[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < FMA_CHAINS; ++c) v[c] = fmaf(v[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) s += v[c];
    if (!isfinite(s)) sink[blockIdx.x * FMA_TPB + threadIdx.x] = s;
}

int fp32_fma_peak(int device, double* tflops) {
    YK_TRY_CUDA(cudaSetDevice(device));
    int sms = 0;
    YK_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    cudaStream_t st;
    YK_TRY_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float* sink = nullptr;
    const int blocks = sms * 8;
    int rc = dev_alloc((void**)&sink, sizeof(float) * blocks * FMA_TPB, st);
    // a = 0.999, b = 1e-3: the chains converge to b / (1 - a) = 1, finite
    const float a = 0.999f, b = 1e-3f;
    const int iters = 4096;
    double best = 0.0;
    for (int rep = 0; rep < 4 && rc == YK_OK; ++rep) {
        cudaEventRecord(e0, st);
        YK_LAUNCH(k_fma_chains, blocks, FMA_TPB, 0, st, a, b, iters, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = YK_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * (double)blocks * FMA_TPB * FMA_CHAINS * 16.0 * iters;
        if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    dev_free(sink, st);
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rc == YK_OK) *tflops = best;
    return rc;
}

}  // namespace yk

extern "C" int yk_fp32_fma_peak(int device, double* tflops) {
    if (!tflops || device < 0) return YK_ERR_ARG;
    return yk::fp32_fma_peak(device, tflops);
}
