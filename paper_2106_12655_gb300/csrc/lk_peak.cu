// Measured FP32 peak of this GPU for the bulk sweep's roofline: a kernel of
// independent packed FP32x2 fused multiply-adds (the instruction the sweep
// spends most of its FMA-pipe cycles on), eight chains per thread and 2,048
// threads per SM, so that nothing but the FMA pipe limits it.  The paper has
// no counterpart; this is measurement support.
#include <cuda_runtime.h>

#include <algorithm>

#include "lk.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;
constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(kPeakThreads) fp32x2_fma_peak_kernel(float2* __restrict__ out, int iters,
                                                                       float2 b, float2 c) {
    float2 a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = make_float2(1e-3f * threadIdx.x + k, 0.5f * k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
    }
    float2 s = a[0];
#pragma unroll
    for (int k = 1; k < kPeakChains; ++k) s = __fadd2_rn(s, a[k]);
    out[(size_t)blockIdx.x * kPeakThreads + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" lk_status lk_measure_fp32_peak(double* tflops, double* ms, void* cuda_stream) {
    if (!tflops) return LK_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LK_ERR_CUDA;
    const int blocks = sms * kPeakBlocksPerSm;
    const int iters = 1 << 17;     // about 16 ms at 80 TFLOP/s on 152 SMs
    float2* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * kPeakThreads * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return LK_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    const float2 b = make_float2(0.999999f, 0.9999995f), c = make_float2(1e-6f, 2e-6f);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, s);
        fp32x2_fma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, iters, b, c);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float m = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, m);   // the first launch warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return LK_ERR_CUDA;
    // per thread and iteration: kPeakChains packed FMAs = 2 lanes x 2 flops each
    const double flops = (double)blocks * kPeakThreads * (double)iters * kPeakChains * 4.0;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return LK_OK;
}
