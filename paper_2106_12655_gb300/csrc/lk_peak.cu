// Measured FP32 peak of this GPU, reported beside the bulk sweep's roofline:
// kernels of independent fused multiply-adds, packed FP32x2 (the instruction
// the sweep spends most of its FMA-pipe cycles on; eight chains per thread)
// and scalar (sixteen chains), 2,048 threads per SM, so that nothing but the
// FMA pipe limits them; the faster counts.  The paper has no counterpart;
// this is measurement support.
#include <cuda_runtime.h>

#include "lk.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;

// Packed: CH chains of __ffma2_rn per thread (4 flops each per iteration).
template <int CH>
__global__ void __launch_bounds__(kPeakThreads) fp32x2_fma_peak_kernel(float2* __restrict__ out, int iters,
                                                                       float2 b, float2 c) {
    float2 a[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = make_float2(1e-3f * threadIdx.x + k, 0.5f * k);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CH; ++k) a[k] = __ffma2_rn(a[k], b, c);
    }
    float2 s = a[0];
#pragma unroll
    for (int k = 1; k < CH; ++k) s = __fadd2_rn(s, a[k]);
    out[(size_t)blockIdx.x * kPeakThreads + threadIdx.x] = s;   // keeps the chains live
}

// Scalar: CH chains of fmaf per thread (2 flops each per iteration).
template <int CH>
__global__ void __launch_bounds__(kPeakThreads) fp32_fma_peak_kernel(float2* __restrict__ out, int iters, float b,
                                                                     float c) {
    float a[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = 1e-3f * threadIdx.x + k;
#pragma unroll 2
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CH; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = a[0];
#pragma unroll
    for (int k = 1; k < CH; ++k) s += a[k];
    out[(size_t)blockIdx.x * kPeakThreads + threadIdx.x] = make_float2(s, s);
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
    // the faster of the packed and the scalar form, each the fastest of three
    // launches after a warm-up
    double best_tf = 0.0;
    float best_ms = 0.0f;
    for (int variant = 0; variant < 2 && e == cudaSuccess; ++variant) {
        const double flops_per_iter = variant == 0 ? 8 * 4.0 : 16 * 2.0;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            if (variant == 0)
                fp32x2_fma_peak_kernel<8><<<blocks, kPeakThreads, 0, s>>>(out, iters, make_float2(0.999999f, 0.9999995f),
                                                                         make_float2(1e-6f, 2e-6f));
            else
                fp32_fma_peak_kernel<16><<<blocks, kPeakThreads, 0, s>>>(out, iters, 0.999999f, 1e-6f);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float m = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&m, e0, e1);
            if (e == cudaSuccess && rep > 0 && m > 0.0f) {
                const double tf = (double)blocks * kPeakThreads * (double)iters * flops_per_iter / (m * 1e-3) / 1e12;
                if (tf > best_tf) {
                    best_tf = tf;
                    best_ms = m;
                }
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return LK_ERR_CUDA;
    *tflops = best_tf;
    if (ms) *ms = best_ms;
    return LK_OK;
}
