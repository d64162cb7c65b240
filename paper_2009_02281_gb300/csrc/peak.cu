// FP32 arithmetic peak of the current device, measured with CUDA events.
//
// The product's FFT passes execute FP32 adds, multiplies and FMAs on the CUDA
// cores; their ALU roofline needs the rate those cores actually reach here,
// not a datasheet figure.  The kernels below run long chains of independent
// FMAs (scalar FFMA, or the packed two-lane form that the register FFTs use for
// their butterfly sums) on every SM and report FLOP/s, an FMA counting as two.

#include "aimx_internal.h"

namespace aimx {

constexpr int kPeakChains = 16;   // independent accumulators per thread (hides the FMA latency)

__global__ void __launch_bounds__(256) k_peak_ffma(float* out, float a, float b, int iters) {
    float acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = (float)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += acc[c];
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_ffma2(float* out, float a, float b, int iters) {
    float2 acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = make_float2((float)(threadIdx.x + c), (float)c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) acc[c] = __ffma2_rn(acc[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += acc[c].x + acc[c].y;
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace aimx

using namespace aimx;

// variant 0: scalar FMA, 1: packed two-lane FMA.  Writes FP32 TFLOP/s (an FMA
// is two FLOPs; a packed FMA four).  Synchronous; allocates 4 bytes.
extern "C" int aimx_measure_fp32_peak(int variant, double* tflops) {
    if (!tflops || variant < 0 || variant > 1) return AIMX_E_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_CUDA;
    }
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * 4) != cudaSuccess) {
        cudaGetLastError();
        return AIMX_E_NOMEM;
    }
    const int threads = 256, blocks = 8 * sms;   // 2048 threads per SM: full occupancy
    const int iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(e0);
        if (variant == 0)
            k_peak_ffma<<<blocks, threads>>>(out, 0.999f, 1e-3f, iters);
        else
            k_peak_ffma2<<<blocks, threads>>>(out, 0.999f, 1e-3f, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = ms < best ? ms : best;   // the first launch is a warm-up
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return AIMX_E_CUDA;
    const double flop_per_inst = variant == 0 ? 2.0 : 4.0;
    const double flops = flop_per_inst * (double)blocks * threads * iters * kPeakChains;
    *tflops = flops / (best * 1e-3) / 1e12;
    return AIMX_OK;
}
