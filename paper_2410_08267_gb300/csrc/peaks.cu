// Arithmetic-throughput microbenchmarks of the GPU, used as the measured
// roofline denominators of the trajectory kernel (an FP32 ALU-bound path):
// scalar FP32 FMA, packed FP32x2 FMA, the special-function unit's reciprocal
// square root and base-2 logarithm, and FP64 FMA (for the FP64 mode).  Every thread runs 8
// independent dependency chains so that the pipes, not latency, bound the
// rate; the grid fills every SM several times over.
#include <cuda_runtime.h>

#include "nuprof_internal.h"

namespace nuprof {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) ffma_kernel(float* out, float a, float b)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1.2345f) out[blockIdx.x] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(kBlock) ffma2_kernel(float* out, float a, float b)
{
    unsigned long long v[kChains];
    const float2 ab = make_float2(a, a), bb = make_float2(b, b);
    const unsigned long long A = *reinterpret_cast<const unsigned long long*>(&ab);
    const unsigned long long B = *reinterpret_cast<const unsigned long long*>(&bb);
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float2 f = make_float2(threadIdx.x * 1e-3f + c, c + 0.5f);
        v[c] = *reinterpret_cast<unsigned long long*>(&f);
    }
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[c]) : "l"(A), "l"(B));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float2 f = *reinterpret_cast<float2*>(&v[c]);
        s += f.x + f.y;
    }
    if (s == 1.2345f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) dfma_kernel(float* out, double a, double b, int iters)
{
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1.2345) out[blockIdx.x] = (float)s;
}

__global__ void __launch_bounds__(kBlock) rsqrt_kernel(float* out)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = 1.0f + threadIdx.x * 1e-3f + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1.2345f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) lg2_kernel(float* out)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = 3.0f + threadIdx.x * 1e-3f + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1.2345f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace nuprof

using namespace nuprof;

extern "C" int nu_measure_peaks(void* stream, nu_peaks* out)
{
    if (!out) return NU_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, clk = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    const int grid = sms * 8;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&sink, grid * sizeof(float)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (sink) cudaFree(sink);
        return NU_ECUDA;
    }
    float ms[5] = {0, 0, 0, 0, 0};
    int rc = NU_OK;
    for (int which = 0; which < 5 && rc == NU_OK; ++which) {
        for (int rep = 0; rep < 2 && rc == NU_OK; ++rep) {   // first pass warms up
            cudaEventRecord(e0, s);
            switch (which) {
            case 0: ffma_kernel<<<grid, kBlock, 0, s>>>(sink, 0.999f, 1e-3f); break;
            case 1: ffma2_kernel<<<grid, kBlock, 0, s>>>(sink, 0.999f, 1e-3f); break;
            case 2: rsqrt_kernel<<<grid, kBlock, 0, s>>>(sink); break;
            case 3: lg2_kernel<<<grid, kBlock, 0, s>>>(sink); break;
            default: dfma_kernel<<<grid, kBlock, 0, s>>>(sink, 0.999, 1e-3, kIters / 16); break;
            }
            count_launch();
            cudaEventRecord(e1, s);
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms[which], e0, e1) != cudaSuccess)
                rc = NU_ECUDA;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != NU_OK) {
        cudaGetLastError();
        return rc;
    }
    const double threads = (double)grid * kBlock;
    const double ops = threads * kChains * kIters;
    out->ffma_tflops = 2.0 * ops / (ms[0] * 1e-3) / 1e12;
    out->ffma2_tflops = 4.0 * ops / (ms[1] * 1e-3) / 1e12;
    out->rsqrt_gops = ops / (ms[2] * 1e-3) / 1e9;
    out->lg2_gops = ops / (ms[3] * 1e-3) / 1e9;
    out->dfma_tflops = 2.0 * ops / 16.0 / (ms[4] * 1e-3) / 1e12;   // a sixteenth of the iterations
    out->sm_count = sms;
    out->clock_mhz_nominal = clk / 1000;
    return NU_OK;
}
