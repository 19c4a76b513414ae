// ucp_peaks.cu -- arithmetic-throughput microbenchmarks of the units the tree
// walk is bound by (FP32 FMA, packed FP32x2 FMA, reciprocal square root, FP64
// FMA), so that walk throughput can be stated as a fraction of a throughput
// measured on the same GPU at the same clocks.  Each thread runs 8 independent
// dependency chains; the grid is 4 blocks of 256 threads per SM.
#include "ucp.h"
#include "ucp_internal.cuh"

#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kThreads) k_peak_ffma(float* out, float a, float b, int iters)
{
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_ffma2(float* out, float a, float b, int iters)
{
    float2 x[8];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = make_float2(1e-3f * (float)(threadIdx.x + k), 0.5f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k].x + x[k].y;
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_rsqrt(float* out, float a, float b, int iters)
{
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = a + (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = rsqrtf(x[k]);
    float s = b;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_dfma(float* out, float a, float b, int iters)
{
    double x[8];
    const double ad = a, bd = b;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], ad, bd);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * kThreads + threadIdx.x] = (float)s;
}

}  // namespace

extern "C" int ucp_measure_peaks(double out[4], void* stream)
{
    if (!out) return UCP_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm < 1)
        return UCP_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = 4 * nsm;
    const double threads = (double)blocks * kThreads;
    float* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess) {
        cudaGetLastError();
        return UCP_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // iterations sized for roughly 5-20 ms per launch on a 152-SM GPU
    const int it_f32 = 8000, it_f64 = 200, it_rsq = 1000;
    auto best_ms = [&](int which, int iters) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {  // the first launch is a warm-up
            cudaEventRecord(e0, s);
            ucp::count_launch(1);
            switch (which) {
            case 0: k_peak_ffma<<<blocks, kThreads, 0, s>>>(buf, 0.9999f, 1e-4f, iters); break;
            case 1: k_peak_ffma2<<<blocks, kThreads, 0, s>>>(buf, 0.9999f, 1e-4f, iters); break;
            case 2: k_peak_rsqrt<<<blocks, kThreads, 0, s>>>(buf, 1.5f, 0.f, iters); break;
            default: k_peak_dfma<<<blocks, kThreads, 0, s>>>(buf, 0.9999f, 1e-4f, iters); break;
            }
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        return (double)best;
    };
    const double per = (double)kUnroll * 8.0 * threads;  // operations per iteration
    out[0] = 2.0 * per * it_f32 / (best_ms(0, it_f32) * 1e-3) / 1e12;
    out[1] = 4.0 * per * it_f32 / (best_ms(1, it_f32) * 1e-3) / 1e12;
    out[2] = per * it_rsq / (best_ms(2, it_rsq) * 1e-3) / 1e9;
    out[3] = 2.0 * per * it_f64 / (best_ms(3, it_f64) * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    return e == cudaSuccess ? UCP_OK : UCP_ECUDA;
}
