// FP32 arithmetic peak of the device, measured: the roofline that bounds the
// mixed-precision element kernels is the FP32 pipe, and its denominator is
// this measurement (not a figure derived from unit counts and the clock).
//
// Every thread runs eight independent multiply-add chains (sixteen steps
// per loop trip, so the chains hide the FMA latency), either scalar FFMA or
// paired FFMA2 on float2; grid = 8 CTAs of 256 threads per SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fea_internal.h"

namespace fea {
namespace {

constexpr int kChains = 8, kSteps = 16;

__global__ void __launch_bounds__(256) k_fma_chain(float *sink, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = threadIdx.x * 1e-6f + (float)j;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int r = 0; r < kSteps; ++r)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 1234.5f) sink[0] = s;   // keeps the chains live; never true for the inputs used
}

__global__ void __launch_bounds__(256) k_fma2_chain(float *sink, int iters, float b, float c) {
    float2 a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = make_float2(threadIdx.x * 1e-6f + (float)j, 0.5f * (float)j);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int r = 0; r < kSteps; ++r)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], bb, cc);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j].x + a[j].y;
    if (s == 1234.5f) sink[0] = s;
}

}  // namespace

cudaError_t measure_fp32_peak(int sms, cudaStream_t s, double *tflops_ffma, double *tflops_ffma2) {
    float *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int grid = 8 * std::max(sms, 1), threads = 256, iters = 2000;
    const double flops = 2.0 * (double)grid * threads * iters * kSteps * kChains;   // a multiply-add counts 2
    double best[2] = {0.0, 0.0};
    if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
        for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
                if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
                if (kind == 0)
                    k_fma_chain<<<grid, threads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
                else
                    k_fma2_chain<<<grid, threads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
                if ((e = cudaGetLastError()) != cudaSuccess) break;
                if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                float ms = 0.f;
                if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
                const double per_flop = kind == 0 ? 1.0 : 2.0;   // FFMA2: two multiply-adds per step
                if (rep > 0 && ms > 0.f) best[kind] = std::max(best[kind], per_flop * flops / (ms * 1e-3) / 1e12);
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    *tflops_ffma = best[0];
    *tflops_ffma2 = best[1];
    return cudaSuccess;
}

}  // namespace fea
