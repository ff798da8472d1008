// pf_peak.cu -- measured arithmetic peaks of the device (measurement helper
// for the roofline of the passes that arithmetic, not memory, bounds).
//
// Every thread runs eight independent multiply-add chains (x <- x a + b) in
// the requested precision -- scalar FP32, paired FP32 (fma.rn.f32x2, two
// lanes per instruction) or FP64 -- over a grid of eight 256-thread CTAs per
// SM; the rate is 2 flops per multiply-add over the CUDA-event time of the
// launch, the best of several launches after warm-up.
#include <cuda_runtime.h>

#include "pf.h"
#include "pf_f2.cuh"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* sink, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(256) k_fma2_chains(float* sink, int iters, float a, float b) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((threadIdx.x + c) * 1e-3f, (threadIdx.x + 2 * c) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = pfk::ffma2(x[c], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1.f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int pf_fma_peak(int kind, double* flop_per_s, void* stream) {
    if (!flop_per_s || kind < 0 || kind > 2) return PF_EINVAL;
    *flop_per_s = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PF_ECUDA;
    const int blocks = nsm * 8, threads = 256;
    // about a millisecond of work per launch at the nominal rates
    const int iters = kind == 2 ? 256 : 8192;
    double* sink = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    cudaEvent_t e0, e1;
    int r = PF_OK;
    if (cudaEventCreate(&e0) != cudaSuccess) r = PF_ECUDA;
    if (r == PF_OK && cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        r = PF_ECUDA;
    }
    if (r != PF_OK) {
        cudaFree(sink);
        return r;
    }
    auto launch = [&]() {
        if (kind == 0) k_fma_chains<float><<<blocks, threads, 0, st>>>((float*)sink, iters, 0.9999999f, 1e-7f);
        else if (kind == 1) k_fma2_chains<<<blocks, threads, 0, st>>>((float*)sink, iters, 0.9999999f, 1e-7f);
        else k_fma_chains<double><<<blocks, threads, 0, st>>>(sink, iters, 0.9999999, 1e-7);
        return cudaGetLastError();
    };
    float best = -1.f;
    for (int rep = 0; rep < 13 && r == PF_OK; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess || launch() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) {
            r = PF_ECUDA;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = PF_ECUDA;
        if (rep >= 3 && ms > 0.f && (best < 0.f || ms < best)) best = ms;  // three warm-up launches
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (r != PF_OK || best <= 0.f) return r != PF_OK ? r : PF_ECUDA;
    const double lanes = kind == 1 ? 2.0 : 1.0;
    const double fmas = (double)blocks * threads * kChains * iters * lanes;
    *flop_per_s = 2.0 * fmas / (best * 1e-3);
    return PF_OK;
}
