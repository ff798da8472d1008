// pf_static.cu -- pf_ms_residual_static: the residual reduction of the
// Moulinec-Suquet pass without any device allocation.
//
// Its per-CTA partial sums and its result live in one file-scope
// __device__ array (g_scratch below, 256 KB + 16 bytes).  Every GPU that loads
// this library holds that array until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress while that device is
// current, and every later call on the device reuses it.
#include <cuda_runtime.h>

#include <mutex>

#include "pf.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int kVoxPerBlock = kThreads * kPerThread;  // 4096 voxels per CTA
constexpr int kMaxBlocks = 16384;
constexpr long long kMaxVoxels = (long long)kMaxBlocks * kVoxPerBlock;  // 67,108,864
constexpr int kMaxDevices = 64;

// [0, 2*kMaxBlocks): per-CTA partial sums; [2*kMaxBlocks, +2): the result.
// Every slot a call reads is written earlier in the same call, so nothing
// has to be cleared between calls.
static __device__ __align__(256) double g_scratch[2 * kMaxBlocks + 2];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (looked up once).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Sum over the CTA's voxels of w_c (new_c - old_c)^2 and w_c new_c^2,
// w = 1 for normal and 2 for shear components (Frobenius norm of the tensor).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_resid_partials(const T* __restrict__ nw, const T* __restrict__ od,
                                                             long long n, double* part) {
    T a0 = 0, a1 = 0;
    const long long base = (long long)blockIdx.x * kVoxPerBlock + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const T w = c < 3 ? (T)1 : (T)2;
#pragma unroll 4
        for (int k = 0; k < kPerThread; ++k) {
            const long long i = base + (long long)k * kThreads;
            if (i < n) {
                const T v = nw[c * n + i];
                const T d = v - od[c * n + i];
                a0 += w * d * d;
                a1 += w * v * v;
            }
        }
    }
    __shared__ double red[kThreads / 32][2];
    double s0 = (double)a0, s1 = (double)a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = s0;
        red[threadIdx.x >> 5][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0;
        for (int wi = 0; wi < kThreads / 32; ++wi) s += red[wi][threadIdx.x];
        part[2 * blockIdx.x + threadIdx.x] = s;
    }
}

// Fixed-order sum of the partials into part[2 * kMaxBlocks + {0, 1}].
__global__ void __launch_bounds__(kThreads) k_resid_final(double* part, int nb) {
    __shared__ double sh[kThreads];
    for (int k = 0; k < 2; ++k) {
        double s = 0;
        for (int b = threadIdx.x; b < nb; b += kThreads) s += part[2 * b + k];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = kThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[2 * kMaxBlocks + k] = sh[0];
        __syncthreads();
    }
}

}  // namespace

extern "C" int pf_ms_residual_static(const void* eps_new, const void* eps_old, long long n_voxels, int precision,
                                     double out[2], void* stream) {
    if (!eps_new || !eps_old || !out || n_voxels < 1) return PF_EINVAL;
    if (precision != PF_FP32 && precision != PF_FP64) return PF_EINVAL;
    if (n_voxels > kMaxVoxels) return PF_EINVAL;  // beyond the fixed scratch array
    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return PF_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = (int)((n_voxels + kVoxPerBlock - 1) / kVoxPerBlock);
    if (precision == PF_FP32)
        k_resid_partials<float><<<nb, kThreads, 0, st>>>(static_cast<const float*>(eps_new),
                                                          static_cast<const float*>(eps_old), n_voxels, scratch);
    else
        k_resid_partials<double><<<nb, kThreads, 0, st>>>(static_cast<const double*>(eps_new),
                                                           static_cast<const double*>(eps_old), n_voxels, scratch);
    if (cudaGetLastError() != cudaSuccess) return PF_ECUDA;
    k_resid_final<<<1, kThreads, 0, st>>>(scratch, nb);
    if (cudaGetLastError() != cudaSuccess) return PF_ECUDA;
    if (cudaMemcpyAsync(out, scratch + 2 * kMaxBlocks, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PF_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PF_ECUDA;
    return PF_OK;
}
