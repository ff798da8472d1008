// pf_yzfix.cuh -- FP32 passes along y and z with compile-time transform
// plans and tile widths (kernel templates; pf_yzfix.cu instantiates the
// power-of-two plans, pf_yzfix_pfa.cu those with a prime-factor radix).
//
// The tiles are the TMA boxes of the generic passes (pf_k_yz.cu): TW kx
// columns x N planes of one component (y) or of every component (z), kx
// innermost, element i of column p at i * TW + p.  For the lengths the
// workloads use most (64 = 8 x 8, 128 = 16 x 8 or 8 x 16, 256 = 16 x 16;
// 80 = 16 x 5, 96 = 16 x 6, 120 = 12 x 10, 160 = 16 x 10; 512 = 16 x 32) the two Stockham
// stages run with the plan, the tile width and the component pitch as
// compile-time constants, so each shared-memory access is a per-thread base
// plus an immediate offset.  Threads take the column fastest, then the
// butterfly, then the component, so a warp sweeps contiguous tile rows; a
// pencil spans warps, so the stages are separated by CTA barriers.  The
// per-mode operators of the z pass are those of the generic pass.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf_device.cuh"
#include "pf_dft32.cuh"
#include "pf_pfa.cuh"

namespace pfk {

namespace {

__device__ __forceinline__ int freq_fix(int k, int n) { return (2 * k < n) ? k : k - n; }
__device__ __forceinline__ bool nyq_fix(int k, int n) { return (n % 2 == 0) && (2 * k == n); }

// complex elements between component tiles (128-byte aligned)
template <int N, int TW> constexpr int comp_pitch() { return (N * TW * 8 + 127) / 128 * 128 / 8; }

// Two-stage transform of the nc component tiles at s (pitch CS): thread t
// serves column t % TW, butterfly (t / TW) % TPP of component t / (TW TPP)
// of each round of components.  tw[m] = exp(-2 pi i m / N).  Every thread of
// the CTA must call it.
//
// Between the stages, output k1 of stage-1 butterfly n1 sits in tile row
// n1 R1 + (k1 ^ (n1 & SW)) instead of n1 R1 + k1.  A 128-byte bank line holds
// 16 / TW tile rows; a warp's stage-1 store (one k1, 32 / TW consecutive n1)
// would otherwise put all its rows R1 apart, in the same part of the line
// (2 x the shared-memory wavefronts for TW = 8).  The swizzle permutes k1
// within aligned groups of SW + 1 (the largest power of two up to 16 / TW
// that divides R1), so the stage-2 loads of a warp (consecutive k1, one n1)
// still cover whole lines.  Each residue of the unrolled index mod SW + 1
// gets its own base pointer, so every access keeps an immediate offset.
// the radices of the compile-time plans: dft_any, and 32 (pf_dft32.cuh)
template <int R, bool INV> __device__ __forceinline__ void dft_tile(float2* v) {
    if constexpr (R == 32) dft32<float, INV>(v);
    else dft_any<float, R, INV>(v);
}

template <int R1, int TW> constexpr int swizzle_mask(int g = 16) {
    return (g <= 1) ? 0 : ((g <= 16 / TW && R1 % g == 0) ? g - 1 : swizzle_mask<R1, TW>(g / 2));
}

template <int N, int R1, int R2, int TW, int CS, bool INV>
__device__ __forceinline__ void fft_tile(float2* s, int nc, const float2* __restrict__ tw) {
    constexpr int nb1 = N / R1, nb2 = N / R2;
    static_assert(nb2 == R1, "two-stage plan");
    constexpr int TPP = nb1 > nb2 ? nb1 : nb2;
    constexpr int SW = swizzle_mask<R1, TW>();
    static_assert(R1 % (SW + 1) == 0 && (TPP * TW) % 32 == 0 && 32 % TW == 0 && TPP % (32 / TW) == 0,
                  "a warp covers whole swizzle groups of one component");
    constexpr int PER = TW * TPP;  // threads per component
    const int cpr = (int)blockDim.x / PER;
    const int p = threadIdx.x % TW;
    const int j = (threadIdx.x / TW) % TPP;
    const int cr = threadIdx.x / PER;
    for (int c0 = 0; c0 < nc; c0 += cpr) {
        const int c = c0 + cr;
        const bool live = cr < cpr && c < nc;
        float2* sp = s + (live ? c : 0) * CS + p;
        float2 v[R1 > R2 ? R1 : R2];
        const bool a1 = live && j < nb1;
        if (a1) {
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = sp[(j + r * nb1) * TW];
            dft_tile<R1, INV>(v);
        }
        __syncthreads();
        if (a1) {
            float2* b[SW + 1];
#pragma unroll
            for (int q = 0; q <= SW; ++q) b[q] = sp + (j * R1 + ((q ^ (j & SW)) - q)) * TW;
#pragma unroll
            for (int r = 0; r < R1; ++r) b[r & SW][r * TW] = v[r];
        }
        __syncthreads();
        const bool a2 = live && j < nb2;
        if (a2) {
            const float2* b[SW + 1];
#pragma unroll
            for (int q = 0; q <= SW; ++q) b[q] = sp + (j ^ q) * TW;
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = b[r & SW][r * R1 * TW];
#pragma unroll
            for (int r = 1; r < R2; ++r) {
                const float2 w = __ldg(&tw[r * j]);
                v[r] = INV ? cmulc<float>(v[r], w) : cmul<float>(v[r], w);
            }
            dft_tile<R2, INV>(v);
        }
        __syncthreads();
        if (a2) {
#pragma unroll
            for (int r = 0; r < R2; ++r) sp[(j + r * R1) * TW] = v[r];
        }
        __syncthreads();
    }
}

template <int N, int R1, int R2> constexpr int tpp_of() { return (N / R1) > (N / R2) ? (N / R1) : (N / R2); }

// ---------------------------------------------------------------------------
// y pass: TW columns of one z plane of one component, one transform round
// ---------------------------------------------------------------------------
template <int N, int R1, int R2, int TW, bool INV>
__global__ void __launch_bounds__(TW * tpp_of<N, R1, R2>()) k_y_fix(YArgs a, const __grid_constant__ CUtensorMap tm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
    __shared__ __align__(8) uint64_t bar;
    const int by = a.box;
    const int kx0 = blockIdx.x * TW;
    const int zc = blockIdx.z * a.g.nz + blockIdx.y;
    // PF_CHECK: the tile inside the field and the launch's shared memory
    if (!pf_check(kx0 < a.g.nxh && a.g.ny == N && (int)blockIdx.y < a.g.nz, a.err) ||
        !pf_check_smem(smem_raw, s + N * TW, a.err))
        return;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, (uint32_t)(N * TW * sizeof(float2)));
        for (int y0 = 0; y0 < N; y0 += by) tma_load_3d(s + y0 * TW, &tm, &bar, 2 * kx0, y0, zc);
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    fft_tile<N, R1, R2, TW, N * TW, INV>(s, 1, (const float2*)a.tw);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int y0 = 0; y0 < N; y0 += by) tma_store_3d(&tm, s + y0 * TW, 2 * kx0, y0, zc);
        bulk_commit();
        bulk_wait_read_all();
    }
}

// eps_hat = -Gamma0 : tau_hat at one mode, frequencies m = xi / (2 pi) per
// axis: K_ik = sum_m B[ik][m] q_m (sB, q = (x^2, y^2, z^2, yz, xz, xy)),
// N = K^-1 by cofactors, t = tau_hat m, u = -N t, eps_hat = sym(u (x) m).
// Components in Voigt order (xx, yy, zz, yz, xz, xy).
__device__ __forceinline__ void green_mode(const float* sB, float mx, float my, float mz, const float2 (&tt)[6],
                                           float2 (&o)[6]) {
    const float q[6] = {mx * mx, my * my, mz * mz, my * mz, mx * mz, mx * my};
    float K[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float t = 0;
#pragma unroll
        for (int jj = 0; jj < 6; ++jj) t += sB[i * 6 + jj] * q[jj];
        K[i] = t;
    }
    // K = [[K0 K5 K4] [K5 K1 K3] [K4 K3 K2]]
    const float c00 = K[1] * K[2] - K[3] * K[3];
    const float c11 = K[0] * K[2] - K[4] * K[4];
    const float c22 = K[0] * K[1] - K[5] * K[5];
    const float c01 = K[4] * K[3] - K[5] * K[2];
    const float c02 = K[5] * K[3] - K[4] * K[1];
    const float c12 = K[5] * K[4] - K[0] * K[3];
    const float inv = 1.f / (K[0] * c00 + K[5] * c01 + K[4] * c02);
    const float2 txx = tt[0], tyy = tt[1], tzz = tt[2], tyz = tt[3], txz = tt[4], txy = tt[5];
    const float2 t0 = make_float2(txx.x * mx + txy.x * my + txz.x * mz, txx.y * mx + txy.y * my + txz.y * mz);
    const float2 t1 = make_float2(txy.x * mx + tyy.x * my + tyz.x * mz, txy.y * mx + tyy.y * my + tyz.y * mz);
    const float2 t2 = make_float2(txz.x * mx + tyz.x * my + tzz.x * mz, txz.y * mx + tyz.y * my + tzz.y * mz);
    const float n00 = -c00 * inv, n11 = -c11 * inv, n22 = -c22 * inv;
    const float n01 = -c01 * inv, n02 = -c02 * inv, n12 = -c12 * inv;
    const float2 u0 = make_float2(n00 * t0.x + n01 * t1.x + n02 * t2.x, n00 * t0.y + n01 * t1.y + n02 * t2.y);
    const float2 u1 = make_float2(n01 * t0.x + n11 * t1.x + n12 * t2.x, n01 * t0.y + n11 * t1.y + n12 * t2.y);
    const float2 u2 = make_float2(n02 * t0.x + n12 * t1.x + n22 * t2.x, n02 * t0.y + n12 * t1.y + n22 * t2.y);
    const float h = 0.5f;
    o[0] = make_float2(u0.x * mx, u0.y * mx);
    o[1] = make_float2(u1.x * my, u1.y * my);
    o[2] = make_float2(u2.x * mz, u2.y * mz);
    o[3] = make_float2(h * (u1.x * mz + u2.x * my), h * (u1.y * mz + u2.y * my));
    o[4] = make_float2(h * (u0.x * mz + u2.x * mx), h * (u0.y * mz + u2.y * mx));
    o[5] = make_float2(h * (u0.x * my + u1.x * mx), h * (u0.y * my + u1.y * mx));
}

// ---------------------------------------------------------------------------
// z pass: TW columns of one ky of every component, forward transform, the
// per-mode operator, inverse transform
// ---------------------------------------------------------------------------
constexpr int kZThreads = 256;
// The Green pass (six components, two 98 KB CTAs per SM) runs 384 threads:
// three components per transform round instead of two (1/3 fewer CTA
// barriers, 24 warps per SM); the per-component passes, split into
// three-component CTAs at four per SM, keep 256.
template <int MODE> constexpr int z_threads() { return MODE == Z_GREEN ? 384 : kZThreads; }

template <int N, int R1, int R2, int TW, int MODE>
__device__ __forceinline__ void z_fix_body(const ZArgs& a, const CUtensorMap& tm) {
    constexpr int ZT = z_threads<MODE>();
    constexpr int CS = comp_pitch<N, TW>();
    constexpr int LOGTW = TW == 16 ? 4 : TW == 8 ? 3 : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
    __shared__ float sB[36];  // K_ik = sum_m B[ik][m] q_m, q = (x^2, y^2, z^2, yz, xz, xy)
    __shared__ __align__(8) uint64_t bar;
    const GridDesc g = a.g;
    // components cb .. cb + nc - 1 of the field (a per-component operator may
    // split them over blockIdx.z; the Green operator takes all six)
    const int cb = blockIdx.z * a.cpc;
    const int nc = min(a.cpc, a.ncomp - cb), ny = g.ny, bz = a.box;
    const int kx0 = blockIdx.x * TW;
    const int ky = blockIdx.y;
    const int ncol = min(TW, g.nxh - kx0);
    // PF_CHECK: the tile inside the field and the launch's shared memory
    if (!pf_check(kx0 < g.nxh && ky < ny && g.nz == N && nc >= 1 && nc <= 6 && a.cstride == CS &&
                      (MODE != Z_GREEN || (cb == 0 && nc == 6)) && (MODE != Z_ENERGY || gridDim.z == 1),
                  a.err) ||
        !pf_check_smem(smem_raw, s + nc * CS, a.err))
        return;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    if (MODE == Z_GREEN && threadIdx.x < 36) {
        // B[(i,k)][(j,l)] = C0_ijkl (+ C0_ilkj for j != l), C0 in Voigt form
        const int pair = threadIdx.x / 6, mono = threadIdx.x % 6;
        const int PI[6] = {0, 1, 2, 1, 0, 0}, PK[6] = {0, 1, 2, 2, 2, 1};
        const int i = PI[pair], k = PK[pair];
        const int jj = PI[mono], l = PK[mono];
        auto vo = [](int p, int q) { return p == q ? p : 6 - p - q; };
        double b = a.C0[vo(i, jj) * 6 + vo(k, l)];
        if (jj != l) b += a.C0[vo(i, l) * 6 + vo(k, jj)];
        sB[threadIdx.x] = (float)b;
    }
    if (MODE != Z_GREEN && a.A && threadIdx.x < 6 * nc) sB[threadIdx.x] = (float)a.A[6 * cb + threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, (uint32_t)(nc * N * TW * sizeof(float2)));
        for (int c = 0; c < nc; ++c)
            for (int z0 = 0; z0 < N; z0 += bz) tma_load_4d(s + c * CS + z0 * TW, &tm, &bar, 2 * kx0, ky, z0, cb + c);
        // the tile of the CTA that will start pf_dist CTAs later (linear
        // order x, y, z of the grid), into L2
        if (a.pf_dist > 0) {
            const unsigned pb = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z) + (unsigned)a.pf_dist;
            if (pb < gridDim.x * gridDim.y * gridDim.z) {
                const int pbx = (int)(pb % gridDim.x), rest = (int)(pb / gridDim.x);
                const int pby = rest % (int)gridDim.y, pbz = rest / (int)gridDim.y;
                const int pcb = pbz * a.cpc, pnc = min(a.cpc, a.ncomp - pcb);
                for (int c = 0; c < pnc; ++c)
                    for (int z0 = 0; z0 < N; z0 += bz) tma_prefetch_4d(&tm, 2 * pbx * TW, pby, z0, pcb + c);
            }
        }
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    fft_tile<N, R1, R2, TW, CS, false>(s, nc, (const float2*)a.tw);

    float acc = 0;
    const float two_pi = 6.283185307179586477f;
    const float rnx = 1.f / (float)g.nx, rnz = 1.f / (float)N;
    const float my = (float)freq_fix(ky, ny) * (1.f / (float)ny);
    const bool nyq_y = nyq_fix(ky, ny);
    for (int e = threadIdx.x; e < N * TW; e += ZT) {
        const int p = e & (TW - 1), z = e >> LOGTW;
        if (p >= ncol) continue;
        const int kx = kx0 + p;
        const float mx = (float)kx * rnx, mz = (float)freq_fix(z, N) * rnz;
        float2* m = s + e;
        if (MODE == Z_GREEN) {
            const bool zero = (kx == 0 && ky == 0 && z == 0) || nyq_fix(kx, g.nx) || nyq_y || nyq_fix(z, N);
            if (zero) {
#pragma unroll
                for (int c = 0; c < 6; ++c) m[c * CS] = make_float2(0.f, 0.f);
                continue;
            }
            const float2 tt[6] = {m[0], m[CS], m[2 * CS], m[3 * CS], m[4 * CS], m[5 * CS]};
            float2 o[6];
            green_mode(sB, mx, my, mz, tt, o);
#pragma unroll
            for (int c = 0; c < 6; ++c) m[c * CS] = o[c];
        } else {
            const float kx2 = two_pi * mx, ky2 = two_pi * my, kz2 = two_pi * mz;
            const float k2 = kx2 * kx2 + ky2 * ky2 + kz2 * kz2;
            // anisotropic symbol xi.A_c.xi: squares, and cross terms only where
            // neither index is at the Nyquist frequency
            float q[6];
            if (a.A) {
                const bool ox = !nyq_fix(kx, g.nx), oy = !nyq_y, oz = !nyq_fix(z, N);
                q[0] = kx2 * kx2;
                q[1] = ky2 * ky2;
                q[2] = kz2 * kz2;
                q[3] = (oy && oz) ? 2.f * ky2 * kz2 : 0.f;
                q[4] = (ox && oz) ? 2.f * kx2 * kz2 : 0.f;
                q[5] = (ox && oy) ? 2.f * kx2 * ky2 : 0.f;
            }
            auto symbol = [&](int c) {
                float t = 0;
#pragma unroll
                for (int i = 0; i < 6; ++i) t += sB[c * 6 + i] * q[i];
                return t;
            };
            if (MODE == Z_HELM) {
                if (a.A) {
                    for (int c = 0; c < nc; ++c)
                        m[c * CS] = cscale<float>(m[c * CS], 1.f / (1.f + (float)a.dtc3 * symbol(c)));
                } else {
                    const float fac = 1.f / (1.f + (float)a.helm * k2);
                    for (int c = 0; c < nc; ++c) m[c * CS] = cscale<float>(m[c * CS], fac);
                }
            } else if (MODE == Z_LAPL) {  // the gradient operator: -c2 |xi|^2 or -xi.A.xi
                for (int c = 0; c < nc; ++c)
                    m[c * CS] = cscale<float>(m[c * CS], -(a.A ? symbol(c) : (float)a.c2 * k2));
            } else {  // Z_ENERGY: half-spectrum weight 2 except kx = 0 and kx = nx/2
                const float w = (kx == 0 || nyq_fix(kx, g.nx)) ? 1.f : 2.f;
                float sum = 0;
                for (int c = 0; c < nc; ++c) {
                    const float2 v = m[c * CS];
                    sum += (a.A ? symbol(c) : k2) * (v.x * v.x + v.y * v.y);
                }
                acc += w * sum;
            }
        }
    }
    if (MODE == Z_ENERGY) {
        const float d[1] = {acc};
        block_sum_store<1, float>(d, a.partials + (size_t)(blockIdx.y * gridDim.x + blockIdx.x));
        return;
    }
    __syncthreads();
    fft_tile<N, R1, R2, TW, CS, true>(s, nc, (const float2*)a.tw);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < nc; ++c)
            for (int z0 = 0; z0 < N; z0 += bz) tma_store_4d(&tm, s + c * CS + z0 * TW, 2 * kx0, ky, z0, cb + c);
        bulk_commit();
        bulk_wait_read_all();
    }
}

template <int N, int R1, int R2, int TW>
cudaError_t y_plan(bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    constexpr int threads = TW * tpp_of<N, R1, R2>();
    if (inv) {
        allow_smem(k_y_fix<N, R1, R2, TW, true>, smem);
        k_y_fix<N, R1, R2, TW, true><<<grid, threads, smem, st>>>(a, tm);
    } else {
        allow_smem(k_y_fix<N, R1, R2, TW, false>, smem);
        k_y_fix<N, R1, R2, TW, false><<<grid, threads, smem, st>>>(a, tm);
    }
    return cudaGetLastError();
}

// tile widths a plan is built for: a warp covers whole swizzle groups of
// one component (TPP * TW a multiple of 32)
template <int N, int R1, int R2, int TW> constexpr bool tw_ok() { return (tpp_of<N, R1, R2>() * TW) % 32 == 0; }

template <int N, int R1, int R2>
cudaError_t y_tw(bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    switch (a.tx) {
        case 8:
            if constexpr (tw_ok<N, R1, R2, 8>()) return y_plan<N, R1, R2, 8>(inv, a, tm, grid, smem, st);
            return cudaErrorNotSupported;
        case 16:
            if constexpr (tw_ok<N, R1, R2, 16>()) return y_plan<N, R1, R2, 16>(inv, a, tm, grid, smem, st);
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

template <int N, int R1, int R2, int TW, int MODE>
__global__ void __launch_bounds__(z_threads<MODE>()) k_z_fix(ZArgs a, const __grid_constant__ CUtensorMap tm) {
    z_fix_body<N, R1, R2, TW, MODE>(a, tm);
}

// The 512-point plan: its radix-32 stage left the compiler free to take
// 100-170 registers, one CTA per SM; this copy is compiled for two (80
// registers for the Green pass, 128 for the others).
template <int N, int R1, int R2, int TW, int MODE>
__global__ void __launch_bounds__(z_threads<MODE>(), 2) k_z_fix2(ZArgs a, const __grid_constant__ CUtensorMap tm) {
    z_fix_body<N, R1, R2, TW, MODE>(a, tm);
}

template <int N, int R1, int R2, int TW, int MODE>
cudaError_t z_launch(const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    if constexpr (N == 512) {
        allow_smem(k_z_fix2<N, R1, R2, TW, MODE>, smem);
        k_z_fix2<N, R1, R2, TW, MODE><<<grid, z_threads<MODE>(), smem, st>>>(a, tm);
    } else {
        allow_smem(k_z_fix<N, R1, R2, TW, MODE>, smem);
        k_z_fix<N, R1, R2, TW, MODE><<<grid, z_threads<MODE>(), smem, st>>>(a, tm);
    }
    return cudaGetLastError();
}

template <int N, int R1, int R2, int TW>
cudaError_t z_plan(int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    switch (mode) {
        case Z_GREEN: return z_launch<N, R1, R2, TW, Z_GREEN>(a, tm, grid, smem, st);
        case Z_HELM: return z_launch<N, R1, R2, TW, Z_HELM>(a, tm, grid, smem, st);
        case Z_LAPL: return z_launch<N, R1, R2, TW, Z_LAPL>(a, tm, grid, smem, st);
        default: return z_launch<N, R1, R2, TW, Z_ENERGY>(a, tm, grid, smem, st);
    }
}

template <int N, int R1, int R2>
cudaError_t z_tw(int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    switch (a.tz) {
        case 4:
            if constexpr (tw_ok<N, R1, R2, 4>()) return z_plan<N, R1, R2, 4>(mode, a, tm, grid, smem, st);
            return cudaErrorNotSupported;
        case 8:
            if constexpr (tw_ok<N, R1, R2, 8>()) return z_plan<N, R1, R2, 8>(mode, a, tm, grid, smem, st);
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

}  // namespace

// launchers of the plans with a prime-factor radix (pf_yzfix_pfa.cu); id as
// returned by plan_id
cudaError_t launch_y_fix_pfa(int id, bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                             cudaStream_t st);
cudaError_t launch_z_fix_pfa(int id, int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                             cudaStream_t st);

}  // namespace pfk
