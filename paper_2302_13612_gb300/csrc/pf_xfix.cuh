// pf_xfix.cuh -- FP32 passes along x with compile-time transform plans
// (kernel templates; pf_xfix.cu instantiates the power-of-two plans of up to
// 256 points, pf_xfix_pfa.cu those of 80, 96, 120, 160 and 512 points).
//
// For the row lengths the workloads use most (N = 64, 128, 256 as two radix
// stages R1 x R2 with R1, R2 in {8, 16}; 80 = 16 x 5, 96 = 16 x 6,
// 120 = 12 x 10 and 160 = 16 x 10, the radices 6, 10 and 12 as prime-factor
// DFTs; 512 = 16 x 32,
// one warp per pencil) the x passes run
// a two-stage Stockham transform whose lengths, radices and strides are
// compile-time constants.  The pencils sit pencil-major in shared memory
// (pencil q at q * kPitch, element i at padded(i) = i + i / 16), so every
// shared-memory access is a per-thread base plus an immediate offset, and
// each pencil is served by the N / min(R1, R2) threads of one warp (16
// lanes for 120 = 12 x 10, of which 12 work)
// (stages separated by __syncwarp).  The element-wise producers
// (polarisation, driving force) and consumers (strain and residual, fields,
// pad corrections) are the same device functions as in the generic passes
// (pf_k_xfwd.cu, pf_k_xinv.cu); inputs and outputs move by cp.async.bulk as
// there.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf_device.cuh"
#include "pf_dft32.cuh"
#include "pf_pfa.cuh"

namespace pfk {

namespace {

// the radices of the compile-time plans: dft_any, and 32 (pf_dft32.cuh)
template <int R, bool INV> __device__ __forceinline__ void dft_x(float2* v) {
    if constexpr (R == 32) dft32<float, INV>(v);
    else dft_any<float, R, INV>(v);
}

// Lanes that serve one pencil: its TPP = N / min(R1, R2) butterfly threads,
// rounded up to a power of two so that a pencil never straddles two warps
// (120 = 12 x 10: 12 threads on 16 lanes); equal to TPP for the other plans.
template <int N, int R1, int R2> constexpr int fix_lanes() {
    constexpr int tpp = N / (R1 < R2 ? R1 : R2);
    return tpp <= 4 ? 4 : tpp <= 8 ? 8 : tpp <= 16 ? 16 : 32;
}

// row and column of voxel e of a row block (unsigned: shifts and masks when
// N is a power of two)
template <int N> __device__ __forceinline__ int row_of(int e) { return (int)((unsigned)e / (unsigned)N); }
template <int N> __device__ __forceinline__ int col_of(int e) { return (int)((unsigned)e % (unsigned)N); }


constexpr int kFixThreads = 256;

template <int N> struct Fix {
    static constexpr int kPitch = N + N / 16;  // complex elements per pencil
};

// Two Stockham stages over one pencil starting at sp (butterfly j of each
// stage; threads j >= the stage's butterfly count idle).  Stage 1 (radix
// R1, no twiddles) maps x[j + r N/R1] to y[j R1 + r]; stage 2 (radix R2,
// span R1) multiplies y[j + r R1] by exp(-+2 pi i r j / N) (table tws,
// [r - 1][j]) and leaves X[j + r R1] in natural order.  Every thread of the
// warp must call it.
template <int N, int R1, int R2, bool INV>
__device__ __forceinline__ void fft_fix(float2* sp, int j, bool live, const float2* __restrict__ tws) {
    constexpr int nb1 = N / R1, nb2 = N / R2;
    static_assert(nb2 == R1, "two-stage plan");
    float2 v[R1 > R2 ? R1 : R2];
    const bool a1 = live && j < nb1;
    if (a1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = sp[padded(j + r * nb1)];
        dft_x<R1, INV>(v);
    }
    __syncwarp();
    if (a1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) sp[padded(j * R1 + r)] = v[r];
    }
    __syncwarp();
    const bool a2 = live && j < nb2;
    if (a2) {
#pragma unroll
        for (int r = 0; r < R2; ++r) v[r] = sp[padded(j + r * R1)];
#pragma unroll
        for (int r = 1; r < R2; ++r) {
            const float2 w = __ldg(&tws[(r - 1) * R1 + j]);
            v[r] = INV ? cmulc<float>(v[r], w) : cmul<float>(v[r], w);
        }
        dft_x<R2, INV>(v);
    }
    __syncwarp();
    if (a2) {
#pragma unroll
        for (int r = 0; r < R2; ++r) sp[padded(j + r * R1)] = v[r];
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// forward pass: producer, R2C transform of packed pairs, split, bulk store
// ---------------------------------------------------------------------------
// Shared memory: [staging | pencils]; the staging holds the inputs (twin
// fractions by group position, strain, plastic strain, grain ids) and then
// the output rows [c][r][P].
// Resident CTAs per SM the forward pass is compiled for: four (64 registers)
// except the driving force, whose longer per-voxel state runs faster at
// three (80 registers), and the 512-point plan, whose radix-32 stage holds 32
// complex values per thread (two, 128 registers).
template <int N, int MODE> constexpr int fwd_min_ctas() { return N == 512 ? 2 : MODE == X_DRIVE ? 3 : 4; }
// the inverse passes: four, two for the radix-32 stage of 512 points
template <int N> constexpr int inv_min_ctas() { return N == 512 ? 2 : 4; }

// FULL: all six variant ids evolved (three groups of two), so the material
// model's group loops have compile-time bounds (the polarisation passes).
template <int N, int R1, int R2, int MODE, bool FULL>
__global__ void __launch_bounds__(kFixThreads, fwd_min_ctas<N, MODE>()) k_x_fwd_fix(XFwdArgs a) {
    using T = float;
    constexpr int TPP = fix_lanes<N, R1, R2>();
    constexpr int PPR = kFixThreads / TPP;  // pencils per round
    constexpr int PITCH = Fix<N>::kPitch;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) T sC0[24];
    const GridDesc g = a.g;
    const int nfin = a.nfin;
    const int npen = (a.ncomp + 1) / 2;
    const int nP = a.rows * npen;
    const int row0 = blockIdx.x * a.rows;
    const int nrow = min(a.rows, g.nrows - row0);
    const int RN = a.rows * N;
    const long long off = (long long)row0 * N;
    const bool stage_grain = a.grain && a.stage_grain;
    T* s_f = reinterpret_cast<T*>(base);  // twin fractions by position
    T* s_eps = s_f + nfin * RN;
    T* s_ep = s_eps + (MODE == X_PLAIN ? 0 : 6 * RN);
    uint16_t* s_g = reinterpret_cast<uint16_t*>(s_ep + (a.eps_p ? 6 * RN : 0));
    float2* s = reinterpret_cast<float2*>(base + a.stage_bytes);
    // PF_CHECK: staging in and out of the buffer, pencils inside the launch's shared memory
    if (!pf_check(row0 < g.nrows && nfin <= 6 && a.ncomp <= 6 && g.P == (N / 2 + 1 + 3) / 4 * 4 &&
                      (size_t)(nfin + (MODE == X_PLAIN ? 0 : 6 + (a.eps_p ? 6 : 0))) * RN * sizeof(T) +
                              (MODE != X_PLAIN && stage_grain ? (size_t)RN * 2 : 0) <=
                          (size_t)a.stage_bytes &&
                      (size_t)a.ncomp * a.rows * g.P * sizeof(float2) <= (size_t)a.stage_bytes,
                  a.err) ||
        !pf_check_smem(smem_raw, s + nP * PITCH, a.err))
        return;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    if ((MODE == X_TAU || MODE == X_TAU_SIG) && threadIdx.x < 24) load_c0<T>(a.C0, sC0);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t rb = (uint32_t)(nrow * N * sizeof(T));
        uint32_t total = 0;
        for (int p = 0; p < nfin; ++p) total += a.fin_slot[p] >= 0 ? rb : 0;
        if (MODE != X_PLAIN) total += 6 * rb + (a.eps_p ? 6 * rb : 0);
        if (MODE != X_PLAIN && stage_grain) total += (uint32_t)(nrow * N * 2);
        mbar_expect_tx(&bar, total);
        const T* f = (const T*)a.f;
        for (int p = 0; p < nfin; ++p)
            if (a.fin_slot[p] >= 0) bulk_load(s_f + p * RN, f + a.fin_slot[p] * g.N + off, rb, &bar);
        if (MODE != X_PLAIN) {
            const T* eps = (const T*)a.eps;
            for (int c = 0; c < 6; ++c) bulk_load(s_eps + c * RN, eps + c * g.N + off, rb, &bar);
            if (a.eps_p) {
                const T* ep = (const T*)a.eps_p;
                for (int c = 0; c < 6; ++c) bulk_load(s_ep + c * RN, ep + c * g.N + off, rb, &bar);
            }
            if (stage_grain) bulk_load(s_g, a.grain + off, (uint32_t)(nrow * N * 2), &bar);
        }
        // the rows of the CTA that will start pf_dist CTAs later, into L2
        const int pb = (int)blockIdx.x + a.pf_dist;
        if (a.pf_dist > 0 && pb < (int)gridDim.x) {
            const int prow0 = pb * a.rows;
            const uint32_t prb = (uint32_t)(min(a.rows, g.nrows - prow0) * N * sizeof(T));
            const long long poff = (long long)prow0 * N;
            for (int p = 0; p < nfin; ++p)
                if (a.fin_slot[p] >= 0) bulk_prefetch_l2(f + a.fin_slot[p] * g.N + poff, prb);
            if (MODE != X_PLAIN) {
                const T* eps = (const T*)a.eps;
                for (int c = 0; c < 6; ++c) bulk_prefetch_l2(eps + c * g.N + poff, prb);
                if (a.eps_p)
                    for (int c = 0; c < 6; ++c) bulk_prefetch_l2((const T*)a.eps_p + c * g.N + poff, prb);
            }
        }
    }
    // grain ids read from global memory one voxel ahead (the first before
    // the rows arrive), so their latency hides under the previous voxel
    const bool gpre = a.grain && !stage_grain && MODE != X_PLAIN;
    int gnext = -1;
    if (gpre) {
        const int e0 = threadIdx.x;
        gnext = (e0 < RN && row_of<N>(e0) < nrow) ? (int)a.grain[off + e0] : 0;
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint16_t* gp = a.grain ? (stage_grain ? s_g : a.grain + off) : nullptr;
    const T* ep = a.eps_p ? s_ep : nullptr;
    for (int e = threadIdx.x; e < a.rows * N; e += kFixThreads) {
        const int r = row_of<N>(e), x = col_of<N>(e);
        const int gcur = gnext;
        if (gpre) {
            const int en = e + kFixThreads;
            gnext = (en < RN && row_of<N>(en) < nrow) ? (int)a.grain[off + en] : 0;
        }
        T out[6] = {0, 0, 0, 0, 0, 0};
        if (r < nrow)
            xfwd_voxel<T, MODE, int, FULL>(a, s_f, nullptr, s_eps, ep, gp, RN, e, off + e, sC0, out, acc, gcur);
        // the polarisation stress always has six components (three pencils)
        constexpr bool SIX = MODE == X_TAU || MODE == X_TAU_SIG;
        float2* row = s + (r * (SIX ? 3 : npen)) * PITCH + padded(x);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (SIX || c < npen) row[c * PITCH] = make_float2(out[2 * c], out[2 * c + 1]);
    }
    __syncthreads();
    // transform and split, each pencil by the TPP threads of one warp; the
    // half-spectrum row (N / 2 + 1 values, padded to 4) is compile-time
    constexpr int P = (N / 2 + 1 + 3) / 4 * 4, nxh = N / 2 + 1;
    float2* o = reinterpret_cast<float2*>(base);
    const int j = threadIdx.x % TPP, qo = threadIdx.x / TPP;
    for (int q0 = 0; q0 < nP; q0 += PPR) {
        const int q = q0 + qo;
        const bool live = q < nP;
        float2* sp = s + (live ? q : 0) * PITCH;
        fft_fix<N, R1, R2, false>(sp, j, live, (const float2*)a.tws);
        if (live) {
            const int r = div_npen(q, npen);
            const int c = q - r * npen;
            float2* oa = o + ((2 * c) * a.rows + r) * P;
            float2* ob = o + ((2 * c + 1) * a.rows + r) * P;
            const bool wb = 2 * c + 1 < a.ncomp;
#pragma unroll
            for (int k0 = 0; k0 < P; k0 += TPP) {
                const int k = k0 + j;
                if (k >= P) break;
                float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
                if (k < nxh) {
                    // A_k = (Z_k + conj Z_{N-k}) / 2, B_k = (Z_k - conj Z_{N-k}) / 2i
                    const float2 z1 = sp[padded(k)];
                    const float2 z2 = sp[padded(k == 0 ? 0 : N - k)];
                    A = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
                    B = make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
                }
                oa[k] = A;
                if (wb) ob[k] = B;
            }
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        float2* spec = (float2*)a.spec;
        const long long cstride = (long long)g.nrows * P;
        for (int c = 0; c < a.ncomp; ++c)
            if (a.out_slot[c] >= 0)
                bulk_store(spec + a.out_slot[c] * cstride + (long long)row0 * P, o + (size_t)c * a.rows * P,
                           (uint32_t)(nrow * P * sizeof(float2)));
        bulk_commit();
    }
    if (MODE == X_DRIVE || MODE == X_TAU_SIG)
        block_sum_store_w<8, T, kFixThreads / 32>(acc, a.partials + (size_t)blockIdx.x * 8);
    if (threadIdx.x == 0) bulk_wait_read_all();
}

// ---------------------------------------------------------------------------
// inverse pass: unpack, C2R transform of packed pairs, consumer, bulk store
// ---------------------------------------------------------------------------
// Shared memory: [spectral rows ncomp x rows x P | old values | pencils];
// the output rows [c][r][N] reuse the spectral staging.
// SIX6: six components (the strain, or six twin fractions) at compile time.
template <int N, int R1, int R2, int MODE, bool SIX6>
__global__ void __launch_bounds__(kFixThreads, inv_min_ctas<N>()) k_x_inv_fix(XInvArgs a) {
    using T = float;
    constexpr int TPP = fix_lanes<N, R1, R2>();
    constexpr int PPR = kFixThreads / TPP;
    constexpr int PITCH = Fix<N>::kPitch;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t bar;
    __shared__ T sE[6];
    const GridDesc g = a.g;
    constexpr int P = (N / 2 + 1 + 3) / 4 * 4, nxh = N / 2 + 1;  // the FP32 half-spectrum row
    const int npen = (a.ncomp + 1) / 2;
    const int nP = a.rows * npen;
    const int row0 = blockIdx.x * a.rows;
    const int nrow = min(a.rows, g.nrows - row0);
    const int RN = a.rows * N;
    float2* s_spec = reinterpret_cast<float2*>(base);
    T* s_old = reinterpret_cast<T*>(base + a.spec_bytes);
    float2* s = reinterpret_cast<float2*>(base + a.stage_bytes);
    // PF_CHECK: spectral rows, old values and output rows inside the staging,
    // pencils inside the launch's shared memory
    {
        const int nold = MODE == XI_EPS ? 6 : MODE == XI_FRES ? a.ncomp : 0;
        if (!pf_check(row0 < g.nrows && a.ncomp <= 6 && g.P == P &&
                          (size_t)a.ncomp * a.rows * P * sizeof(float2) <= (size_t)a.spec_bytes &&
                          (size_t)a.ncomp * RN * sizeof(T) <= (size_t)a.spec_bytes &&
                          (size_t)a.spec_bytes + (size_t)nold * RN * sizeof(T) <= (size_t)a.stage_bytes,
                      a.err) ||
            !pf_check_smem(smem_raw, s + nP * PITCH, a.err))
            return;
    }
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    if (MODE == XI_EPS && threadIdx.x < 6) sE[threadIdx.x] = (T)a.E[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t sb = (uint32_t)(nrow * P * sizeof(float2));
        const uint32_t rb = (uint32_t)(nrow * N * sizeof(T));
        mbar_expect_tx(&bar, a.ncomp * sb + (MODE == XI_EPS ? 6 * rb : MODE == XI_FRES ? a.ncomp * rb : 0));
        const float2* spec = (const float2*)a.spec;
        const long long cstride = (long long)g.nrows * P;
        for (int c = 0; c < a.ncomp; ++c)
            bulk_load(s_spec + (size_t)c * a.rows * P, spec + c * cstride + (long long)row0 * P, sb, &bar);
        if (MODE == XI_EPS || MODE == XI_FRES) {
            const T* old = (const T*)a.out + (long long)row0 * N;
            const int nold = MODE == XI_EPS ? 6 : a.ncomp;
            for (int c = 0; c < nold; ++c) bulk_load(s_old + c * RN, old + c * g.N, rb, &bar);
        }
        // the rows of the CTA that will start pf_dist CTAs later, into L2
        const int pb = (int)blockIdx.x + a.pf_dist;
        if (a.pf_dist > 0 && pb < (int)gridDim.x) {
            const int prow0 = pb * a.rows;
            const int pn = min(a.rows, g.nrows - prow0);
            for (int c = 0; c < a.ncomp; ++c)
                bulk_prefetch_l2(spec + c * cstride + (long long)prow0 * P, (uint32_t)(pn * P * sizeof(float2)));
            if (MODE == XI_EPS || MODE == XI_FRES) {
                const T* old = (const T*)a.out + (long long)prow0 * N;
                const int nold = MODE == XI_EPS ? 6 : a.ncomp;
                for (int c = 0; c < nold; ++c) bulk_prefetch_l2(old + c * g.N, (uint32_t)(pn * N * sizeof(T)));
            }
        }
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    // unpack Z = A + iB (Z_{N-k} = conj A_k + i conj B_k) and transform back,
    // each pencil by the TPP threads of one warp
    const int j = threadIdx.x % TPP, qo = threadIdx.x / TPP;
    for (int q0 = 0; q0 < nP; q0 += PPR) {
        const int q = q0 + qo;
        const bool live = q < nP;
        float2* sp = s + (live ? q : 0) * PITCH;
        if (live) {
            const int r = div_npen(q, npen);
            const int c = q - r * npen;
            const float2* ra = s_spec + ((size_t)(2 * c) * a.rows + r) * P;
            const float2* rb = s_spec + ((size_t)(2 * c + 1) * a.rows + r) * P;
            const bool hb = 2 * c + 1 < a.ncomp && r < nrow;
#pragma unroll
            for (int k0 = 0; k0 < nxh; k0 += TPP) {
                const int k = k0 + j;
                if (k >= nxh) break;
                const float2 A = r < nrow ? ra[k] : make_float2(0.f, 0.f);
                const float2 B = hb ? rb[k] : make_float2(0.f, 0.f);
                sp[padded(k)] = make_float2(A.x - B.y, A.y + B.x);
                if (k >= 1 && 2 * k < N) sp[padded(N - k)] = make_float2(A.x + B.y, B.x - A.y);
            }
        }
        __syncwarp();
        fft_fix<N, R1, R2, true>(sp, j, live, (const float2*)a.tws);
    }
    __syncthreads();
    T* o = reinterpret_cast<T*>(base);  // output rows [comp][r][N] over the spectral staging
    T acc[2] = {0, 0};
    const T invN = (T)(1.0 / (double)g.N);
    const T c3dt = (T)a.c3dt;
    const long long gbase = (long long)row0 * N;
    constexpr bool SIX = SIX6;
    for (int e = threadIdx.x; e < nrow * N; e += kFixThreads) {
        const int r = row_of<N>(e), x = col_of<N>(e);
        const float2* row = s + (r * (SIX ? 3 : npen)) * PITCH + padded(x);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (SIX || c < npen) {
                const float2 z = row[c * PITCH];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int comp = 2 * c + h;
                    if (SIX || comp < a.ncomp) {
                        T v = (h == 0 ? z.x : z.y) * invN;
                        if (MODE == XI_EPS) {
                            v += sE[comp];
                            const T w = comp < 3 ? (T)1 : (T)2;
                            const T d = v - s_old[comp * RN + e];
                            acc[0] += w * d * d;
                            acc[1] += w * v * v;
                        } else if (MODE == XI_FRES) {
                            const T d = v - s_old[comp * RN + e];
                            acc[0] += d * d;
                            acc[1] += v * v;
                        } else if (MODE == XI_PAD) {
                            // v = L f^(k); rhs = g + c3 dt (M - 1) L f^(k)
                            const long long gi = gbase + e;
                            const T m = ((const T*)a.mob)[gi];
                            v = ((const T*)a.g_in)[(size_t)comp * g.N + gi] + c3dt * (m - (T)1) * v;
                        }
                        o[comp * RN + e] = v;
                    }
                }
            }
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        T* out = (T*)a.out + (long long)row0 * N;
        for (int c = 0; c < a.ncomp; ++c) bulk_store(out + c * g.N, o + c * RN, (uint32_t)(nrow * N * sizeof(T)));
        bulk_commit();
    }
    if (MODE == XI_EPS || MODE == XI_FRES) block_sum_store<2, T>(acc, a.partials + (size_t)blockIdx.x * 2);
    if (threadIdx.x == 0) bulk_wait_read_all();
}

template <int N, int R1, int R2, int MODE, bool FULL>
cudaError_t fwd_launch(const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    allow_smem(k_x_fwd_fix<N, R1, R2, MODE, FULL>, smem);
    k_x_fwd_fix<N, R1, R2, MODE, FULL><<<nblocks, kFixThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N, int R1, int R2>
cudaError_t fwd_plan(int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    const bool full = a.gr.ng == 3 && a.gr.both[0] && a.gr.both[1] && a.gr.both[2];
    switch (mode) {
        case X_TAU:
            return full ? fwd_launch<N, R1, R2, X_TAU, true>(a, nblocks, smem, st)
                        : fwd_launch<N, R1, R2, X_TAU, false>(a, nblocks, smem, st);
        case X_TAU_SIG:
            return full ? fwd_launch<N, R1, R2, X_TAU_SIG, true>(a, nblocks, smem, st)
                        : fwd_launch<N, R1, R2, X_TAU_SIG, false>(a, nblocks, smem, st);
        case X_DRIVE:  // (the compile-time form spilled at the pass's 80 registers and gained nothing)
            return fwd_launch<N, R1, R2, X_DRIVE, false>(a, nblocks, smem, st);
        default: return fwd_launch<N, R1, R2, X_PLAIN, false>(a, nblocks, smem, st);
    }
}

template <int N, int R1, int R2, int MODE, bool SIX6>
cudaError_t inv_launch(const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    allow_smem(k_x_inv_fix<N, R1, R2, MODE, SIX6>, smem);
    k_x_inv_fix<N, R1, R2, MODE, SIX6><<<nblocks, kFixThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N, int R1, int R2>
cudaError_t inv_plan(int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (mode) {
        case XI_EPS: return inv_launch<N, R1, R2, XI_EPS, true>(a, nblocks, smem, st);
        case XI_PAD: return inv_launch<N, R1, R2, XI_PAD, false>(a, nblocks, smem, st);
        case XI_FRES: return inv_launch<N, R1, R2, XI_FRES, false>(a, nblocks, smem, st);
        default:
            return a.ncomp == 6 ? inv_launch<N, R1, R2, XI_F, true>(a, nblocks, smem, st)
                                : inv_launch<N, R1, R2, XI_F, false>(a, nblocks, smem, st);
    }
}

}  // namespace

// launchers of the 80-, 96- and 160-point plans (pf_xfix_pfa.cu); id as
// returned by fix_id
cudaError_t launch_x_fwd_fix_pfa(int id, int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st);
cudaError_t launch_x_inv_fix_pfa(int id, int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st);

}  // namespace pfk
