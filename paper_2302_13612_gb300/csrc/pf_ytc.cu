// pf_ytc.cu -- the transform along y with both radix-16 stages on the BF16
// tensor cores (the mixed-precision arm, PF_MIXED).
//
// A tile holds TW = 8 kx columns x 256 y planes of one component (element i
// of column p at i * 8 + p, the TMA box of the y pass).  A radix-16 Stockham
// stage is, over the tile, the complex product Y = F X with F the 16 x 16
// DFT matrix and X[r][(j, p)] = x_p[j + 16 r] (twiddled by w^(r j) in the
// second stage); in real form
//     [Y_re; Y_im] = [[F_re, -F_im], [F_im, F_re]] [X_re; X_im],
// a 32 x 32 by 32 x 128 product: two m16 tiles (real and imaginary rows),
// two k16 steps (real and imaginary inputs) and 16 n8 tiles (8 columns p of
// one butterfly j each) of mma.sync m16n8k16.  The FP32 inputs and the
// FP32-rounded DFT matrix are split exactly into BF16 terms
// (x = x_h + x_m + x_l); with three terms the products of order <= 2
// (hh, hm, mh, hl, mm, lh) are accumulated in FP32, which keeps the stage at
// the FP32 level (the dropped products are O(2^-24) of the result); with two
// terms (hh, hm, mh) it is O(2^-16).  Stage outputs go to the other tile
// buffer (out of place), so one CTA barrier separates the stages.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf_device.cuh"
#include "pf_mma.cuh"

namespace pfk {

namespace {

constexpr int kTcN = 256, kTcTW = 8, kTcThreads = 128;  // 4 warps x 4 n8 tiles per stage

// One radix-16 stage from tile `in` to tile `out` for the four n8 tiles
// (butterflies j = 4 w .. 4 w + 3, w the warp) of this warp.  SECOND:
// multiply by the twiddles w^(r j) first and store in natural order
// (j + 16 k); otherwise store at j * 16 + k.
template <int TERMS, bool INV, bool SECOND>
__device__ __forceinline__ void tc_stage(const float2* __restrict__ in, float2* __restrict__ out,
                                         const uint32_t (&af)[TERMS][2][2][4], const float2* __restrict__ tw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int j = warp * 4 + i;
        // B operand: column p = g of butterfly j, rows r = 2 tq, 2 tq + 1, 2 tq + 8, 2 tq + 9
        float re[4], im[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = 2 * tq + (u & 1) + 8 * (u >> 1);
            float2 v = in[(j + 16 * r) * kTcTW + g];
            if (SECOND) {
                const float2 w = __ldg(&tw[r * j]);
                v = INV ? cmulc<float>(v, w) : cmul<float>(v, w);
            }
            re[u] = v.x;
            im[u] = v.y;
        }
        // the terms of the split, packed as k16 x n8 B fragments per k step
        uint32_t bf[TERMS][2][2];
        {
            Split3 sr[4], si[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                sr[u] = split3(re[u]);
                si[u] = split3(im[u]);
            }
#pragma unroll
            for (int tm = 0; tm < TERMS; ++tm) {
                auto pick = [&](const Split3& s) { return tm == 0 ? s.h : tm == 1 ? s.m : s.l; };
                bf[tm][0][0] = bf16x2(pick(sr[0]), pick(sr[1]));
                bf[tm][0][1] = bf16x2(pick(sr[2]), pick(sr[3]));
                bf[tm][1][0] = bf16x2(pick(si[0]), pick(si[1]));
                bf[tm][1][1] = bf16x2(pick(si[2]), pick(si[3]));
            }
        }
        float d[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int c = 0; c < 4; ++c) d[mt][c] = 0.f;
        // products of total order <= TERMS - 1, smallest first
#pragma unroll
        for (int ord = TERMS - 1; ord >= 0; --ord)
#pragma unroll
            for (int ta = 0; ta < TERMS; ++ta) {
                const int tb = ord - ta;
                if (tb < 0 || tb >= TERMS) continue;
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) mma_16816(d[mt], af[ta][mt][ks], bf[tb][ks][0], bf[tb][ks][1]);
            }
        // D: rows k = g, g + 8 (real part from m tile 0, imaginary from 1), columns p = 2 tq, 2 tq + 1
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = g + 8 * (c >> 1), p = 2 * tq + (c & 1);
            const int o = SECOND ? j + 16 * k : j * 16 + k;
            out[o * kTcTW + p] = make_float2(d[0][c], d[1][c]);
        }
    }
}

template <int TERMS, bool INV>
__global__ void __launch_bounds__(kTcThreads) k_y_tc(YArgs a, const __grid_constant__ CUtensorMap tm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s0 = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
    float2* s1 = s0 + kTcN * kTcTW;
    __shared__ __align__(8) uint64_t bar;
    const int by = a.box;
    const int kx0 = blockIdx.x * kTcTW;
    const int zc = blockIdx.z * a.g.nz + blockIdx.y;
    // PF_CHECK: the tile inside the field, both tile buffers inside the launch's shared memory
    if (!pf_check(kx0 < a.g.nxh && a.g.ny == kTcN && (int)blockIdx.y < a.g.nz, a.err) ||
        !pf_check_smem(smem_raw, s1 + kTcN * kTcTW, a.err))
        return;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, (uint32_t)(kTcN * kTcTW * sizeof(float2)));
        for (int y0 = 0; y0 < kTcN; y0 += by) tma_load_3d(s0 + y0 * kTcTW, &tm, &bar, 2 * kx0, y0, zc);
    }
    // the lane's A fragments (terms x m tiles x k steps) while the tile arrives
    uint32_t af[TERMS][2][2][4];
    {
        const int lane = threadIdx.x & 31;
        const uint4* src = reinterpret_cast<const uint4*>(a.tc_a) + (INV ? 3 * 2 * 2 * 32 : 0);
#pragma unroll
        for (int t = 0; t < TERMS; ++t)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint4 v = __ldg(&src[((t * 2 + mt) * 2 + ks) * 32 + lane]);
                    af[t][mt][ks][0] = v.x;
                    af[t][mt][ks][1] = v.y;
                    af[t][mt][ks][2] = v.z;
                    af[t][mt][ks][3] = v.w;
                }
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    const float2* tw = (const float2*)a.tw;
    tc_stage<TERMS, INV, false>(s0, s1, af, tw);
    __syncthreads();
    tc_stage<TERMS, INV, true>(s1, s0, af, tw);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int y0 = 0; y0 < kTcN; y0 += by) tma_store_3d(&tm, s0 + y0 * kTcTW, 2 * kx0, y0, zc);
        bulk_commit();
        bulk_wait_read_all();
    }
}

template <int TERMS>
cudaError_t launch_terms(bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, cudaStream_t st) {
    const size_t smem = 2 * kTcN * kTcTW * sizeof(float2) + 128;
    if (inv) {
        allow_smem(k_y_tc<TERMS, true>, smem);
        k_y_tc<TERMS, true><<<grid, kTcThreads, smem, st>>>(a, tm);
    } else {
        allow_smem(k_y_tc<TERMS, false>, smem);
        k_y_tc<TERMS, false><<<grid, kTcThreads, smem, st>>>(a, tm);
    }
    return cudaGetLastError();
}

}  // namespace

bool y_tc_ok(const FftPlan& p, int tx) {
    return p.n == kTcN && p.nst == 2 && p.radix[0] == 16 && p.radix[1] == 16 && tx == kTcTW;
}

size_t y_tc_smem() { return 2 * kTcN * kTcTW * sizeof(float2) + 128; }

cudaError_t launch_y_tc(bool inv, int terms, const YArgs& a, const CUtensorMap& tm, dim3 grid, cudaStream_t st) {
    if (!y_tc_ok(a.plan, a.tx) || !a.tc_a) return cudaErrorNotSupported;
    return terms == 2 ? launch_terms<2>(inv, a, tm, grid, st) : launch_terms<3>(inv, a, tm, grid, st);
}

}  // namespace pfk
