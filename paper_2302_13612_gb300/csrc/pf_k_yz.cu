// pf_k_yz.cu -- the complex transforms along y and the z pass with the per-mode
// operator (Green contraction, Helmholtz division, energy, Laplacian).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "pf_device.cuh"

namespace pfk {

// ---------------------------------------------------------------------------
// pass along y: tx consecutive kx columns of one z plane of one component,
// moved in and out of shared memory by TMA
// ---------------------------------------------------------------------------
template <typename T, bool INV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_y(YArgs a, const __grid_constant__ CUtensorMap tm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));  // TMA tiles: 128-byte aligned
    __shared__ __align__(8) uint64_t bar;
    const int tx = a.tx, ny = a.g.ny, by = a.box;
    const int kx0 = blockIdx.x * tx;
    const int zc = blockIdx.z * a.g.nz + blockIdx.y;
    // PF_CHECK: the tile inside the field and the launch's shared memory
    if (!pf_check(kx0 < a.g.nxh && (int)blockIdx.y < a.g.nz, a.err) || !pf_check_smem(smem_raw, s + ny * tx, a.err))
        return;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, (uint32_t)(ny * tx * sizeof(cx<T>)));
        for (int y0 = 0; y0 < ny; y0 += by) tma_load_3d(s + y0 * tx, &tm, &bar, 2 * kx0, y0, zc);
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    {
        // more columns than one round of the CTA's threads covers go in rounds
        const int tpp = a.plan.nst ? a.plan.n / a.plan.rmin : 1;
        const int mnr = min(tx, (int)blockDim.x / tpp);
        fft_smem<T, INV>(s, tx, mnr, mnr, tx, a.plan, (const cx<T>*)a.tw);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int y0 = 0; y0 < ny; y0 += by) tma_store_3d(&tm, s + y0 * tx, 2 * kx0, y0, zc);
        bulk_commit();
        bulk_wait_read_all();
    }
}

// ---------------------------------------------------------------------------
// pass along z with the per-mode operator between forward and inverse
// ---------------------------------------------------------------------------
__device__ __forceinline__ int freq(int k, int n) { return (2 * k < n) ? k : k - n; }
__device__ __forceinline__ bool nyquist(int k, int n) { return (n % 2 == 0) && (2 * k == n); }

template <typename T, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_z(ZArgs a, const __grid_constant__ CUtensorMap tm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));  // TMA tiles: 128-byte aligned
    __shared__ T sB[36];  // K_ik = sum_m B[ik][m] q_m, q = (x^2, y^2, z^2, yz, xz, xy)
    __shared__ __align__(8) uint64_t bar;
    const GridDesc g = a.g;
    const int tz = a.tz, nc = a.ncomp, nz = g.nz, ny = g.ny, bz = a.box;
    const int cs = a.cstride;  // complex elements between component tiles
    const int kx0 = blockIdx.x * tz;
    const int ky = blockIdx.y;
    const int ncol = min(tz, g.nxh - kx0);
    // PF_CHECK: the tile inside the field, component tiles apart by at least
    // a tile, all inside the launch's shared memory
    if (!pf_check(kx0 < g.nxh && ky < ny && nc >= 1 && nc <= 6 && cs >= nz * tz, a.err) ||
        !pf_check_smem(smem_raw, s + (size_t)nc * cs, a.err))
        return;

    if (threadIdx.x == 0) mbar_init(&bar, 1);
    if (MODE == Z_GREEN && threadIdx.x < 36) {
        // B[(i,k)][(j,l)] = C0_ijkl (+ C0_ilkj for j != l), C0 in Voigt form
        const int pair = threadIdx.x / 6, mono = threadIdx.x % 6;
        const int PI[6] = {0, 1, 2, 1, 0, 0}, PK[6] = {0, 1, 2, 2, 2, 1};
        const int i = PI[pair], k = PK[pair];
        const int j = PI[mono], l = PK[mono];
        auto vo = [](int p, int q) { return p == q ? p : 6 - p - q; };
        double b = a.C0[vo(i, j) * 6 + vo(k, l)];
        if (j != l) b += a.C0[vo(i, l) * 6 + vo(k, j)];
        sB[threadIdx.x] = (T)b;
    }
    // anisotropic gradient tensors A_c (xx, yy, zz, yz, xz, xy) for HELM / ENERGY
    if (MODE != Z_GREEN && a.A && threadIdx.x < 6 * nc) sB[threadIdx.x] = (T)a.A[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, (uint32_t)(nc * nz * tz * sizeof(cx<T>)));
        for (int c = 0; c < nc; ++c)
            for (int z0 = 0; z0 < nz; z0 += bz) tma_load_4d(s + c * cs + z0 * tz, &tm, &bar, 2 * kx0, ky, z0, c);
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    fft_smem<T, false>(s, nc * tz, tz, cs, tz, a.plan, (const cx<T>*)a.tw);

    T acc = 0;
    const T two_pi = (T)6.283185307179586477;
    // reciprocal lengths once per CTA: m = k / n as k * (1 / n)
    const T rnx = (T)1 / (T)g.nx, rnz = (T)1 / (T)nz;
    const T my = (T)freq(ky, ny) * ((T)1 / (T)ny);
    const bool nyq_y = nyquist(ky, ny);
    RowCursor rc(threadIdx.x, blockDim.x, tz);
    for (int e = threadIdx.x; e < nz * tz; e += blockDim.x, rc.next()) {
        const int p = rc.x, z = rc.r;
        if (p >= ncol) continue;
        const int kx = kx0 + p;
        const T mx = (T)kx * rnx, mz = (T)freq(z, nz) * rnz;
        cx<T>* m = s + z * tz + p;
        if (MODE == Z_GREEN) {
            const bool zero = (kx == 0 && ky == 0 && z == 0) || nyquist(kx, g.nx) || nyq_y || nyquist(z, nz);
            if (zero) {
#pragma unroll
                for (int c = 0; c < 6; ++c) m[c * cs] = mk<T>(0, 0);
                continue;
            }
            const T q[6] = {mx * mx, my * my, mz * mz, my * mz, mx * mz, mx * my};
            T K[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                T t = 0;
#pragma unroll
                for (int j = 0; j < 6; ++j) t += sB[i * 6 + j] * q[j];
                K[i] = t;
            }
            // K = [[K0 K5 K4] [K5 K1 K3] [K4 K3 K2]]; N = K^-1 by cofactors
            const T c00 = K[1] * K[2] - K[3] * K[3];
            const T c11 = K[0] * K[2] - K[4] * K[4];
            const T c22 = K[0] * K[1] - K[5] * K[5];
            const T c01 = K[4] * K[3] - K[5] * K[2];
            const T c02 = K[5] * K[3] - K[4] * K[1];
            const T c12 = K[5] * K[4] - K[0] * K[3];
            const T inv = (T)1 / (K[0] * c00 + K[5] * c01 + K[4] * c02);
            const cx<T> txx = m[0], tyy = m[cs], tzz = m[2 * cs], tyz = m[3 * cs], txz = m[4 * cs],
                        txy = m[5 * cs];
            // t = tau_hat xi
            const cx<T> t0 = mk<T>(txx.x * mx + txy.x * my + txz.x * mz, txx.y * mx + txy.y * my + txz.y * mz);
            const cx<T> t1 = mk<T>(txy.x * mx + tyy.x * my + tyz.x * mz, txy.y * mx + tyy.y * my + tyz.y * mz);
            const cx<T> t2 = mk<T>(txz.x * mx + tyz.x * my + tzz.x * mz, txz.y * mx + tyz.y * my + tzz.y * mz);
            // u = -N t (the minus sign of eps_hat = -Gamma0 : tau_hat)
            const T n00 = -c00 * inv, n11 = -c11 * inv, n22 = -c22 * inv;
            const T n01 = -c01 * inv, n02 = -c02 * inv, n12 = -c12 * inv;
            const cx<T> u0 = mk<T>(n00 * t0.x + n01 * t1.x + n02 * t2.x, n00 * t0.y + n01 * t1.y + n02 * t2.y);
            const cx<T> u1 = mk<T>(n01 * t0.x + n11 * t1.x + n12 * t2.x, n01 * t0.y + n11 * t1.y + n12 * t2.y);
            const cx<T> u2 = mk<T>(n02 * t0.x + n12 * t1.x + n22 * t2.x, n02 * t0.y + n12 * t1.y + n22 * t2.y);
            const T h = (T)0.5;
            m[0] = mk<T>(u0.x * mx, u0.y * mx);
            m[cs] = mk<T>(u1.x * my, u1.y * my);
            m[2 * cs] = mk<T>(u2.x * mz, u2.y * mz);
            m[3 * cs] = mk<T>(h * (u1.x * mz + u2.x * my), h * (u1.y * mz + u2.y * my));
            m[4 * cs] = mk<T>(h * (u0.x * mz + u2.x * mx), h * (u0.y * mz + u2.y * mx));
            m[5 * cs] = mk<T>(h * (u0.x * my + u1.x * mx), h * (u0.y * my + u1.y * mx));
        } else {
            const T kx2 = two_pi * mx, ky2 = two_pi * my, kz2 = two_pi * mz;
            const T k2 = kx2 * kx2 + ky2 * ky2 + kz2 * kz2;
            // anisotropic symbol xi.A_c.xi: squares, and cross terms only where
            // neither index is at the Nyquist frequency
            T q[6];
            if (a.A) {
                const bool ox = !nyquist(kx, g.nx), oy = !nyq_y, oz = !nyquist(z, nz);
                q[0] = kx2 * kx2;
                q[1] = ky2 * ky2;
                q[2] = kz2 * kz2;
                q[3] = (oy && oz) ? (T)2 * ky2 * kz2 : (T)0;
                q[4] = (ox && oz) ? (T)2 * kx2 * kz2 : (T)0;
                q[5] = (ox && oy) ? (T)2 * kx2 * ky2 : (T)0;
            }
            auto symbol = [&](int c) {
                T t = 0;
#pragma unroll
                for (int i = 0; i < 6; ++i) t += sB[c * 6 + i] * q[i];
                return t;
            };
            if (MODE == Z_HELM) {
                if (a.A) {
                    for (int c = 0; c < nc; ++c)
                        m[c * cs] = cscale<T>(m[c * cs], (T)1 / ((T)1 + (T)a.dtc3 * symbol(c)));
                } else {
                    const T fac = (T)1 / ((T)1 + (T)a.helm * k2);
                    for (int c = 0; c < nc; ++c) m[c * cs] = cscale<T>(m[c * cs], fac);
                }
            } else if (MODE == Z_LAPL) {  // the gradient operator: -c2 |xi|^2 or -xi.A.xi
                for (int c = 0; c < nc; ++c)
                    m[c * cs] = cscale<T>(m[c * cs], -(a.A ? symbol(c) : (T)a.c2 * k2));
            } else {  // Z_ENERGY: half-spectrum weight 2 except kx = 0 and kx = nx/2
                const T w = (kx == 0 || nyquist(kx, g.nx)) ? (T)1 : (T)2;
                T sum = 0;
                for (int c = 0; c < nc; ++c) {
                    const cx<T> v = m[c * cs];
                    sum += (a.A ? symbol(c) : k2) * (v.x * v.x + v.y * v.y);
                }
                acc += w * sum;
            }
        }
    }
    if (MODE == Z_ENERGY) {
        const T d[1] = {acc};
        block_sum_store<1, T>(d, a.partials + (size_t)(blockIdx.y * gridDim.x + blockIdx.x));
        return;
    }
    __syncthreads();
    fft_smem<T, true>(s, nc * tz, tz, cs, tz, a.plan, (const cx<T>*)a.tw);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < nc; ++c)
            for (int z0 = 0; z0 < nz; z0 += bz) tma_store_4d(&tm, s + c * cs + z0 * tz, 2 * kx0, ky, z0, c);
        bulk_commit();
        bulk_wait_read_all();
    }
}

template <typename T>
static cudaError_t y_t(bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    if (inv) {
        allow_smem(k_y<T, true>, smem);
        k_y<T, true><<<grid, a.nthreads, smem, st>>>(a, tm);
    } else {
        allow_smem(k_y<T, false>, smem);
        k_y<T, false><<<grid, a.nthreads, smem, st>>>(a, tm);
    }
    return cudaGetLastError();
}

cudaError_t launch_y(int prec, bool inv, const YArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                     cudaStream_t st) {
    return prec ? y_t<float>(inv, a, tm, grid, smem, st) : y_t<double>(inv, a, tm, grid, smem, st);
}

template <typename T>
static cudaError_t z_t(int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
    switch (mode) {
        case Z_GREEN:
            allow_smem(k_z<T, Z_GREEN>, smem);
            k_z<T, Z_GREEN><<<grid, a.nthreads, smem, st>>>(a, tm);
            break;
        case Z_HELM:
            allow_smem(k_z<T, Z_HELM>, smem);
            k_z<T, Z_HELM><<<grid, a.nthreads, smem, st>>>(a, tm);
            break;
        case Z_LAPL:
            allow_smem(k_z<T, Z_LAPL>, smem);
            k_z<T, Z_LAPL><<<grid, a.nthreads, smem, st>>>(a, tm);
            break;
        default:
            allow_smem(k_z<T, Z_ENERGY>, smem);
            k_z<T, Z_ENERGY><<<grid, a.nthreads, smem, st>>>(a, tm);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_z(int prec, int mode, const ZArgs& a, const CUtensorMap& tm, dim3 grid, size_t smem,
                     cudaStream_t st) {
    return prec ? z_t<float>(mode, a, tm, grid, smem, st) : z_t<double>(mode, a, tm, grid, smem, st);
}


}  // namespace pfk
