// pf_k_xinv.cu -- inverse passes along x (complex-to-real) with their
// element-wise consumers (strain and residual, fields, pad corrections).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "pf_device.cuh"

namespace pfk {

// ---------------------------------------------------------------------------
// inverse pass along x (complex-to-real, two real rows per complex pencil)
// ---------------------------------------------------------------------------
// Rebuild the full complex row Z = A + iB from the half spectra of two real
// rows (Z_{n-k} = conj A_k + i conj B_k) and transform it back.  A and B are
// read through spec_at(c, r, k).
template <typename T, typename Get>
__device__ __forceinline__ void xinv_consume(const XInvArgs& a, cx<T>* s, int es, int npen, Get spec_at) {
    const int nx = a.g.nx, nxh = a.g.nxh;
    const int nP = a.rows * npen;
    pencil_items(a, nP, nxh, [&](int q, int k) {
        const int r = div_npen(q, npen);
        const int c = q - r * npen;
        const cx<T> A = spec_at(2 * c, r, k);
        const cx<T> B = (2 * c + 1 < a.ncomp) ? spec_at(2 * c + 1, r, k) : mk<T>(0, 0);
        s[pel(k, a.wl) * es + q] = mk<T>(A.x - B.y, A.y + B.x);
        if (k >= 1 && 2 * k < nx) s[pel(nx - k, a.wl) * es + q] = mk<T>(A.x + B.y, B.x - A.y);
    });
    if (a.wl) {
        // each pencil was unpacked by the threads that transform it
        __syncwarp();
        fft_smem_wl<T, true>(s, nP, es, a.plan, (const cx<T>*)a.tws);
        return;
    }
    __syncthreads();
    const int tpp = a.plan.nst ? a.plan.n / a.plan.rmin : 1;
    const int mnr = min(nP, (int)blockDim.x / tpp);
    fft_smem<T, true>(s, nP, mnr, mnr, es, a.plan, (const cx<T>*)a.tw);
}

// Real outputs of the row block: v = z / N (+ E for the strain); the strain
// pass also sums |eps_new - eps_old|^2 and |eps_new|^2 (Frobenius weights).
// `old` and `dst` address component 0 of the row block, component stride cst.
template <typename T, int MODE, typename I>
__device__ __forceinline__ void xinv_emit(const XInvArgs& a, const cx<T>* s, int es, int npen, int nrow,
                                          const T* old, T* dst, I cst, const T* sE, T (&acc)[2],
                                          long long gbase) {
    const int nx = a.g.nx;
    const T invN = (T)(1.0 / (double)a.g.N);
    const T c3dt = (T)a.c3dt;
    RowCursor rc(threadIdx.x, blockDim.x, nx);
    for (int e = threadIdx.x; e < nrow * nx; e += blockDim.x, rc.next()) {
        const int r = rc.r, x = rc.x;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c < npen) {
                const cx<T> z = s[pel(x, a.wl) * es + r * npen + c];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int comp = 2 * c + h;
                    if (comp < a.ncomp) {
                        T v = (h == 0 ? z.x : z.y) * invN;
                        if (MODE == XI_EPS) {
                            v += sE[comp];
                            const T w = comp < 3 ? (T)1 : (T)2;
                            const T d = v - old[comp * cst + e];
                            acc[0] += w * d * d;
                            acc[1] += w * v * v;
                        } else if (MODE == XI_FRES) {
                            const T d = v - old[comp * cst + e];
                            acc[0] += d * d;
                            acc[1] += v * v;
                        } else if (MODE == XI_PAD) {
                            // v = L f^(k); rhs = g + c3 dt (M - 1) L f^(k)
                            const long long gi = gbase + e;
                            const T m = ((const T*)a.mob)[gi];
                            v = ((const T*)a.g_in)[(size_t)comp * a.g.N + gi] + c3dt * (m - (T)1) * v;
                        }
                        dst[comp * cst + e] = v;
                    }
                }
            }
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kMaxThreads) k_x_inv(XInvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
    const GridDesc g = a.g;
    const int npen = (a.ncomp + 1) / 2;
    const int es = (a.rows * npen) | 1;
    const int row0 = blockIdx.x * a.rows;
    const int nrow = min(a.rows, g.nrows - row0);
    const cx<T>* spec = (const cx<T>*)a.spec;
    const long long cstride = (long long)g.nrows * g.P;
    __shared__ T sE[6];
    if (MODE == XI_EPS && threadIdx.x < 6) sE[threadIdx.x] = (T)a.E[threadIdx.x];
    xinv_consume<T>(a, s, es, npen, [&](int c, int r, int k) {
        return (r < nrow) ? spec[c * cstride + (long long)(row0 + r) * g.P + k] : mk<T>(0, 0);
    });
    // outputs go to registers first so that no load of the old strain waits
    // behind a store to the same array
    T acc[2] = {0, 0};
    T* out = (T*)a.out + (long long)row0 * g.nx;
    if (MODE == XI_EPS) {
        const int nx = g.nx;
        const T invN = (T)(1.0 / (double)g.N);
        RowCursor rc(threadIdx.x, blockDim.x, nx);
        for (int e = threadIdx.x; e < nrow * nx; e += blockDim.x, rc.next()) {
            const int r = rc.r, x = rc.x;
            T v[6], o[6];
#pragma unroll
            for (int comp = 0; comp < 6; ++comp) o[comp] = out[comp * g.N + e];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const cx<T> z = s[pel(x, a.wl) * es + r * 3 + c];
                v[2 * c] = z.x * invN + sE[2 * c];
                v[2 * c + 1] = z.y * invN + sE[2 * c + 1];
            }
#pragma unroll
            for (int comp = 0; comp < 6; ++comp) {
                const T w = comp < 3 ? (T)1 : (T)2;
                const T d = v[comp] - o[comp];
                acc[0] += w * d * d;
                acc[1] += w * v[comp] * v[comp];
                out[comp * g.N + e] = v[comp];
            }
        }
        block_sum_store<2, T>(acc, a.partials + (size_t)blockIdx.x * 2);
    } else {
        xinv_emit<T, MODE, long long>(a, s, es, npen, nrow, MODE == XI_FRES ? out : nullptr, out, g.N, sE, acc,
                                      (long long)row0 * g.nx);
        if (MODE == XI_FRES) block_sum_store<2, T>(acc, a.partials + (size_t)blockIdx.x * 2);
    }
}

// Bulk-staged form: the CTA's spectral rows (and, for the strain, its old
// strain rows) arrive by cp.async.bulk; the real rows leave by bulk stores.
// Shared memory: [spectral rows ncomp x rows x P | old strain 6 x rows x nx |
// FFT pencils]; the output rows reuse the spectral staging.
template <typename T, int MODE>
__global__ void __launch_bounds__(kMaxThreads) k_x_inv_bulk(XInvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t bar;
    const GridDesc g = a.g;
    const int nx = g.nx, P = g.P;
    const int npen = (a.ncomp + 1) / 2;
    const int es = (a.rows * npen) | 1;
    const int row0 = blockIdx.x * a.rows;
    const int nrow = min(a.rows, g.nrows - row0);
    const long long RN = (long long)a.rows * nx;
    cx<T>* s_spec = reinterpret_cast<cx<T>*>(base);
    T* s_old = reinterpret_cast<T*>(base + a.spec_bytes);
    cx<T>* s = reinterpret_cast<cx<T>*>(base + a.stage_bytes);
    __shared__ T sE[6];
    // PF_CHECK: spectral rows, old values and output rows inside the staging,
    // the pencils inside the launch's shared memory
    {
        const int nold = MODE == XI_EPS ? 6 : MODE == XI_FRES ? a.ncomp : 0;
        if (!pf_check(row0 < g.nrows && a.ncomp <= 6 &&
                          (size_t)a.ncomp * a.rows * P * sizeof(cx<T>) <= (size_t)a.spec_bytes &&
                          (size_t)a.ncomp * RN * sizeof(T) <= (size_t)a.spec_bytes &&
                          (size_t)a.spec_bytes + (size_t)nold * RN * sizeof(T) <= (size_t)a.stage_bytes,
                      a.err) ||
            !pf_check_smem(smem_raw, s + (size_t)(pel(nx - 1, a.wl) + 1) * es, a.err))
            return;
    }
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    if (MODE == XI_EPS && threadIdx.x < 6) sE[threadIdx.x] = (T)a.E[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t sb = (uint32_t)(nrow * P * sizeof(cx<T>));
        const uint32_t rb = (uint32_t)(nrow * nx * sizeof(T));
        mbar_expect_tx(&bar, a.ncomp * sb + (MODE == XI_EPS ? 6 * rb : MODE == XI_FRES ? a.ncomp * rb : 0));
        const cx<T>* spec = (const cx<T>*)a.spec;
        const long long cstride = (long long)g.nrows * P;
        for (int c = 0; c < a.ncomp; ++c)
            bulk_load(s_spec + (size_t)c * a.rows * P, spec + c * cstride + (long long)row0 * P, sb, &bar);
        if (MODE == XI_EPS || MODE == XI_FRES) {
            const T* old = (const T*)a.out + (long long)row0 * nx;
            const int nold = MODE == XI_EPS ? 6 : a.ncomp;
            for (int c = 0; c < nold; ++c) bulk_load(s_old + c * RN, old + c * g.N, rb, &bar);
        }
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    xinv_consume<T>(a, s, es, npen, [&](int c, int r, int k) {
        return (r < nrow) ? s_spec[((size_t)c * a.rows + r) * P + k] : mk<T>(0, 0);
    });
    T* o = reinterpret_cast<T*>(base);  // output rows [comp][r][nx] over the spectral staging
    T acc[2] = {0, 0};
    xinv_emit<T, MODE, int>(a, s, es, npen, nrow, s_old, o, (int)RN, sE, acc, (long long)row0 * nx);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        T* out = (T*)a.out + (long long)row0 * nx;
        for (int c = 0; c < a.ncomp; ++c)
            bulk_store(out + c * g.N, o + c * RN, (uint32_t)(nrow * nx * sizeof(T)));
        bulk_commit();
    }
    if (MODE == XI_EPS || MODE == XI_FRES) block_sum_store<2, T>(acc, a.partials + (size_t)blockIdx.x * 2);
    if (threadIdx.x == 0) bulk_wait_read_all();
}

template <typename T>
static cudaError_t x_inv_t(int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (mode) {
        case XI_EPS:
            allow_smem(k_x_inv<T, XI_EPS>, smem);
            k_x_inv<T, XI_EPS><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case XI_PAD:
            allow_smem(k_x_inv<T, XI_PAD>, smem);
            k_x_inv<T, XI_PAD><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case XI_FRES:
            allow_smem(k_x_inv<T, XI_FRES>, smem);
            k_x_inv<T, XI_FRES><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        default:
            allow_smem(k_x_inv<T, XI_F>, smem);
            k_x_inv<T, XI_F><<<nblocks, a.nthreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t x_inv_bulk_t(int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (mode) {
        case XI_EPS:
            allow_smem(k_x_inv_bulk<T, XI_EPS>, smem);
            k_x_inv_bulk<T, XI_EPS><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case XI_PAD:
            allow_smem(k_x_inv_bulk<T, XI_PAD>, smem);
            k_x_inv_bulk<T, XI_PAD><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case XI_FRES:
            allow_smem(k_x_inv_bulk<T, XI_FRES>, smem);
            k_x_inv_bulk<T, XI_FRES><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        default:
            allow_smem(k_x_inv_bulk<T, XI_F>, smem);
            k_x_inv_bulk<T, XI_F><<<nblocks, a.nthreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_x_inv(int prec, int mode, const XInvArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    if (a.bulk)
        return prec ? x_inv_bulk_t<float>(mode, a, nblocks, smem, st)
                    : x_inv_bulk_t<double>(mode, a, nblocks, smem, st);
    return prec ? x_inv_t<float>(mode, a, nblocks, smem, st) : x_inv_t<double>(mode, a, nblocks, smem, st);
}


}  // namespace pfk
