// pf_k_xfwd.cu -- forward passes along x: the element-wise producers (polarisation,
// driving force, plain fields) fused with the real-to-complex transform.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "pf_device.cuh"

namespace pfk {

// ---------------------------------------------------------------------------
// forward pass along x (fused elementwise producer + real-to-complex)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void store_drive_stats(const T (&acc)[8], double* out) {
    block_sum_store<8, T>(acc, out);
}

// Element-wise phase into the interleaved pencils, then the forward x FFT.
template <typename T, int MODE, typename I>
__device__ __forceinline__ void xfwd_produce(const XFwdArgs& a, cx<T>* s, int es, int npen, int row0, const T* f,
                                             const int* fmap, const T* eps, const T* ep, const uint16_t* grain,
                                             I cst, const T* sC0, T (&acc)[8]) {
    const int nx = a.g.nx;
    RowCursor rc(threadIdx.x, blockDim.x, nx);
    for (int e = threadIdx.x; e < a.rows * nx; e += blockDim.x, rc.next()) {
        const int r = rc.r, x = rc.x;
        T out[6] = {0, 0, 0, 0, 0, 0};
        if (row0 + r < a.g.nrows)
            xfwd_voxel<T, MODE, I>(a, f, fmap, eps, ep, grain, cst, (I)e, (long long)row0 * nx + e, sC0, out, acc);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (c < npen) s[pel(x, a.wl) * es + r * npen + c] = mk<T>(out[2 * c], out[2 * c + 1]);
    }
    __syncthreads();
    const int nP = a.rows * npen;
    if (a.wl) {
        // the split that follows reads each pencil with the threads that
        // transformed it
        fft_smem_wl<T, false>(s, nP, es, a.plan, (const cx<T>*)a.tws, false);
        return;
    }
    const int tpp = a.plan.nst ? a.plan.n / a.plan.rmin : 1;
    const int mnr = min(nP, (int)blockDim.x / tpp);
    fft_smem<T, false>(s, nP, mnr, mnr, es, a.plan, (const cx<T>*)a.tw);
}

// Split the packed transform Z = A + iB of two real rows:
// A_k = (Z_k + conj Z_{n-k}) / 2, B_k = (Z_k - conj Z_{n-k}) / 2i.
template <typename T>
__device__ __forceinline__ void split_pair(const cx<T>* s, int es, int nx, int k, int q, cx<T>& A, cx<T>& B,
                                           int wl) {
    const T half = (T)0.5;
    const cx<T> z1 = s[pel(k, wl) * es + q];
    const cx<T> z2 = s[pel((k == 0) ? 0 : nx - k, wl) * es + q];
    A = mk<T>(half * (z1.x + z2.x), half * (z1.y - z2.y));
    B = mk<T>(half * (z1.y + z2.y), half * (z2.x - z1.x));
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kMaxThreads) k_x_fwd(XFwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
    __shared__ __align__(16) T sC0[24];
    const GridDesc g = a.g;
    const int nx = g.nx;
    const int npen = (a.ncomp + 1) / 2;
    const int nP = a.rows * npen;
    const int es = nP | 1;
    const int row0 = blockIdx.x * a.rows;
    if ((MODE == X_TAU || MODE == X_TAU_SIG) && threadIdx.x < 24) load_c0<T>(a.C0, sC0);
    __syncthreads();
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long off = (long long)row0 * nx;
    const T* eps = (const T*)a.eps;
    const T* ep = (const T*)a.eps_p;
    // twin fractions are read in place: position p is slot fin_slot[p]
    xfwd_produce<T, MODE, long long>(a, s, es, npen, row0, (const T*)a.f + off, a.fin_slot,
                                     eps ? eps + off : nullptr, ep ? ep + off : nullptr,
                                     a.grain ? a.grain + off : nullptr, g.N, sC0, acc);
    const int nxh = g.nxh;
    cx<T>* spec = (cx<T>*)a.spec;
    const long long cstride = (long long)g.nrows * g.P;
    pencil_items(a, nP, nxh, [&](int q, int k) {
        const int r = div_npen(q, npen);
        const int c = q - r * npen;
        const int row = row0 + r;
        if (row >= g.nrows) return;
        cx<T> A, B;
        split_pair<T>(s, es, nx, k, q, A, B, a.wl);
        const int sa = a.out_slot[2 * c];
        const int sb = 2 * c + 1 < a.ncomp ? a.out_slot[2 * c + 1] : -1;
        if (sa >= 0) spec[sa * cstride + (long long)row * g.P + k] = A;
        if (sb >= 0) spec[sb * cstride + (long long)row * g.P + k] = B;
    });
    if (MODE == X_DRIVE || MODE == X_TAU_SIG)
        store_drive_stats<T>(acc, a.partials + (size_t)blockIdx.x * 8);
}

// Same pass with the CTA's rows staged through shared memory by bulk copies:
// every input component of the row block arrives with one cp.async.bulk, the
// packed spectra leave with one bulk store per component.
// Shared memory: [staging | FFT pencils]; staging holds the inputs
// (eps 6, f V, eps_p 6, grain) and is reused for the output rows [c][r][P].
template <typename T, int MODE>
__global__ void __launch_bounds__(kMaxThreads) k_x_fwd_bulk(XFwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) T sC0[24];
    const GridDesc g = a.g;
    const int nx = g.nx, nfin = a.nfin;
    const int npen = (a.ncomp + 1) / 2;
    const int nP = a.rows * npen;
    const int es = nP | 1;
    const int row0 = blockIdx.x * a.rows;
    const int nrow = min(a.rows, g.nrows - row0);
    const long long RN = (long long)a.rows * nx;
    const long long off = (long long)row0 * nx;
    const bool stage_grain = a.grain && a.stage_grain;
    // staging layout
    T* s_f = reinterpret_cast<T*>(base);  // twin fractions by position
    T* s_eps = s_f + nfin * RN;
    T* s_ep = s_eps + (MODE == X_PLAIN ? 0 : 6 * RN);
    uint16_t* s_g = reinterpret_cast<uint16_t*>(s_ep + (a.eps_p ? 6 * RN : 0));
    cx<T>* s = reinterpret_cast<cx<T>*>(base + a.stage_bytes);
    // PF_CHECK: staging in and out of its area, the pencils (element
    // pel(nx - 1) of the last pencil) inside the launch's shared memory
    if (!pf_check(row0 < g.nrows && nfin <= 6 && a.ncomp <= 6 &&
                      (size_t)(nfin + (MODE == X_PLAIN ? 0 : 6 + (a.eps_p ? 6 : 0))) * RN * sizeof(T) +
                              (MODE != X_PLAIN && stage_grain ? (size_t)RN * 2 : 0) <=
                          (size_t)a.stage_bytes &&
                      (size_t)a.ncomp * a.rows * g.P * sizeof(cx<T>) <= (size_t)a.stage_bytes,
                  a.err) ||
        !pf_check_smem(smem_raw, s + (size_t)(pel(nx - 1, a.wl) + 1) * es, a.err))
        return;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    if ((MODE == X_TAU || MODE == X_TAU_SIG) && threadIdx.x < 24) load_c0<T>(a.C0, sC0);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t rb = (uint32_t)(nrow * nx * sizeof(T));
        uint32_t total = 0;
        for (int p = 0; p < nfin; ++p) total += a.fin_slot[p] >= 0 ? rb : 0;
        if (MODE != X_PLAIN) total += 6 * rb + (a.eps_p ? 6 * rb : 0);
        if (MODE != X_PLAIN && stage_grain) total += (uint32_t)(nrow * nx * 2);
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
            if (stage_grain) bulk_load(s_g, a.grain + off, (uint32_t)(nrow * nx * 2), &bar);
        }
    }
    if (!cta_wait(&bar, 0, a.err)) return;
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint16_t* gp = a.grain ? (stage_grain ? s_g : a.grain + off) : nullptr;
    xfwd_produce<T, MODE, int>(a, s, es, npen, row0, s_f, nullptr, s_eps, a.eps_p ? s_ep : nullptr, gp, (int)RN,
                               sC0, acc);
    // split into [c][r][P] rows in the (now free) staging area, zero padding
    const int nxh = g.nxh, P = g.P;
    cx<T>* o = reinterpret_cast<cx<T>*>(base);
    pencil_items(a, nP, P, [&](int q, int k) {
        const int r = div_npen(q, npen);
        const int c = q - r * npen;
        cx<T> A = mk<T>(0, 0), B = mk<T>(0, 0);
        if (k < nxh) split_pair<T>(s, es, nx, k, q, A, B, a.wl);
        o[((2 * c) * a.rows + r) * P + k] = A;
        if (2 * c + 1 < a.ncomp) o[((2 * c + 1) * a.rows + r) * P + k] = B;
    });
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        cx<T>* spec = (cx<T>*)a.spec;
        const long long cstride = (long long)g.nrows * P;
        for (int c = 0; c < a.ncomp; ++c)
            if (a.out_slot[c] >= 0)
                bulk_store(spec + a.out_slot[c] * cstride + (long long)row0 * P, o + (size_t)c * a.rows * P,
                           (uint32_t)(nrow * P * sizeof(cx<T>)));
        bulk_commit();
    }
    if (MODE == X_DRIVE || MODE == X_TAU_SIG)
        store_drive_stats<T>(acc, a.partials + (size_t)blockIdx.x * 8);
    if (threadIdx.x == 0) bulk_wait_read_all();
}

template <typename T>
static cudaError_t x_fwd_t(int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (mode) {
        case X_TAU:
            allow_smem(k_x_fwd<T, X_TAU>, smem);
            k_x_fwd<T, X_TAU><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case X_TAU_SIG:
            allow_smem(k_x_fwd<T, X_TAU_SIG>, smem);
            k_x_fwd<T, X_TAU_SIG><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case X_DRIVE:
            allow_smem(k_x_fwd<T, X_DRIVE>, smem);
            k_x_fwd<T, X_DRIVE><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        default:
            allow_smem(k_x_fwd<T, X_PLAIN>, smem);
            k_x_fwd<T, X_PLAIN><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t x_fwd_bulk_t(int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    switch (mode) {
        case X_TAU:
            allow_smem(k_x_fwd_bulk<T, X_TAU>, smem);
            k_x_fwd_bulk<T, X_TAU><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case X_TAU_SIG:
            allow_smem(k_x_fwd_bulk<T, X_TAU_SIG>, smem);
            k_x_fwd_bulk<T, X_TAU_SIG><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        case X_DRIVE:
            allow_smem(k_x_fwd_bulk<T, X_DRIVE>, smem);
            k_x_fwd_bulk<T, X_DRIVE><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
        default:
            allow_smem(k_x_fwd_bulk<T, X_PLAIN>, smem);
            k_x_fwd_bulk<T, X_PLAIN><<<nblocks, a.nthreads, smem, st>>>(a);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_x_fwd(int prec, int mode, const XFwdArgs& a, int nblocks, size_t smem, cudaStream_t st) {
    if (a.bulk)
        return prec ? x_fwd_bulk_t<float>(mode, a, nblocks, smem, st)
                    : x_fwd_bulk_t<double>(mode, a, nblocks, smem, st);
    return prec ? x_fwd_t<float>(mode, a, nblocks, smem, st) : x_fwd_t<double>(mode, a, nblocks, smem, st);
}


}  // namespace pfk
