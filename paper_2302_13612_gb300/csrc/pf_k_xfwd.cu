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
// Entry threadIdx.x (< 36) of the shared copy of C0: row-major C0 in FP64;
// in FP32, -C0 as row pairs, (p, j) -> (-C0[2p][j], -C0[2p+1][j]).
template <typename T>
__device__ __forceinline__ void load_c0(const double* C0, T* sC0) {
    const int t = threadIdx.x;
    if constexpr (sizeof(T) == 4) {
        const int pj = t >> 1, h = t & 1;
        const int p = pj / 6, j = pj - p * 6;
        sC0[t] = (T)(-C0[(2 * p + h) * 6 + j]);
    } else {
        sC0[t] = (T)C0[t];
    }
}

// Produce the real fields of one voxel: tau (TAU), g = f + dt c3 d (DRIVE) or
// f (PLAIN).  Field pointers address component 0 of the voxel's row block;
// component c lives at c * cst.  DRIVE also accumulates <sigma>, G_dw, G_me.
template <typename T, int MODE, typename I>
__device__ __forceinline__ void xfwd_voxel(const XFwdArgs& a, const T* f, const T* eps, const T* ep,
                                           const uint16_t* grain, I cst, I li, long long gi, const T* sC0,
                                           T (&out)[6], T (&acc)[8]) {
    const int V = a.m.V;
    VoxelState<T> vs;
    load_f<T, I>(vs, f, cst, li, V);
    if (MODE == X_PLAIN) {
#pragma unroll
        for (int i = 0; i < 6; ++i) out[i] = vs.f[i];
        return;
    }
    T quad_a[6];  // DRIVE: e:(C_tw^a - C_hex):e
    XtalState<T> xs;
    const int gid = grain ? (int)grain[li] : 0;
    xtal_material<T, MODE == X_DRIVE, I>(xs, a, vs.f, gid, eps, ep, cst, li, quad_a);
    if (MODE == X_TAU || MODE == X_TAU_SIG) {
        if (MODE == X_TAU_SIG) {
#pragma unroll
            for (int i = 0; i < 6; ++i) acc[i] += xs.sig[i];
        }
        // tau = sigma - C0 : eps (engineering shears for the Voigt product)
        T ee[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const T x0 = eps[i * cst + li];
            ee[i] = (i < 3) ? x0 : (T)2 * x0;
        }
        if constexpr (sizeof(T) == 4) {
            // sC0 holds -C0 as row pairs: entry (p, j) = (-C0[2p][j], -C0[2p+1][j])
            const float2* nC = reinterpret_cast<const float2*>(sC0);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                float2 t = f2(xs.sig[2 * p], xs.sig[2 * p + 1]);
#pragma unroll
                for (int j = 0; j < 6; ++j) t = ffma2(nC[p * 6 + j], f2(ee[j]), t);
                out[2 * p] = t.x;
                out[2 * p + 1] = t.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                T t = xs.sig[i];
#pragma unroll
                for (int j = 0; j < 6; ++j) t -= sC0[i * 6 + j] * ee[j];
                out[i] = t;
            }
        }
        return;
    }
    // X_DRIVE: d_a of Eq. fRate2 over all phases, the matrix f0 included
    const T c1 = (T)a.c1, c3dt = (T)a.c3dt, gam = (T)a.m.gamma;
    const T mf = a.mob ? ((const T*)a.mob)[gi] : (T)1;  // pad-layer mobility factor
    const T f0 = (T)1 - vs.fsum;
    const XtalTab<T>& t = xtab<T>(a);
    // sum over the other phases b (matrix included) of f_b (f_b - f_a)
    // = S2 - f_a S1 with S1 = sum_b f_b and S2 = sum_b f_b^2 over all phases
    T S1 = f0, S2 = f0 * f0;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        if (b < V) {
            S1 += vs.f[b];
            S2 += vs.f[b] * vs.f[b];
        }
    }
#pragma unroll
    for (int al = 0; al < 6; ++al) {
        if (al < V) {
            const T fa = vs.f[al];
            const T chem = -c1 * fa * (S2 - fa * S1);
            // sigma:S_a (S with tensor shears, so shear terms count twice)
            T rss = 0;
#pragma unroll
            for (int i = 0; i < 6; ++i) rss += ((i < 3) ? (T)1 : (T)2) * xs.sc[i] * t.S[al][i];
            const T d = chem + gam * rss - (T)0.5 * quad_a[al];
            out[al] = (a.f_base ? ((const T*)a.f_base)[(size_t)al * a.g.N + gi] : fa) + c3dt * mf * d;
            if (a.g_out) ((T*)a.g_out)[(size_t)al * a.g.N + gi] = out[al];
        } else {
            out[al] = 0;
        }
    }
    // statistics: <sigma>, G_dw, G_me
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[i] += xs.sig[i];
    T gdw = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        if (b < V) {
            const T fb2 = vs.f[b] * vs.f[b];
            gdw += f0 * f0 * fb2;
#pragma unroll
            for (int c = b + 1; c < 6; ++c)
                if (c < V) gdw += fb2 * vs.f[c] * vs.f[c];
        }
    }
    acc[6] += (T)0.5 * c1 * gdw;
    T gme = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) gme += xs.sc[i] * xs.ee[i];
    acc[7] += (T)0.5 * gme;
}

template <typename T>
__device__ __forceinline__ void store_drive_stats(const T (&acc)[8], double* out) {
    block_sum_store<8, T>(acc, out);
}

// Element-wise phase into the interleaved pencils, then the forward x FFT.
template <typename T, int MODE, typename I>
__device__ __forceinline__ void xfwd_produce(const XFwdArgs& a, cx<T>* s, int es, int npen, int row0, const T* f,
                                             const T* eps, const T* ep, const uint16_t* grain, I cst,
                                             const T* sC0, T (&acc)[8]) {
    const int nx = a.g.nx;
    RowCursor rc(threadIdx.x, blockDim.x, nx);
    for (int e = threadIdx.x; e < a.rows * nx; e += blockDim.x, rc.next()) {
        const int r = rc.r, x = rc.x;
        T out[6] = {0, 0, 0, 0, 0, 0};
        if (row0 + r < a.g.nrows)
            xfwd_voxel<T, MODE, I>(a, f, eps, ep, grain, cst, (I)e, (long long)row0 * nx + e, sC0, out, acc);
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
    __shared__ __align__(8) T sC0[36];
    const GridDesc g = a.g;
    const int nx = g.nx;
    const int npen = (a.ncomp + 1) / 2;
    const int nP = a.rows * npen;
    const int es = nP | 1;
    const int row0 = blockIdx.x * a.rows;
    if ((MODE == X_TAU || MODE == X_TAU_SIG) && threadIdx.x < 36) load_c0<T>(a.C0, sC0);
    __syncthreads();
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long off = (long long)row0 * nx;
    const T* eps = (const T*)a.eps;
    const T* ep = (const T*)a.eps_p;
    xfwd_produce<T, MODE, long long>(a, s, es, npen, row0, (const T*)a.f + off, eps ? eps + off : nullptr,
                                     ep ? ep + off : nullptr, a.grain ? a.grain + off : nullptr, g.N, sC0, acc);
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
        spec[(2 * c) * cstride + (long long)row * g.P + k] = A;
        if (2 * c + 1 < a.ncomp) spec[(2 * c + 1) * cstride + (long long)row * g.P + k] = B;
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
    __shared__ __align__(8) T sC0[36];
    const GridDesc g = a.g;
    const int nx = g.nx, V = a.m.V;
    const int npen = (a.ncomp + 1) / 2;
    const int nP = a.rows * npen;
    const int es = nP | 1;
    const int row0 = blockIdx.x * a.rows;
    const int nrow = min(a.rows, g.nrows - row0);
    const long long RN = (long long)a.rows * nx;
    const long long off = (long long)row0 * nx;
    const bool stage_grain = a.grain && a.stage_grain;
    // staging layout
    T* s_f = reinterpret_cast<T*>(base);
    T* s_eps = s_f + V * RN;
    T* s_ep = s_eps + (MODE == X_PLAIN ? 0 : 6 * RN);
    uint16_t* s_g = reinterpret_cast<uint16_t*>(s_ep + (a.eps_p ? 6 * RN : 0));
    cx<T>* s = reinterpret_cast<cx<T>*>(base + a.stage_bytes);
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    if ((MODE == X_TAU || MODE == X_TAU_SIG) && threadIdx.x < 36) load_c0<T>(a.C0, sC0);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t rb = (uint32_t)(nrow * nx * sizeof(T));
        uint32_t total = V * rb;
        if (MODE != X_PLAIN) total += 6 * rb + (a.eps_p ? 6 * rb : 0);
        if (MODE != X_PLAIN && stage_grain) total += (uint32_t)(nrow * nx * 2);
        mbar_expect_tx(&bar, total);
        const T* f = (const T*)a.f;
        for (int c = 0; c < V; ++c) bulk_load(s_f + c * RN, f + c * g.N + off, rb, &bar);
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
    xfwd_produce<T, MODE, int>(a, s, es, npen, row0, s_f, s_eps, a.eps_p ? s_ep : nullptr, gp, (int)RN, sC0, acc);
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
            bulk_store(spec + c * cstride + (long long)row0 * P, o + (size_t)c * a.rows * P,
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
