// pf_kernels.cu -- sm_103a kernels of the phase-field twin step: the C0 sum,
// the stress field, reductions, the warm start and the device-side step
// control.  The transform passes live in pf_k_xfwd.cu, pf_k_yz.cu and
// pf_k_xinv.cu, their shared device code in pf_device.cuh.
//
// One Moulinec-Suquet pass is five launches over the half spectrum:
//   k_x_fwd<TAU>   polarisation tau = C(x):(eps - eps*) - C0:eps (Eq. stiffM and
//                  the twin eigenstrain of Sec. 2.1.3) fused with the real-to-
//                  complex transform along x (two real fields packed per
//                  complex pencil);
//   k_y<fwd>       complex transform along y;
//   k_z<GREEN>     forward transform along z, eps_hat = -Gamma0(xi):tau_hat
//                  formed on the fly from C0 and xi, inverse transform along z;
//   k_y<inv>;
//   k_x_inv<EPS>   complex-to-real along x, mean strain added back, FP64
//                  partial sums of the residual norms.
// The phase-field update reuses the same passes: k_x_fwd<DRIVE> evaluates the
// driving force of Eq. fRate2 and forms g = f + dt c3 d, k_z<HELM> divides by
// 1 + dt c3 c2 |xi|^2 (Eq. fRate3), k_x_inv<F> writes f^{n+1}.
// Reductions are per-CTA FP64 partials summed by k_finalize in a fixed order,
// so results are bitwise reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "pf_device.cuh"

namespace pfk {

// ---------------------------------------------------------------------------
// C0 = <C(x)>: per-CTA sums of the 21 packed entries of C(x)
// ---------------------------------------------------------------------------
// Sums of C(x) = C_m(g) + sum_a f_a (C_tw^a(g) - C_m(g)) over voxels.  The
// mixture is linear in f, so each lane sums f over a run of voxels of one
// grain and the grain's tables apply once per run.  A run is applied by the
// whole warp, lane i < 21 taking packed entry i (one coalesced table row per
// term), so a lane that changes grain costs the warp a few instructions, not
// a divergent 21 x 7 multiply-add.  Every member is called by all 32 lanes
// of a warp the same number of times.
// NV: the variant count when known at compile time (6), else 0 (m.V).
template <typename T, int NV = 0>
struct C0Run {
    T fs[6];   // twin fractions summed over the lane's open run
    T acc;     // lane i < 21: entry i of the warp's sum of C(x)
    int cnt;   // voxels in the open run
    int gcur;  // grain of the open run (-1: none yet)
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 6; ++i) fs[i] = 0;
        acc = 0;
        cnt = 0;
        gcur = -1;
    }
    // add the open runs of the lanes in mask, in ascending lane order
    __device__ __forceinline__ void apply(const MatDesc& m, unsigned mask) {
        const unsigned full = 0xffffffffu;
        const int lane = threadIdx.x & 31;
        const int li = lane < 21 ? lane : 0;
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const int g = __shfl_sync(full, gcur, src);
            const T c = (T)__shfl_sync(full, cnt, src);
            T v = c * ((const T*)m.Cm)[g * kCRow + li];
            const T* dC = (const T*)m.dC + (size_t)g * m.V * kCRow + li;
#pragma unroll
            for (int al = 0; al < 6; ++al) {
                if (al < (NV ? NV : m.V)) v += __shfl_sync(full, fs[al], src) * dC[al * kCRow];
            }
            if (lane < 21) acc += v;
        }
    }
    // next voxel of the lane (grain gid) when active; the caller then adds its
    // twin fractions to fs
    __device__ __forceinline__ void voxel(const MatDesc& m, int gid, bool active) {
        const bool change = active && gid != gcur;
        const unsigned mask = __ballot_sync(0xffffffffu, change && cnt > 0);
        if (mask) apply(m, mask);
        if (change) {
#pragma unroll
            for (int i = 0; i < 6; ++i) fs[i] = 0;
            cnt = 0;
            gcur = gid;
        }
        if (active) ++cnt;
    }
    // close the open runs; when all lanes are in one grain they pool their
    // runs and the warp applies the tables once
    __device__ __forceinline__ void finish(const MatDesc& m) {
        const unsigned full = 0xffffffffu;
        const int g0 = __shfl_sync(full, gcur, 0);
        unsigned mask;
        if (__all_sync(full, gcur == g0 && g0 >= 0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    if (i < (NV ? NV : m.V)) fs[i] += __shfl_xor_sync(full, fs[i], o);
                cnt += __shfl_xor_sync(full, cnt, o);
            }
            mask = 1u;
        } else {
            mask = __ballot_sync(full, cnt > 0);
        }
        apply(m, mask);
    }
    // the CTA's 21 sums (FP64 across warps) into out[0..20]; all threads call
    __device__ __forceinline__ void store(double* out) const {
        __shared__ double red[kMaxThreads / 32][21];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane < 21) red[warp][lane] = (double)acc;
        __syncthreads();
        if (threadIdx.x < 21) {
            const int nw = (blockDim.x + 31) >> 5;
            double s = 0;
            for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
            out[threadIdx.x] = s;
        }
    }
};

// Per-CTA sums of C(x) over a contiguous voxel range: each lane's voxels are
// blockDim.x apart, mostly in one grain, and its runs go through C0Run.
// Loads of four voxels are issued before any run is applied; the warp walks
// together, lanes past the end inactive.
template <typename T, int NV>
__global__ void __launch_bounds__(kMaxThreads) k_c0(C0Args a) {
    const long long N = a.g.N;
    const int V = NV ? NV : a.m.V;
    const T* f = (const T*)a.f;
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    const long long v0 = (long long)blockIdx.x * per;
    const long long v1 = v0 + per < N ? v0 + per : N;
    C0Run<T, NV> run;
    run.init();
    constexpr int B = 4;
    const long long step = (long long)blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long vb = v0 + (threadIdx.x - lane); vb < v1; vb += B * step) {
        T fv[B][6];
        int gv[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const long long vi = vb + lane + u * step;
            const bool in = vi < v1;
            gv[u] = in ? (a.grain ? (int)a.grain[vi] : 0) : -2;
#pragma unroll
            for (int al = 0; al < 6; ++al) fv[u][al] = (in && al < V) ? f[al * N + vi] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const bool in = gv[u] != -2;
            run.voxel(a.m, gv[u], in);
            if (in) {
#pragma unroll
                for (int al = 0; al < 6; ++al) run.fs[al] += fv[u][al];
            }
        }
    }
    run.finish(a.m);
    run.store(a.partials + (size_t)blockIdx.x * 21);
}

// ---------------------------------------------------------------------------
// stress field of the solved pair and its per-CTA sums
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kMaxThreads) k_stress(StressArgs a) {
    const long long N = a.g.N;
    T acc[6] = {0, 0, 0, 0, 0, 0};
    T* sig = (T*)a.sigma;
    for (long long vi = (long long)blockIdx.x * blockDim.x + threadIdx.x; vi < N;
         vi += (long long)gridDim.x * blockDim.x) {
        VoxelState<T> vs;
        load_f<T>(vs, (const T*)a.f, N, vi, a.m.V);
        material<T>(vs, a.m, (const T*)a.eps, (const T*)a.eps_p, a.grain, N, vi, true);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            acc[i] += vs.sig[i];
            if (sig) sig[i * N + vi] = vs.sig[i];
        }
    }
    block_sum_store<6, T>(acc, a.partials + (size_t)blockIdx.x * 6);
}

template <typename T>
__global__ void k_fill(T* eps, long long N, T e0, T e1, T e2, T e3, T e4, T e5) {
    for (long long vi = (long long)blockIdx.x * blockDim.x + threadIdx.x; vi < N;
         vi += (long long)gridDim.x * blockDim.x) {
        eps[vi] = e0;
        eps[N + vi] = e1;
        eps[2 * N + vi] = e2;
        eps[3 * N + vi] = e3;
        eps[4 * N + vi] = e4;
        eps[5 * N + vi] = e5;
    }
}

// Fixed-order sum of per-CTA partials, K values per CTA, by gridDim.x CTAs:
// CTA c sums the partials of blocks [c chunk, (c + 1) chunk) (thread t takes
// blocks t, t + 256, ... of the range; warp shuffles; the 8 warp sums in
// order) into stage[c][k]; the CTA that finishes last (a ticket from an
// atomic counter, after a fence that publishes its sums) adds the CTA sums
// in the order c = 0, 1, ... and resets the counter for the next call.  The
// grouping depends only on nb and the CTA count, so the result is bitwise
// reproducible.  (One CTA reading ~22k partials of 8 values took ~67 us:
// the round trips of a single SM.)
constexpr int kFinalThreads = 256, kFinalCtas = 64;
template <int K>
__global__ void __launch_bounds__(kFinalThreads) k_finalize(const double* __restrict__ part, int nb, int chunk,
                                                            double scale, int expand_c0, double* out,
                                                            double* stage, unsigned* count) {
    __shared__ double red[kFinalThreads / 32][K];
    __shared__ double res[K];
    __shared__ int last;
    const int b0 = blockIdx.x * chunk;
    const int b1 = min(nb, b0 + chunk);
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = 0.0;
#pragma unroll 4
    for (int b = b0 + threadIdx.x; b < b1; b += kFinalThreads) {
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] += part[(size_t)b * K + k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = s[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double x = 0.0;
        for (int w = 0; w < kFinalThreads / 32; ++w) x += red[w][threadIdx.x];
        stage[blockIdx.x * K + threadIdx.x] = x;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < K) {
        const volatile double* st = stage;
        double x = 0.0;
        for (unsigned c = 0; c < gridDim.x; ++c) x += st[c * K + threadIdx.x];
        res[threadIdx.x] = x * scale;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (expand_c0) {
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) out[i * 6 + j] = res[sym_idx(i, j)];
        } else {
            for (int k = 0; k < K; ++k) out[k] = res[k];
        }
        *count = 0;
    }
}

// ---------------------------------------------------------------------------
// device-side control of the step loop (CUDA graph conditional nodes)
// ---------------------------------------------------------------------------
// Start of a step: pick this step's mean strain and open the
// Moulinec-Suquet loop.
__global__ void k_step_begin(StepCtl* c, const double* E_all, double* E_cur, double* E_user, int mixed,
                             cudaGraphConditionalHandle ms) {
    const int k = c->step;
    // strain control: E of the step; uniaxial loading: E_user carries the
    // prescribed axial strain and E_cur keeps the corrected mean strain
    const bool set_cur = !mixed || !c->have_E;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        E_user[i] = E_all[6 * k + i];
        if (set_cur) E_cur[i] = E_all[6 * k + i];
    }
    c->have_E = 1;
    c->it = 0;
    cudaGraphSetConditional(ms, 1);
}

// After each pass: residual from the two FP64 sums, and whether to iterate
// (tol > 0: until r <= tol or max_it passes; tol = 0: exactly max_it).
__global__ void k_ms_decide(StepCtl* c, const double* red, double tol, int max_it, cudaGraphConditionalHandle ms) {
    const double r = red[1] > 0.0 ? sqrt(red[0] / red[1]) : sqrt(red[0]);
    const int it = ++c->it;
    c->resid = r;
    int more;
    if (!isfinite(r)) {
        c->status = -5;  // PF_ENAN
        more = 0;
    } else {
        more = (tol > 0.0 ? (r > tol) : 1) && it < max_it;
        if (!more && tol > 0.0 && r > tol && c->status == 0) c->status = -4;  // PF_ENOCONV
    }
    if (!more) {
        c->n_ms_last = it;
        c->n_ms_total += it;
    }
    cudaGraphSetConditional(ms, more);
}

// End of a step.  The loop body runs the steps in pairs (A then B); after A
// the kernel decides whether B runs (`pair`) and whether another pair follows
// (`outer`); a non-finite residual stops both.
__global__ void k_step_end(StepCtl* c, int first_of_pair, cudaGraphConditionalHandle pair,
                           cudaGraphConditionalHandle outer) {
    const int done = ++c->step;
    if (!first_of_pair) return;
    const int rem = c->nsteps - done;
    const int ok = c->status != -5;
    cudaGraphSetConditional(pair, ok && rem > 0);
    cudaGraphSetConditional(outer, ok && rem > 1);
}

// Uniaxial mixed loading: correct the mean strain after a polarisation pass.
// In the frame whose third axis is the load axis (rows of Q), the five
// stress-free components take Delta E_F = -(C0_FF)^-1 <sigma>_F (engineering
// shears) and the axial component takes its prescribed value d.E_user.d.
// One thread, FP64.
__global__ void k_mixed_update(const double* sums, double invN, const double* C0, const double* E_user, double* E_cur,
                               MixedFrame fr) {
    const int P[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
    const int Vo[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    double sig[3][3], E[3][3], Eu[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            sig[i][j] = sums[Vo[i][j]] * invN;
            E[i][j] = E_cur[Vo[i][j]];
            Eu[i][j] = E_user[Vo[i][j]];
        }
    const double* Q = fr.Q;  // row-major, rows = frame axes
    auto rot2 = [&](const double (*A)[3], double (*B)[3]) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double t = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) t += Q[3 * i + k] * A[k][l] * Q[3 * j + l];
                B[i][j] = t;
            }
    };
    double sr[3][3], Er[3][3];
    rot2(sig, sr);
    rot2(E, Er);
    // axial strain prescribed: d.E_user.d with d = third row of Q
    double edd = 0;
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) edd += Q[6 + k] * Eu[k][l] * Q[6 + l];
    // C0 in the frame: C'_ijkl = Q_ia Q_jb Q_kc Q_ld C_abcd, then Voigt
    double Cr[6][6];
    for (int A = 0; A < 6; ++A)
        for (int B = 0; B < 6; ++B) {
            const int i = P[A][0], j = P[A][1], k = P[B][0], l = P[B][1];
            double t = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const double qab = Q[3 * i + a] * Q[3 * j + b];
                    for (int c = 0; c < 3; ++c)
                        for (int d = 0; d < 3; ++d) t += qab * Q[3 * k + c] * Q[3 * l + d] * C0[Vo[a][b] * 6 + Vo[c][d]];
                }
            Cr[A][B] = t;
        }
    const int F[5] = {0, 1, 3, 4, 5};
    double M[5][6];
    for (int r = 0; r < 5; ++r) {
        for (int c = 0; c < 5; ++c) M[r][c] = Cr[F[r]][F[c]];
        M[r][5] = sr[P[F[r]][0]][P[F[r]][1]];
    }
    // Gaussian elimination with partial pivoting
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        for (int r = c + 1; r < 5; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 6; ++k) {
                const double t = M[c][k];
                M[c][k] = M[piv][k];
                M[piv][k] = t;
            }
        for (int r = c + 1; r < 5; ++r) {
            const double m = M[r][c] / M[c][c];
            for (int k = c; k < 6; ++k) M[r][k] -= m * M[c][k];
        }
    }
    double x[5];
    for (int r = 4; r >= 0; --r) {
        double t = M[r][5];
        for (int k = r + 1; k < 5; ++k) t -= M[r][k] * x[k];
        x[r] = t / M[r][r];
    }
    for (int r = 0; r < 5; ++r) {
        const int i = P[F[r]][0], j = P[F[r]][1];
        const double de = -x[r] * (F[r] < 3 ? 1.0 : 0.5);  // engineering -> tensor shear
        Er[i][j] += de;
        if (i != j) Er[j][i] += de;
    }
    Er[2][2] = edd;
    // back to the sample frame: E = Q^T E' Q
    for (int A = 0; A < 6; ++A) {
        const int i = P[A][0], j = P[A][1];
        double t = 0;
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) t += Q[3 * k + i] * Er[k][l] * Q[3 * l + j];
        E_cur[A] = t;
    }
}

// Extrapolated warm start over the n = 6N strain elements (grid-stride, 16-byte
// vectors with a scalar tail).  The count k is read once per thread before any
// thread could change it (*nh is advanced by k_hist_count, launched after this
// kernel); histories that are not held are never read.
template <typename T> __device__ __forceinline__ T warm_w(const WarmWeights& W, int k, int i);
template <> __device__ __forceinline__ float warm_w<float>(const WarmWeights& W, int k, int i) { return W.wf[k][i]; }
template <> __device__ __forceinline__ double warm_w<double>(const WarmWeights& W, int k, int i) { return W.wd[k][i]; }

template <typename T, int W>
__device__ __forceinline__ void extrapolate_at(T* __restrict__ eps, const WarmHist& H, const WarmWeights& Wt,
                                               long long i, int k, int slots, int head) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    union U {
        V v;
        T t[W];
    };
    auto ld = [&](const T* p) {
        U u;
        if constexpr (W > 1) u.v = *reinterpret_cast<const V*>(p + i);
        else u.t[0] = p[i];
        return u;
    };
    auto st = [&](T* p, const U& u) {
        if constexpr (W > 1) *reinterpret_cast<V*>(p + i) = u.v;
        else p[i] = u.t[0];
    };
    // v[0] = s_n (eps), v[j] = h_j = s_{n-j} in ring slot (head + j - 1) mod slots
    U v[kMaxWarmDegree + 1];
    v[0] = ld(eps);
#pragma unroll
    for (int j = 1; j <= kMaxWarmDegree; ++j)
        if (j < k) v[j] = ld((const T*)H.h[(head + j - 1) % slots]);
    U r;
    if (k >= 2) {
        // weighted sum of the held solutions, newest first
        const T w0 = warm_w<T>(Wt, k, 0);
#pragma unroll
        for (int j = 0; j < W; ++j) r.t[j] = w0 * v[0].t[j];
#pragma unroll
        for (int q = 1; q <= kMaxWarmDegree; ++q) {
            if (q < k) {
                const T c = warm_w<T>(Wt, k, q);
#pragma unroll
                for (int j = 0; j < W; ++j) r.t[j] = r.t[j] + c * v[q].t[j];
            }
        }
    }
    // s_n becomes the newest history in the slot of the oldest (dropped) one;
    // k_hist_count moves the ring head there
    st((T*)H.h[(head + slots - 1) % slots], v[0]);
    if (k >= 2) st(eps, r);
}

template <typename T>
__global__ void __launch_bounds__(256) k_extrapolate(T* __restrict__ eps, WarmHist H, WarmWeights Wt, long long n,
                                                     const int* nh, int slots) {
    constexpr int W = 16 / sizeof(T);
    const int k = nh[0], head = nh[1];
    if (k == 0) return;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nv = n / W;
    for (long long v = tid; v < nv; v += stride) extrapolate_at<T, W>(eps, H, Wt, v * W, k, slots, head);
    for (long long i = nv * W + tid; i < n; i += stride) extrapolate_at<T, 1>(eps, H, Wt, i, k, slots, head);
}

// One more solution held (up to cap); once s_n has been stored, the ring
// head moves to its slot.
__global__ void k_hist_count(int* nh, int cap) {
    const int slots = cap - 1;
    if (nh[0] >= 1) nh[1] = (nh[1] + slots - 1) % slots;
    if (nh[0] < cap) nh[0] += 1;
}

cudaError_t launch_extrapolate(int prec, void* eps, const WarmHist& H, const WarmWeights& W, long long n,
                               const int* nh, int slots, cudaStream_t st) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256;
    const int grid = (int)(want < (long long)nsm * 8 ? want : (long long)nsm * 8);
    if (slots < 1 || slots > kMaxWarmDegree) return cudaErrorInvalidValue;
    if (prec) k_extrapolate<float><<<grid, 256, 0, st>>>((float*)eps, H, W, n, nh, slots);
    else k_extrapolate<double><<<grid, 256, 0, st>>>((double*)eps, H, W, n, nh, slots);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_diff_sums(const T* __restrict__ a, const T* __restrict__ b, long long n,
                                                   double* partials) {
    T acc[2] = {0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const T x = a[i], d = x - b[i];
        acc[0] += d * d;
        acc[1] += x * x;
    }
    block_sum_store<2, T>(acc, partials + (size_t)blockIdx.x * 2);
}

cudaError_t launch_diff_sums(int prec, const void* a, const void* b, long long n, double* partials, int nblocks,
                             cudaStream_t st) {
    if (prec) k_diff_sums<float><<<nblocks, 256, 0, st>>>((const float*)a, (const float*)b, n, partials);
    else k_diff_sums<double><<<nblocks, 256, 0, st>>>((const double*)a, (const double*)b, n, partials);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_clamp(T* __restrict__ f, int V, long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        T v[6], tot = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            if (a < V) {
                const T x = f[a * N + i];
                v[a] = x < (T)0 ? (T)0 : (x > (T)1 ? (T)1 : x);
                tot += v[a];
            }
        }
        const T sc = tot > (T)1 ? (T)1 / tot : (T)1;
#pragma unroll
        for (int a = 0; a < 6; ++a)
            if (a < V) f[a * N + i] = v[a] * sc;
    }
}

cudaError_t launch_clamp(int prec, void* f, int V, long long N, int nblocks, cudaStream_t st) {
    if (prec) k_clamp<float><<<nblocks, 256, 0, st>>>((float*)f, V, N);
    else k_clamp<double><<<nblocks, 256, 0, st>>>((double*)f, V, N);
    return cudaGetLastError();
}

cudaError_t launch_hist_count(int* nh, int cap, cudaStream_t st) {
    k_hist_count<<<1, 1, 0, st>>>(nh, cap);
    return cudaGetLastError();
}

cudaError_t launch_mixed_update(const double* sums, double invN, const double* C0, const double* E_user,
                                double* E_cur, const MixedFrame& fr, cudaStream_t st) {
    k_mixed_update<<<1, 1, 0, st>>>(sums, invN, C0, E_user, E_cur, fr);
    return cudaGetLastError();
}

cudaError_t launch_step_begin(StepCtl* c, const double* E_all, double* E_cur, double* E_user, int mixed,
                              cudaGraphConditionalHandle ms, cudaStream_t st) {
    k_step_begin<<<1, 1, 0, st>>>(c, E_all, E_cur, E_user, mixed, ms);
    return cudaGetLastError();
}

cudaError_t launch_ms_decide(StepCtl* c, const double* red, double tol, int max_it, cudaGraphConditionalHandle ms,
                             cudaStream_t st) {
    k_ms_decide<<<1, 1, 0, st>>>(c, red, tol, max_it, ms);
    return cudaGetLastError();
}

cudaError_t launch_step_end(StepCtl* c, int first_of_pair, cudaGraphConditionalHandle pair,
                            cudaGraphConditionalHandle outer, cudaStream_t st) {
    k_step_end<<<1, 1, 0, st>>>(c, first_of_pair, pair, outer);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t max_dynamic_smem() { return 200 * 1024; }

int c0_ctas_per_sm(int prec, int nthreads) {
    int n = 0;
    const cudaError_t e = prec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_c0<float, 0>, nthreads, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_c0<double, 0>, nthreads, 0);
    return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t launch_c0(int prec, const C0Args& a, int nblocks, cudaStream_t st) {
    // six variants (the full set): loops with compile-time bounds
    if (prec) {
        if (a.m.V == 6) k_c0<float, 6><<<nblocks, a.nthreads, 0, st>>>(a);
        else k_c0<float, 0><<<nblocks, a.nthreads, 0, st>>>(a);
    } else {
        k_c0<double, 0><<<nblocks, a.nthreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_stress(int prec, const StressArgs& a, int nblocks, cudaStream_t st) {
    if (prec) k_stress<float><<<nblocks, a.nthreads, 0, st>>>(a);
    else k_stress<double><<<nblocks, a.nthreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fill(int prec, void* eps, long long N, const double* E, cudaStream_t st) {
    const int nb = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
    if (prec)
        k_fill<float><<<nb, 256, 0, st>>>((float*)eps, N, (float)E[0], (float)E[1], (float)E[2], (float)E[3],
                                          (float)E[4], (float)E[5]);
    else
        k_fill<double><<<nb, 256, 0, st>>>((double*)eps, N, E[0], E[1], E[2], E[3], E[4], E[5]);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblocks, int K, double scale, int expand_c0, double* out,
                            double* stage, unsigned* count, cudaStream_t st) {
    int ctas = (nblocks + 4 * kFinalThreads - 1) / (4 * kFinalThreads);
    ctas = ctas < 1 ? 1 : ctas > kFinalCtas ? kFinalCtas : ctas;
    const int chunk = (nblocks + ctas - 1) / ctas;
    switch (K) {
#define PF_FIN(KK)                                                                                        \
    case KK:                                                                                              \
        k_finalize<KK><<<ctas, kFinalThreads, 0, st>>>(partials, nblocks, chunk, scale, expand_c0, out, stage, \
                                                        count);                                           \
        break;
        PF_FIN(1)
        PF_FIN(2)
        PF_FIN(6)
        PF_FIN(8)
        PF_FIN(21)
#undef PF_FIN
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pfk
