// pf_kernels.cu -- sm_103a kernels of the phase-field twin step.
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

#include "pf_fft.cuh"
#include "pf_f2.cuh"
#include "pf_internal.h"
#include "pf_tma.cuh"

namespace pfk {

constexpr int kMaxThreads = 512;

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int sym_idx(int a, int b) {
    return a <= b ? a * (11 - a) / 2 + b : b * (11 - b) / 2 + a;
}

// out = C v for a symmetric 6x6 stored as 21 packed entries
template <typename T>
__device__ __forceinline__ void sym6_mv(const T* c, const T* v, T* out) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T s = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) s += c[sym_idx(i, j)] * v[j];
        out[i] = s;
    }
}

template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Block-wide sum of K values per thread; threads k < K write out[k] (fixed
// order).  The 32 lanes of a warp are summed in the field precision T (GB300
// runs FP64 at a small fraction of its FP32 rate, and a 5-level FP32 sum of
// a warp adds no more than the per-thread FP32 sums already do); the warp
// sums are combined in FP64.
template <int K, typename T>
__device__ __forceinline__ void block_sum_store(const T (&v)[K], double* out) {
    __shared__ double red[kMaxThreads / 32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][k] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0;
        for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Row r and column x of the element e = r * n + x, stepped by `step`
// elements at a time without an integer division per element.
struct RowCursor {
    int r, x, dr, dx, n;
    __device__ __forceinline__ RowCursor(int e0, int step, int n_) : n(n_) {
        r = e0 / n;
        x = e0 - r * n;
        dr = step / n;
        dx = step - dr * n;
    }
    __device__ __forceinline__ void next() {
        x += dx;
        r += dr;
        if (x >= n) {
            x -= n;
            ++r;
        }
    }
};

// Position of pencil element i in the x passes' shared memory: padded for
// the warp-local transform (wl), plain otherwise.
__device__ __forceinline__ int pel(int i, int wl) { return wl ? padded(i) : i; }

// q / npen for npen in {1, 2, 3} and 0 <= q < 131072 without a division
// (multiply-shift by the rounded-up reciprocal, Granlund & Montgomery 1994).
__device__ __forceinline__ int div_npen(int q, int npen) {
    return npen == 3 ? (int)(((unsigned)q * 43691u) >> 17) : (npen == 2 ? q >> 1 : q);
}

// ---------------------------------------------------------------------------
// local material model of one voxel
// ---------------------------------------------------------------------------
// Reads f_a, the strain, the plastic strain and the grain id of voxel vi;
// returns the elastic strain e = eps - eps* (tensor shears), the engineering
// form ee, C(x) (21 packed) and sigma = C(x) ee.
template <typename T>
struct VoxelState {
    T f[6];
    T fsum;
    T e[6];
    T ee[6];
    T cx[21];
    T sig[6];
    int gid;
};

// I: index type (int for rows staged in shared memory, long long for global fields)
template <typename T, typename I>
__device__ __forceinline__ void load_f(VoxelState<T>& s, const T* __restrict__ f, I N, I vi, int V) {
    s.fsum = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        s.f[a] = (a < V) ? f[a * N + vi] : (T)0;
        s.fsum += s.f[a];
    }
}

// Table rows are padded to 16-byte multiples (24 entries for a packed
// stiffness, 8 for S) and read as vectors.
template <int NV>
__device__ __forceinline__ void load_row(const float* p, float* out) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < NV / 4; ++i) {
        const float4 v = __ldg(q + i);
        out[4 * i] = v.x;
        out[4 * i + 1] = v.y;
        out[4 * i + 2] = v.z;
        out[4 * i + 3] = v.w;
    }
}
template <int NV>
__device__ __forceinline__ void load_row(const double* p, double* out) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) {
        const double2 v = __ldg(q + i);
        out[2 * i] = v.x;
        out[2 * i + 1] = v.y;
    }
}

constexpr int kCRow = 24;  // padded packed-stiffness row
constexpr int kSRow = 8;   // padded Schmid row

template <typename T, typename I>
__device__ __forceinline__ void material(VoxelState<T>& s, const MatDesc& m, const T* __restrict__ eps,
                                         const T* __restrict__ ep, const uint16_t* __restrict__ grain,
                                         I N, I vi, bool want_stress, T* quad = nullptr) {
    const int V = m.V;
    s.gid = grain ? (int)grain[vi] : 0;
    const T* Cm = (const T*)m.Cm + s.gid * kCRow;
    const T* dC = (const T*)m.dC + (size_t)s.gid * V * kCRow;
    const T* S = (const T*)m.S + (size_t)s.gid * V * kSRow;
    const T gam = (T)m.gamma;
    if constexpr (sizeof(T) == 4) {
        // FP32: the eigenstrain first, then one pass over the C_tw - C_m rows
        // for the mixture (and, when quad is given, e:(C_tw - C_m):e per
        // variant), two entries per instruction
        float2 e2[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            e2[p] = eps ? f2(eps[(2 * p) * N + vi], eps[(2 * p + 1) * N + vi]) : f2(0.f);
            if (ep) e2[p] = ffma2(f2(ep[(2 * p) * N + vi], ep[(2 * p + 1) * N + vi]), f2(-1.f), e2[p]);
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            if (a < V) {
                const float4* r = reinterpret_cast<const float4*>(S + a * kSRow);
                const float4 s0 = __ldg(r), s1 = __ldg(r + 1);
                const float2 g = f2(-gam * s.f[a]);
                e2[0] = ffma2(f2(s0.x, s0.y), g, e2[0]);
                e2[1] = ffma2(f2(s0.z, s0.w), g, e2[1]);
                e2[2] = ffma2(f2(s1.x, s1.y), g, e2[2]);
            }
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            s.e[2 * p] = e2[p].x;
            s.e[2 * p + 1] = e2[p].y;
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) s.ee[i] = (i < 3) ? s.e[i] : (T)2 * s.e[i];
        // pp = (w_ij e_i e_j) in packed order, entries 21..23 zero
        float2 pp[12];
        if (quad) {
            float w[24];
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = i; j < 6; ++j) w[sym_idx(i, j)] = ((i == j) ? 1.f : 2.f) * s.ee[i] * s.ee[j];
            w[21] = w[22] = w[23] = 0.f;
#pragma unroll
            for (int k = 0; k < 12; ++k) pp[k] = f2(w[2 * k], w[2 * k + 1]);
        }
        float2 c2[12];
        {
            const float4* q = reinterpret_cast<const float4*>(Cm);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const float4 v = __ldg(q + i);
                c2[2 * i] = f2(v.x, v.y);
                c2[2 * i + 1] = f2(v.z, v.w);
            }
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            if (a < V) {
                const float2 fa = f2(s.f[a]);
                const float4* q = reinterpret_cast<const float4*>(dC + a * kCRow);
                float2 u = f2(0.f);
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const float4 v = __ldg(q + i);
                    c2[2 * i] = ffma2(f2(v.x, v.y), fa, c2[2 * i]);
                    c2[2 * i + 1] = ffma2(f2(v.z, v.w), fa, c2[2 * i + 1]);
                    if (quad) {
                        u = ffma2(f2(v.x, v.y), pp[2 * i], u);
                        u = ffma2(f2(v.z, v.w), pp[2 * i + 1], u);
                    }
                }
                if (quad) quad[a] = u.x + u.y;
            }
        }
#pragma unroll
        for (int i = 0; i < 21; ++i) s.cx[i] = (i & 1) ? c2[i >> 1].y : c2[i >> 1].x;
        if (want_stress) sym6_mv<T>(s.cx, s.ee, s.sig);
        return;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T x = eps ? eps[i * N + vi] : (T)0;
        if (ep) x -= ep[i * N + vi];
        s.e[i] = x;
    }
    {
        T row[kCRow];
        load_row<kCRow>(Cm, row);
#pragma unroll
        for (int i = 0; i < 21; ++i) s.cx[i] = row[i];
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        if (a < V) {
            const T fa = s.f[a];
            T row[kCRow];
            load_row<kCRow>(dC + a * kCRow, row);
#pragma unroll
            for (int i = 0; i < 21; ++i) s.cx[i] += fa * row[i];
            T sr[kSRow];
            load_row<kSRow>(S + a * kSRow, sr);
            const T g = gam * fa;
#pragma unroll
            for (int i = 0; i < 6; ++i) s.e[i] -= g * sr[i];
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) s.ee[i] = (i < 3) ? s.e[i] : (T)2 * s.e[i];
    if (want_stress) sym6_mv<T>(s.cx, s.ee, s.sig);
}

// ---------------------------------------------------------------------------
// local material model in the grain's crystal frame (x forward pass)
// ---------------------------------------------------------------------------
// Every grain holds the same HCP crystal and the same twin variants, seen
// through its rotation R (crystal -> sample).  The pass rotates the strain
// into the crystal frame, evaluates the mixture with the grain-independent
// tables (kernel arguments: constant operands, nine rotation entries loaded
// per voxel instead of the 216 sample-frame table entries) and rotates the
// stress back: sigma = R [C_c (R^T eps R - eps*_c)] R^T, the same sigma as
// material() up to rounding.  Contractions (sigma:S_a, e:dC_a:e, sigma:e)
// are frame-invariant and taken in the crystal frame.
template <typename T>
struct XtalState {
    T ee[6];   // elastic strain, crystal frame, engineering shears
    T sc[6];   // stress, crystal frame
    T sig[6];  // stress, sample frame
};

template <typename T> __device__ __forceinline__ const XtalTab<T>& xtab(const XFwdArgs& a);
template <> __device__ __forceinline__ const XtalTab<float>& xtab<float>(const XFwdArgs& a) { return a.xt.f; }
template <> __device__ __forceinline__ const XtalTab<double>& xtab<double>(const XFwdArgs& a) { return a.xt.d; }

// Voigt pairs (xx yy zz yz xz xy): component v is tensor entry (vi(v), vj(v))
__host__ __device__ constexpr int vi(int v) { return v < 3 ? v : (v == 3 ? 1 : 0); }
__host__ __device__ constexpr int vj(int v) { return v < 3 ? v : (v == 5 ? 1 : 2); }

// out = R^T E R for the symmetric tensor E given as Voigt components with
// tensor shears (sample -> crystal frame)
template <typename T>
__device__ __forceinline__ void rot_to_crystal(const T (&R)[12], const T (&e)[6], T (&out)[6]) {
    const T E[3][3] = {{e[0], e[5], e[4]}, {e[5], e[1], e[3]}, {e[4], e[3], e[2]}};
    T M[3][3];  // E R
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = E[i][0] * R[j] + E[i][1] * R[4 + j] + E[i][2] * R[8 + j];
#pragma unroll
    for (int v = 0; v < 6; ++v) {
        const int i = vi(v), j = vj(v);
        out[v] = R[i] * M[0][j] + R[4 + i] * M[1][j] + R[8 + i] * M[2][j];
    }
}

// out = R S R^T (crystal -> sample frame), same component convention
template <typename T>
__device__ __forceinline__ void rot_to_sample(const T (&R)[12], const T (&s)[6], T (&out)[6]) {
    const T Sm[3][3] = {{s[0], s[5], s[4]}, {s[5], s[1], s[3]}, {s[4], s[3], s[2]}};
    T M[3][3];  // R S
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = R[4 * i] * Sm[0][j] + R[4 * i + 1] * Sm[1][j] + R[4 * i + 2] * Sm[2][j];
#pragma unroll
    for (int v = 0; v < 6; ++v) {
        const int i = vi(v), j = vj(v);
        out[v] = M[i][0] * R[4 * j] + M[i][1] * R[4 * j + 1] + M[i][2] * R[4 * j + 2];
    }
}

// R of grain gid: three rows of four entries (the fourth is padding)
template <typename T>
__device__ __forceinline__ void load_rot(const MatDesc& m, int gid, T (&R)[12]) {
    load_row<12>((const T*)m.R + gid * 12, R);
}

// Elastic state of one voxel (twin fractions f, grain gid); with QUAD also
// quad[a] = e:(C_tw^a - C_hex):e in the crystal frame.
template <typename T, bool QUAD, typename I>
__device__ __forceinline__ void xtal_material(XtalState<T>& xs, const XFwdArgs& a, const T (&f)[6], int gid,
                                              const T* __restrict__ eps, const T* __restrict__ ep, I N, I vi,
                                              T (&quad)[6]) {
    const XtalTab<T>& t = xtab<T>(a);
    const int V = a.m.V;
    T R[12];
    load_rot<T>(a.m, gid, R);
    T es[6], e[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T x = eps ? eps[i * N + vi] : (T)0;
        if (ep) x -= ep[i * N + vi];
        es[i] = x;
    }
    rot_to_crystal<T>(R, es, e);
    const T gam = (T)a.m.gamma;
    // eigenstrain
    if constexpr (sizeof(T) == 4) {
        float2 e2[3] = {f2(e[0], e[1]), f2(e[2], e[3]), f2(e[4], e[5])};
#pragma unroll
        for (int al = 0; al < 6; ++al) {
            if (al < V) {
                const float2 g = f2(-gam * f[al]);
#pragma unroll
                for (int k = 0; k < 3; ++k) e2[k] = ffma2(f2(t.S[al][2 * k], t.S[al][2 * k + 1]), g, e2[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            e[2 * k] = e2[k].x;
            e[2 * k + 1] = e2[k].y;
        }
    } else {
#pragma unroll
        for (int al = 0; al < 6; ++al) {
            if (al < V) {
                const T g = gam * f[al];
#pragma unroll
                for (int k = 0; k < 6; ++k) e[k] -= g * t.S[al][k];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) xs.ee[i] = (i < 3) ? e[i] : (T)2 * e[i];
    const T* ee = xs.ee;
    if (QUAD) {
        // q_a = (C_tw^a - C_hex) ee serves both sigma = C_hex ee + sum_a f_a q_a
        // and quad_a = ee . q_a
        T sc[6];
        sc[0] = t.Ch[0] * ee[0] + t.Ch[1] * ee[1] + t.Ch[2] * ee[2];
        sc[1] = t.Ch[1] * ee[0] + t.Ch[0] * ee[1] + t.Ch[2] * ee[2];
        sc[2] = t.Ch[2] * (ee[0] + ee[1]) + t.Ch[3] * ee[2];
        sc[3] = t.Ch[4] * ee[3];
        sc[4] = t.Ch[4] * ee[4];
        sc[5] = t.Ch[5] * ee[5];
        if constexpr (sizeof(T) == 4) {
            // FP32: q_a two rows per instruction from the row-pair table
            float2 ee2[6], sc2[3];
#pragma unroll
            for (int j = 0; j < 6; ++j) ee2[j] = f2(ee[j]);
#pragma unroll
            for (int p = 0; p < 3; ++p) sc2[p] = f2(sc[2 * p], sc[2 * p + 1]);
#pragma unroll
            for (int al = 0; al < 6; ++al) {
                if (al < V) {
                    float2 q2[3];
#pragma unroll
                    for (int p = 0; p < 3; ++p) {
                        q2[p] = fmul2(f2(t.dCp[al][p * 12], t.dCp[al][p * 12 + 1]), ee2[0]);
#pragma unroll
                        for (int j = 1; j < 6; ++j)
                            q2[p] = ffma2(f2(t.dCp[al][p * 12 + 2 * j], t.dCp[al][p * 12 + 2 * j + 1]), ee2[j], q2[p]);
                    }
                    float2 u = fmul2(q2[0], f2(ee[0], ee[1]));
                    u = ffma2(q2[1], f2(ee[2], ee[3]), u);
                    u = ffma2(q2[2], f2(ee[4], ee[5]), u);
                    quad[al] = u.x + u.y;
                    const float2 fa = f2(f[al]);
#pragma unroll
                    for (int p = 0; p < 3; ++p) sc2[p] = ffma2(fa, q2[p], sc2[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                sc[2 * p] = sc2[p].x;
                sc[2 * p + 1] = sc2[p].y;
            }
        } else {
#pragma unroll
            for (int al = 0; al < 6; ++al) {
                if (al < V) {
                    T q[6];
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        T x = 0;
#pragma unroll
                        for (int j = 0; j < 6; ++j) x += t.dC[al][sym_idx(i, j)] * ee[j];
                        q[i] = x;
                    }
                    T qq = 0;
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        qq += q[i] * ee[i];
                        sc[i] += f[al] * q[i];
                    }
                    quad[al] = qq;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) xs.sc[i] = sc[i];
    } else {
        // C(x) in the crystal frame: the HCP pattern plus the twin corrections
        T cx[22];
#pragma unroll
        for (int i = 0; i < 22; ++i) cx[i] = (T)0;
        cx[sym_idx(0, 0)] = t.Ch[0];
        cx[sym_idx(1, 1)] = t.Ch[0];
        cx[sym_idx(0, 1)] = t.Ch[1];
        cx[sym_idx(0, 2)] = t.Ch[2];
        cx[sym_idx(1, 2)] = t.Ch[2];
        cx[sym_idx(2, 2)] = t.Ch[3];
        cx[sym_idx(3, 3)] = t.Ch[4];
        cx[sym_idx(4, 4)] = t.Ch[4];
        cx[sym_idx(5, 5)] = t.Ch[5];
        if constexpr (sizeof(T) == 4) {
            // two entries per instruction
            float2 c2[11];
#pragma unroll
            for (int k = 0; k < 11; ++k) c2[k] = f2(cx[2 * k], cx[2 * k + 1]);
#pragma unroll
            for (int al = 0; al < 6; ++al) {
                if (al < V) {
                    const float2 fa = f2(f[al]);
#pragma unroll
                    for (int k = 0; k < 11; ++k) c2[k] = ffma2(f2(t.dC[al][2 * k], t.dC[al][2 * k + 1]), fa, c2[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                cx[2 * k] = c2[k].x;
                cx[2 * k + 1] = c2[k].y;
            }
        } else {
#pragma unroll
            for (int al = 0; al < 6; ++al) {
                if (al < V) {
#pragma unroll
                    for (int i = 0; i < 21; ++i) cx[i] += f[al] * t.dC[al][i];
                }
            }
        }
        sym6_mv<T>(cx, xs.ee, xs.sc);
    }
    rot_to_sample<T>(R, xs.sc, xs.sig);
}

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

// Work items (pencil q, index k < len) of the split or unpack around an x
// transform: with the warp-local transform each pencil stays with the threads
// that transform it (k = butterfly, butterfly + tpp, ...), otherwise all
// threads sweep all items with k fastest.
template <typename Args, typename F>
__device__ __forceinline__ void pencil_items(const Args& a, int nP, int len, F&& f) {
    if (a.wl) {
        const int tpp = a.plan.n / a.plan.rmin;
        const int ppr = blockDim.x / tpp;
        const int j = threadIdx.x % tpp;
        for (int q = threadIdx.x / tpp; q < nP; q += ppr)
            for (int k = j; k < len; k += tpp) f(q, k);
    } else {
        RowCursor rc(threadIdx.x, blockDim.x, len);
        for (int e = threadIdx.x; e < nP * len; e += blockDim.x, rc.next()) f(rc.r, rc.x);
    }
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
template <typename T>
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
                if (al < m.V) v += __shfl_sync(full, fs[al], src) * dC[al * kCRow];
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
                    if (i < m.V) fs[i] += __shfl_xor_sync(full, fs[i], o);
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
template <typename T>
__global__ void __launch_bounds__(kMaxThreads) k_c0(C0Args a) {
    const long long N = a.g.N;
    const int V = a.m.V;
    const T* f = (const T*)a.f;
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    const long long v0 = (long long)blockIdx.x * per;
    const long long v1 = v0 + per < N ? v0 + per : N;
    C0Run<T> run;
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

// Fixed-order sum of per-CTA partials, K values per CTA: thread t sums
// b = t, t + 256, ... for every k, then warp shuffles and the 8 warp sums in
// order.  One small kernel per K keeps the code (and its instruction fetch on
// a cold SM) short.
constexpr int kFinalThreads = 256;
template <int K>
__global__ void __launch_bounds__(kFinalThreads) k_finalize(const double* __restrict__ part, int nb, double scale,
                                                            int expand_c0, double* out) {
    __shared__ double red[kFinalThreads / 32][K];
    __shared__ double res[K];
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = 0.0;
#pragma unroll 4
    for (int b = threadIdx.x; b < nb; b += kFinalThreads) {
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

template <typename KernelT>
static void allow_smem(KernelT kern, size_t smem) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

int c0_ctas_per_sm(int prec, int nthreads) {
    int n = 0;
    const cudaError_t e = prec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_c0<float>, nthreads, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_c0<double>, nthreads, 0);
    return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t launch_c0(int prec, const C0Args& a, int nblocks, cudaStream_t st) {
    if (prec) k_c0<float><<<nblocks, a.nthreads, 0, st>>>(a);
    else k_c0<double><<<nblocks, a.nthreads, 0, st>>>(a);
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
                            cudaStream_t st) {
    switch (K) {
        case 1: k_finalize<1><<<1, kFinalThreads, 0, st>>>(partials, nblocks, scale, expand_c0, out); break;
        case 2: k_finalize<2><<<1, kFinalThreads, 0, st>>>(partials, nblocks, scale, expand_c0, out); break;
        case 6: k_finalize<6><<<1, kFinalThreads, 0, st>>>(partials, nblocks, scale, expand_c0, out); break;
        case 8: k_finalize<8><<<1, kFinalThreads, 0, st>>>(partials, nblocks, scale, expand_c0, out); break;
        case 21: k_finalize<21><<<1, kFinalThreads, 0, st>>>(partials, nblocks, scale, expand_c0, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pfk
