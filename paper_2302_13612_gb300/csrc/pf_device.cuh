// pf_device.cuh -- device helpers shared by the kernel translation units:
// reductions, row cursors, the local material models (sample frame and the
// grain's crystal frame) and the launch helper for large shared memory.
#pragma once
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

template <typename KernelT>
inline void allow_smem(KernelT kern, size_t smem) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace pfk
