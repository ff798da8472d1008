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
// sums are combined in FP64.  NW bounds the CTA's warps (the shared
// array's rows); block_sum_store takes the library's largest CTA.
template <int K, typename T, int NW>
__device__ __forceinline__ void block_sum_store_w(const T (&v)[K], double* out) {
    __shared__ double red[NW][K];
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

template <int K, typename T>
__device__ __forceinline__ void block_sum_store(const T (&v)[K], double* out) {
    block_sum_store_w<K, T, kMaxThreads / 32>(v, out);
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

// The pair model.  Variant ids k and k + 3 (k = 0, 1, 2) are images of each
// other under the 180-degree rotation about c, which reverses the yz and xz
// Voigt components: C_twin^(k+3) - C_hex = D (C_twin^k - C_hex) D and
// S_(k+3) = D S_k, D = diag(1, 1, 1, -1, -1, 1).  The evolved variants form
// groups (a pair, or one variant alone); group g owns internal positions 2g
// (its first id) and 2g + 1 (the partner, when evolved) and one table set.
// With p_g = f_2g + f_(2g+1) and m_g = f_2g - f_(2g+1),
//   sum_a f_a (C_twin^a - C_hex) = sum_g dC_g o (p_g where D_i D_j = 1, else m_g),
//   sum_a f_a S_a                = sum_g S_g o (p_g where D_i = 1, else m_g),
// entrywise, so six variants cost three table applications.

// Voigt components reversed by the 180-degree rotation about c (yz, xz)
__host__ __device__ constexpr bool odd_c(int v) { return v == 3 || v == 4; }
// packed entry (i, j) takes the pair difference m_g
__host__ __device__ constexpr bool flips(int i, int j) { return odd_c(i) != odd_c(j); }
// entry (i <= j) of the HCP stiffness as an index into XtalTab::Ch, -1 where zero
__host__ __device__ constexpr int ch_idx(int i, int j) {
    return (i == j) ? (i < 2 ? 0 : i == 2 ? 3 : i < 5 ? 4 : 5)
                    : (i == 0 && j == 1) ? 1 : ((i < 2 && j == 2) ? 2 : -1);
}

// Elastic strain of one voxel in the crystal frame (tensor shears),
// e = R^T (eps - eps_p) R - gamma sum_g S_g o (p_g or m_g), and the twin
// fractions at the group positions (fpos(p): fraction at position p).
// FULL: three groups of two variants (all six ids), known at compile time.
template <typename T, bool FULL = false, typename FP>
__device__ __forceinline__ void xtal_strain(const XtalTab<T>& t, const XGroups& gr, const T (&R)[12],
                                            const T (&es)[6], FP&& fpos, T (&e)[6], T (&fa)[3], T (&fb)[3]) {
    rot_to_crystal<T>(R, es, e);
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        fa[g] = fb[g] = (T)0;
        if (FULL || g == 0 || g < gr.ng) {  // group 0 always exists (V >= 1)
            fa[g] = fpos(2 * g);
            if (FULL || gr.both[g]) fb[g] = fpos(2 * g + 1);
            const T sp = fa[g] + fb[g], dm = fa[g] - fb[g];
#pragma unroll
            for (int i = 0; i < 6; ++i) e[i] -= t.S[g][i] * (odd_c(i) ? dm : sp);
        }
    }
}

// Stress of one voxel, sample frame: sigma = R [C(f) (e)] R^T with the
// mixture C(f) = C_hex + sum_g dC_g o (p_g or m_g) formed once (21 entries).
template <typename T, bool FULL = false, typename FP>
__device__ __forceinline__ void xtal_stress(const XtalTab<T>& t, const XGroups& gr, const T (&R)[12],
                                            const T (&es)[6], FP&& fpos, T (&sig)[6]) {
    T e[6], fa[3], fb[3];
    xtal_strain<T, FULL>(t, gr, R, es, fpos, e, fa, fb);
    // group 0 always exists (V >= 1): its terms start the mixture from C_hex
    T M[21];
    {
        const T sp = fa[0] + fb[0], dm = fa[0] - fb[0];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = i; j < 6; ++j) {
                const T c = ch_idx(i, j) >= 0 ? t.Ch[ch_idx(i, j)] : (T)0;
                M[sym_idx(i, j)] = t.dC[0][sym_idx(i, j)] * (flips(i, j) ? dm : sp) + c;
            }
    }
#pragma unroll
    for (int g = 1; g < 3; ++g) {
        if (FULL || g < gr.ng) {
            const T sp = fa[g] + fb[g], dm = fa[g] - fb[g];
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = i; j < 6; ++j) M[sym_idx(i, j)] += t.dC[g][sym_idx(i, j)] * (flips(i, j) ? dm : sp);
        }
    }
    T ee[6], sc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        ee[i] = (i < 3) ? e[i] : (T)2 * e[i];
        sc[i] = (T)0;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) {
            sc[i] += M[sym_idx(i, j)] * ee[j];
            if (i != j) sc[j] += M[sym_idx(i, j)] * ee[i];
        }
    rot_to_sample<T>(R, sc, sig);
}

// Driving-force state of one voxel in the crystal frame: with a_g, b_g the
// products of ee with the even and odd parts of dC_g, the two members of a
// group have q = dC ee = a_g + b_g and a_g - b_g, so
//   sigma_c = C_hex ee + sum_g (p_g a_g + m_g b_g),
//   quad_p  = ee . q_p              (e : (C_twin - C_hex) : e),
//   rss_p   = sigma_c : S_p         (tensor S, shear terms twice).
// Positions of absent partners get zeros.
template <typename T, bool FULL = false, typename FP>
__device__ __forceinline__ void xtal_drive(XtalState<T>& xs, const XtalTab<T>& t, const XGroups& gr,
                                           const T (&R)[12], const T (&es)[6], FP&& fpos, T (&fp)[6],
                                           T (&quad)[6], T (&rss)[6]) {
    T e[6], fa[3], fb[3];
    xtal_strain<T, FULL>(t, gr, R, es, fpos, e, fa, fb);
    T* ee = xs.ee;
#pragma unroll
    for (int i = 0; i < 6; ++i) ee[i] = (i < 3) ? e[i] : (T)2 * e[i];
    T sc[6];
    sc[0] = t.Ch[0] * ee[0] + t.Ch[1] * ee[1] + t.Ch[2] * ee[2];
    sc[1] = t.Ch[1] * ee[0] + t.Ch[0] * ee[1] + t.Ch[2] * ee[2];
    sc[2] = t.Ch[2] * (ee[0] + ee[1]) + t.Ch[3] * ee[2];
    sc[3] = t.Ch[4] * ee[3];
    sc[4] = t.Ch[4] * ee[4];
    sc[5] = t.Ch[5] * ee[5];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        fp[2 * g] = fa[g];
        fp[2 * g + 1] = fb[g];
        quad[2 * g] = quad[2 * g + 1] = (T)0;
        if (FULL || g == 0 || g < gr.ng) {  // group 0 always exists
            T av[6], bv[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) av[i] = bv[i] = (T)0;
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = i; j < 6; ++j) {
                    const T d = t.dC[g][sym_idx(i, j)];
                    if (flips(i, j)) {
                        bv[i] += d * ee[j];
                        bv[j] += d * ee[i];
                    } else {
                        av[i] += d * ee[j];
                        if (i != j) av[j] += d * ee[i];
                    }
                }
            T ea = 0, eb = 0;
            const T sp = fa[g] + fb[g], dm = fa[g] - fb[g];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                ea += ee[i] * av[i];
                eb += ee[i] * bv[i];
                sc[i] += sp * av[i] + dm * bv[i];
            }
            quad[2 * g] = ea + eb;
            quad[2 * g + 1] = ea - eb;
        }
    }
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        rss[2 * g] = rss[2 * g + 1] = (T)0;
        if (FULL || g == 0 || g < gr.ng) {  // group 0 always exists
            T u = 0, v = 0;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const T w = (i < 3 ? (T)1 : (T)2) * sc[i] * t.S1[g][i];
                if (odd_c(i)) v += w;
                else u += w;
            }
            rss[2 * g] = u + v;
            rss[2 * g + 1] = u - v;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) xs.sc[i] = sc[i];
    rot_to_sample<T>(R, xs.sc, xs.sig);
}

// ---------------------------------------------------------------------------
// element-wise producer of the forward x passes
// ---------------------------------------------------------------------------
// Entry threadIdx.x (< 24) of the shared copy of C0: the 21 packed entries
// of the symmetric Voigt 6x6 (upper triangle, row by row), zero-padded to 24
// so that the table reads as 16-byte vectors.
template <typename T>
__device__ __forceinline__ void load_c0(const double* C0, T* sC0) {
    const int t = threadIdx.x;
    int i = 0, k = t;
    while (i < 6 && k >= 6 - i) {
        k -= 6 - i;
        ++i;
    }
    sC0[t] = t < 21 ? (T)C0[i * 6 + i + k] : (T)0;
}

// tau = sig - C0 : ee for the symmetric C0 held packed in shared memory
template <typename T>
__device__ __forceinline__ void c0_contract(const T* sC0, const T (&sig)[6], const T (&ee)[6], T (&out)[6]) {
    T c[24];
    if constexpr (sizeof(T) == 4) {
        const float4* q = reinterpret_cast<const float4*>(sC0);
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            const float4 x = q[v];
            c[4 * v] = x.x;
            c[4 * v + 1] = x.y;
            c[4 * v + 2] = x.z;
            c[4 * v + 3] = x.w;
        }
    } else {
        const double2* q = reinterpret_cast<const double2*>(sC0);
#pragma unroll
        for (int v = 0; v < 12; ++v) {
            const double2 x = q[v];
            c[2 * v] = x.x;
            c[2 * v + 1] = x.y;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = sig[i];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) {
            out[i] -= c[sym_idx(i, j)] * ee[j];
            if (i != j) out[j] -= c[sym_idx(i, j)] * ee[i];
        }
}

// Produce the real fields of one voxel: tau (TAU), g = f + dt c3 d (DRIVE) or
// f (PLAIN).  Field pointers address component 0 of the voxel's row block;
// component c lives at c * cst.  Twin fractions are read by internal
// position p at f + map(p) * cst (map = fmap when given, else the identity:
// rows staged by position).  Output p of DRIVE belongs to the variant at
// position p.  DRIVE also accumulates <sigma>, G_dw, G_me.
template <typename T, int MODE, typename I, bool FULL = false>
__device__ __forceinline__ void xfwd_voxel(const XFwdArgs& a, const T* f, const int* fmap, const T* eps, const T* ep,
                                           const uint16_t* grain, I cst, I li, long long gi, const T* sC0,
                                           T (&out)[6], T (&acc)[8], int gid_in = -1) {
    auto fpos = [&](int p) { return f[(I)(fmap ? fmap[p] : p) * cst + li]; };
    if (MODE == X_PLAIN) {
#pragma unroll
        for (int p = 0; p < 6; ++p) out[p] = p < a.nfin ? fpos(p) : (T)0;
        return;
    }
    const XtalTab<T>& t = xtab<T>(a);
    // the grain id (gid_in >= 0: already loaded by the caller)
    const int gid = gid_in >= 0 ? gid_in : grain ? (int)grain[li] : 0;
    T R[12];
    load_rot<T>(a.m, gid, R);
    T ev[6], es[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) es[i] = ev[i] = eps[i * cst + li];
    if (ep) {
#pragma unroll
        for (int i = 0; i < 6; ++i) es[i] -= ep[i * cst + li];
    }
    if (MODE == X_TAU || MODE == X_TAU_SIG) {
        T sig[6];
        xtal_stress<T, FULL>(t, a.gr, R, es, fpos, sig);
        if (MODE == X_TAU_SIG) {
#pragma unroll
            for (int i = 0; i < 6; ++i) acc[i] += sig[i];
        }
        // tau = sigma - C0 : eps (engineering shears for the Voigt product)
        T ee[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) ee[i] = (i < 3) ? ev[i] : (T)2 * ev[i];
        c0_contract<T>(sC0, sig, ee, out);
        return;
    }
    // X_DRIVE: d_a of Eq. fRate2 over all phases, the matrix f0 included
    XtalState<T> xs;
    T fp[6], quad[6], rss[6];
    xtal_drive<T, FULL>(xs, t, a.gr, R, es, fpos, fp, quad, rss);
    const T c1 = (T)a.c1, c3dt = (T)a.c3dt, gam = (T)a.m.gamma;
    const T mf = a.mob ? ((const T*)a.mob)[gi] : (T)1;  // pad-layer mobility factor
    T fsum = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p) fsum += fp[p];
    const T f0 = (T)1 - fsum;
    // sum over the other phases b (matrix included) of f_b (f_b - f_a)
    // = S2 - f_a S1 with S1 = sum_b f_b and S2 = sum_b f_b^2 over all phases
    // (positions without a variant hold 0 and add nothing)
    T S1 = f0 + fsum, S2 = f0 * f0;
#pragma unroll
    for (int p = 0; p < 6; ++p) S2 += fp[p] * fp[p];
    // d_a and g_a = f_a + dt c3 M d_a; positions without a variant give 0.
    // One test per voxel chooses between the plain update and the one of the
    // pad layer / Picard iterations (f_base, g_out)
    T dd[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        const T fa = fp[p];
        const T chem = -c1 * fa * (S2 - fa * S1);
        dd[p] = chem + gam * rss[p] - (T)0.5 * quad[p];
    }
    if (!a.f_base && !a.g_out) {
#pragma unroll
        for (int p = 0; p < 6; ++p) out[p] = (FULL || a.out_slot[p] >= 0) ? fp[p] + c3dt * mf * dd[p] : (T)0;
    } else {
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            const int slot = a.out_slot[p];
            if (FULL || slot >= 0) {
                out[p] = (a.f_base ? ((const T*)a.f_base)[(size_t)slot * a.g.N + gi] : fp[p]) + c3dt * mf * dd[p];
                if (a.g_out) ((T*)a.g_out)[(size_t)slot * a.g.N + gi] = out[p];
            } else {
                out[p] = 0;
            }
        }
    }
    // statistics: <sigma>; G_dw and G_me only for pf_energy
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[i] += xs.sig[i];
    if (!a.energy) return;
    T gdw = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const T fb2 = fp[b] * fp[b];
        gdw += f0 * f0 * fb2;
#pragma unroll
        for (int c = b + 1; c < 6; ++c) gdw += fb2 * fp[c] * fp[c];
    }
    acc[6] += (T)0.5 * c1 * gdw;
    T gme = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) gme += xs.sc[i] * xs.ee[i];
    acc[7] += (T)0.5 * gme;
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
