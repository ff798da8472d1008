// pf_fft.cuh -- complex arithmetic, radix-2/3/4/5/8/16 butterflies and the
// in-place Stockham passes over pencils held in shared memory.
//
// A pencil is one 1-D transform of length n; a CTA holds nP pencils in shared
// memory at s[q + i*es] (pencil q = 0..nP-1, element i = 0..n-1, element
// stride es >= nP), i.e. pencils interleaved so that consecutive threads touch
// consecutive addresses.  The Stockham autosort stage for radix R, with Ns the
// product of the radices already applied, takes butterfly j (0 <= j < n/R):
//     k = j mod Ns,  v_r = x[j + r n/R] * w_n^{r k n/(Ns R)},  V = DFT_R(v),
//     y[(j - k) R + k + r Ns] = V_r,
// and leaves the transform in natural order after the last stage.  Every
// thread keeps its butterfly in registers across a barrier, so one shared
// buffer suffices; pencils are processed in groups small enough that every
// butterfly of a group has its own thread.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pfk {

template <typename T> struct cx_of;
template <> struct cx_of<float> { typedef float2 type; };
template <> struct cx_of<double> { typedef double2 type; };
template <typename T> using cx = typename cx_of<T>::type;

template <typename T> __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// a * w and a * conj(w)
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> w) {
    return mk<T>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
template <typename T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> w) {
    return mk<T>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cx<T> rot_mi(cx<T> a) {
    return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// cos and sin of 2 pi e / 16, e = 0..15 (exact values of the 16th roots of unity).
constexpr double kC1 = 0.92387953251128675613;  // cos(pi/8)
constexpr double kS1 = 0.38268343236508977173;  // sin(pi/8)
constexpr double kR2 = 0.70710678118654752440;  // sqrt(2)/2
__host__ __device__ constexpr double cos16(int e) {
    return e == 0 ? 1.0 : e == 1 ? kC1 : e == 2 ? kR2 : e == 3 ? kS1 : e == 4 ? 0.0 :
           e == 5 ? -kS1 : e == 6 ? -kR2 : e == 7 ? -kC1 : e == 8 ? -1.0 : e == 9 ? -kC1 :
           e == 10 ? -kR2 : e == 11 ? -kS1 : e == 12 ? 0.0 : e == 13 ? kS1 : e == 14 ? kR2 : kC1;
}
__host__ __device__ constexpr double sin16(int e) { return cos16((e + 12) & 15); }

// v * exp(-+ 2 pi i E / N) for N in {8, 16}, E a compile-time constant.
template <typename T, int N, int E, bool INV>
__device__ __forceinline__ cx<T> twc(cx<T> v) {
    constexpr int e = (E % N) * (16 / N);  // in 16ths of a turn
    if constexpr (e == 0) {
        return v;
    } else if constexpr (e == 8) {
        return mk<T>(-v.x, -v.y);
    } else if constexpr (e == 4) {
        return rot_mi<T, INV>(v);
    } else if constexpr (e == 12) {
        return rot_mi<T, !INV>(v);
    } else {
        const T c = (T)cos16(e), s = (T)sin16(e);
        // forward multiplies by (c - i s), inverse by (c + i s)
        return INV ? mk<T>(v.x * c - v.y * s, v.y * c + v.x * s)
                   : mk<T>(v.x * c + v.y * s, v.y * c - v.x * s);
    }
}

template <typename T, bool INV> __device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
    cx<T> t = a;
    a = cadd<T>(t, b);
    b = csub<T>(t, b);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cx<T>& v0, cx<T>& v1, cx<T>& v2, cx<T>& v3) {
    cx<T> t0 = cadd<T>(v0, v2), t1 = csub<T>(v0, v2);
    cx<T> t2 = cadd<T>(v1, v3), t3 = rot_mi<T, INV>(csub<T>(v1, v3));
    v0 = cadd<T>(t0, t2);
    v2 = csub<T>(t0, t2);
    v1 = cadd<T>(t1, t3);
    v3 = csub<T>(t1, t3);
}

template <typename T, bool INV> __device__ __forceinline__ void dft3(cx<T>* v) {
    const T s = (T)0.86602540378443864676;  // sin(2 pi / 3)
    cx<T> t1 = cadd<T>(v[1], v[2]);
    cx<T> t2 = cscale<T>(csub<T>(v[1], v[2]), s);
    cx<T> m = mk<T>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
    v[0] = cadd<T>(v[0], t1);
    cx<T> it = rot_mi<T, INV>(t2);
    v[1] = cadd<T>(m, it);
    v[2] = csub<T>(m, it);
}

template <typename T, bool INV> __device__ __forceinline__ void dft5(cx<T>* v) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
    cx<T> t1 = cadd<T>(v[1], v[4]), t2 = cadd<T>(v[2], v[3]);
    cx<T> t3 = csub<T>(v[1], v[4]), t4 = csub<T>(v[2], v[3]);
    cx<T> a1 = mk<T>(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    cx<T> a2 = mk<T>(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    cx<T> b1 = rot_mi<T, INV>(mk<T>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    cx<T> b2 = rot_mi<T, INV>(mk<T>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    v[0] = mk<T>(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
    v[1] = cadd<T>(a1, b1);
    v[4] = csub<T>(a1, b1);
    v[2] = cadd<T>(a2, b2);
    v[3] = csub<T>(a2, b2);
}

// DFT of length 8 = 2 x 4: inner length-2 transforms over inputs 4 r1 + r2,
// twiddle w_8^{r2 q1}, outer length-4 transforms; output q1 + 2 q2.
template <typename T, bool INV> __device__ __forceinline__ void dft8(cx<T>* v) {
    cx<T> y[4][2];
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) {
        y[r2][0] = v[r2];
        y[r2][1] = v[r2 + 4];
        dft2<T, INV>(y[r2][0], y[r2][1]);
    }
    y[1][1] = twc<T, 8, 1, INV>(y[1][1]);
    y[2][1] = twc<T, 8, 2, INV>(y[2][1]);
    y[3][1] = twc<T, 8, 3, INV>(y[3][1]);
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1) {
        dft4<T, INV>(y[0][q1], y[1][q1], y[2][q1], y[3][q1]);
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) v[q1 + 2 * q2] = y[q2][q1];
    }
}

// DFT of length 16 = 4 x 4, same index map with twiddle w_16^{r2 q1}.
template <typename T, bool INV> __device__ __forceinline__ void dft16(cx<T>* v) {
    cx<T> y[4][4];
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) {
        y[r2][0] = v[r2];
        y[r2][1] = v[r2 + 4];
        y[r2][2] = v[r2 + 8];
        y[r2][3] = v[r2 + 12];
        dft4<T, INV>(y[r2][0], y[r2][1], y[r2][2], y[r2][3]);
    }
    y[1][1] = twc<T, 16, 1, INV>(y[1][1]);
    y[1][2] = twc<T, 16, 2, INV>(y[1][2]);
    y[1][3] = twc<T, 16, 3, INV>(y[1][3]);
    y[2][1] = twc<T, 16, 2, INV>(y[2][1]);
    y[2][2] = twc<T, 16, 4, INV>(y[2][2]);
    y[2][3] = twc<T, 16, 6, INV>(y[2][3]);
    y[3][1] = twc<T, 16, 3, INV>(y[3][1]);
    y[3][2] = twc<T, 16, 6, INV>(y[3][2]);
    y[3][3] = twc<T, 16, 9, INV>(y[3][3]);
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) {
        dft4<T, INV>(y[0][q1], y[1][q1], y[2][q1], y[3][q1]);
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) v[q1 + 4 * q2] = y[q2][q1];
    }
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dft_r(cx<T>* v) {
    if constexpr (R == 2) dft2<T, INV>(v[0], v[1]);
    else if constexpr (R == 3) dft3<T, INV>(v);
    else if constexpr (R == 4) dft4<T, INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) dft5<T, INV>(v);
    else if constexpr (R == 8) dft8<T, INV>(v);
    else dft16<T, INV>(v);
}

struct FftPlan {
    int n;          // transform length
    int nst;        // number of stages (0 for n == 1)
    int rmin;       // smallest radix; n / rmin threads serve one pencil
    int radix[8];   // radices in stage order
    unsigned code;  // the same radices, 4 bits per stage (the radix itself, 16 as 0)
};

// One Stockham stage on the pencil starting at sp (element stride es),
// butterfly j; both barriers are inside, so every thread of the CTA must call
// it.
template <typename T, int R, bool INV>
__device__ __forceinline__ void stage(cx<T>* sp, int j, bool live, int es, int n, int Ns, int tws,
                                      const cx<T>* __restrict__ tw) {
    const int nb = n / R;
    const bool act = live && j < nb;
    cx<T> v[R];
    int k = 0;
    if (act) {
        k = (Ns & (Ns - 1)) == 0 ? (j & (Ns - 1)) : j % Ns;
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sp[(j + r * nb) * es];
        if (Ns > 1) {
            const int step = k * tws;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const cx<T> w = __ldg(&tw[r * step]);
                v[r] = INV ? cmulc<T>(v[r], w) : cmul<T>(v[r], w);
            }
        }
        dft_r<T, R, INV>(v);
    }
    __syncthreads();
    if (act) {
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sp[(base + r * Ns) * es] = v[r];
    }
    __syncthreads();
}

// All stages of the plan on one pencil (butterfly j of every stage).
template <typename T, bool INV>
__device__ __forceinline__ void fft_stages(cx<T>* sp, int j, bool live, int es, const FftPlan& pl,
                                           const cx<T>* __restrict__ tw) {
    const int n = pl.n;
    // Ns: span of the finished sub-transforms; rem = n / Ns, so the twiddle
    // step n / (Ns R) is rem / R with R a compile-time constant
    int Ns = 1, rem = n;
    for (int st = 0; st < pl.nst; ++st) {
        const int c = (pl.code >> (4 * st)) & 15u;
        switch (c) {
            case 2: rem /= 2; stage<T, 2, INV>(sp, j, live, es, n, Ns, rem, tw); Ns *= 2; break;
            case 3: rem /= 3; stage<T, 3, INV>(sp, j, live, es, n, Ns, rem, tw); Ns *= 3; break;
            case 4: rem /= 4; stage<T, 4, INV>(sp, j, live, es, n, Ns, rem, tw); Ns *= 4; break;
            case 5: rem /= 5; stage<T, 5, INV>(sp, j, live, es, n, Ns, rem, tw); Ns *= 5; break;
            case 8: rem /= 8; stage<T, 8, INV>(sp, j, live, es, n, Ns, rem, tw); Ns *= 8; break;
            default: rem /= 16; stage<T, 16, INV>(sp, j, live, es, n, Ns, rem, tw); Ns *= 16; break;
        }
    }
}

// In-place transform of nP pencils held in shared memory.  Pencil
// q = maj * minor + m (0 <= m < minor) starts at s[maj * mstride + m] and its
// elements are es apart.  Threads take m fastest, then the butterfly index,
// then maj, so a warp sweeps contiguous rows.  tw holds exp(-2 pi i t / n),
// t = 0..n-1; the inverse uses its conjugate and is unnormalised.  Requires
// minor * (n / pl.rmin) <= blockDim.x.  Every thread of the CTA must call it.
template <typename T, bool INV>
__device__ __forceinline__ void fft_smem(cx<T>* s, int nP, int minor, int mstride, int es, const FftPlan& pl,
                                         const cx<T>* __restrict__ tw) {
    if (pl.nst == 0) return;
    const int tpp = pl.n / pl.rmin;
    const int span = minor * tpp;
    const int majg = blockDim.x / span;
    const int nmaj = (nP + minor - 1) / minor;
    const int tid = threadIdx.x;
    const int m = tid % minor;
    const int j = (tid / minor) % tpp;
    const int mo = tid / span;
    for (int g0 = 0; g0 < nmaj; g0 += majg) {
        const int maj = g0 + mo;
        const bool live = (mo < majg) && (maj * minor + m < nP);
        cx<T>* sp = s + (live ? maj * mstride + m : 0);
        fft_stages<T, INV>(sp, j, live, es, pl, tw);
    }
}

// ---------------------------------------------------------------------------
// Warp-local form for pencils served by at most 32 threads (n / rmin divides
// 32): the threads of one pencil sit in one warp, butterfly index fastest, so
// the stages need only __syncwarp.  Element i of a pencil is stored at
// padded position i + (i >> 4), which spreads a radix-8 or radix-16 first
// stage's strided stores over all banks.  Stage twiddles come from a table
// laid out per stage as [r - 1][k] (k = butterfly mod Ns fastest), so the
// lanes of a pencil read consecutive entries: exp(-2 pi i r k / (Ns R)),
// r = 1..R-1, k = 0..Ns-1, for every stage with Ns > 1, in plan order.
__device__ __forceinline__ int padded(int i) { return i + (i >> 4); }

template <typename T, int R, bool INV>
__device__ __forceinline__ void stage_wl(cx<T>* sp, int j, bool live, int es, int n, int Ns,
                                         const cx<T>* __restrict__ tws) {
    const int nb = n / R;
    const bool act = live && j < nb;
    cx<T> v[R];
    int k = 0;
    if (act) {
        k = (Ns & (Ns - 1)) == 0 ? (j & (Ns - 1)) : j % Ns;
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sp[padded(j + r * nb) * es];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const cx<T> w = __ldg(&tws[(r - 1) * Ns + k]);
                v[r] = INV ? cmulc<T>(v[r], w) : cmul<T>(v[r], w);
            }
        }
        dft_r<T, R, INV>(v);
    }
    __syncwarp();
    if (act) {
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sp[padded(base + r * Ns) * es] = v[r];
    }
    __syncwarp();
}

// In-place transform of nP pencils, pencil q at s[q], element i at
// s[padded(i) * es + q]; thread t serves pencils t / tpp + m * (blockDim.x /
// tpp), butterfly t % tpp.  Every thread of the CTA must call it; it ends with
// a CTA barrier, or (cta_end false) with a warp barrier only, for a caller
// that goes on with the same thread-to-pencil map.
template <typename T, bool INV>
__device__ __forceinline__ void fft_smem_wl(cx<T>* s, int nP, int es, const FftPlan& pl,
                                            const cx<T>* __restrict__ tws, bool cta_end = true) {
    if (pl.nst > 0) {
        const int n = pl.n;
        const int tpp = n / pl.rmin;
        const int ppr = blockDim.x / tpp;  // pencils per round
        const int j = threadIdx.x % tpp;
        const int qo = threadIdx.x / tpp;
        for (int q0 = 0; q0 < nP; q0 += ppr) {
            const int q = q0 + qo;
            const bool live = qo < ppr && q < nP;
            cx<T>* sp = s + (live ? q : 0);
            int Ns = 1;
            const cx<T>* t = tws;
            for (int st = 0; st < pl.nst; ++st) {
                const int c = (pl.code >> (4 * st)) & 15u;
                switch (c) {
                    case 2: stage_wl<T, 2, INV>(sp, j, live, es, n, Ns, t); t += Ns > 1 ? Ns : 0; Ns *= 2; break;
                    case 3: stage_wl<T, 3, INV>(sp, j, live, es, n, Ns, t); t += Ns > 1 ? 2 * Ns : 0; Ns *= 3; break;
                    case 4: stage_wl<T, 4, INV>(sp, j, live, es, n, Ns, t); t += Ns > 1 ? 3 * Ns : 0; Ns *= 4; break;
                    case 5: stage_wl<T, 5, INV>(sp, j, live, es, n, Ns, t); t += Ns > 1 ? 4 * Ns : 0; Ns *= 5; break;
                    case 8: stage_wl<T, 8, INV>(sp, j, live, es, n, Ns, t); t += Ns > 1 ? 7 * Ns : 0; Ns *= 8; break;
                    default: stage_wl<T, 16, INV>(sp, j, live, es, n, Ns, t); t += Ns > 1 ? 15 * Ns : 0; Ns *= 16; break;
                }
            }
        }
    }
    if (cta_end) __syncthreads();
}

}  // namespace pfk
