// pf_dft32.cuh -- the length-32 DFT of the compile-time-plan y and z passes of
// 512 points (16 x 32): 32 = 2 x 16 with the index map of dft8 and dft16 in
// pf_fft.cuh (inner length-2 transforms over inputs 16 r1 + r2, twiddle
// w_32^(r2 q1), outer length-16 transforms, output q1 + 2 q2).
#pragma once
#include "pf_fft.cuh"

namespace pfk {

// cos(2 pi e / 32), e = 0..31, from the values at e = 0..8 (cos of multiples
// of pi / 16) by symmetry
__host__ __device__ constexpr double cos32(int e) {
    const double c[9] = {1.0,
                         0.98078528040323044913,
                         0.92387953251128675613,
                         0.83146961230254523708,
                         0.70710678118654752440,
                         0.55557023301960222474,
                         0.38268343236508977173,
                         0.19509032201612826785,
                         0.0};
    e &= 31;
    return e <= 8 ? c[e] : e <= 16 ? -c[16 - e] : e <= 24 ? -c[e - 16] : c[32 - e];
}
__host__ __device__ constexpr double sin32(int e) { return cos32((e + 24) & 31); }

// v * exp(-+ 2 pi i E / 32) for a compile-time E (forward multiplies by
// c - i s, inverse by c + i s)
template <typename T, int E, bool INV> __device__ __forceinline__ cx<T> tw32(cx<T> v) {
    constexpr int e = E & 31;
    if constexpr (e == 0) {
        return v;
    } else if constexpr (e % 2 == 0) {
        return twc<T, 16, e / 2, INV>(v);
    } else {
        const T c = (T)cos32(e), s = (T)sin32(e);
        return INV ? mk<T>(v.x * c - v.y * s, v.y * c + v.x * s) : mk<T>(v.x * c + v.y * s, v.y * c - v.x * s);
    }
}

template <typename T, bool INV> __device__ __forceinline__ void dft32(cx<T>* v) {
    cx<T> y[16][2];
#pragma unroll
    for (int r2 = 0; r2 < 16; ++r2) {
        y[r2][0] = v[r2];
        y[r2][1] = v[r2 + 16];
        dft2<T, INV>(y[r2][0], y[r2][1]);
    }
    y[1][1] = tw32<T, 1, INV>(y[1][1]);
    y[2][1] = tw32<T, 2, INV>(y[2][1]);
    y[3][1] = tw32<T, 3, INV>(y[3][1]);
    y[4][1] = tw32<T, 4, INV>(y[4][1]);
    y[5][1] = tw32<T, 5, INV>(y[5][1]);
    y[6][1] = tw32<T, 6, INV>(y[6][1]);
    y[7][1] = tw32<T, 7, INV>(y[7][1]);
    y[8][1] = tw32<T, 8, INV>(y[8][1]);
    y[9][1] = tw32<T, 9, INV>(y[9][1]);
    y[10][1] = tw32<T, 10, INV>(y[10][1]);
    y[11][1] = tw32<T, 11, INV>(y[11][1]);
    y[12][1] = tw32<T, 12, INV>(y[12][1]);
    y[13][1] = tw32<T, 13, INV>(y[13][1]);
    y[14][1] = tw32<T, 14, INV>(y[14][1]);
    y[15][1] = tw32<T, 15, INV>(y[15][1]);
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1) {
        cx<T> z[16];
#pragma unroll
        for (int r2 = 0; r2 < 16; ++r2) z[r2] = y[r2][q1];
        dft16<T, INV>(z);
#pragma unroll
        for (int q2 = 0; q2 < 16; ++q2) v[q1 + 2 * q2] = z[q2];
    }
}

}  // namespace pfk
