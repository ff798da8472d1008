// pf_pfa.cuh -- DFTs of length 6, 10 and 12 by the prime-factor
// (Good-Thomas) algorithm, for the compile-time-plan y and z passes whose
// lengths have factors 3 and 5 (96 = 16 x 6, 120 = 12 x 10, 160 = 16 x 10).
#pragma once
#include "pf_fft.cuh"

namespace pfk {

// a^-1 mod m for coprime a and m >= 2
__host__ __device__ constexpr int inv_mod(int a, int m, int x = 1) {
    return x >= m ? 1 : ((a * x) % m == 1 ? x : inv_mod(a, m, x + 1));
}

// DFT of length N = N1 N2, N1 and N2 coprime: input n = (N2 n1 + N1 n2) mod N,
// length-N2 transforms over n2, then length-N1 transforms over n1, output
// k = (N2 a k1 + N1 b k2) mod N with a = N2^-1 mod N1 and b = N1^-1 mod N2.
// By the Chinese remainder theorem these index maps take the place of the
// twiddle factors between the two transforms; all of them are compile-time.
template <typename T, int N1, int N2, bool INV> __device__ __forceinline__ void dft_pfa(cx<T>* v) {
    constexpr int N = N1 * N2;
    constexpr int A = inv_mod(N2 % N1, N1), B = inv_mod(N1 % N2, N2);
    cx<T> y[N1][N2];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) y[n1][n2] = v[(N2 * n1 + N1 * n2) % N];
        dft_r<T, N2, INV>(y[n1]);
    }
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
        cx<T> c[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) c[n1] = y[n1][k2];
        dft_r<T, N1, INV>(c);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[(N2 * A * k1 + N1 * B * k2) % N] = c[k1];
    }
}

// dft_r extended by the radices 6 = 2 x 3, 10 = 2 x 5 and 12 = 4 x 3
template <typename T, int R, bool INV> __device__ __forceinline__ void dft_any(cx<T>* v) {
    if constexpr (R == 6) dft_pfa<T, 2, 3, INV>(v);
    else if constexpr (R == 10) dft_pfa<T, 2, 5, INV>(v);
    else if constexpr (R == 12) dft_pfa<T, 4, 3, INV>(v);
    else dft_r<T, R, INV>(v);
}

}  // namespace pfk
