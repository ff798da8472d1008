// pf_mma.cuh -- warp-level BF16 tensor-core products (mma.sync m16n8k16, FP32
// accumulation) and the exact split of FP32 values into BF16 terms.
//
// Fragment layouts of mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32
// (PTX ISA), with g = lane / 4 and t = lane % 4; each .b32 register holds two
// BF16 values, the lower index in the low half:
//   A (16 x 16, row-major): a0 = (g, 2t..2t+1), a1 = (g + 8, 2t..2t+1),
//                           a2 = (g, 2t+8..2t+9), a3 = (g + 8, 2t+8..2t+9)
//   B (16 x 8, column):     b0 = (2t..2t+1, g), b1 = (2t+8..2t+9, g)
//   C, D (16 x 8, FP32):    d0, d1 = (g, 2t..2t+1), d2, d3 = (g + 8, 2t..2t+1)
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pfk {

// d += A b
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two floats as a BF16 pair (x in the low half), rounded to nearest
__device__ __forceinline__ uint32_t bf16x2(float x, float y) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// x = h + m + l with BF16 terms, each the nearest BF16 to what the previous
// terms leave; three terms hold every bit of an FP32 significand, so the sum
// is x exactly (barring exponent underflow of the last term).
struct Split3 {
    float h, m, l;
};
__device__ __forceinline__ Split3 split3(float x) {
    Split3 s;
    s.h = __bfloat162float(__float2bfloat16_rn(x));
    const float r = x - s.h;  // exact
    s.m = __bfloat162float(__float2bfloat16_rn(r));
    s.l = r - s.m;            // exact; representable in BF16 up to rounding
    return s;
}

}  // namespace pfk
