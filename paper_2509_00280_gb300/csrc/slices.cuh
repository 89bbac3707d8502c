// slices.cuh -- exact signed 7-bit integer slices of FP64 values on a
// power-of-two scale, the operands of the sliced tensor-core kernels
// (gram_oz.cu, solve_oz.cu).
//
// On the scale of an exponent field E (the largest field of the row or
// column the value belongs to), x = q 2^(E - 1077) with |q| < 2^55, q
// truncated toward zero; |q| = sum_{k<8} d_k 2^(7 (7 - k)), d_k in [0, 127],
// and slice k is sign(x) d_k, an integer that BF16 represents exactly.
#pragma once
#include <cstdint>

namespace relate {
namespace sl {

// Exponent field of x (0: zero or subnormal, 0x7ff: Inf or NaN).
__device__ __forceinline__ int expo_of(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }

// The 8 slices of x on the scale of E (E >= the field of x) as BF16 bit
// patterns, slice 0 the most significant. Subnormal x counts as 0.
__device__ __forceinline__ void slices8(double x, int E, uint32_t (&u)[8]) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    uint64_t q = 0;
    if (e != 0) {
        const uint64_t mant = (b & 0xfffffffffffffull) | (1ull << 52);
        const int sh = max(E - e - 2, -2);  // e <= E: |q| < 2^55
        q = sh >= 0 ? (sh < 64 ? mant >> sh : 0ull) : mant << (-sh);
    }
    // two 28-bit halves: slices 0..3 from the high one, 4..7 from the low one
    const uint32_t hi = (uint32_t)(q >> 28), lo = (uint32_t)q & 0x0fffffffu;
    const uint32_t sg = (uint32_t)(b >> 63) << 15;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const uint32_t d = ((k < 4 ? hi : lo) >> (7 * (3 - (k & 3)))) & 127u;
        const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;  // d exactly, as FP32
        u[k] = (__float_as_uint(f) >> 16) | sg;                          // its top half: the BF16 pattern
    }
}

// Exact 64-bit word of four group sums a_0..a_3 (|a| < 2^23, integers held
// in FP32): sum_j a_j 2^(7 (3 - j)), formed as two 32-bit pairs.
__device__ __forceinline__ long long word4(float a0, float a1, float a2, float a3) {
    const int p01 = __float2int_rn(a0) * 128 + __float2int_rn(a1);  // |p| < 2^31
    const int p23 = __float2int_rn(a2) * 128 + __float2int_rn(a3);
    return (long long)p01 * 16384 + p23;
}

}  // namespace sl
}  // namespace relate
