// Device helpers shared by the CUDA-core kernels: float64 <-> float32
// conversions by integer operations, packed f32x2 FMAs and compensated sums.
#pragma once
#include <cuda_runtime.h>

namespace kx {

// Conversions between float64 and float32 with integer operations: on this
// GPU the hardware conversions run on the float64 pipe, which is slow enough
// that they, not memory, would bound the kernels that use them.  Finite values in the
// float32 normal range convert as IEEE rounding would, up to the tie rule
// (half-ulp ties round away from zero); magnitudes below 2^-126 become zero
// or a float32 subnormal below 2^-146, magnitudes beyond the float32 range a
// non-finite value.
__device__ __forceinline__ float f64_to_f32(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned lo = (unsigned)u;
    unsigned hi = (unsigned)(u >> 32);
    const unsigned lo_r = lo + 0x10000000u;  // half of the last kept mantissa bit
    hi += (lo_r < lo) ? 1u : 0u;             // its carry
    // float64 exponent 896 + e is float32 exponent e: clamp to 0 .. 255, rebias
    const unsigned ax = min(max(hi & 0x7fffffffu, 896u << 20), 1151u << 20) - (896u << 20);
    return __uint_as_float((hi & 0x80000000u) | (ax << 3) | (lo_r >> 29));
}

__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sgn = b & 0x80000000u, ax = b & 0x7fffffffu;
    unsigned hi = sgn, lo = 0u;
    if (ax >= 0x7f800000u) {
        hi = sgn | 0x7ff00000u;
    } else if (ax >= 0x00800000u) {
        hi = sgn | ((ax >> 3) + (896u << 20));
        lo = ax << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// s += a * b on both lanes of a float pair, one packed instruction.
__device__ __forceinline__ void fma2(float2 &s, float2 a, float2 b) {
    unsigned long long rs = *reinterpret_cast<unsigned long long *>(&s);
    asm("fma.rn.f32x2 %0, %1, %2, %0;"
        : "+l"(rs)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    s = *reinterpret_cast<float2 *>(&rs);
}

// (hi, lo) += v with the rounding error of the float32 addition kept in lo.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v) {
    const float t = hi + v;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (v - bp);
    hi = t;
}

}  // namespace kx
