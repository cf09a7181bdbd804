// FP64 reciprocal and square root by one third-order correction of the hardware's
// single-precision estimates (PTX rcp.approx.ftz.f32 / rsqrt.approx.ftz.f32, relative
// error about 2^-23).  The FP64 unit is the scarce resource of the propagation kernel, so
// the range guard and the double <-> float conversions around the estimate are done on
// the integer pipe: the seed is taken from x with its mantissa truncated to 20 bits
// (relative error <= 2^-20, so seeds are good to about 2^-20), and one step of third
// order triples the correct bits (20 -> 60): three FP64 instructions for the reciprocal,
// five for the square root.  Results are within a few ulp of the IEEE operations
// (checked by pch_selftest_math).  Inputs outside [2^-99, 2^99) (where a
// single-precision seed could leave the normal range) use the IEEE operations instead.
#pragma once
#include <cuda_runtime.h>

namespace pch {

__device__ __forceinline__ float rcp_approx_f32(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_approx_f32(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 2^-99 <= |x| < 2^99, from the biased exponent field.
__device__ __forceinline__ bool nr_range(double x) {
    const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
    return e - (1023u - 99u) < 198u;
}
// 2^-99 <= x < 2^99 (the sign bit lands above the exponent field and fails the test).
__device__ __forceinline__ bool nr_range_pos(double x) {
    const unsigned e = (unsigned)__double2hiint(x) >> 20;
    return e - (1023u - 99u) < 198u;
}

// x in the guarded range as a float: exponent rebiased (1023 -> 127), mantissa cut to
// its top 20 bits.
__device__ __forceinline__ float narrow_seed(double x) {
    const unsigned hi = (unsigned)__double2hiint(x);
    return __uint_as_float((hi & 0x80000000u) | (((hi & 0x7fffffffu) - (896u << 20)) << 3));
}

// A normal float as the exactly equal double.
__device__ __forceinline__ double widen_normal(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(b << 29));
}

// 1 / x from the seed r (|1 - x r| <= about 2^-20): with e = 1 - x r, 1 / x = r / (1 - e)
// = r (1 + e + e^2 + ...); one step of third order (the Newton-Raphson iteration carried to
// the quadratic term of that series) leaves a truncation of about e^3 <= 2^-59.
__device__ __forceinline__ double rcp_nr(double x) {
    if (!nr_range(x)) return 1.0 / x;
    const double r = widen_normal(rcp_approx_f32(narrow_seed(x)));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// sqrt(x) from Goldschmidt's coupled start for the square root as given by P. Markstein,
// "Software Division and Square Root Using Goldschmidt's Algorithms" (Proc. 6th Conference
// on Real Numbers and Computers, 2004), and in his "IA-64 and Elementary Functions"
// (Prentice Hall, 2000): from the seed y ~ 1/sqrt(x), g = x y ~ sqrt(x) and h = y / 2 ~
// 1 / (2 sqrt(x)); with r = 1/2 - g h, (2 g h) = 1 - 2 r and sqrt(x) = g (1 - 2 r)^(-1/2)
// = g (1 + r + 3/2 r^2 + ...).  Carried to the quadratic term (one step of third order;
// Goldschmidt's own step stops at the linear term) the truncation is about 5/2 r^3 <=
// 2^-58, and the rounding of g cancels to first order in the correction.
__device__ __forceinline__ double sqrt_nr(double x) {
    if (!nr_range_pos(x)) return sqrt(x);
    const float y = rsqrt_approx_f32(narrow_seed(x));
    const double g = x * widen_normal(y);
    const double h = widen_normal(0.5f * y);
    const double r = fma(-g, h, 0.5);
    return fma(g, r * fma(1.5, r, 1.0), g);
}

}  // namespace pch
