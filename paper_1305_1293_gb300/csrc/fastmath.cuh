// FP64 reciprocal and square root by Newton-Raphson iteration from the hardware's
// single-precision estimates (PTX rcp.approx.ftz.f32 / rsqrt.approx.ftz.f32, relative
// error about 2^-23).  Each step roughly doubles the correct bits (23 -> 46 -> 92), so two
// steps reach the limit of FP64 rounding; results are within a few ulp of the IEEE
// operations (checked by pch_selftest_math).  Inputs outside [1e-30, 1e30] (where the
// single-precision seed would underflow or overflow) use the IEEE operations instead.
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

// 1 / x: r <- r + r (1 - x r), twice.
__device__ __forceinline__ double rcp_nr(double x) {
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    double r = (double)rcp_approx_f32((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// sqrt(x) for x > 0: y ~ 1/sqrt(x) refined by y <- y (3/2 - x y^2 / 2) twice, then
// s = x y and one correction s + (x - s^2) y / 2.
__device__ __forceinline__ double sqrt_nr(double x) {
    if (!(x > 1e-30 && x < 1e30)) return sqrt(x);
    double y = (double)rsqrt_approx_f32((float)x);
    const double h = 0.5 * x;
    y = y * fma(-h * y, y, 1.5);
    y = y * fma(-h * y, y, 1.5);
    const double s = x * y;
    return fma(fma(-s, s, x), 0.5 * y, s);
}

}  // namespace pch
