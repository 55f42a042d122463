// fastmath.cuh -- square root and reciprocal square root for the FP64 pipe-bound
// kernels of GB300, where FP64 runs at 1/64 of the FP32 rate.
//
// Both start from the hardware single-precision reciprocal-square-root
// approximation (PTX rsqrt.approx.ftz.f32, on the SFU), reach it through
// integer bit manipulation instead of FP64<->FP32 conversions, and finish with
// one Newton-Raphson step in FP64:
//   rsqrt:  y1 = y0 + y0 (1 - a y0^2) / 2                          (3 FP64 ops)
//   sqrt :  s0 = a y0,  s1 = s0 + (a - s0^2) y0 / 2   (Heron step)  (3 FP64 ops)
// With |y0 sqrt(a) - 1| = e <= ~2^-22 the refined results carry a relative
// error of O(e^2) ~ 1e-13, against ~10 FP64-pipe instructions for the correctly
// rounded library routines.  Arguments outside the single-precision exponent
// range go to the library routines (sqrt of a value below 2^-126 returns 0,
// an absolute error below 1.1e-19).
#pragma once

#include <stdint.h>

namespace chs {

// Offset between the FP64 and FP32 exponent biases (1023 - 127), in the position
// of the FP64 exponent field of the high word.
constexpr int kBiasShift = (1023 - 127) << 20;

__device__ __forceinline__ float rsqrt_approx_f32(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// For a positive normal double a with 2^-126 <= a < 2^128: the float whose bits
// are a's exponent (rebiased) and the top 23 mantissa bits (truncated).
__device__ __forceinline__ float f64_to_f32_trunc(int hi, int lo)
{
    return __int_as_float(((hi - kBiasShift) << 3) | (int)((unsigned)lo >> 29));
}

// Exact widening of a positive normal float to double, on the integer pipe.
__device__ __forceinline__ double f32_to_f64_bits(float f)
{
    const int b = __float_as_int(f);
    return __hiloint2double((b >> 3) + kBiasShift, b << 29);
}

// True when a is a positive normal double inside the FP32 exponent range.
__device__ __forceinline__ bool in_f32_range(int hi)
{
    return (unsigned)(hi - ((1023 - 126) << 20)) < (unsigned)(((1023 + 127) - (1023 - 126)) << 20);
}

// Round-to-nearest FP64 -> FP32 on the integer pipe (no FP64-pipe conversion):
// values below FLT_MIN flush to zero, values beyond FLT_MAX become infinity.
__device__ __forceinline__ float f32_from_f64(double a)
{
    const long long r = __double_as_longlong(a) + (1LL << 28);
    const int hi = (int)(r >> 32);
    const unsigned lo = (unsigned)r;
    const int sgn = hi & (int)0x80000000;
    const int ah = hi & 0x7fffffff;
    int fb = ((ah - kBiasShift) << 3) | (int)(lo >> 29);
    fb = ah < ((1023 - 126) << 20) ? 0 : fb;
    fb = ah >= ((1023 + 128) << 20) ? 0x7f800000 : fb;
    return __int_as_float(fb | sgn);
}

// sqrt(a) for a >= 0, relative error ~1e-13.
__device__ __forceinline__ double sqrt_nr(double a)
{
    const int hi = __double2hiint(a), lo = __double2loint(a);
    if (in_f32_range(hi)) {
        const float yf = rsqrt_approx_f32(f64_to_f32_trunc(hi, lo));
        const double y = f32_to_f64_bits(yf);
        const double hy = f32_to_f64_bits(0.5f * yf);
        const double s0 = a * y;
        const double r = fma(-s0, s0, a);
        return fma(r, hy, s0);
    }
    return hi < ((1023 - 126) << 20) ? 0.0 : sqrt(a);
}

// 1/sqrt(a) for a > 0, relative error ~1e-13.
__device__ __forceinline__ double rsqrt_nr(double a)
{
    const int hi = __double2hiint(a), lo = __double2loint(a);
    if (in_f32_range(hi)) {
        const float yf = rsqrt_approx_f32(f64_to_f32_trunc(hi, lo));
        const double y = f32_to_f64_bits(yf);
        const double hy = f32_to_f64_bits(0.5f * yf);
        const double t = a * y;
        const double e = fma(-t, y, 1.0);
        return fma(hy, e, y);
    }
    return rsqrt(a);
}

}  // namespace chs
