// fastmath.cuh -- square root and reciprocal square root for the FP64 pipe-bound
// kernels of GB300, where FP64 runs at 1/64 of the FP32 rate.
//
// Every routine starts from the hardware single-precision reciprocal-square-
// root approximation (PTX rsqrt.approx.ftz.f32, on the SFU), reached through
// integer bit manipulation instead of FP64<->FP32 conversions.  rsqrt_nr
// finishes with one Newton-Raphson step in FP64,
//   y1 = y0 + y0 (1 - a y0^2) / 2                                   (3 FP64 ops)
// (with |y0 sqrt(a) - 1| = e <= ~2^-22 the result carries a relative error of
// O(e^2) ~ 1e-13, against ~10 FP64-pipe instructions for the correctly rounded
// library routine; arguments outside the single-precision exponent range go to
// the library); the double-float routines below keep even that step off the
// FP64 pipe.
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

// --------------------------------------------------------------------------
// Double-float arithmetic for the LD integrand and the renormalisation
//
// A value is carried as an unevaluated sum hi + lo of two floats (about 48
// significant bits; Dekker's double-length arithmetic).  The input double is
// split on the integer pipe, the square root takes one Newton (Heron) step from
// the SFU estimate in FP32, sums use Knuth's error-free two-sum (TAOCP vol. 2,
// Sec. 4.2.2), products the exact FMA product error (Muller et al., Handbook of
// Floating-Point Arithmetic, Sec. 4.4), and only the final widening back to a
// double uses the FP64 pipe (one addition).  Relative error of a square root
// ~2^-44, of a reciprocal square root ~2^-43.
// --------------------------------------------------------------------------

struct FF {
    float hi, lo;
};

// a >= 0 split into hi + lo (hi = a rounded to 24 bits, lo = the remainder
// rounded to 24 bits), on the integer pipe.  a < 2^-126 gives 0; the remainder
// is dropped for a < 2^-74 (relative error 2^-25 there); a non-finite a gives NaN.
__device__ __forceinline__ FF ff_split(double a)
{
    const long long A = __double_as_longlong(a);
    const int E = (int)(A >> 52);  // biased exponent (a >= 0)
    if (E < 1023 - 126) return FF{0.0f, 0.0f};
    if (E >= 1023 + 128) return FF{__int_as_float(0x7fc00000), 0.0f};
    const long long M = (A & ((1LL << 52) - 1)) | (1LL << 52);
    const long long Mh = (M + (1LL << 28)) >> 29;  // 24 bits (2^24 after a carry)
    const int D = (int)(M - (Mh << 29));           // |D| <= 2^28
    // hi = Mh 2^(E - 1023 - 23): the carry of Mh = 2^24 moves into the exponent field
    const float hi = __int_as_float(((E - (1023 - 127)) << 23) + (int)(Mh - (1LL << 23)));
    const int es = E - (1023 + 52 - 127);  // exponent field of 2^(E - 1075)
    const float lo = es >= 1 ? __int2float_rn(D) * __int_as_float(es << 23) : 0.0f;
    return FF{hi, lo};
}

// Exact widening of a finite float of either sign to double (integer pipe);
// zero and subnormal floats give 0.
__device__ __forceinline__ double f32_to_f64_signed(float f)
{
    const int b = __float_as_int(f);
    const int mag = b & 0x7fffffff;
    if (mag < 0x00800000) return 0.0;
    const int sgn = b & (int)0x80000000;
    return __hiloint2double(((mag >> 3) + kBiasShift) | sgn, b << 29);
}

__device__ __forceinline__ double ff_to_f64(FF a)
{
    return f32_to_f64_signed(a.hi) + f32_to_f64_signed(a.lo);
}

// sqrt(hi + lo) for hi >= 2^-126 (else 0): s0 = hi y with y ~ 1/sqrt(hi) from
// the SFU, then one Newton (Heron) step s0 + (a - s0^2) y / 2 with the residual
// formed exactly by an FMA.
__device__ __forceinline__ FF ff_sqrt(FF a)
{
    if (!(a.hi >= 1.17549435e-38f)) return FF{a.hi != a.hi ? a.hi : 0.0f, 0.0f};
    const float y = rsqrt_approx_f32(a.hi);
    const float s0 = a.hi * y;
    const float r = fmaf(-s0, s0, a.hi) + a.lo;
    return FF{s0, r * (0.5f * y)};
}

// acc += w (hi, lo) with w a power of two: two-sum of the high parts, the
// rounding error and the low parts into acc.lo.
__device__ __forceinline__ void ff_acc(FF& acc, FF x, float w)
{
    const float xh = w * x.hi;
    const float s = acc.hi + xh;
    const float bb = s - acc.hi;
    const float err = (acc.hi - (s - bb)) + (xh - bb);
    acc.hi = s;
    acc.lo = acc.lo + (err + w * x.lo);
}

// sum_i sqrt|f_i| in double-float.
template <int D>
__device__ __forceinline__ FF ff_sum_sqrt_abs(const double* f)
{
    FF acc{0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < D; ++i) ff_acc(acc, ff_sqrt(ff_split(fabs(f[i]))), 1.0f);
    return acc;
}

// 1 / sqrt(a) for a > 0 in the FP32 exponent range, relative error ~2^-43, with
// one FP64 addition: y ~ 1/sqrt(hi) from the SFU, e = 1 - a y^2 in double-float
// (hi y = p + p_lo exactly by an FMA), result y + y e / 2.  Falls back to the
// library rsqrt outside that range.
__device__ __forceinline__ double rsqrt_ff(double a)
{
    const int hi32 = __double2hiint(a);
    if (!in_f32_range(hi32) || hi32 >= ((1023 + 126) << 20)) return rsqrt(a);
    const FF x = ff_split(a);
    const float y = rsqrt_approx_f32(x.hi);
    const float p = x.hi * y;
    const float p_lo = fmaf(x.hi, y, -p);
    const float q = fmaf(-p, y, 1.0f);
    const float e = fmaf(-fmaf(x.lo, y, p_lo), y, q);
    return f32_to_f64_bits(y) + f32_to_f64_signed(0.5f * y * e);
}

}  // namespace chs
