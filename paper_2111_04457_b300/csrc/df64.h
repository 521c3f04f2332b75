// Double-float ("df64") arithmetic: a real number as an unevaluated sum
// hi + lo of two FP32 values (|lo| <= ulp(hi)/2), about 48 significant bits.
// B300's FP64 pipe runs at ~1.1 TFLOP/s while its FP32 pipe runs at ~70, so
// operator applications that need close-to-FP64 accuracy but not FP64
// exactness (the intermediate defects of the FP64 outer loop) run faster in
// this form on the FP32 pipe.
//
// Building blocks are the error-free transformations of Knuth (TwoSum) and
// Dekker (FastTwoSum), with the product error taken from a fused multiply-add
// (TwoProd).  Addition is the cheaper variant that adds the two low parts into
// the error term (relative error ~2^-44 of the larger operand) and does not
// renormalise (see operator+), which is ample for defects down to 1e-12.
#pragma once

#include <cuda_runtime.h>

namespace bpp {

// The FP64 route of the split for magnitudes outside 2^-74 .. 2^100, kept
// out of line so that the compiler does not if-convert it into every split
// (its FP64 conversions would then occupy the slow FP64 pipe for all values).
static __device__ __noinline__ void split_rare(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

struct df64 {
    float hi, lo;
    __host__ __device__ df64() {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ df64(int v) : hi((float)v), lo(0.f) {}
    // Split of an FP64 value with integer operations (the FP64 pipe is slow on
    // this GPU): hi = v truncated to 24 significant bits (exact in FP32), lo =
    // the remaining 29 bits rounded once to FP32, so hi + lo = v to 2^-48.
    // Zero, and magnitudes outside 2^-74 .. 2^100 (where 2^(e - 1075) would not
    // be a normal FP32 number), take the FP64 route.
    __device__ explicit df64(double v) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const int e = (int)((b >> 52) & 0x7FF);
        if ((b << 1) == 0ULL) {
            hi = lo = __uint_as_float((unsigned)(b >> 32));   // +-0
        } else if (e < 949 || e > 1023 + 100) {
            split_rare(v, hi, lo);
        } else {
            const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
            hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
            const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);   // 2^(e - 1075)
            const float l = __uint2float_rn((unsigned)(b & 0x1FFFFFFFu)) * scale;
            lo = sign ? -l : l;
        }
    }
    __device__ double to_double() const { return f2d(hi) + f2d(lo); }
    // FP32 -> FP64 is exact; the FP64 pattern is built with integer
    // operations only (the FP64 pipe then carries just the one add of
    // to_double): normal numbers rebias the exponent (+1023 - 127) and shift
    // the significand up by 29 bits; subnormals are normalised with a count
    // of leading zeros; zero keeps its sign; infinities and NaN get the
    // all-ones exponent.  Branch-free (selects), so no FP64 conversion is
    // issued on any path.
    static __device__ __forceinline__ double f2d(float f) {
        const unsigned u = __float_as_uint(f);
        const unsigned e = (u >> 23) & 0xFFu;
        const unsigned m = u & 0x7FFFFFu;
        const int lz = __clz(m) - 8;   // subnormal: shift bringing the leading one to bit 23
        const unsigned mn = e == 0u ? ((m << lz) & 0x7FFFFFu) : m;
        const unsigned en = e == 0u ? (m == 0u ? 0u : (unsigned)(897 - lz)) : (e == 0xFFu ? 2047u : e + 896u);
        const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                     ((unsigned long long)en << 52) | ((unsigned long long)mn << 29);
        return __longlong_as_double((long long)d);
    }
};

__device__ __forceinline__ df64 quick_two_sum(float a, float b) {
    const float s = a + b;
    return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return df64(s, (a - (s - bb)) + (b - bb));
}

// Addition leaves the result unnormalised: (TwoSum of the high parts, its
// error plus both low parts).  hi + lo is the sum to ~2^-48 as before; |lo| may
// exceed half an ulp of hi, which products (TwoProd with both cross terms) and
// further additions tolerate.  Products, fma and stores renormalise.
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    const df64 s = two_sum(a.hi, b.hi);
    return df64(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df64 normalized(df64 a) { return quick_two_sum(a.hi, a.lo); }

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}

// Exact-match overloads so that unqualified fma() inside this namespace keeps
// resolving to the hardware FMA for float and double arguments.
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }

// a * b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const df64 s = two_sum(p, c.hi);
    return quick_two_sum(s.hi, s.lo + (e + c.lo));
}

}  // namespace bpp
