// Double-word FP32 storage and arithmetic: a 64-bit format for GB300.
//
// On GB300 the FP64 pipe runs at a small fraction of the FP32 rate, which
// makes the FP64 step ALU-bound far below its HBM roofline (even converting
// FP64 loads to FP32 pairs saturates that pipe).  This format stores every
// population as a pair of FP32 numbers x = hi + lo (|lo| <= ulp(hi) / 2; 8
// bytes, like FP64) and evaluates the collision on such pairs, about 48
// significant bits, with FP32 instructions only.  The
// algorithms are the classical error-free transformations -- Knuth's TwoSum,
// Dekker's FastTwoSum and the FMA-based TwoProduct -- assembled as in Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic" (ACM TOMS 44(2), 2017): the "sloppy" sum
// (absolute error ~ 2^-48 (|x| + |y|), enough here because every sum of the
// collision is bounded by O(1) operands) and the double-word product.  The
// reciprocal is one Newton step from the FP32 reciprocal.
#pragma once
#include <cuda_runtime.h>

namespace trt {

struct df64 {
    float hi, lo;

    df64() = default;   // trivial, so that __shared__ arrays of pairs need no constructor
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ df64(int v) : hi((float)v), lo(0.f) {}
    // split of a double: hi = fl32(x), lo = fl32(x - hi); exact to ~2^-48 |x|
    __host__ __device__ df64(double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// The primitives use __fadd_rn / __fsub_rn / __fmul_rn, which the compiler
// never contracts into FMAs: the error-free transformations rely on every
// operation being rounded exactly once.

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// p + e = a * b exactly (FMA)
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ df64 operator+(const df64& x, const df64& y) {
    float sh, sl;
    two_sum(x.hi, y.hi, sh, sl);
    const float w = __fadd_rn(sl, __fadd_rn(x.lo, y.lo));
    df64 z;
    fast_two_sum(sh, w, z.hi, z.lo);
    return z;
}
__device__ __forceinline__ df64 operator-(const df64& x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(const df64& x, const df64& y) { return x + (-y); }
__device__ __forceinline__ df64 operator*(const df64& x, const df64& y) {
    float ch, cl;
    two_prod(x.hi, y.hi, ch, cl);
    const float t = fmaf(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
    df64 z;
    fast_two_sum(ch, __fadd_rn(cl, t), z.hi, z.lo);
    return z;
}
// 1 / y: FP32 reciprocal r, then r + r (1 - y r) in double-word arithmetic
__device__ __forceinline__ df64 recip(const df64& y) {
    const float r = __frcp_rn(y.hi);
    const df64 e = df64(1.0f, 0.0f) - y * df64(r, 0.0f);
    return df64(r, 0.0f) + df64(r, 0.0f) * e;
}
__device__ __forceinline__ df64 operator/(const df64& x, const df64& y) { return x * recip(y); }
__device__ __forceinline__ df64& operator+=(df64& x, const df64& y) { return x = x + y; }
__device__ __forceinline__ df64& operator-=(df64& x, const df64& y) { return x = x - y; }

// A double as a double-word pair without FP64 instructions, which GB300 runs
// at a small fraction of the FP32 rate: hi takes the top 24 significant bits
// of x and lo the next 23 (truncated, |x - hi - lo| < 2^-46 |x|), both by bit
// manipulation and one exact FP32 subtraction (2^e (1 + m 2^-23) - 2^e).
// Magnitudes outside [2^-103, 2^128) other than zero, where lo would leave
// the normal FP32 range, take the FP64 conversion of df64(double).
// The FP64 conversion as a call of its own, so that the compiler does not
// evaluate it alongside the bit manipulation and select (this is the rare
// path).
static __device__ __noinline__ df64 df64_of_double(double x) { return df64(x); }

__device__ __forceinline__ df64 df64_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    if ((b << 1) == 0ull) return df64(0.f, 0.f);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int dexp = (int)((hw >> 20) & 0x7ffu);
    if (dexp < 1023 - 103 || dexp > 1023 + 127) return df64_of_double(x);
    const unsigned sign = hw & 0x80000000u;
    const unsigned e = (unsigned)(dexp - 1023 + 127);              // biased FP32 exponent of x
    const unsigned mhi = ((hw & 0xfffffu) << 3) | (lw >> 29);      // mantissa bits 51..29
    const unsigned mlo = (lw >> 6) & 0x7fffffu;                    // mantissa bits 28..6
    const float hi = __uint_as_float(sign | (e << 23) | mhi);
    const float unit = __uint_as_float(sign | ((e - 23u) << 23));  // the last place of hi
    const float lo = __fsub_rn(__uint_as_float(sign | ((e - 23u) << 23) | mlo), unit);
    return df64(hi, lo);
}

// A float widened to double from its bits: exact, like the conversion, but
// without an FP64 instruction.  Subnormal, infinite and NaN inputs take the
// conversion (out of line, so that it is not evaluated alongside).
static __device__ __noinline__ double f64_of_float_slow(float x) { return (double)x; }
__device__ __forceinline__ double f64_of_float(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if (e == 0u && (b & 0x7fffffu) == 0u) return __longlong_as_double((long long)sign);   // +-0
    if (e == 0u || e == 0xffu) return f64_of_float_slow(x);
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}
// hi + lo in double: the same sum as (double)hi + (double)lo, one FP64 add.
__device__ __forceinline__ double dw_to_double(df64 v) { return f64_of_float(v.hi) + f64_of_float(v.lo); }

// storage tag: a double-word pair in memory (hi at the lower address)
struct __align__(8) f64dw {
    float hi, lo;
};

template <typename S> struct Fmt;
template <> struct Fmt<f64dw> {
    using C = df64;
    static __device__ __forceinline__ df64 ld(f64dw s) { return df64(s.hi, s.lo); }
    static __device__ __forceinline__ f64dw st(df64 c) { return f64dw{c.hi, c.lo}; }
};

}  // namespace trt
