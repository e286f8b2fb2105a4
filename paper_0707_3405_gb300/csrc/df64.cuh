// Double-FP32 ("double-word") real scalar for the FP64-class dense algebra of
// the Rayleigh-Ritz step on a GPU whose FP64 units are few: a value is an
// unevaluated pair hi + lo of FP32 numbers with |lo| <= ulp(hi) / 2, which
// carries about 48 significant bits in the FP32 exponent range.
//
// Building blocks (the error-free transformations of floating-point
// arithmetic):
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, s = fl(a + b);
//   FastTwoSum (Dekker 1971): the same when |a| >= |b|, in three operations;
//   TwoProd through one FMA: p + e = a b exactly, p = fl(a b).
// Addition is the accurate double-word sum (both parts through TwoSum, two
// renormalisations), multiplication TwoProd plus the two cross terms,
// division three quotient digits from FP32 divisions with double-word
// remainders, square root one Newton correction of the FP32 root.  Relative
// error of each operation: a few units of 2^-48.  Every step uses the _rn
// intrinsics so that the compiler cannot contract or reorder it.
//
// The operators and math functions are hidden friends: they are found only
// for df64 arguments, so they never capture calls on double or float.
#pragma once

#include <cuda_runtime.h>

namespace lg {

struct alignas(8) df64 {
    float hi, lo;

    df64() = default;
    __host__ __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ df64(float f) : hi(f), lo(0.f) {}
    __host__ __device__ __forceinline__ df64(int i) : df64((double)i) {}
    __host__ __device__ __forceinline__ df64(unsigned int i) : df64((double)i) {}
    __host__ __device__ __forceinline__ df64(double d) {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }

    // ---- error-free transformations
    static __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
        s = __fadd_rn(a, b);
        const float bb = __fsub_rn(s, a);
        e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    }
    static __device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
        s = __fadd_rn(a, b);
        e = __fsub_rn(b, __fsub_rn(s, a));
    }
    static __device__ __forceinline__ df64 norm(float a, float b) {
        df64 r;
        fast_two_sum(a, b, r.hi, r.lo);
        return r;
    }

    // ---- arithmetic
    friend __device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
    friend __device__ __forceinline__ df64 operator+(df64 a, df64 b) {
        float s, e, t, f;
        two_sum(a.hi, b.hi, s, e);
        two_sum(a.lo, b.lo, t, f);
        e = __fadd_rn(e, t);
        fast_two_sum(s, e, s, e);
        e = __fadd_rn(e, f);
        return norm(s, e);
    }
    friend __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
    friend __device__ __forceinline__ df64 operator*(df64 a, df64 b) {
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
        return norm(p, e);
    }
    friend __device__ __forceinline__ df64 operator/(df64 a, df64 b) {
        const float q1 = __fdiv_rn(a.hi, b.hi);
        const df64 r = a - b * df64(q1);
        const float q2 = __fdiv_rn(r.hi, b.hi);
        const df64 r2 = r - b * df64(q2);
        const float q3 = __fdiv_rn(r2.hi, b.hi);
        const df64 q = norm(q1, q2);
        return q + df64(q3);
    }
    // a b + c with a single renormalisation (the accumulation form of the GEMM kernels)
    friend __device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
        float s, t;
        two_sum(c.hi, p, s, t);
        t = __fadd_rn(t, __fadd_rn(c.lo, e));
        return norm(s, t);
    }
    friend __device__ __forceinline__ df64 sqrt(df64 a) {
        if (!(a.hi > 0.f)) return df64(__fsqrt_rn(a.hi), 0.f);  // 0 -> 0, negative -> NaN
        const float s = __fsqrt_rn(a.hi);
        const float p = __fmul_rn(s, s);
        const float e = __fmaf_rn(s, s, -p);
        const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
        return norm(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
    }
    friend __device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
    friend __device__ __forceinline__ df64 copysign(df64 a, df64 b) {
        return (signbit(a.hi) != signbit(b.hi)) ? -a : a;
    }

    // ---- comparisons (normalised pairs compare lexicographically)
    friend __device__ __forceinline__ bool operator<(df64 a, df64 b) {
        return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
    }
    friend __device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
    friend __device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
    friend __device__ __forceinline__ bool operator>=(df64 a, df64 b) { return b <= a; }
    friend __device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
    friend __device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }
    friend __device__ __forceinline__ df64 fmax(df64 a, df64 b) { return (a < b) ? b : a; }
    friend __device__ __forceinline__ df64 fmin(df64 a, df64 b) { return (b < a) ? b : a; }

    friend __device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
    friend __device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
    friend __device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }
    friend __device__ __forceinline__ df64 &operator/=(df64 &a, df64 b) { return a = a / b; }

    // ---- warp exchange
    friend __device__ __forceinline__ df64 __shfl_xor_sync(unsigned mask, df64 v, int m) {
        return df64(__shfl_xor_sync(mask, v.hi, m), __shfl_xor_sync(mask, v.lo, m));
    }
    friend __device__ __forceinline__ df64 __shfl_sync(unsigned mask, df64 v, int src) {
        return df64(__shfl_sync(mask, v.hi, src), __shfl_sync(mask, v.lo, src));
    }
};

static_assert(sizeof(df64) == 8, "df64 is two floats");

// The same pair with the "sloppy" double-word sum (one TwoSum on the high parts, the low parts
// added, one renormalisation: 11 instead of 20 FP32 operations).  Its error is bounded by a few
// units of 2^-48 of |a| + |b| rather than of |a + b|: enough wherever the error analysis is
// norm-wise, as in the butterflies of an FFT, whose outputs carry errors relative to the
// transform's norm anyway.  Multiplication and the conversions are df64's.
struct alignas(8) df64f {
    float hi, lo;

    df64f() = default;
    __host__ __device__ __forceinline__ df64f(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ df64f(float f) : hi(f), lo(0.f) {}
    __host__ __device__ __forceinline__ df64f(int i) : df64f((double)i) {}
    __host__ __device__ __forceinline__ df64f(double d) {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }

    friend __device__ __forceinline__ df64f operator-(df64f a) { return df64f(-a.hi, -a.lo); }
    friend __device__ __forceinline__ df64f operator+(df64f a, df64f b) {
        float s, e;
        df64::two_sum(a.hi, b.hi, s, e);
        e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
        df64f r;
        df64::fast_two_sum(s, e, r.hi, r.lo);
        return r;
    }
    friend __device__ __forceinline__ df64f operator-(df64f a, df64f b) { return a + (-b); }
    friend __device__ __forceinline__ df64f operator*(df64f a, df64f b) {
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
        df64f r;
        df64::fast_two_sum(p, e, r.hi, r.lo);
        return r;
    }
    friend __device__ __forceinline__ df64f &operator+=(df64f &a, df64f b) { return a = a + b; }
    friend __device__ __forceinline__ df64f &operator-=(df64f &a, df64f b) { return a = a - b; }
    friend __device__ __forceinline__ df64f &operator*=(df64f &a, df64f b) { return a = a * b; }
};

static_assert(sizeof(df64f) == 8, "df64f is two floats");

}  // namespace lg
