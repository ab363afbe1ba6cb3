// arith.cuh -- scalar and complex arithmetic for the three working precisions
// of the FFT-Newton path: FP64 (double), FP32 (float) and double-float (dd,
// an unevaluated sum hi + lo of two floats, ~48-bit significand).
//
// The double-float operations are built from the classical error-free
// transformations: Knuth's TwoSum (TAOCP vol. 2, 4.2.2), Dekker's
// FastTwoSum (Dekker 1971) and the FMA form of TwoProd (the exact product
// error is fma(a, b, -fl(a*b))).  Every step uses explicitly rounded
// intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn) so the compiler cannot contract
// or reassociate them.  Addition is the "sloppy" variant (one TwoSum on the
// high parts, low parts added once), whose error is a small multiple of
// 2^-46 (|x| + |y|): the normwise bound the FFT and matrix-product error
// analysis of Proposition 2.1 needs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct dd {
    float hi, lo;
};

template <class T>
struct __align__(2 * sizeof(T)) cx {
    T re, im;
};

__device__ __forceinline__ dd dd_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dd dd_fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ dd dd_add(dd x, dd y)
{
    dd s = dd_two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return dd_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

__device__ __forceinline__ dd dd_mul(dd x, dd y)
{
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return dd_fast_two_sum(p, e);
}

// x + y without the final normalisation: hi is the rounded sum of the high
// parts, lo collects their exact error and both low parts, and |lo| may
// exceed half an ulp of hi.  Chains of these inside one small DFT are
// normalised once at its end (dd_norm); every operation here accepts such
// unnormalised operands, and the error stays a small multiple of
// 2^-48 (|x| + |y|).
__device__ __forceinline__ dd dd_add_nn(dd x, dd y)
{
    const dd s = dd_two_sum(x.hi, y.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ dd dd_norm(dd x) { return dd_fast_two_sum(x.hi, x.lo); }

// a*b + c*d with one TwoSum: the two high products and their exact errors
// (FMA), the four cross terms folded into the low part, one normalisation
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d)
{
    const float p1 = __fmul_rn(a.hi, b.hi), p2 = __fmul_rn(c.hi, d.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p1);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float f = __fmaf_rn(c.hi, d.hi, -p2);
    f = __fmaf_rn(c.hi, d.lo, f);
    f = __fmaf_rn(c.lo, d.hi, f);
    const dd s = dd_two_sum(p1, p2);
    return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, f)));
}

// a*b + c with one normalisation
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    dd s = dd_two_sum(p, c.hi);
    float t = __fadd_rn(s.lo, __fadd_rn(e, c.lo));
    return dd_fast_two_sum(s.hi, t);
}

// ---------------------------------------------------------------------------
// Conversions between binary64 and the FP32-based formats done with integer
// operations on the two 32-bit halves, so they stay off the (narrow) FP64
// pipe.  Magnitudes below 2^-126 are flushed to a signed zero: every use here
// compares absolute errors far above that.

// binary64 -> nearest binary32 (ties to even).  Outside the normal binary32
// range: below it a signed zero, above it a signed infinity (NaN stays a
// quiet NaN) -- selected with integer operations too, so that no predicated
// FP64 instruction is left in the FFT kernels that call this per element.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sg = hw & 0x80000000u;
    const int ex = (int)((hw >> 20) & 0x7ffu);
    const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
    const unsigned rem = lw & 0x1fffffffu;
    const unsigned up = (rem + 0x0fffffffu + (m23 & 1u)) >> 29;  // round half to even: rem > 2^28, or = 2^28 and m23 odd
    unsigned fb = sg | ((((unsigned)(ex - 896)) << 23) + m23 + up);  // a carry may round up to infinity
    const unsigned big = sg | 0x7f800000u | ((ex == 2047 && ((hw & 0xfffffu) | lw)) ? 0x00400000u : 0u);
    fb = ex < 897 ? sg : fb;
    fb = ex > 1150 ? big : fb;
    return __uint_as_float(fb);
}

// binary64 -> double-float (hi = nearest binary32, lo = the rest rounded to
// binary32; lo flushes to zero below 2^-126), integer operations only.
__device__ __forceinline__ dd dd_from_double(double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sg = hw & 0x80000000u;
    const int ex = (int)((hw >> 20) & 0x7ffu);
    const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
    const unsigned rem = lw & 0x1fffffffu;
    const unsigned up = (rem + 0x0fffffffu + (m23 & 1u)) >> 29;  // round half to even: rem > 2^28, or = 2^28 and m23 odd
    unsigned fb = sg | ((((unsigned)(ex - 896)) << 23) + m23 + up);
    // x - hi = (rem - up 2^29) 2^(ex - 1075), with the sign of x
    const int r = (int)rem - (int)(up << 29);
    float lo = __int2float_rn(sg ? -r : r) * __uint_as_float(((unsigned)max(ex - 948, 1)) << 23);
    lo = (ex >= 949 && ex <= 1150) ? lo : 0.0f;
    const unsigned big = sg | 0x7f800000u | ((ex == 2047 && ((hw & 0xfffffu) | lw)) ? 0x00400000u : 0u);
    fb = ex < 897 ? sg : fb;
    fb = ex > 1150 ? big : fb;
    return {__uint_as_float(fb), lo};
}

// binary32 -> binary64, exact (binary32 subnormals flush to zero; infinities
// and NaNs keep their class), integer operations only
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e8 = (u >> 23) & 0xffu, sg = u & 0x80000000u, m = u & 0x7fffffu;
    const unsigned e11 = e8 == 0xffu ? 0x7ffu : e8 + 896u;
    unsigned hw = sg | (e11 << 20) | (m >> 3), lw = m << 29;
    hw = e8 == 0u ? sg : hw;
    lw = e8 == 0u ? 0u : lw;
    return __longlong_as_double(((long long)hw << 32) | lw);
}

// the sum of two exact binary64 conversions is exact (at most 48 significant
// bits): one FP64 add, used only where a double-float result is stored as FP64
__device__ __forceinline__ double dd_to_double(dd x) { return f32_to_f64(x.hi) + f32_to_f64(x.lo); }

// ---------------------------------------------------------------------------
// Real arithmetic traits.  scal(a, s) multiplies by a host scalar s that is a
// signed power of two (1/M, -1/M, 0.5): exact in every precision.
template <class T>
struct Ar;

template <>
struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double neg(double a) { return -a; }
    static __device__ __forceinline__ double scal(double a, double s) { return a * s; }
    static __device__ __forceinline__ double scal_f(double a, float s) { return a * (double)s; }
    static __device__ __forceinline__ double from_d(double x) { return x; }
    static __device__ __forceinline__ double to_d(double x) { return x; }
    static __device__ __forceinline__ double from_f(float x) { return f32_to_f64(x); }
    static __device__ __forceinline__ float to_f(double x) { return f64_to_f32_rn(x); }
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double one() { return 1.0; }
    static __device__ __forceinline__ double add_nn(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub_nn(double a, double b) { return a - b; }
    static __device__ __forceinline__ double norm(double a) { return a; }
    static __device__ __forceinline__ double rsqrt2() { return 0.70710678118654752440; }
};

template <>
struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
    static __device__ __forceinline__ float scal(float a, double s) { return a * (float)s; }
    static __device__ __forceinline__ float scal_f(float a, float s) { return a * s; }
    static __device__ __forceinline__ float from_d(double x) { return f64_to_f32_rn(x); }
    static __device__ __forceinline__ double to_d(float x) { return f32_to_f64(x); }
    static __device__ __forceinline__ float from_f(float x) { return x; }
    static __device__ __forceinline__ float to_f(float x) { return x; }
    static __device__ __forceinline__ float zero() { return 0.0f; }
    static __device__ __forceinline__ float one() { return 1.0f; }
    static __device__ __forceinline__ float add_nn(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub_nn(float a, float b) { return a - b; }
    static __device__ __forceinline__ float norm(float a) { return a; }
    static __device__ __forceinline__ float rsqrt2() { return 0x1.6a09e6p-1f; }
};

template <>
struct Ar<dd> {
    static __device__ __forceinline__ dd add(dd a, dd b) { return dd_add(a, b); }
    static __device__ __forceinline__ dd sub(dd a, dd b) { return dd_sub(a, b); }
    static __device__ __forceinline__ dd mul(dd a, dd b) { return dd_mul(a, b); }
    static __device__ __forceinline__ dd fma(dd a, dd b, dd c) { return dd_fma(a, b, c); }
    static __device__ __forceinline__ dd neg(dd a) { return dd_neg(a); }
    static __device__ __forceinline__ dd scal(dd a, double s)
    {
        float f = (float)s;
        return {a.hi * f, a.lo * f};
    }
    static __device__ __forceinline__ dd scal_f(dd a, float f) { return {a.hi * f, a.lo * f}; }
    static __device__ __forceinline__ dd from_d(double x) { return dd_from_double(x); }
    static __device__ __forceinline__ double to_d(dd x) { return dd_to_double(x); }
    static __device__ __forceinline__ dd from_f(float x) { return {x, 0.0f}; }
    static __device__ __forceinline__ float to_f(dd x) { return x.hi + x.lo; }
    static __device__ __forceinline__ dd zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ dd one() { return {1.0f, 0.0f}; }
    static __device__ __forceinline__ dd add_nn(dd a, dd b) { return dd_add_nn(a, b); }
    static __device__ __forceinline__ dd sub_nn(dd a, dd b) { return dd_add_nn(a, dd_neg(b)); }
    static __device__ __forceinline__ dd norm(dd a) { return dd_norm(a); }
    // sqrt(1/2) = hi + lo within 4e-16
    static __device__ __forceinline__ dd rsqrt2() { return {0x1.6a09e6p-1f, 0x1.9fcef4p-27f}; }
};

// ---------------------------------------------------------------------------
// Complex helpers
template <class T>
__device__ __forceinline__ cx<T> c_zero() { return {Ar<T>::zero(), Ar<T>::zero()}; }
template <class T>
__device__ __forceinline__ cx<T> c_add(cx<T> a, cx<T> b) { return {Ar<T>::add(a.re, b.re), Ar<T>::add(a.im, b.im)}; }
template <class T>
__device__ __forceinline__ cx<T> c_sub(cx<T> a, cx<T> b) { return {Ar<T>::sub(a.re, b.re), Ar<T>::sub(a.im, b.im)}; }
template <class T>
__device__ __forceinline__ cx<T> c_conj(cx<T> a) { return {a.re, Ar<T>::neg(a.im)}; }
template <class T>
__device__ __forceinline__ cx<T> c_neg(cx<T> a) { return {Ar<T>::neg(a.re), Ar<T>::neg(a.im)}; }
template <class T>
__device__ __forceinline__ cx<T> c_scal(cx<T> a, double s) { return {Ar<T>::scal(a.re, s), Ar<T>::scal(a.im, s)}; }
// a * b
template <class T>
__device__ __forceinline__ cx<T> c_mul(cx<T> a, cx<T> b)
{
    return {Ar<T>::fma(a.re, b.re, Ar<T>::neg(Ar<T>::mul(a.im, b.im))),
            Ar<T>::fma(a.re, b.im, Ar<T>::mul(a.im, b.re))};
}
// double-float a * b: each component one dot product with one normalisation
__device__ __forceinline__ cx<dd> c_mul(cx<dd> a, cx<dd> b)
{
    return {dd_dot2(a.re, b.re, dd_neg(a.im), b.im), dd_dot2(a.re, b.im, a.im, b.re)};
}
// sums without the final normalisation (see dd_add_nn) and the normalisation
template <class T>
__device__ __forceinline__ cx<T> c_add_nn(cx<T> a, cx<T> b) { return {Ar<T>::add_nn(a.re, b.re), Ar<T>::add_nn(a.im, b.im)}; }
template <class T>
__device__ __forceinline__ cx<T> c_sub_nn(cx<T> a, cx<T> b) { return {Ar<T>::sub_nn(a.re, b.re), Ar<T>::sub_nn(a.im, b.im)}; }
template <class T>
__device__ __forceinline__ cx<T> c_norm(cx<T> a) { return {Ar<T>::norm(a.re), Ar<T>::norm(a.im)}; }
// c += a * b
template <class T>
__device__ __forceinline__ void c_mac(cx<T> &c, cx<T> a, cx<T> b)
{
    c.re = Ar<T>::fma(a.re, b.re, c.re);
    c.re = Ar<T>::fma(Ar<T>::neg(a.im), b.im, c.re);
    c.im = Ar<T>::fma(a.re, b.im, c.im);
    c.im = Ar<T>::fma(a.im, b.re, c.im);
}
// i * a
template <class T>
__device__ __forceinline__ cx<T> c_mul_i(cx<T> a) { return {Ar<T>::neg(a.im), a.re}; }

template <class T>
__device__ __forceinline__ cx<T> c_from_d(double re, double im) { return {Ar<T>::from_d(re), Ar<T>::from_d(im)}; }
template <class T>
__device__ __forceinline__ cx<T> c_from_f(float re, float im) { return {Ar<T>::from_f(re), Ar<T>::from_f(im)}; }
