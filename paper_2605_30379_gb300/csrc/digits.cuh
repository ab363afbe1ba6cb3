// digits.cuh -- exact base-256 digit splitting of scaled FP32 and
// double-float values for the integer tensor-core products (ozaki.cu with
// mma.sync, ozaki_tc.cu with tcgen05), and the power-of-two helpers around it.
//
// A value v scaled so that |v| <= 1/2 is written as S balanced digits
// v ~ sum_s q_s 2^(8s - 8S), |q_s| <= 128, each exactly a BF16 integer; the
// product of two such values is then an exact sum of digit products
// q_s r_t 2^(8(s+t) - 16S), which the tensor cores form exactly in FP32
// (products <= 2^14).  Pairs with s + t < GMIN are dropped.  This is the
// error-free splitting idea of Ozaki et al. (2012).
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace mrc_digits {

// Digits per value and smallest digit-pair weight group kept, per precision:
// double-float 6 digits (48 bits), groups s + t >= 5; FP32 5 digits (40 bits
// relative to the row/column maximum), groups s + t >= 5.  Fewer FP32 digits
// are not enough: the level products cancel heavily (A*B = e0 + small), and
// with 3 or 4 digits the error relative to the row maximum left max|rho_L|
// at 1e-5 and 5e-10 after one refinement sweep at d = 33..64, against
// 3e-14 with 5 digits (8.7e-14 with FP32 SIMT products).
#ifndef MRC_OZ_F32_DIGITS
#define MRC_OZ_F32_DIGITS 5
#endif
// (Five double-float digits, 15 pairs, were measured: pairmul_dd 70 -> 62 ms
// at d = 64, N = 2^18, but the residual error rose from ~1e-13 to ~2e-11.)
#ifndef MRC_OZ_DD_DIGITS
#define MRC_OZ_DD_DIGITS 6
#endif
template <class T> struct OzP;
template <> struct OzP<dd> { static constexpr int S = MRC_OZ_DD_DIGITS, GMIN = MRC_OZ_DD_DIGITS - 1; };
template <> struct OzP<float> { static constexpr int S = MRC_OZ_F32_DIGITS, GMIN = MRC_OZ_F32_DIGITS; };
// Six balanced base-256 digits of v = hi + lo, |v| <= 1/2: digit s has weight
// 2^(8s-48) and |q_s| <= 128.  t = (x + C) - C with C = 1.5 * 2^k rounds x to
// the nearest multiple of 2^(k-23) (|x| <= 2^(k-1)) and x - t is exact.  lo
// joins after two digits through an exact TwoSum (y + e = rest + lo, |y| <=
// 2^-17 + 2^-26, |e| <= 2^-41); e joins after four digits, where the rest is
// <= 2^-33.  Each digit therefore stays within 128 (+ at most 1/2 before
// rounding to an integer).
__device__ __forceinline__ void digits6(float hi, float lo, float (&q)[6])
{
    float x = hi, t;
    t = __fsub_rn(__fadd_rn(x, 49152.0f), 49152.0f);            // grid 2^-8
    q[5] = t * 256.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 192.0f), 192.0f);                // grid 2^-16
    q[4] = t * 65536.0f;
    x = __fsub_rn(x, t);
    const dd ye = dd_two_sum(x, lo);                            // exact: x + lo = y + e
    x = ye.hi;
    t = __fsub_rn(__fadd_rn(x, 0.75f), 0.75f);                  // grid 2^-24
    q[3] = t * 16777216.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-9f), 0x1.8p-9f);          // grid 2^-32
    q[2] = t * 0x1p32f;
    x = __fadd_rn(__fsub_rn(x, t), ye.lo);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-17f), 0x1.8p-17f);        // grid 2^-40
    q[1] = t * 0x1p40f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-25f), 0x1.8p-25f);        // grid 2^-48
    q[0] = t * 0x1p48f;
}

// Three balanced base-256 digits of an FP32 value |x| <= 1/2 (weights 2^-8,
// 2^-16, 2^-24; the rest, below 2^-25, is dropped as FP32 rounding).
__device__ __forceinline__ void digits3(float x, float (&q)[3])
{
    float t;
    t = __fsub_rn(__fadd_rn(x, 49152.0f), 49152.0f);
    q[2] = t * 256.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 192.0f), 192.0f);
    q[1] = t * 65536.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 0.75f), 0.75f);
    q[0] = t * 16777216.0f;
}

__device__ __forceinline__ float hi_part(float x) { return x; }
__device__ __forceinline__ float hi_part(dd x) { return x.hi; }

__device__ __forceinline__ void split_digits(dd v, float sc, float (&q)[6]) { digits6(v.hi * sc, v.lo * sc, q); }

// Five digits of a double-float value (weights 2^-8 .. 2^-40), same folding
// of lo and of the TwoSum error as digits6.
__device__ __forceinline__ void split_digits(dd v, float sc, float (&q)[5])
{
    float x = v.hi * sc, t;
    t = __fsub_rn(__fadd_rn(x, 49152.0f), 49152.0f);
    q[4] = t * 256.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 192.0f), 192.0f);
    q[3] = t * 65536.0f;
    x = __fsub_rn(x, t);
    const dd ye = dd_two_sum(x, v.lo * sc);
    x = ye.hi;
    t = __fsub_rn(__fadd_rn(x, 0.75f), 0.75f);
    q[2] = t * 16777216.0f;
    x = __fsub_rn(x, t);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-9f), 0x1.8p-9f);
    q[1] = t * 0x1p32f;
    x = __fadd_rn(__fsub_rn(x, t), ye.lo);
    t = __fsub_rn(__fadd_rn(x, 0x1.8p-17f), 0x1.8p-17f);
    q[0] = t * 0x1p40f;
}
__device__ __forceinline__ void split_digits(float v, float sc, float (&q)[3]) { digits3(v * sc, q); }
__device__ __forceinline__ void split_digits(float v, float sc, float (&q)[5])
{
    float r[3];
    float x = v * sc;
    digits3(x, r);
    float rest = __fsub_rn(__fsub_rn(__fsub_rn(x, r[2] * 0x1p-8f), r[1] * 0x1p-16f), r[0] * 0x1p-24f);
    float t = __fsub_rn(__fadd_rn(rest, 0x1.8p-9f), 0x1.8p-9f);  // grid 2^-32
    q[1] = t * 0x1p32f;
    rest = __fsub_rn(rest, t);
    t = __fsub_rn(__fadd_rn(rest, 0x1.8p-17f), 0x1.8p-17f);      // grid 2^-40
    q[0] = t * 0x1p40f;
    q[2] = r[0];
    q[3] = r[1];
    q[4] = r[2];
}
__device__ __forceinline__ void split_digits(float v, float sc, float (&q)[4])
{
    float r[3];
    float x = v * sc;
    digits3(x, r);
    // fourth digit from the rest below 2^-24
    const float rest = __fsub_rn(__fsub_rn(__fsub_rn(x, r[2] * 0x1p-8f), r[1] * 0x1p-16f), r[0] * 0x1p-24f);
    const float t = __fsub_rn(__fadd_rn(rest, 0x1.8p-9f), 0x1.8p-9f);
    q[0] = t * 0x1p32f;
    q[1] = r[0];
    q[2] = r[1];
    q[3] = r[2];
}

__device__ __forceinline__ unsigned short bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// 2^e as a float for e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }

// multiply by 2^e with e possibly outside one float exponent's range
__device__ __forceinline__ float scale2(float x, int e)
{
    int e1 = e / 2, e2 = e - e1;
    e1 = max(-126, min(127, e1));
    e2 = max(-126, min(127, e2));
    return x * pow2f(e1) * pow2f(e2);
}

// exponent sigma with max|.| <= b < 2^(sigma - 1), i.e. scaled values <= 1/2
__device__ __forceinline__ int scale_exp(float b)
{
    if (!(b > 0x1p-120f)) return 0;  // zero (or negligible) row: all digits vanish
    int e;
    frexpf(b * (1.0f + 0x1p-20f), &e);  // b < 2^e
    return e + 1;
}

template <class T>
__device__ __forceinline__ T from_int(long long v, int ex);
template <>
__device__ __forceinline__ dd from_int<dd>(long long v, int ex)
{
    const float h = __ll2float_rn(v);
    const float l = __ll2float_rn(v - __float2ll_rn(h));
    return dd_fast_two_sum(scale2(h, ex), scale2(l, ex));
}
template <>
__device__ __forceinline__ float from_int<float>(long long v, int ex) { return scale2(__ll2float_rn(v), ex); }


} // namespace mrc_digits
