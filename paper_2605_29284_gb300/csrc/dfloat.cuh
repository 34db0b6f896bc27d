// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// floats (about 48 significant bits), built from error-free transformations:
// Knuth's TwoSum, Dekker's FastTwoSum (|a| >= |b|) and the FMA product
// error (a * b - fl(a * b) = fma(a, b, -fl(a * b)) exactly).  GB300 runs FP32
// at 64x its FP64 rate, so sums that need more than FP32 but not full FP64
// precision (the exact low-frequency block of the FP32 path, which only has
// to be far below the FP32 transform's rounding) are cheaper this way.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace rk {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_make(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}

// float -> double from the IEEE 754 encodings (binary32 -> binary64: the
// exponent rebiased by 1023 - 127, the significand moved up 52 - 23 bits):
// exact for normal floats; zeros and subnormals give a signed zero,
// infinities and NaNs keep their class.  Integer instructions only: the
// conversion instruction runs on GB300's FP64 pipe (1/64 of the FP32 rate).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned ed = e == 0u ? 0u : e == 0xffu ? 0x7ffu : e + 896u;
  const unsigned m = e == 0u ? 0u : (u & 0x7fffffu);
  const unsigned hi = (u & 0x80000000u) | (ed << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}

// hi + lo in double: one FP64 addition
__device__ __forceinline__ double df_double(dfl a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, e);
}

// a * b + c
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
  float s, e;
  two_sum(p, c.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  return fast_two_sum(s, e);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

// A sum of double-float products kept as an unnormalised pair: each term's
// exact high product joins s by TwoSum and everything else (the product's
// error and cross terms, TwoSum's error) collects in e; one FastTwoSum at
// the end.  12 instructions per term instead of df_fma's 15, for long dot
// products (e holds a few dozen terms' small parts without losing them).
struct dfacc {
  float s = 0.f, e = 0.f;
};

__device__ __forceinline__ void dfacc_fma(dfacc& c, dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
  float s, t;
  two_sum(c.s, p, s, t);
  c.s = s;
  c.e = __fadd_rn(c.e, __fadd_rn(t, pe));
}

__device__ __forceinline__ dfl dfacc_value(const dfacc& c) { return fast_two_sum(c.s, c.e); }

// a * b
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
  return fast_two_sum(p, pe);
}

// sqrt(a) for a >= 0: the rounded single-precision root s, then one Newton
// step s + (a - s^2) / (2 s) with a - s^2 formed exactly (s^2 = p + pe by the
// FMA product error; a.hi - p is exact by Sterbenz's lemma).
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float s = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -p);
  const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
  return fast_two_sum(s, __fmul_rn(res, __fdividef(0.5f, s)));
}

// e^{-d} for d >= 0 (0 beyond d = 80, below 2^-115): Cody and Waite's
// reduction d = k ln 2 + r, |r| <= ln(2) / 2 + rounding, so e^{-d} = 2^{-k}
// e^{-r}, and the Taylor series of e^{-r} to degree 12 (remainder below
// 0.35^13 / 13! < 2e-16) by Horner's rule: degrees 8-12, which stay below
// 6e-9, in single precision, degrees 0-7 in double-float.  The error stays
// within a few 1e-15 absolute (ln 2 held to about 2^-48 gives a relative
// error growing like 2^-48 k, on a value below 2^-k).
__device__ __forceinline__ dfl df_exp_neg(dfl d) {
  if (!(d.hi <= 80.f)) return {0.f, 0.f};
  constexpr double kLn2 = 0.69314718055994530942;
  constexpr float kLn2Hi = (float)kLn2;
  constexpr float kLn2Lo = (float)(kLn2 - (double)kLn2Hi);
  const float k = rintf(d.hi * 1.44269504f);
  const dfl r = df_fma({-k, 0.f}, {kLn2Hi, kLn2Lo}, d);
  const dfl nr = df_neg(r);
  float t = (float)(1.0 / 479001600.0);                        // 1 / 12!
  t = __fmaf_rn(t, nr.hi, (float)(1.0 / 39916800.0));
  t = __fmaf_rn(t, nr.hi, (float)(1.0 / 3628800.0));
  t = __fmaf_rn(t, nr.hi, (float)(1.0 / 362880.0));
  t = __fmaf_rn(t, nr.hi, (float)(1.0 / 40320.0));               // 1 / 8!
  constexpr double c[8] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720,
                           1.0 / 5040};
  dfl e = {t, 0.f};
#pragma unroll
  for (int j = 7; j >= 0; --j) {
    const float ch = (float)c[j];
    e = df_fma(e, nr, {ch, (float)(c[j] - (double)ch)});
  }
  const float sc = __int_as_float((127 - (int)k) << 23);         // 2^{-k}, k in [0, 116]
  return {e.hi * sc, e.lo * sc};
}

// Two unnormalised pair sums side by side, each component in one half of
// float2 registers, for the packed FP32 instructions: the operations of
// dfacc_fma on both components at once (12 instructions for the two).
// c_k += a_k b_k for k = 0, 1 with a = ahi + alo, b = bhi + blo componentwise
// and nahi = -ahi (formed once where a is reused): np = -fl(a b) exactly, the
// product error a b - fl(a b) = fma(ahi, bhi, np), the two-sum of c.s and
// -np, and the cross terms and errors into c.e.
struct dfacc2 {
  float2 s = {0.f, 0.f}, e = {0.f, 0.f};
};
__device__ __forceinline__ void dfacc2_fma(dfacc2& c, float2 ahi, float2 nahi, float2 alo,
                                           float2 bhi, float2 blo) {
  const float2 np = f2_mul(nahi, bhi);
  float2 pe = f2_fma(ahi, bhi, np);
  pe = f2_fma(alo, bhi, f2_fma(ahi, blo, pe));
  const float2 s = f2_sub(c.s, np);                  // c.s + p
  const float2 bb = f2_sub(s, c.s);
  const float2 t = f2_sub(f2_sub(c.s, f2_sub(s, bb)), f2_add(np, bb));   // two-sum error
  c.s = s;
  c.e = f2_add(c.e, f2_add(t, pe));
}
__device__ __forceinline__ dfl dfacc2_x(const dfacc2& c) { return fast_two_sum(c.s.x, c.e.x); }
__device__ __forceinline__ dfl dfacc2_y(const dfacc2& c) { return fast_two_sum(c.s.y, c.e.y); }

// complex double-float: (re.hi, re.lo, im.hi, im.lo) in a float4
__device__ __forceinline__ float4 cdf_pack(dfl re, dfl im) {
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}
// the same as packed pairs: (re.hi, im.hi, re.lo, im.lo), the hi and lo
// halves of a complex value each one float2 for the packed instructions
__device__ __forceinline__ float4 cdf_pack_pairs(dfl re, dfl im) {
  return make_float4(re.hi, im.hi, re.lo, im.lo);
}

}  // namespace rk
