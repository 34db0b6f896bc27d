// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// floats (about 48 significant bits), built from error-free transformations:
// Knuth's TwoSum, Dekker's FastTwoSum (|a| >= |b|) and the FMA product
// error (a * b - fl(a * b) = fma(a, b, -fl(a * b)) exactly).  GB300 runs FP32
// at 64x its FP64 rate, so sums that need more than FP32 but not full FP64
// precision (the exact low-frequency block of the FP32 path, which only has
// to be far below the FP32 transform's rounding) are cheaper this way.
#pragma once

#include <cuda_runtime.h>

namespace rk {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_make(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}

__device__ __forceinline__ double df_double(dfl a) { return (double)a.hi + (double)a.lo; }

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

// complex double-float: (re.hi, re.lo, im.hi, im.lo) in a float4
__device__ __forceinline__ float4 cdf_pack(dfl re, dfl im) {
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

}  // namespace rk
