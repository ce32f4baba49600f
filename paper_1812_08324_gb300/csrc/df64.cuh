// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats (|lo| <= ulp(hi)/2), about 48 significant bits.  Built from the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2,
// 4.2.2): two-sum, fast-two-sum and the FMA two-product.  Every operation
// uses the __f*_rn intrinsics so that the compiler never contracts or
// reorders the steps the error terms depend on.
//
// On this GPU an FP32 instruction issues every cycle per SM sub-partition
// (latency 4 cycles) while an FP64 instruction occupies it for 64 cycles, so
// serial small dense factorizations run several times faster in double-float
// than in FP64.
#pragma once

#include <cuda_runtime.h>

namespace hm {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dfl df_from(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}

__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = df_two_sum(a.hi, b.hi);
  const dfl t = df_two_sum(a.lo, b.lo);
  s = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);          // exact error of the product of the high parts
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// c - a b and c + a b
__device__ __forceinline__ dfl df_fms(dfl c, dfl a, dfl b) { return df_sub(c, df_mul(a, b)); }
__device__ __forceinline__ dfl df_fma(dfl c, dfl a, dfl b) { return df_add(c, df_mul(a, b)); }

// a / b: float quotient, then one correction from the double-float remainder
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfl r = df_sub(a, df_mul({q1, 0.f}, b));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return df_fast_two_sum(q1, q2);
}

// sqrt(a), a >= 0: float root, then one Newton correction (a - x^2) / (2x)
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float x = __fsqrt_rn(a.hi);
  const dfl r = df_sub(a, df_mul({x, 0.f}, {x, 0.f}));
  return df_fast_two_sum(x, __fdiv_rn(r.hi, __fmul_rn(2.f, x)));
}

__device__ __forceinline__ dfl df_mul2(dfl a, float k) {  // a * k for k a power of two
  return {__fmul_rn(a.hi, k), __fmul_rn(a.lo, k)};
}

}  // namespace hm
