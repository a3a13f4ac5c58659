// Float-float ("double-word") arithmetic for the macroscopic quantities of
// the FP32 path: a value is hi + lo with |lo| <= ulp(hi)/2, about 48
// significant bits.  GB300 issues FP32 adds 60x faster than FP64 ones, so
// the density, the Poisson prefix sum and the moment combination use these
// error-free transformations instead of double.
//
// Algorithms: TwoSum (Knuth, TAOCP vol. 2), Fast2Sum (Dekker 1971), TwoProd
// by FMA, and the double-word sums/products of Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44(2), 2017 (Algorithms 6, 4 and 9).  Every step
// uses explicitly rounded intrinsics so that no contraction or
// reassociation can change them.
#pragma once
#include <cuda_runtime.h>

namespace mmk {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float x) { return {x, 0.0f}; }

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// double-word + double-word (accurate version)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  const float c = __fadd_rn(s.lo, t.hi);
  const ff v = fast_two_sum(s.hi, c);
  const float w = __fadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}

// double-word + float
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  const ff s = two_sum(a.hi, b);
  const float v = __fadd_rn(a.lo, s.lo);
  return fast_two_sum(s.hi, v);
}

// double-word + double-word, "sloppy" form (Dekker 1971): one TwoSum of the
// high parts, the low parts added in float.  Its error is bounded in
// absolute terms, about 2^-47 (|a| + |b|), not relative to the result: what
// a finite-difference stencil over values of similar size needs, at about
// half the cost of ff_add.
__device__ __forceinline__ ff ff_add_abs(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  const float w = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, w);
}
__device__ __forceinline__ ff ff_sub_abs(ff a, ff b) {
  const ff s = two_sum(a.hi, -b.hi);
  const float w = __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// double-word * float
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float ch = __fmul_rn(a.hi, b);
  float cl = __fmaf_rn(a.hi, b, -ch);
  cl = __fmaf_rn(a.lo, b, cl);
  return fast_two_sum(ch, cl);
}

// double-word * double-word
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float ch = __fmul_rn(a.hi, b.hi);
  float cl = __fmaf_rn(a.hi, b.hi, -ch);
  cl = __fmaf_rn(a.hi, b.lo, cl);
  cl = __fmaf_rn(a.lo, b.hi, cl);
  return fast_two_sum(ch, cl);
}

__device__ __forceinline__ double ff_to_double(ff a) {
  return (double)a.hi + (double)a.lo;
}

__device__ __forceinline__ ff ff_from_double(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return {hi, lo};
}

__device__ __forceinline__ ff ff_shfl_up(ff a, int d) {
  return {__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ ff ff_shfl_down(ff a, int d) {
  return {__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ ff ff_shfl_xor(ff a, int m) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}
__device__ __forceinline__ ff ff_shfl(ff a, int src) {
  return {__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
}

}  // namespace mmk
