// Float-float ("double-single") arithmetic on the FP32 pipe.
//
// GB300 runs FP64 at 1/58 of its FP32 rate, so FP64-accurate inner loops are
// written with unevaluated sums hi + lo of two FP32 numbers (48 significand
// bits), built from the error-free transformations of Dekker (1971) and Knuth
// (TAOCP vol. 2): two-sum for additions and the fma residual for products.
// Every rounding step that an error term depends on goes through __fadd_rn /
// __fmul_rn, which the compiler never contracts into an FMA.
#pragma once
#include <cuda_runtime.h>

namespace fmpb {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_make(float h) { return {h, 0.f}; }

// exact conversions at the FP64 boundary
__device__ __forceinline__ ff ff_from_d(double a) {
  const float h = __double2float_rn(a);
  return {h, __double2float_rn(a - (double)h)};
}
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return quick_two_sum(s, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);                 // exact residual of the product
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return quick_two_sum(p, e);
}
// a * b with b a plain float
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.h, b);
  const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
  return quick_two_sum(p, e);
}

// a / b: approximate quotient, one residual correction
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = __fdividef(a.h, b.h);
  const ff r = ff_sub(a, ff_mul_f(b, q1));
  const float q2 = __fdividef(r.h, b.h);
  return quick_two_sum(q1, q2);
}
__device__ __forceinline__ ff ff_rcp(ff b) { return ff_div(ff_make(1.f), b); }

// sqrt(a), a > 0: FP32 root, one Newton correction y + (a - y^2) / (2y)
__device__ __forceinline__ ff ff_sqrt(ff a) {
  const float y = sqrtf(a.h);
  const float p = __fmul_rn(y, y);
  const float e = fmaf(y, y, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), e), a.l);
  return quick_two_sum(y, __fdividef(r, 2.f * y));
}

// complex float-float
struct ffc {
  ff re, im;
};
__device__ __forceinline__ ffc ffc_mul(ffc a, ffc b) {
  return {ff_sub(ff_mul(a.re, b.re), ff_mul(a.im, b.im)), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}

}  // namespace fmpb
