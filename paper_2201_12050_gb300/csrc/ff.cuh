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

// ------------------------------------------------ float-float products ----
// GB300 runs FP64 at 1/58 of its FP32 rate, so the operator keeps its
// spectrum as float-float pairs (re_hi, re_lo, im_hi, im_lo): the same 16
// bytes per entry as complex double, hi + lo carrying 48 significand bits.
// Products use exact FP32 products (fma residual) and two-sum accumulation,
// giving FP64-level accuracy (about 2^-47 per product) on the FP32 pipe.
__device__ __forceinline__ float4 split_ff(double2 v) {
  const float rh = __double2float_rn(v.x);
  const float ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (sh, sl) += a * x for a, x float-float complex; re and im separately.
__device__ __forceinline__ void ff_cmac(const float4 a, const float4 x, float& rh, float& rl, float& ih, float& il) {
  // hi x hi products with their exact rounding errors
  const float p1 = __fmul_rn(a.x, x.x), e1 = fmaf(a.x, x.x, -p1);   // ar xr
  const float p2 = __fmul_rn(a.z, x.z), e2 = fmaf(a.z, x.z, -p2);   // ai xi
  const float p3 = __fmul_rn(a.x, x.z), e3 = fmaf(a.x, x.z, -p3);   // ar xi
  const float p4 = __fmul_rn(a.z, x.x), e4 = fmaf(a.z, x.x, -p4);   // ai xr
  // cross terms hi x lo + lo x hi
  const float cr = fmaf(a.x, x.y, fmaf(a.y, x.x, -fmaf(a.z, x.w, a.w * x.z)));
  const float ci = fmaf(a.x, x.w, fmaf(a.y, x.z, fmaf(a.z, x.y, a.w * x.x)));
  float d, ed, s, es;
  two_sum_f(p1, -p2, d, ed);
  two_sum_f(rh, d, s, es);
  rh = s;
  rl += (es + ed) + ((e1 - e2) + cr);
  two_sum_f(p3, p4, d, ed);
  two_sum_f(ih, d, s, es);
  ih = s;
  il += (es + ed) + ((e3 + e4) + ci);
}

// warp sum of a float-float value
__device__ __forceinline__ void ff_warp_sum(float& h, float& l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum_f(h, oh, s, e);
    h = s;
    l = __fadd_rn(__fadd_rn(l, ol), e);
  }
}

// Renormalise a float-float pair so that |lo| <= ulp(hi)/2.
__device__ __forceinline__ float4 ff_norm(float rh, float rl, float ih, float il) {
  const float a = __fadd_rn(rh, rl), b = __fadd_rn(ih, il);
  return make_float4(a, __fsub_rn(rl, __fsub_rn(a, rh)), b, __fsub_rn(il, __fsub_rn(b, ih)));
}

__device__ __forceinline__ double2 ff_to_cd(const float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

}  // namespace fmpb
