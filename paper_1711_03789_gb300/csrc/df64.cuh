// Double-float arithmetic: a real number carried as an unevaluated sum hi + lo of two FP32
// values with |lo| <= ulp(hi) / 2 (about 48 significant bits), built from the error-free
// transformations of Knuth (two-sum), Dekker / FMA (two-product) and the compensated
// summation of Ogita, Rump and Oishi (2005). GB300 runs FP64 at 1/64 of the FP32 rate, so
// the Krylov kernels of the mixed form use this format where FP64 would otherwise be the
// bound. Every operation uses the _rn intrinsics so that no multiply-add contraction can
// change an error-free step.
//
// Storage of a complex double-float value: float4 {re_hi, im_hi, re_lo, im_lo}; the (x, y)
// half is the value rounded to c64.
#pragma once

#include <cuda_runtime.h>

namespace mx {
namespace df {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Compensated accumulator: the sum of the terms is s + e (e collects the rounding errors
// of the running sum and the low parts of the products).
struct Acc {
  float s = 0.f, e = 0.f;
};

// acc += (xh + xl) * u, u an FP32 value
__device__ __forceinline__ void add_prod(Acc& a, float xh, float xl, float u) {
  const float p = __fmul_rn(xh, u);
  float err = __fmaf_rn(xh, u, -p);
  err = __fmaf_rn(xl, u, err);
  float s, se;
  two_sum(a.s, p, s, se);
  a.s = s;
  a.e = __fadd_rn(a.e, __fadd_rn(se, err));
}

// acc += (xh + xl) * (yh + yl) (the xl * yl term is below the format's precision)
__device__ __forceinline__ void add_prod2(Acc& a, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float err = __fmaf_rn(xh, yh, -p);
  err = __fmaf_rn(xh, yl, err);
  err = __fmaf_rn(xl, yh, err);
  float s, se;
  two_sum(a.s, p, s, se);
  a.s = s;
  a.e = __fadd_rn(a.e, __fadd_rn(se, err));
}

// normalised (hi, lo) of an accumulator
__device__ __forceinline__ float2 value(const Acc& a) {
  float h, l;
  fast_two_sum(a.s, a.e, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ double to_double(const Acc& a) { return (double)a.s + (double)a.e; }

// (ah + al) - (bh + bl), normalised
__device__ __forceinline__ float2 sub(float ah, float al, float bh, float bl) {
  float s, e;
  two_sum(ah, -bh, s, e);
  e = __fadd_rn(e, __fsub_rn(al, bl));
  float h, l;
  fast_two_sum(s, e, h, l);
  return make_float2(h, l);
}

// (xh + xl) * (yh + yl), normalised
__device__ __forceinline__ float2 mul(float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float err = __fmaf_rn(xh, yh, -p);
  err = __fmaf_rn(xh, yl, err);
  err = __fmaf_rn(xl, yh, err);
  float h, l;
  fast_two_sum(p, err, h, l);
  return make_float2(h, l);
}

// split of an FP64 value (one FP64 subtraction)
__host__ __device__ inline float2 split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

__device__ __forceinline__ float4 split_c(double2 z) {
  const float2 a = split(z.x), b = split(z.y);
  return make_float4(a.x, b.x, a.y, b.y);
}

__device__ __forceinline__ double2 to_c128(float4 v) {
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

}  // namespace df
}  // namespace mx
