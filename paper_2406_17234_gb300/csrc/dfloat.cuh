// Float-float ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
// GB300 runs FP64 at about 1/64 of its FP32 rate, so the mixed mode keeps the
// quantities that need more than FP32 (S, J, the opacity and rate sums) in
// this form, on the FP32 pipe. The error-free transformations are the
// classical ones: Knuth's two-sum, Dekker's fast two-sum, and the product
// error from a fused multiply-add; the pair arithmetic follows the
// double-double algorithms of Hida, Li and Bailey (QD library paper, 2001),
// written here for float pairs. Every operation uses explicitly rounded
// intrinsics, so the compiler neither contracts nor reorders them.
#pragma once
#include <cuda_runtime.h>

namespace jfnk {

struct df {
  float hi, lo;
};

__host__ __device__ __forceinline__ df df_make(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

#ifdef __CUDACC__
// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}
// p + e = a b exactly (barring underflow)
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

__device__ __forceinline__ df df_add(df a, df b) {
  float e, f;
  const float s = two_sum(a.hi, b.hi, e);
  const float t = two_sum(a.lo, b.lo, f);
  e = __fadd_rn(e, t);
  float g;
  const float s2 = fast_two_sum(s, e, g);
  g = __fadd_rn(g, f);
  float h;
  const float hi = fast_two_sum(s2, g, h);
  return df_make(hi, h);
}
__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// a + b with a float b
__device__ __forceinline__ df df_add_f(df a, float b) {
  float e;
  const float s = two_sum(a.hi, b, e);
  e = __fadd_rn(e, a.lo);
  float h;
  const float hi = fast_two_sum(s, e, h);
  return df_make(hi, h);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  float e;
  const float p = two_prod(a.hi, b.hi, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float h;
  const float hi = fast_two_sum(p, e, h);
  return df_make(hi, h);
}
// a b with a float b
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float e;
  const float p = two_prod(a.hi, b, e);
  e = __fmaf_rn(a.lo, b, e);
  float h;
  const float hi = fast_two_sum(p, e, h);
  return df_make(hi, h);
}
// a + b for operands of the same sign (sums of positive terms): the cheaper
// "sloppy" addition, exact up to the pair's precision when nothing cancels
__device__ __forceinline__ df df_acc(df a, df b) {
  float e;
  const float s = two_sum(a.hi, b.hi, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float h;
  const float hi = fast_two_sum(s, e, h);
  return df_make(hi, h);
}
// a / b: the float quotient q1 from a hardware reciprocal of b.hi, then one
// correction q2 from the remainder a - q1 b (its leading part exact by
// Sterbenz's lemma): relative error about 2^-44, for b whose float parts are
// normal.
__device__ __forceinline__ df df_div(df a, df b) {
  float rb;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rb) : "f"(b.hi));
  const float q1 = __fmul_rn(a.hi, rb);
  float e;
  const float p = two_prod(q1, b.hi, e);
  float r = __fsub_rn(a.hi, p);
  r = __fsub_rn(r, e);
  r = __fadd_rn(r, a.lo);
  r = __fmaf_rn(-q1, b.lo, r);
  const float q2 = __fmul_rn(r, rb);
  float h;
  const float hi = fast_two_sum(q1, q2, h);
  return df_make(hi, h);
}
__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ df df_load(const float2* p, size_t i) {
  const float2 v = p[i];
  return df_make(v.x, v.y);
}
__device__ __forceinline__ void df_store(float2* p, size_t i, df a) { p[i] = make_float2(a.hi, a.lo); }
#endif

// Host and device: the pair nearest a double (hi its float rounding, lo the
// rounded remainder), and back.
__host__ __device__ __forceinline__ df df_from_double(double x) {
  const float hi = (float)x;
  return df_make(hi, (float)(x - (double)hi));
}
__host__ __device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace jfnk
