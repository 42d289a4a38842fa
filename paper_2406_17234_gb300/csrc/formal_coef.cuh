// Shared pieces of the formal-solution kernels: the evaluation mode of a
// column and the piecewise-linear coefficients of App. A.1 in the form the
// difference recurrences use.
#pragma once

#include "internal.cuh"

namespace jfnk {

__device__ __forceinline__ int eval_mode_f(const ColDesc& cd) {
  if (cd.forced_mode >= 0) return cd.forced_mode;
  switch (cd.w.st->phase) {
    case PH_BASE: return EV_BASE;
    case PH_JVP:
    case PH_RESTART: return cd.w.st->fd_scheme ? EV_FD : EV_TANGENT;
    case PH_RH92: return EV_RH92;
    default: return EV_SKIP;
  }
}

// Coefficients of one step of optical depth x: e = exp(-x), w = (1 - e)/x,
// a = 1 - w and bq = (w - e)/x, each from its own Taylor series below
// x = 0.1 (where 1 - e, 1 - w and w - e cancel); r = 1/x is supplied by the
// caller (shared between the rays of a layer).
// FP64 Taylor coefficients: w = sum_{n>=0} (-x)^n/(n+1)!,
// a/x = sum_{n>=0} (-x)^n/(n+2)!, bq = sum_{n>=0} (-x)^n (n+1)/(n+2)!.
__device__ __forceinline__ void pl_series64(double x, double& w, double& a, double& bq) {
  // terms up to n = 5: below x = 1e-3 the first omitted one is < 3e-23 relative
  constexpr double f[8] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040};
  double pw = 0.0, pa = 0.0, pb = 0.0;
#pragma unroll
  for (int m = 5; m >= 0; --m) {
    const double sg = (m & 1) ? -1.0 : 1.0;
    pw = fma(pw, x, sg * f[m + 1]);
    pa = fma(pa, x, sg * f[m + 2]);
    pb = fma(pb, x, sg * (m + 1) * f[m + 2]);
  }
  w = pw;
  a = pa * x;
  bq = pb;
}

// In FP64 the direct forms of w, a and bq lose about 1e-16/x^2 relative
// (1 - e, 1 - w and w - e cancel): 2e-10 at x = 1e-3, so the series takes
// over below x = 1e-3 only.
// exp(-x) in FP64 by the table-driven method of P. T. P. Tang (ACM Trans.
// Math. Softw. 15, 1989): x 32/ln2 = k + f with k the nearest integer,
// r = x - k ln2/32 (Cody-Waite: ln2/32 = L1 + L2 with L1 of 32 significant
// bits, so that k L1 is exact), exp(-x) = 2^-m 2^(-j/32) exp(-r) for
// k = 32 m + j, with 2^(-j/32) tabulated (the values below are those powers
// correctly rounded) and exp(-r), |r| <= ln2/64, from its Taylor polynomial of
// degree 6 (truncation below 4e-18): 11 FP64 operations, the power of two by
// integer arithmetic on the exponent. Within about 2 ulp (tested against the
// IEEE value); 0 above x = 700 (exp(-700) ~ 1e-304); NaN stays NaN.
static __device__ const double kExpTab[32] = {
    0x1.0000000000000p+0, 0x1.f50765b6e4540p-1, 0x1.ea4afa2a490dap-1, 0x1.dfc97337b9b5fp-1,
    0x1.d5818dcfba487p-1, 0x1.cb720dcef9069p-1, 0x1.c199bdd85529cp-1, 0x1.b7f76f2fb5e47p-1,
    0x1.ae89f995ad3adp-1, 0x1.a5503b23e255dp-1, 0x1.9c49182a3f090p-1, 0x1.93737b0cdc5e5p-1,
    0x1.8ace5422aa0dbp-1, 0x1.82589994cce13p-1, 0x1.7a11473eb0187p-1, 0x1.71f75e8ec5f74p-1,
    0x1.6a09e667f3bcdp-1, 0x1.6247eb03a5585p-1, 0x1.5ab07dd485429p-1, 0x1.5342b569d4f82p-1,
    0x1.4bfdad5362a27p-1, 0x1.44e086061892dp-1, 0x1.3dea64c123422p-1, 0x1.371a7373aa9cbp-1,
    0x1.306fe0a31b715p-1, 0x1.29e9df51fdee1p-1, 0x1.2387a6e756238p-1, 0x1.1d4873168b9aap-1,
    0x1.172b83c7d517bp-1, 0x1.11301d0125b51p-1, 0x1.0b5586cf9890fp-1, 0x1.059b0d3158574p-1,
};
__device__ __forceinline__ double exp_neg(double x) {
  if (!(x <= 700.0)) return x > 700.0 ? 0.0 : x;
  const double kInvL = 0x1.71547652b82fep+5;    // 32/ln2
  const double kShift = 0x1.8p+52;              // 1.5 2^52: the low word of x/L + shift is k
  const double kL1 = 0x1.62e42ff000000p-6;      // ln2/32, leading 32 bits
  const double kL2 = -0x1.718432a1b0e26p-40;    // ln2/32 - L1
  const double t = fma(x, kInvL, kShift);
  const int k = __double2loint(t);
  const double kd = t - kShift;
  double r = fma(-kd, kL1, x);
  r = fma(-kd, kL2, r);
  const double s = -r;
  double p = fma(s, 1.0 / 720.0, 1.0 / 120.0);
  p = fma(p, s, 1.0 / 24.0);
  p = fma(p, s, 1.0 / 6.0);
  p = fma(p, s, 0.5);
  p = fma(p, s, 1.0);
  p = fma(p, s, 1.0);
  const double v = kExpTab[k & 31] * p;
  return __hiloint2double(__double2hiint(v) - ((k >> 5) << 20), __double2loint(v));
}

__device__ __forceinline__ void pl_coef_f(double x, double r, double& e, double& w, double& a, double& bq) {
  e = exp_neg(x);
  if (x < 1e-3) {
    pl_series64(x, w, a, bq);
  } else {
    w = (1.0 - e) * r;
    a = 1.0 - w;
    bq = (w - e) * r;
  }
}

__device__ __forceinline__ void pl_coef_f(float x, float r, float& e, float& w, float& a, float& bq) {
  e = __expf(-x);
  if (x < 0.1f) {
    w = fmaf(fmaf(fmaf(fmaf(fmaf(-1.0f / 720.0f, x, 1.0f / 120.0f), x, -1.0f / 24.0f), x, 1.0f / 6.0f), x, -0.5f), x, 1.0f);
    a = x * fmaf(fmaf(fmaf(fmaf(fmaf(-1.0f / 5040.0f, x, 1.0f / 720.0f), x, -1.0f / 120.0f), x, 1.0f / 24.0f), x, -1.0f / 6.0f), x, 0.5f);
    bq = fmaf(fmaf(fmaf(fmaf(1.0f / 144.0f, x, -1.0f / 30.0f), x, 1.0f / 8.0f), x, -1.0f / 3.0f), x, 0.5f);
  } else {
    w = (1.0f - e) * r;
    a = 1.0f - w;
    bq = (w - e) * r;
  }
}

// Every operation of a ray step is an explicitly rounded intrinsic: the
// compiler may not contract or reorder any of them, so the two kernel
// variants below (which see the same values in different registers, lanes
// and orders of issue) produce bit-identical results.
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fma3(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Tangent of the opacity and source function at (nu, k) in FP32 (Eqs. chi,
// eta differentiated; n and J^dagger fixed): per active transition
//   dchi += V (dn_lo - g dn_up),  deta += g V dn_up   (eta normalised by 2 h nu^3/c^2)
// and dS = (deta - S dchi)/chi. Shared by the opacity kernel and the sweeps
// that form it on the fly, so that both give the same bits.
struct TanAcc {
  float dchi = 0.f, deta = 0.f;
};
__device__ __forceinline__ void tan_acc(TanAcc& t, float V, float g, float vlo, float vup) {
  t.dchi = fma3(V, sub(vlo, mul(g, vup)), t.dchi);
  t.deta = fma3(mul(g, V), vup, t.deta);
}
// Hardware reciprocal (1 ulp): a single instruction without a slow-path
// branch, so that loops around it stay one basic block the compiler can
// software-pipeline. Its arguments (opacity sums) are positive normal numbers.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float tan_dS(const TanAcc& t, float S, float chi) {
  return mul(sub(t.deta, mul(S, t.dchi)), rcp_approx(chi));
}

}  // namespace jfnk
