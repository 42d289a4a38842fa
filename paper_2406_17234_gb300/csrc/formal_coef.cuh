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
__device__ __forceinline__ void pl_coef_f(double x, double r, double& e, double& w, double& a, double& bq) {
  e = exp(-x);
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
