// The residual F(n) of Algorithm 1 and its tangent, for every column of a
// batch: opacity/emissivity (Eqs. chi, eta), piecewise-linear formal solution
// along every (nu, mu) ray (Eqs. Iplus/Iminus, App. A), the angle and
// frequency integrals into radiative rates (Eqs. Rij/Rji), the per-depth
// assembly with particle conservation (Eqs. residuals_1/2) and the
// block-Jacobi preconditioner blocks (Sect. 2.5.2).
//
// Precision: ``real`` is double in the FP64 mode and float in the mixed mode
// for chi, I and their tangents. The mixed mode's base evaluations keep S, J
// and the opacity and rate sums in float pairs (dfloat.cuh); the assembly and
// everything after it is double. Intensities and source functions are carried
// normalised by 2 h nu^3 / c^2 so that float keeps range.
#include <cooperative_groups.h>

#include "formal_coef.cuh"

namespace cg = cooperative_groups;

namespace jfnk {

__device__ __forceinline__ int eval_mode(const ColDesc& cd) {
  if (cd.forced_mode >= 0) return cd.forced_mode;
  switch (cd.w.st->phase) {
    case PH_BASE: return EV_BASE;
    case PH_JVP:
    case PH_RESTART: return cd.w.st->fd_scheme ? EV_FD : EV_TANGENT;
    case PH_RH92: return EV_RH92;
    default: return EV_SKIP;
  }
}

__device__ __forceinline__ const double* tangent_dir(const ColDesc& cd) {
  if (cd.forced_mode >= 0) return cd.w.v;
  const int N = cd.t.nz * cd.t.nl;
  return cd.w.st->phase == PH_RESTART ? cd.w.x : cd.w.Vb + (size_t)cd.w.st->j * N;
}

// ---------------------------------------------------------------------------
// a1: opacity and source function per (nu, k), shared by every ray
// ---------------------------------------------------------------------------
// Prefetch of one line into L2 (no register is held while it is in flight).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <typename real>
__device__ __forceinline__ void opacity_point(const ColDesc& cd, int mode, int i);

// Grid-stride over the (nu, k) points of a column: a launch has a few blocks
// per column, so that columns in another evaluation kind cost little.
template <typename real>
__global__ void k_opacity(const ColDesc* __restrict__ cols, int skip_tangent) {
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode(cd);
  if (mode == EV_SKIP || (skip_tangent && mode == EV_TANGENT)) return;
  const int n = cd.t.nq * cd.t.nz;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (sizeof(real) == sizeof(float) && mode != EV_TANGENT && i + stride < n) {
      // the next point's background terms and first transition, into L2
      const ColTables& T = cd.t;
      const int j = i + stride, q = j / T.nz, k = j - q * T.nz;
      prefetch_l2(as_pairs(jdag_ptr(cd)) + j);
      prefetch_l2(T.etac2 + j);
      prefetch_l2(T.chibg2 + j);
      const int m = __ldg(T.qmeta + q);
      if (m >= 0) {
        prefetch_l2(T.V2 + (size_t)(m >> 8) * T.nz + k);
        prefetch_l2(T.gV2 + (size_t)(m >> 8) * T.nz + k);
      }
    }
    opacity_point<real>(cd, mode, i);
  }
}

template <typename real>
__device__ __forceinline__ void opacity_point(const ColDesc& cd, int mode, int i) {
  const ColTables& T = cd.t;
  const int nz = T.nz, nl = T.nl;
  if (mode == EV_TANGENT) {
    // chi and S at the base point are those of the Newton step's base
    // evaluation (n and J^dagger are unchanged): only their tangents are new,
    // in the working precision.
    if (cd.mixed) return;   // k_opacity_tan32
    const int q = i / nz, k = i - q * nz;
    const double* v = tangent_dir(cd) + k * nl;
    real dchi = 0, deta = 0;
    for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
      const int t = T.q_t[s];
      const size_t p = (size_t)(T.t_base[t] + q - T.t_q0[t]) * nz + k;
      const real V = (real)T.V[p], g = (real)T.G[p];
      const real vlo = (real)v[T.t_lo[t]], vup = (real)v[T.t_up[t]];
      dchi += V * (vlo - g * vup);
      deta += g * V * vup;                 // normalised by 2 h nu^3 / c^2
    }
    const real chi = reinterpret_cast<const real*>(cd.w.chi)[i];
    const real S = (real)cd.w.S[i];
    reinterpret_cast<real*>(cd.w.dchi)[i] = dchi;
    cd.w.dS[i] = (double)((deta - S * dchi) / chi);
    return;
  }
  const int q = i / nz, k = i - q * nz;
  if (sizeof(real) == sizeof(float)) {
    // mixed mode: chi is stored in float, S (and the RH92 emissivity) as
    // float pairs; every sum runs in pair arithmetic on the FP32 pipe (GB300's
    // FP64 pipe is 1/64 of it): chi = chi_c + chi_sca + sum V n_lo - sum g V
    // n_up, eta / (2 h nu^3/c^2) = (eta_c + chi_sca J^dagger) c^2/(2 h nu^3)
    // + sum g V n_up (Eqs. chi, eta)
    const float2* n2 = cd.w.n2 + k * nl;
    const df jd = df_load(as_pairs(jdag_ptr(cd)), i);
    const df eta_bg = df_add(df_load(T.etac2, i), df_mul(df_load(T.chisca2, k), jd));
    df chl = df_make(0.f, 0.f), el = df_make(0.f, 0.f);
    if (T.max_overlap <= kQMetaT) {
      // the packed table gives window point and levels in one load
#pragma unroll
      for (int j = 0; j < kQMetaT; ++j) {
        const int m = __ldg(T.qmeta + (size_t)j * T.nq + q);
        if (m < 0) break;
        const size_t p = (size_t)(m >> 8) * nz + k;
        chl = df_add(chl, df_mul(df_load(T.V2, p), df_load(n2, (m >> 4) & 15)));
        el = df_add(el, df_mul(df_load(T.gV2, p), df_load(n2, m & 15)));
      }
    } else {
      for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
        const int t = T.q_t[s];
        const size_t p = (size_t)(T.t_base[t] + q - T.t_q0[t]) * nz + k;
        chl = df_add(chl, df_mul(df_load(T.V2, p), df_load(n2, T.t_lo[t])));
        el = df_add(el, df_mul(df_load(T.gV2, p), df_load(n2, T.t_up[t])));
      }
    }
    const df chi = df_sub(df_add(df_load(T.chibg2, i), chl), el);
    const df etan = df_add(df_mul(eta_bg, df_load(T.rc2p, q)), el);
    reinterpret_cast<float*>(cd.w.chi)[i] = chi.hi;
    df_store(as_pairs(cd.w.S), i, df_div(etan, chi));
    if (mode == EV_RH92) {   // for the RH92 rate sums
      df_store(as_pairs(cd.w.eta), i, df_add(eta_bg, df_mul(el, df_load(T.c2p, q))));
      cd.w.etab32[i] = eta_bg.hi;
    }
    return;
  }
  const double* n = eval_pops(cd, mode) + k * nl;
  const double eta_bg = T.eta_c[i] + T.chi_sca[k] * jdag_ptr(cd)[i];
  const double c2 = T.c2[q];
  // sum V n_lo and sum g V n_up (the latter serves chi and eta alike), two
  // FP64 operations per transition; the packed table gives window point and
  // levels in one load
  double chl = 0.0, el = 0.0;
  if (T.max_overlap <= kQMetaT) {
    for (int j = 0; j < kQMetaT; ++j) {
      const int m = __ldg(T.qmeta + (size_t)j * T.nq + q);
      if (m < 0) break;
      const size_t p = (size_t)(m >> 8) * nz + k;
      chl = fma(T.V[p], n[(m >> 4) & 15], chl);
      el = fma(T.gV[p], n[m & 15], el);
    }
  } else {
    for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
      const int t = T.q_t[s];
      const size_t p = (size_t)(T.t_base[t] + q - T.t_q0[t]) * nz + k;
      chl = fma(T.V[p], n[T.t_lo[t]], chl);
      el = fma(T.gV[p], n[T.t_up[t]], el);
    }
  }
  const double chi = (T.chi_c[i] + T.chi_sca[k]) + (chl - el);
  const double eta = fma(c2, el, eta_bg);
  reinterpret_cast<real*>(cd.w.chi)[i] = (real)chi;
  cd.w.S[i] = eta / (chi * c2);
  if (mode == EV_RH92) cd.w.eta[i] = eta;   // for the RH92 rate sums
}

// Mixed mode, tangent evaluations: dchi and dS in FP32 (tan_acc). A thread
// owns one frequency nu and a run of ``depths`` depths (Batch::optan_depths,
// chosen by the autotuner); consecutive threads
// take consecutive frequencies, so every warp reads and writes coalesced rows
// of the depth-major arrays and line tables. The transitions active at nu
// come from the packed qmeta table, loaded once (the first two held, the
// others read when present), and kOpTanBatch depths' table loads are issued
// before any of their sums use them.
constexpr int kOpTanDepths = 16;   // default run of depths per thread
constexpr int kOpTanBatch = 1;   // depths whose loads are issued together (the L2
                                 // prefetch supplies the memory parallelism; fewer
                                 // registers leave room for six blocks per SM)
constexpr int kOpTanAhead = 4;   // depths ahead whose rows are prefetched into L2

__global__ void __launch_bounds__(256, 6) k_opacity_tan32(const ColDesc* __restrict__ cols, int nqb, int depths) {
  const ColDesc& cd = cols[blockIdx.y];
  if (!cd.mixed || eval_mode(cd) != EV_TANGENT) return;
  const ColTables& T = cd.t;
  const int nq = T.nq, nz = T.nz, nl = T.nl, nwin = T.nwin;
  const int qb = blockIdx.x % nqb, kc = blockIdx.x / nqb;
  const int q = qb * blockDim.x + threadIdx.x, k0 = kc * depths;
  if (q >= nq || k0 >= nz) return;
  const int k1 = min(nz, k0 + depths);
  const size_t pitch = (size_t)col_pitch(nq);
  const int m0 = __ldg(T.qmeta + q), m1 = __ldg(T.qmeta + (size_t)nq + q);
  struct In {
    float V0, G0, l0, u0, V1, G1, l1, u1, S, c;
  };
  auto ld = [&](int k) {
    In r;
    const float2* __restrict__ VG = T.VG32T + (size_t)k * nwin;
    const float* __restrict__ v = cd.w.v32 + (size_t)k * nl;
    const size_t o = (size_t)k * pitch + q;
    r.S = __ldg(cd.w.S32T + o);
    r.c = __ldg(cd.w.chiT + o);
    r.V0 = r.G0 = r.l0 = r.u0 = r.V1 = r.G1 = r.l1 = r.u1 = 0.f;
    if (m0 >= 0) {
      const float2 a = __ldg(VG + (m0 >> 8));
      r.V0 = a.x;
      r.G0 = a.y;
      r.l0 = __ldg(v + ((m0 >> 4) & 15));
      r.u0 = __ldg(v + (m0 & 15));
    }
    if (m1 >= 0) {
      const float2 a = __ldg(VG + (m1 >> 8));
      r.V1 = a.x;
      r.G1 = a.y;
      r.l1 = __ldg(v + ((m1 >> 4) & 15));
      r.u1 = __ldg(v + (m1 & 15));
    }
    return r;
  };
  auto fin = [&](int k, const In& r) {
    TanAcc ta;
    if (m0 >= 0) tan_acc(ta, r.V0, r.G0, r.l0, r.u0);
    if (m1 >= 0) {
      tan_acc(ta, r.V1, r.G1, r.l1, r.u1);
      const float2* __restrict__ VG = T.VG32T + (size_t)k * nwin;
      const float* __restrict__ v = cd.w.v32 + (size_t)k * nl;
#pragma unroll
      for (int j = 2; j < kQMetaT; ++j) {
        const int m = __ldg(T.qmeta + (size_t)j * nq + q);
        if (m < 0) break;
        const float2 a = __ldg(VG + (m >> 8));
        tan_acc(ta, a.x, a.y, __ldg(v + ((m >> 4) & 15)), __ldg(v + (m & 15)));
      }
      if (T.max_overlap > kQMetaT)
        for (int s = T.q_off[q] + kQMetaT; s < T.q_off[q + 1]; ++s) {
          const int t = T.q_t[s];
          const float2 a = __ldg(VG + T.t_base[t] + q - T.t_q0[t]);
          tan_acc(ta, a.x, a.y, __ldg(v + T.t_lo[t]), __ldg(v + T.t_up[t]));
        }
    }
    const size_t o = (size_t)k * pitch + q;
    cd.w.dchiT[o] = ta.dchi;
    cd.w.dS32T[o] = tan_dS(ta, r.S, r.c);
  };
  auto pf = [&](int k) {
    if (k >= k1) return;
    const size_t o = (size_t)k * pitch + q;
    prefetch_l2(cd.w.S32T + o);
    prefetch_l2(cd.w.chiT + o);
    const float2* __restrict__ VG = T.VG32T + (size_t)k * nwin;
    if (m0 >= 0) prefetch_l2(VG + (m0 >> 8));
    if (m1 >= 0) prefetch_l2(VG + (m1 >> 8));
  };
#pragma unroll
  for (int i = 0; i < kOpTanAhead; ++i) pf(k0 + i);
  int k = k0;
  for (; k + kOpTanBatch <= k1; k += kOpTanBatch) {
#pragma unroll
    for (int i = 0; i < kOpTanBatch; ++i) pf(k + kOpTanAhead + i);
    In r[kOpTanBatch];
#pragma unroll
    for (int i = 0; i < kOpTanBatch; ++i) r[i] = ld(k + i);
#pragma unroll
    for (int i = 0; i < kOpTanBatch; ++i) fin(k + i, r[i]);
  }
  for (; k < k1; ++k) fin(k, ld(k));
}

// Mixed mode, tangent evaluations: the tangent rate integrals (Eqs. Rij/Rji
// differentiated: only J moves) in FP32 from the depth-major dJ. One warp per
// (transition, depth): lanes stride over the transition's frequency window
// (coalesced rows of the depth-major tables) and a fixed xor-butterfly adds
// the lanes, so the sums are bit-reproducible.
constexpr int kRateTanWarps = 8;
constexpr int kRateTanDepths = 4;   // depths per warp (independent sums in flight)
__global__ void __launch_bounds__(32 * kRateTanWarps) k_rates_tan32(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.z];
  if (!cd.mixed || eval_mode(cd) != EV_TANGENT) return;
  const ColTables& T = cd.t;
  const int t = blockIdx.y;
  // warp w of the block takes depths k0 + w + d * kRateTanWarps, d < kRateTanDepths
  const int k0 = blockIdx.x * kRateTanWarps * kRateTanDepths + (threadIdx.x >> 5);
  if (t >= T.nt || k0 >= T.nz) return;   // whole warps
  const int lane = threadIdx.x & 31;
  const int nz = T.nz, nwin = T.nwin;
  const size_t pitch = (size_t)col_pitch(T.nq);
  const int q0 = T.t_q0[t], q1 = T.t_q1[t], base = T.t_base[t];
  const float2* __restrict__ VG = T.VG32T + base - q0;
  const float* __restrict__ W32 = T.W32 + base - q0;
  const float* __restrict__ dJ = cd.w.dJ32T;
  float a0[kRateTanDepths], a1[kRateTanDepths];
#pragma unroll
  for (int d = 0; d < kRateTanDepths; ++d) a0[d] = a1[d] = 0.f;
  for (int q = q0 + lane; q <= q1; q += 32) {
    const float W = __ldg(W32 + q);
#pragma unroll
    for (int d = 0; d < kRateTanDepths; ++d) {
      const int k = k0 + d * kRateTanWarps;
      if (k < nz) {
        const float2 vg = __ldg(VG + (size_t)k * nwin + q);
        const float WV = W * vg.x;
        const float x = __ldg(dJ + (size_t)k * pitch + q);
        a0[d] = fmaf(WV, x, a0[d]);
        a1[d] = fmaf(WV * vg.y, x, a1[d]);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < kRateTanDepths; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0[d] += __shfl_xor_sync(0xffffffffu, a0[d], o);
      a1[d] += __shfl_xor_sync(0xffffffffu, a1[d], o);
    }
    const int k = k0 + d * kRateTanWarps;
    if (lane == 0 && k < nz) {
      const size_t i = (size_t)t * nz + k;
      cd.w.dRup[i] = (double)a0[d];
      cd.w.dRdn[i] = (double)a1[d];
    }
  }
}

// Mixed mode: float copy of the tangent direction of every column in a
// tangent evaluation (the opacity tangent then runs entirely in FP32).
__global__ void k_dir32(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  if (!cd.mixed || eval_mode(cd) != EV_TANGENT) return;
  const int N = cd.t.nz * cd.t.nl;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  cd.w.v32[i] = (float)tangent_dir(cd)[i];
}

// Mixed mode: J^dagger as float pairs in the bytes of its FP64 array (after
// the host or the tables filled it in FP64), and J_new back to FP64 for the
// caller; in place, element by element.
__global__ void k_jdag_to_pairs(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const size_t n = (size_t)cd.t.nq * cd.t.nz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!cd.mixed || i >= n) return;
  double* J = const_cast<double*>(jdag_ptr(cd));
  const double x = J[i];
  df_store(as_pairs(J), i, df_from_double(x));
}
__global__ void k_jnew_to_double(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const size_t n = (size_t)cd.t.nq * cd.t.nz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!cd.mixed || i >= n) return;
  double* J = jnew_ptr(cd);
  const float2 p = as_pairs(J)[i];
  J[i] = (double)p.x + (double)p.y;
}
int launch_j_pairs(const ColDesc* d_cols, int ncols, size_t max_qz, cudaStream_t s, bool to_pairs) {
  if (ncols <= 0 || max_qz == 0) return JFNK_OK;
  const dim3 g((unsigned)((max_qz + 255) / 256), ncols);
  if (to_pairs) k_jdag_to_pairs<<<g, 256, 0, s>>>(d_cols);
  else k_jnew_to_double<<<g, 256, 0, s>>>(d_cols);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

// Mixed mode, base and RH92 evaluations: the populations as float pairs for
// the pair arithmetic of the opacity kernel.
__global__ void k_pop_pairs(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  if (!cd.mixed) return;
  const int mode = eval_mode(cd);
  if (mode != EV_BASE && mode != EV_RH92) return;
  const int N = cd.t.nz * cd.t.nl;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  df_store(cd.w.n2, i, df_from_double(cd.w.n[i]));
}

// Differences of the source function (and of its tangent) between adjacent
// depths, formed in FP64 before any rounding to ``real``.
template <typename real>
__global__ void k_source_diff(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode(cd);
  if (mode == EV_SKIP) return;
  const int nz = cd.t.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cd.t.nq * nz) return;
  const int k = i % nz;
  const bool last = (k == nz - 1);
  reinterpret_cast<real*>(cd.w.dSk)[i] = last ? (real)0 : (real)(cd.w.S[i + 1] - cd.w.S[i]);
  if (mode == EV_TANGENT)
    reinterpret_cast<real*>(cd.w.ddSk)[i] = last ? (real)0 : (real)(cd.w.dS[i + 1] - cd.w.dS[i]);
}

// Piecewise-linear coefficients (App. A.1) in the form the difference
// recurrence needs: e = exp(-x), w = (1 - e)/x, a = 1 - w and bq = b/x with
// b = w - e. Below a threshold every one of them comes from its own Taylor
// series, since 1 - e, 1 - w and w - e all cancel there (a = 1 - w loses all
// FP32 digits at x ~ 1e-6): x = 0.1 in FP32, x = 1e-3 in FP64.
__device__ __forceinline__ void pl_coef(double x, double& e, double& w, double& a, double& bq) {
  e = exp(-x);
  if (x < 1e-3) {
    pl_series64(x, w, a, bq);   // see formal_coef.cuh
  } else {
    const double r = 1.0 / x;
    w = (1.0 - e) * r;
    a = 1.0 - w;
    bq = (w - e) * r;
  }
}

__device__ __forceinline__ void pl_coef(float x, float& e, float& w, float& a, float& bq) {
  e = __expf(-x);
  if (x < 0.1f) {
    // the same series to x^5 (truncation below 3e-10 relative)
    w = fmaf(fmaf(fmaf(fmaf(fmaf(-1.0f / 720.0f, x, 1.0f / 120.0f), x, -1.0f / 24.0f), x, 1.0f / 6.0f), x, -0.5f), x, 1.0f);
    a = x * fmaf(fmaf(fmaf(fmaf(fmaf(-1.0f / 5040.0f, x, 1.0f / 720.0f), x, -1.0f / 120.0f), x, 1.0f / 24.0f), x, -1.0f / 6.0f), x, 0.5f);
    bq = fmaf(fmaf(fmaf(fmaf(1.0f / 144.0f, x, -1.0f / 30.0f), x, 1.0f / 8.0f), x, -1.0f / 3.0f), x, 0.5f);
  } else {
    const float r = __frcp_rn(x);
    w = (1.0f - e) * r;
    a = 1.0f - w;
    bq = (w - e) * r;
  }
}

// ---------------------------------------------------------------------------
// a2: formal solution, one thread per (nu, mu, hemisphere) ray.
// The piecewise-linear recurrence of Eqs. Iplus/Iminus is carried for
// D = I - S: with a = 1 - w and b = w - e it becomes
//   D^k = D^{k+1} e^{-dtau^k} + w^k (S^{k+1} - S^k)          (mu > 0)
//   D^k = D^{k-1} e^{-dtau^{k-1}} + w^{k-1} (S^{k-1} - S^k)  (mu < 0)
// identical in exact arithmetic; in FP32 it keeps the precision of I - S,
// which is what the net rates of nearly thermalised layers depend on.
// Outputs per ray r and depth k: 1/2 w_mu D, its tangent, and in base mode
// the local derivatives dI^k/dchi^k and dI^k/deta^k (App. A.2).
// Layout of the per-ray outputs: [r][k][q].
// ---------------------------------------------------------------------------
template <typename real>
__global__ void k_formal(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode(cd);
  if (mode == EV_SKIP) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq, nmu = T.nmu;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * 2 * nmu) return;
  const int q = i % nq, r = i / nq;
  const int up = r < nmu;
  const int m = up ? r : r - nmu;
  const real hw = (real)(0.5 * T.wmu[m]);
  const real inv2mu = (real)(0.5 / T.mu[m]);
  const size_t row = (size_t)q * nz;
  const real* chi = reinterpret_cast<const real*>(cd.w.chi) + row;
  const real* dSk = reinterpret_cast<const real*>(cd.w.dSk) + row;
  const double* S64 = cd.w.S + row;
  const bool tan = (mode == EV_TANGENT);
  const bool der = (mode == EV_BASE || mode == EV_RH92);
  const real* dchi = tan ? reinterpret_cast<const real*>(cd.w.dchi) + row : nullptr;
  const real* ddSk = tan ? reinterpret_cast<const real*>(cd.w.ddSk) + row : nullptr;
  real* H = reinterpret_cast<real*>(cd.w.H) + (size_t)r * nz * nq + q;
  real* HI = der ? reinterpret_cast<real*>(cd.w.HI) + (size_t)r * nz * nq + q : nullptr;
  real* dH = tan ? reinterpret_cast<real*>(cd.w.dH) + (size_t)r * nz * nq + q : nullptr;
  real* LX = der ? reinterpret_cast<real*>(cd.w.LX) + (size_t)r * nz * nq + q : nullptr;
  real* LE = der ? reinterpret_cast<real*>(cd.w.LE) + (size_t)r * nz * nq + q : nullptr;
  const int k0 = up ? nz - 1 : 0;
  const int step = up ? -1 : 1;
  // boundary values: I = B_nu(T_bottom) entering at the bottom, I = 0 at the top
  real D = up ? (real)(T.Bn[row + nz - 1] / T.c2[q] - S64[k0]) : (real)(-S64[k0]);
  real dD = tan ? (real)(-cd.w.dS[row + k0]) : (real)0;
  real chi1 = chi[k0];
  real dchi1 = tan ? dchi[k0] : (real)0;
  // base evaluations also carry I itself, which keeps relative precision where
  // I << S (optically thin, hot layers) and D = I - S cancels
  real I = up ? (real)(T.Bn[row + nz - 1] / T.c2[q]) : (real)0;
  real S1 = (real)S64[k0];
  H[(size_t)k0 * nq] = hw * D;
  if (tan) dH[(size_t)k0 * nq] = hw * dD;
  if (der) { LX[(size_t)k0 * nq] = 0; LE[(size_t)k0 * nq] = 0; HI[(size_t)k0 * nq] = hw * I; }
  real M = D < (real)0 ? -D : D;   // attenuated bound of |D| upstream (base re-anchoring)
  for (int s = 1; s < nz; ++s) {
    const int k = k0 + step * s;
    const int kd = up ? k : k - 1;             // layer between k and its upstream neighbour
    const real chi0 = chi[k];
    const real dS = up ? dSk[k] : -dSk[k - 1];  // S_upstream - S^k
    const real h = (real)T.dz[kd] * inv2mu;
    const real dtau = h * (chi0 + chi1);
    real e, w, a, bq;
    pl_coef(dtau, e, w, a, bq);
    real Dnew = D * e + w * dS;
    if (der) {
      // App. A.2 with S_up - I_up = -D_up
      const real S0 = (real)S64[k];
      LX[(size_t)k * nq] = hw * (-(S0 / chi0) * a - h * (e * D + dS * bq));
      LE[(size_t)k * nq] = hw * (a / chi0);
      I = I * e + a * S0 + (bq * dtau) * S1;   // Eqs. Iplus / Iminus, b = bq dtau
      HI[(size_t)k * nq] = hw * I;
      S1 = S0;
      // re-anchor D on I - S where that is better conditioned
      const real aD = Dnew < (real)0 ? -Dnew : Dnew;
      M = fmax(M * e, aD);
      const real anchor = (I < (real)0 ? -I : I) + (S0 < (real)0 ? -S0 : S0);
      if (anchor < M) {
        Dnew = I - S0;
        M = anchor;
      }
    }
    if (tan) {
      const real dchi0 = dchi[k];
      const real ddS = up ? ddSk[k] : -ddSk[k - 1];
      const real ddtau = h * (dchi0 + dchi1);
      const real dDnew = dD * e - ddtau * (e * D + bq * dS) + w * ddS;
      dH[(size_t)k * nq] = hw * dDnew;
      dD = dDnew;
      dchi1 = dchi0;
    }
    D = Dnew;
    H[(size_t)k * nq] = hw * D;
    chi1 = chi0;
  }
  if (up && der) cd.w.Iem[(size_t)q * nmu + m] = (double)I * T.c2[q];
}

// ---------------------------------------------------------------------------
// a3 (part 1): sums over the 2 n_mu rays -> J, dJ, Lambda_chi, Lambda_eta;
// J = S + sum_r 1/2 w_r D_r (the Gauss-Legendre weights sum to one).
// ---------------------------------------------------------------------------
template <typename real>
__global__ void k_ray_sum(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode(cd);
  if (mode == EV_SKIP) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq, nr = 2 * T.nmu;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // i = k * nq + q
  if (i >= nq * nz) return;
  const int k = i / nq, q = i - k * nq;
  const size_t plane = (size_t)nz * nq;
  const size_t o = (size_t)q * nz + k;
  const double c2 = T.c2[q];
  double s = 0.0, sa = 0.0;
  const real* H = reinterpret_cast<const real*>(cd.w.H) + i;
  for (int r = 0; r < nr; ++r) {
    const double h = (double)H[r * plane];
    s += h;
    sa += fabs(h);
  }
  double J = (cd.w.S[o] + s) * c2;
  if (mode == EV_BASE || mode == EV_RH92) {
    // take the representation with the smaller rounding error: sum |w D| vs sum |w I|
    const real* HI = reinterpret_cast<const real*>(cd.w.HI) + i;
    double si = 0.0;
    for (int r = 0; r < nr; ++r) si += (double)HI[r * plane];
    if (fabs(si) < sa) J = si * c2;   // intensities are non-negative: sum |w I| = sum w I
  }
  if (mode == EV_FD) cd.w.J[o] = J;   // base and RH92 rates read J_new
  if (mode == EV_TANGENT) {
    const real* dH = reinterpret_cast<const real*>(cd.w.dH) + i;
    double ds = 0.0;
    for (int r = 0; r < nr; ++r) ds += (double)dH[r * plane];
    cd.w.dJ[o] = (cd.w.dS[o] + ds) * c2;
  } else if (mode != EV_FD) {
    jnew_ptr(cd)[o] = J;
    const real* LX = reinterpret_cast<const real*>(cd.w.LX) + i;
    const real* LE = reinterpret_cast<const real*>(cd.w.LE) + i;
    double sx = 0.0, se = 0.0;
    for (int r = 0; r < nr; ++r) {
      sx += (double)LX[r * plane];
      se += (double)LE[r * plane];
    }
    cd.w.Lchi[o] = sx * c2;   // dJ/dchi in cgs
    cd.w.Leta[o] = se;        // dJ/deta = a/chi needs no rescaling
  }
}

// ---------------------------------------------------------------------------
// a3 (part 2): frequency integrals per (transition, depth); in base mode also
// the preconditioner sums A^kk_{t, j} = sum_nu W chi_t (beta_j Lchi + gamma_j Leta)
// and in RH92 mode the sums of the preconditioned rate equations.
// ---------------------------------------------------------------------------
constexpr int kRateWarps = 4;
constexpr int kRateSplit = 4;            // most blocks of a cluster sharing one (transition, depth tile)
constexpr int kRateBlocksPerSM = 128;    // blocks of the column loop per multiprocessor

// Per-lane partial sums in dynamic shared memory: racc doubles
// [warp][slot][lane], then (mixed mode) fslots floats [warp][slot][lane].
struct RateSmem {
  double* red;
  float* fsl;
  int racc, fslots;
  __device__ double& d(int w, int j, int lane) const { return red[((size_t)w * racc + j) * 32 + lane]; }
  __device__ float& f(int w, int j, int lane) const { return fsl[((size_t)w * fslots + j) * 32 + lane]; }
};

// The evaluation kind this cluster integrates for column cd, EV_SKIP when it
// has nothing to do there. Uniform over the cluster: its blocks differ only
// in their frequency chunk.
__device__ __forceinline__ int rate_mode(const ColDesc& cd, int t, int tile) {
  const int mode = eval_mode(cd);
  if (mode == EV_SKIP || (mode == EV_TANGENT && cd.mixed) || t >= cd.t.nt || tile * 32 >= cd.t.nz)
    return EV_SKIP;
  return mode;
}

// One (32-depth tile, transition t, column): lanes map to depths (every table
// and J access is coalesced), the ``split`` blocks of the cluster split the
// frequency window into contiguous chunks and their warps stride through the
// chunk; partial sums are reduced through shared memory inside a block and
// through distributed shared memory across the cluster, in a fixed order
// (bit-reproducible, no atomics).
//
// R_ij = sum W V J and R_ji = Rsp + sum W g V J (Eqs. Rij, Rji): in FP64 one
// product per term from the WV, WgV tables; in mixed mode the same sums in
// float pairs (W, V, g V, J pairs), the preconditioner sums (base) and the
// RH92 sums in FP32, and Jeff = J - Psi* eta from the pairs because it cancels
// in optically thick layers.
__device__ void rates_tile(const ColDesc& cd, const int mode, const int t, const int tile, const int rank,
                           const RateSmem& sm, cg::cluster_group& cluster, const SolverOpts* bopts) {
  const ColTables& T = cd.t;
  const int nz = T.nz, nl = T.nl, nt = T.nt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool tan = (mode == EV_TANGENT);
  const bool base_mode = (mode == EV_BASE);
  const bool rh = (mode == EV_RH92);
  const bool mix = cd.mixed != 0;
  const int nacc = tan ? 2 : (base_mode ? 2 + nl : (rh ? 2 + kRhFixed + nt : 2));
  const int k = min(tile * 32 + lane, nz - 1);
  const int q0 = T.t_q0[t], q1 = T.t_q1[t], wbase = T.t_base[t];
  const int nw = q1 - q0 + 1;
  const int split = (int)cluster.num_blocks();
  const int qa = q0 + (int)(((long)nw * rank) / split);
  const int qb = q0 + (int)(((long)nw * (rank + 1)) / split) - 1;
  const double* n = eval_pops(cd, mode) + k * nl;
  const double n_lo = n[T.t_lo[t]], n_up = n[T.t_up[t]];
  // slots indexed by level or transition accumulate in place (lane-private)
  for (int j = 2; j < nacc; ++j) sm.d(wid, j, lane) = 0.0;
  if (mix) for (int j = 0; j < sm.fslots; ++j) sm.f(wid, j, lane) = 0.f;
  // base and RH92 evaluations leave J in J_new, difference evaluations in J
  const double* __restrict__ J = tan ? cd.w.dJ : (mode == EV_FD ? cd.w.J : jnew_ptr(cd));
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a5 = 0.0;
  // mixed mode: J, S and eta are float pairs; the rate sums accumulate in pairs
  const float2* __restrict__ J2 = mix ? as_pairs(jnew_ptr(cd)) : nullptr;
  df s0 = df_make(0.f, 0.f), s1 = df_make(0.f, 0.f);
  float f0 = 0.f, f1 = 0.f, f3 = 0.f;
  if (!base_mode && !rh) {
    // tangent (FP64 mode) or a difference evaluation: the two rate sums only
    for (int q = qa + wid; q <= qb; q += kRateWarps) {
      const size_t pk = (size_t)(wbase + q - q0) * nz + k;
      const double Jq = J[(size_t)q * nz + k];
      a0 = fma(T.WV[pk], Jq, a0);
      a1 = fma(T.WgV[pk], Jq, a1);
    }
  } else if (base_mode && mix) {
    // rate sums in pair arithmetic, preconditioner sums
    // A^kk_{t,j} = sum W chi_t (beta_j Lchi + gamma_j Leta) in FP32
    const float nlo_f = (float)n_lo, nup_f = (float)n_up;
    const int pv = precond_variant(cd, bopts);
    const float sca_f = (float)T.chi_sca[k];
    const bool packed = T.max_overlap <= kQMetaT;
    // one frequency's inputs; two frequencies are loaded before the first is
    // summed, so that their latencies overlap (the sums keep their order)
    struct In {
      df J, w, V, gV;
      float Vf, gf, Wr, Lx, Le, c2f;
      int m0, m1;
      float Vs0, Gs0, Vs1, Gs1;
    };
    auto ld = [&](int q) {
      In r;
      const int p = wbase + q - q0;
      const size_t pk = (size_t)p * nz + k, o = (size_t)q * nz + k;
      r.J = df_load(J2, o);
      r.w = df_load(T.W2, p);
      r.V = df_load(T.V2, pk);
      r.gV = df_load(T.gV2, pk);
      r.Vf = __ldg(T.V32 + pk);
      r.gf = __ldg(T.G32 + pk);
      r.Wr = __ldg(T.Wr32 + p);
      r.Lx = cd.w.Lchi32[o];
      r.Le = cd.w.Leta32[o];
      r.c2f = __ldg(T.c2f + q);
      r.m0 = r.m1 = -1;
      r.Vs0 = r.Gs0 = r.Vs1 = r.Gs1 = 0.f;
      if (packed) {
        // the packed table gives window point and levels in one load
        r.m0 = __ldg(T.qmeta + q);
        r.m1 = __ldg(T.qmeta + (size_t)T.nq + q);
        if (r.m0 >= 0) {
          const size_t ps = (size_t)(r.m0 >> 8) * nz + k;
          r.Vs0 = __ldg(T.V32 + ps);
          r.Gs0 = __ldg(T.G32 + ps);
        }
        if (r.m1 >= 0) {
          const size_t ps = (size_t)(r.m1 >> 8) * nz + k;
          r.Vs1 = __ldg(T.V32 + ps);
          r.Gs1 = __ldg(T.G32 + ps);
        }
      }
      return r;
    };
    auto use = [&](int q, const In& r) {
      s0 = df_acc(s0, df_mul(df_mul(r.w, r.V), r.J));
      s1 = df_acc(s1, df_mul(df_mul(r.w, r.gV), r.J));
      const float Wc0 = r.Wr * (r.Vf * (nlo_f - r.gf * nup_f));
      // third solution of Sect. 2.5.2: d J/d n over 1 - chi_sca Leta
      const float Wc = pv == 3 ? Wc0 / (1.0f - sca_f * r.Le) : Wc0;
      if (pv == 2) {
        // second solution: + chi_sca (d J/d n_j)^dagger Leta for every level
        const float f = Wc0 * sca_f * r.Le;
        const double* Dq = cd.w.dJdn + ((size_t)q * nz + k) * nl;
        for (int j = 0; j < nl; ++j) sm.f(wid, j, lane) = fmaf(f, (float)Dq[j], sm.f(wid, j, lane));
      }
      const float cLx = Wc * r.Lx, cU = Wc * (r.c2f * r.Le - r.Lx);
      // beta_j (Sect. 2.5.1, read from Eq. chi) and gamma_j (Eq. der_eta_n)
      // of every transition active at nu
      auto add_terms = [&](int m, float Vs, float Gs) {
        float& zl = sm.f(wid, (m >> 4) & 15, lane);
        zl = fmaf(cLx, Vs, zl);
        float& zu = sm.f(wid, m & 15, lane);
        zu = fmaf(cU, Gs * Vs, zu);
      };
      if (packed) {
        if (r.m0 >= 0) add_terms(r.m0, r.Vs0, r.Gs0);
        if (r.m1 >= 0) {
          add_terms(r.m1, r.Vs1, r.Gs1);
          for (int j = 2; j < kQMetaT; ++j) {
            const int m = __ldg(T.qmeta + (size_t)j * T.nq + q);
            if (m < 0) break;
            const size_t ps = (size_t)(m >> 8) * nz + k;
            add_terms(m, __ldg(T.V32 + ps), __ldg(T.G32 + ps));
          }
        }
      } else {
        for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
          const int ts = T.q_t[s];
          const size_t ps = (size_t)(T.t_base[ts] + q - T.t_q0[ts]) * nz + k;
          add_terms((T.t_lo[ts] << 4) | T.t_up[ts], T.V32[ps], T.G32[ps]);
        }
      }
    };
    int q = qa + wid;
    for (; q + kRateWarps <= qb; q += 2 * kRateWarps) {
      const In r0 = ld(q), r1 = ld(q + kRateWarps);
      use(q, r0);
      use(q + kRateWarps, r1);
    }
    if (q <= qb) use(q, ld(q));
  } else if (base_mode) {
    const int pv = precond_variant(cd, bopts);
    const double sca = T.chi_sca[k];
    for (int q = qa + wid; q <= qb; q += kRateWarps) {
      const size_t pk = (size_t)(wbase + q - q0) * nz + k, o = (size_t)q * nz + k;
      const double Jq = J[o];
      const double wv = T.WV[pk], wgv = T.WgV[pk];
      a0 = fma(wv, Jq, a0);
      a1 = fma(wgv, Jq, a1);
      const double Wc0 = wv * n_lo - wgv * n_up;     // W chi_t
      const double Lx = cd.w.Lchi[o], Le = cd.w.Leta[o], c2 = T.c2[q];
      // third solution of Sect. 2.5.2: d J/d n over 1 - chi_sca Leta
      const double Wc = pv == 3 ? Wc0 / (1.0 - sca * Le) : Wc0;
      if (pv == 2) {
        // second solution: + chi_sca (d J/d n_j)^dagger Leta for every level
        const double f = Wc0 * sca * Le;
        const double* Dq = cd.w.dJdn + o * nl;
        for (int j = 0; j < nl; ++j) sm.d(wid, 2 + j, lane) += f * Dq[j];
      }
      for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
        const int ts = T.q_t[s];
        const size_t ps = (size_t)(T.t_base[ts] + q - T.t_q0[ts]) * nz + k;
        const double Vs = T.V[ps], gs = T.G[ps];
        sm.d(wid, 2 + T.t_lo[ts], lane) += Wc * (Vs * Lx);
        sm.d(wid, 2 + T.t_up[ts], lane) += Wc * (-gs * Vs * Lx + c2 * gs * Vs * Le);
      }
    }
  } else if (mix) {
    // RH92 (full preconditioning): N_t(n') = sum W [chi_t(n') Jeff + chi_t(n) Psi eta(n') - eta_t(n')]
    const float nlo_f = (float)n_lo, nup_f = (float)n_up;
    const bool packed = T.max_overlap <= kQMetaT;
    const float2* __restrict__ eta2 = as_pairs(cd.w.eta);
    // one frequency's inputs; two frequencies are loaded before the first is
    // summed, so that their latencies overlap (the sums keep their order)
    struct In {
      df J, w, V, gV, eta;
      float Le, Wf, Vf, gf, c2f, etab;
      int m0, t0, m1, t1;
      float GV0, GV1;
    };
    auto ld = [&](int q) {
      In r;
      const int p = wbase + q - q0;
      const size_t pk = (size_t)p * nz + k, o = (size_t)q * nz + k;
      r.J = df_load(J2, o);
      r.w = df_load(T.W2, p);
      r.V = df_load(T.V2, pk);
      r.gV = df_load(T.gV2, pk);
      r.eta = df_load(eta2, o);
      r.Le = cd.w.Leta32[o];
      r.Wf = __ldg(T.Wr32 + p);
      r.Vf = __ldg(T.V32 + pk);
      r.gf = __ldg(T.G32 + pk);
      r.c2f = __ldg(T.c2f + q);
      r.etab = cd.w.etab32[o];
      r.m0 = r.m1 = r.t0 = r.t1 = -1;
      r.GV0 = r.GV1 = 0.f;
      if (packed) {
        // the packed tables give window point and transition in two loads
        r.m0 = __ldg(T.qmeta + q);
        r.m1 = __ldg(T.qmeta + (size_t)T.nq + q);
        r.t0 = __ldg(T.qtr + q);
        r.t1 = __ldg(T.qtr + (size_t)T.nq + q);
        if (r.m0 >= 0) {
          const size_t ps = (size_t)(r.m0 >> 8) * nz + k;
          r.GV0 = __ldg(T.G32 + ps) * __ldg(T.V32 + ps);
        }
        if (r.m1 >= 0) {
          const size_t ps = (size_t)(r.m1 >> 8) * nz + k;
          r.GV1 = __ldg(T.G32 + ps) * __ldg(T.V32 + ps);
        }
      }
      return r;
    };
    auto use = [&](int q, const In& r) {
      s0 = df_acc(s0, df_mul(df_mul(r.w, r.V), r.J));
      s1 = df_acc(s1, df_mul(df_mul(r.w, r.gV), r.J));
      // Jeff = J - Psi* eta cancels in optically thick layers: formed from the pairs
      const float Jf = df_to_float(df_sub(r.J, df_mul_f(r.eta, r.Le)));
      const float WVf = r.Wf * r.Vf;
      f0 = fmaf(WVf, Jf, f0);
      f1 = fmaf(WVf * r.gf, Jf, f1);
      const float wcp = r.Wf * (r.Vf * (nlo_f - r.gf * nup_f)) * r.Le;
      f3 = fmaf(wcp, r.etab, f3);
      const float wcu = wcp * r.c2f;
      if (packed) {
        if (r.m0 >= 0) {
          float& z = sm.f(wid, r.t0, lane);
          z = fmaf(wcu, r.GV0, z);
        }
        if (r.m1 >= 0) {
          float& z = sm.f(wid, r.t1, lane);
          z = fmaf(wcu, r.GV1, z);
          for (int j = 2; j < kQMetaT; ++j) {
            const int m = __ldg(T.qmeta + (size_t)j * T.nq + q);
            if (m < 0) break;
            const size_t ps = (size_t)(m >> 8) * nz + k;
            float& zj = sm.f(wid, __ldg(T.qtr + (size_t)j * T.nq + q), lane);
            zj = fmaf(wcu, __ldg(T.G32 + ps) * __ldg(T.V32 + ps), zj);
          }
        }
      } else {
        for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
          const int ts = T.q_t[s];
          const size_t ps = (size_t)(T.t_base[ts] + q - T.t_q0[ts]) * nz + k;
          float& z = sm.f(wid, ts, lane);
          z = fmaf(wcu, T.G32[ps] * T.V32[ps], z);
        }
      }
    };
    int q = qa + wid;
    for (; q + kRateWarps <= qb; q += 2 * kRateWarps) {
      const In r0 = ld(q), r1 = ld(q + kRateWarps);
      use(q, r0);
      use(q + kRateWarps, r1);
    }
    if (q <= qb) use(q, ld(q));
  } else {
    const double* Jd = jdag_ptr(cd);
    for (int q = qa + wid; q <= qb; q += kRateWarps) {
      const size_t pk = (size_t)(wbase + q - q0) * nz + k, o = (size_t)q * nz + k;
      const double Jq = J[o];
      const double wv = T.WV[pk], wgv = T.WgV[pk];
      a0 = fma(wv, Jq, a0);
      a1 = fma(wgv, Jq, a1);
      const double Le = cd.w.Leta[o];
      const double Jeff = fma(-Le, cd.w.eta[o], Jq);
      a2 = fma(wv, Jeff, a2);
      a3 = fma(wgv, Jeff, a3);
      const double wcp = (wv * n_lo - wgv * n_up) * Le;
      a5 = fma(wcp, T.eta_c[o] + T.chi_sca[k] * Jd[o], a5);
      const double wcu = wcp * T.c2[q];
      for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
        const int ts = T.q_t[s];
        const size_t ps = (size_t)(T.t_base[ts] + q - T.t_q0[ts]) * nz + k;
        sm.d(wid, 2 + kRhFixed + ts, lane) += wcu * (T.G[ps] * T.V[ps]);
      }
    }
  }
  const bool pairs = mix && (base_mode || rh);
  sm.d(wid, 0, lane) = pairs ? df_to_double(s0) : a0;
  sm.d(wid, 1, lane) = pairs ? df_to_double(s1) : a1;
  if (rh) {
    // slot 2 + 2 (sum W U, U = 2 h nu^3/c^2 g V) is the spontaneous table, added below
    sm.d(wid, 2, lane) = mix ? (double)f0 : a2;
    sm.d(wid, 3, lane) = mix ? (double)f1 : a3;
    sm.d(wid, 5, lane) = mix ? (double)f3 : a5;
    if (mix)
      for (int j = 0; j < nt; ++j) sm.d(wid, 2 + kRhFixed + j, lane) = (double)sm.f(wid, j, lane);
  } else if (base_mode && mix) {
    for (int j = 0; j < nl; ++j) sm.d(wid, 2 + j, lane) = (double)sm.f(wid, j, lane);
  }
  __syncthreads();
  if (wid == 0)
    for (int j = 0; j < nacc; ++j) {
      double v = sm.d(0, j, lane);
      for (int w = 1; w < kRateWarps; ++w) v += sm.d(w, j, lane);
      sm.d(0, j, lane) = v;
    }
  cluster.sync();
  if (rank == 0 && wid == 0) {
    const int kw = tile * 32 + lane;
    if (kw < nz) {
      double acc[2 + kRhFixed + kMaxT > 2 + kMaxL ? 2 + kRhFixed + kMaxT : 2 + kMaxL];
      for (int j = 0; j < nacc; ++j) acc[j] = sm.d(0, j, lane);
      for (int r = 1; r < split; ++r) {
        const double* peer = cluster.map_shared_rank(sm.red, r);
        for (int j = 0; j < nacc; ++j) acc[j] += peer[(size_t)j * 32 + lane];
      }
      const size_t i = (size_t)t * nz + kw;
      if (tan) {
        cd.w.dRup[i] = acc[0];
        cd.w.dRdn[i] = acc[1];
      } else {
        const double rsp = T.Rsp[i];
        cd.w.Rup[i] = acc[0];
        cd.w.Rdn[i] = acc[1] + rsp;
        if (base_mode)
          for (int j = 0; j < nl; ++j) cd.w.Apart[i * nl + j] = acc[2 + j];
        if (rh) {
          acc[4] = rsp;
          for (int j = 0; j < kRhFixed + nt; ++j) cd.w.rh[i * kRhStride + j] = acc[2 + j];
        }
      }
    }
  }
  cluster.sync();   // peers keep their shared memory until rank 0 has read it
}

// A persistent-style loop over the batch's columns: each cluster owns one
// (depth tile, transition) and walks the columns 32 at a time, lane l testing
// column c0 + l * step, so that columns in another evaluation kind cost one
// load each instead of a cluster launch.
__global__ void __launch_bounds__(32 * kRateWarps) k_rates(const ColDesc* __restrict__ cols, int ncols,
                                                           int racc, int fslots, const SolverOpts* bopts) {
  extern __shared__ __align__(16) unsigned char rate_smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  RateSmem sm;
  sm.red = reinterpret_cast<double*>(rate_smem);
  sm.fsl = reinterpret_cast<float*>(sm.red + (size_t)kRateWarps * racc * 32);
  sm.racc = racc;
  sm.fslots = fslots;
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.y, tile = blockIdx.x;
  const int split = (int)cluster.num_blocks();
  const int step = gridDim.z / split;
  for (int c0 = blockIdx.z / split; c0 < ncols; c0 += 32 * step) {
    const int cl = c0 + lane * step;
    const int ml = cl < ncols ? rate_mode(cols[cl], t, tile) : EV_SKIP;
    unsigned act = __ballot_sync(0xffffffffu, ml != EV_SKIP);   // the same in every warp of the cluster
    while (act) {
      const int l = __ffs(act) - 1;
      act &= act - 1;
      const int mode = __shfl_sync(0xffffffffu, ml, l);
      rates_tile(cols[c0 + l * step], mode, t, tile, rank, sm, cluster, bopts);
    }
  }
}

// Kernel attributes, set once per device when a context is created (outside
// any stream capture): the rate kernel's largest dynamic shared memory.
int prepare_kernels() {
  const int max_smem = (int)((size_t)kRateWarps * 32 * ((2 + kRhFixed + kMaxT) * sizeof(double) +
                                                       std::max(kMaxT, kMaxL) * sizeof(float)));
  JFNK_CUDA(cudaFuncSetAttribute(k_rates, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  return JFNK_OK;
}

static int launch_rates(const Batch& b, cudaStream_t s) {
  const int tiles = (b.max_nz + 31) / 32;
  const int racc = 2 + std::max(kRhFixed + b.max_nt, kMaxL);
  const int fslots = b.mixed ? std::max(b.max_nt, kMaxL) : 0;
  const size_t smem = (size_t)kRateWarps * 32 * (racc * sizeof(double) + fslots * sizeof(float));
  const long sms = std::max(b.n_sm, 1);
  const long per = (long)tiles * std::max(b.max_nt, 1);
  // a frequency window is split over a cluster only when the (tile,
  // transition, column) units alone leave the multiprocessors short of blocks
  const int split = (long)b.ncols * per >= 32 * sms ? 1 : kRateSplit;
  const long want = kRateBlocksPerSM * sms / split;
  const int cz = (int)std::max(1L, std::min<long>(b.ncols, (want + per - 1) / per));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles, b.max_nt, cz * split);
  cfg.blockDim = dim3(32 * kRateWarps);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = split;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  JFNK_CUDA(cudaLaunchKernelEx(&cfg, k_rates, (const ColDesc*)b.d_cols, b.ncols, racc, fslots,
                               (const SolverOpts*)b.d_opts));
  return JFNK_OK;
}

// Second solution of Sect. 2.5.2: after a base evaluation (whose rate kernel
// has used the previous estimate) the lagged d J_nu^k/d n_j^k is renewed as
// beta_j Lchi + (gamma_j + chi_sca D_j) Leta, beta_j = d chi/d n_j,
// gamma_j = d eta/d n_j from the transitions active at nu; thread per (nu, k).
__global__ void k_dJdn_update(const ColDesc* __restrict__ cols, const SolverOpts* bopts) {
  const ColDesc& cd = cols[blockIdx.y];
  if (eval_mode(cd) != EV_BASE || precond_variant(cd, bopts) != 2) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nl = T.nl;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.nq * nz; i += gridDim.x * blockDim.x) {
    const int q = i / nz, k = i - q * nz;
    double beta[kMaxL], gamma[kMaxL];
    for (int j = 0; j < nl; ++j) beta[j] = gamma[j] = 0.0;
    for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
      const int t = T.q_t[s];
      const size_t pk = (size_t)(T.t_base[t] + q - T.t_q0[t]) * nz + k;
      const double V = T.V[pk], gV = T.G[pk] * V;
      beta[T.t_lo[t]] += V;
      beta[T.t_up[t]] -= gV;
      gamma[T.t_up[t]] += T.c2[q] * gV;
    }
    const double Lx = cd.mixed ? (double)cd.w.Lchi32[i] : cd.w.Lchi[i];
    const double Le = cd.mixed ? (double)cd.w.Leta32[i] : cd.w.Leta[i];
    const double sca = T.chi_sca[k];
    double* D = cd.w.dJdn + (size_t)i * nl;
    for (int j = 0; j < nl; ++j) D[j] = beta[j] * Lx + (gamma[j] + sca * D[j]) * Le;
  }
}

static void launch_dJdn_update(const Batch& b, cudaStream_t s) {
  if (!b.has_dJdn) return;
  const long pts = (long)b.max_nq * b.max_nz;
  k_dJdn_update<<<dim3((unsigned)std::min<long>((pts + 255) / 256, 1024), b.ncols), 256, 0, s>>>(
      b.d_cols, b.d_opts);
}

// ---------------------------------------------------------------------------
// a4: per-depth assembly of F (or J_F v) and, in base mode, of P^k; one warp
// per depth: lanes first take transitions (net rates), then levels (F) and
// matrix entries (P), each sum in a fixed order. Solver evaluations also
// LU-factorise P^k in place (lane 0), explicit evaluations leave it as is.
// ---------------------------------------------------------------------------
constexpr int kAsmWarps = 4;

// Tangent evaluations: the directional derivative of F only (no block of the
// preconditioner), one thread per (depth, level) with the level on the grid's
// z axis, so that the per-(transition, depth) rates are read in coalesced
// rows; each level's sum runs over its own transitions in index order, the
// additions of the warp-per-depth kernel.
constexpr int kAsmTanThreads = 128;
__global__ void __launch_bounds__(kAsmTanThreads) k_assemble_tan(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  if (eval_mode(cd) != EV_TANGENT) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nl = T.nl, nt = T.nt;
  const int k = blockIdx.x * kAsmTanThreads + threadIdx.x, l = blockIdx.z;
  if (k >= nz || l >= nl) return;
  const double* n = cd.w.n + (size_t)k * nl;
  const double* v = tangent_dir(cd) + (size_t)k * nl;
  const double* C = T.C + (size_t)k * nl * nl;
  double f = 0.0;
  if (l == cd.w.istar[k]) {
    for (int j = 0; j < nl; ++j) f += v[j];
    f = -f;
  } else {
    const int* inc = T.lvl_inc + l * (nt + 1);
    for (int e = 0; e < nt; ++e) {
      const int m = __ldg(inc + e);
      if (m < 0) break;
      const int t = m >> 1;
      const int lo = __ldg(T.t_lo + t), up = __ldg(T.t_up + t);
      const size_t o = (size_t)t * nz + k;
      const double ur = C[lo * nl + up] + cd.w.Rup[o];
      const double dr = C[up * nl + lo] + cd.w.Rdn[o];
      const double kp = v[lo] * ur + n[lo] * cd.w.dRup[o] - v[up] * dr - n[up] * cd.w.dRdn[o];
      f += (m & 1) ? -kp : kp;
    }
  }
  cd.w.dF[(size_t)k * nl + l] = f;
}

__global__ void __launch_bounds__(32 * kAsmWarps) k_assemble(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode(cd);
  if (mode == EV_SKIP || mode == EV_TANGENT) return;   // k_assemble_tan
  const ColTables& T = cd.t;
  const int nz = T.nz, nl = T.nl, nt = T.nt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int k = blockIdx.x * kAsmWarps + wid;
  if (k >= nz) return;
  __shared__ double s_up[kAsmWarps][kMaxT], s_dn[kAsmWarps][kMaxT], s_kap[kAsmWarps][kMaxT];
  __shared__ double s_P[kAsmWarps][kMaxL * kMaxL];
  const bool fd = (mode == EV_FD);
  const double* n = eval_pops(cd, mode) + k * nl;
  const double* C = T.C + (size_t)k * nl * nl;
  const bool tan = (mode == EV_TANGENT);
  int is;
  if (!tan && !fd) {
    // conservation row at the most populated level (lowest index on ties)
    is = 0;
    for (int l = 1; l < nl; ++l)
      if (n[l] > n[is]) is = l;
    if (lane == 0) cd.w.istar[k] = is;
  } else {
    is = cd.w.istar[k];
  }
  const double* v = tan ? tangent_dir(cd) + k * nl : nullptr;
  for (int t = lane; t < nt; t += 32) {
    const int lo = T.t_lo[t], up = T.t_up[t];
    const size_t o = (size_t)t * nz + k;
    const double ur = C[lo * nl + up] + cd.w.Rup[o];
    const double dr = C[up * nl + lo] + cd.w.Rdn[o];
    if (tan)
      s_kap[wid][t] = v[lo] * ur + n[lo] * cd.w.dRup[o] - v[up] * dr - n[up] * cd.w.dRdn[o];
    else
      s_kap[wid][t] = n[lo] * ur - n[up] * dr;
    s_up[wid][t] = ur;
    s_dn[wid][t] = dr;
  }
  __syncwarp();
  if (lane < nl) {
    // the level's own transitions in index order (the same additions as a scan
    // over every transition, without the FP64 instructions that add nothing)
    double f = 0.0;
    const int* inc = T.lvl_inc + lane * (nt + 1);
    for (int e = 0; e < nt; ++e) {
      const int m = inc[e];
      if (m < 0) break;
      const double kp = s_kap[wid][m >> 1];
      f += (m & 1) ? -kp : kp;
    }
    if (lane == is) {
      double sv = 0.0;
      if (tan) {
        for (int l = 0; l < nl; ++l) sv += v[l];
        f = -sv;
      } else {
        for (int l = 0; l < nl; ++l) sv += n[l];
        f = T.ntot[k] - sv;
      }
    }
    (tan || fd ? cd.w.dF : cd.w.F)[k * nl + lane] = f;
  }
  if (mode != EV_BASE) return;
  // P^k = Gamma^k + A^kk (Sect. 2.5.1), conservation row -1
  for (int e = lane; e < nl * nl; e += 32) {
    const int i = e / nl, j = e - i * nl;
    double pv = 0.0;
    const int* inc = T.lvl_inc + i * (nt + 1);   // the transitions of level i, in index order
    for (int ee = 0; ee < nt; ++ee) {
      const int m = inc[ee];
      if (m < 0) break;
      const int t = m >> 1;
      const int lo = T.t_lo[t], up = T.t_up[t];
      double g = cd.w.Apart[((size_t)t * nz + k) * nl + j];
      if (j == lo) g += s_up[wid][t];
      if (j == up) g -= s_dn[wid][t];
      pv += (m & 1) ? -g : g;   // i is the lower level (+) or the upper one (-)
    }
    s_P[wid][e] = (i == is) ? -1.0 : pv;
  }
  __syncwarp();
  double* P = cd.w.P + (size_t)k * nl * nl;
  if (cd.forced_mode >= 0) {
    for (int e = lane; e < nl * nl; e += 32) P[e] = s_P[wid][e];
    return;
  }
  // explicit inverse of P^k, so that the Krylov step applies P^{-1} as a fully
  // parallel small mat-vec: Gauss-Jordan elimination with partial pivoting on
  // [P | I], lane j owning column j (2 nl <= 32 lanes); every lane finds the
  // same pivot from the same shared data, one reciprocal per column
  __shared__ double s_aug[kAsmWarps][kMaxL * 2 * kMaxL];
  double* G = s_aug[wid];
  const int w2 = 2 * nl;
  for (int e = lane; e < nl * w2; e += 32) {
    const int r = e / w2, j = e - r * w2;
    G[e] = j < nl ? s_P[wid][r * nl + j] : (j - nl == r ? 1.0 : 0.0);
  }
  __syncwarp();
  const bool own = lane < w2;
  for (int c = 0; c < nl; ++c) {
    int pr = c;
    double best = fabs(G[c * w2 + c]);
    for (int r = c + 1; r < nl; ++r) {
      const double vv = fabs(G[r * w2 + c]);
      if (vv > best) { best = vv; pr = r; }
    }
    __syncwarp();   // every lane has read column c before rows move
    if (own && pr != c) {
      const double tmp = G[c * w2 + lane];
      G[c * w2 + lane] = G[pr * w2 + lane];
      G[pr * w2 + lane] = tmp;
    }
    __syncwarp();
    const double rd = 1.0 / G[c * w2 + c];
    double f[kMaxL];
#pragma unroll
    for (int r = 0; r < kMaxL; ++r) f[r] = r < nl ? G[r * w2 + c] : 0.0;
    __syncwarp();   // the pivot row and column are read before they change
    if (own) {
      const double pc = G[c * w2 + lane] * rd;
      G[c * w2 + lane] = pc;
#pragma unroll
      for (int r = 0; r < kMaxL; ++r)
        if (r < nl && r != c) G[r * w2 + lane] = fma(-f[r], pc, G[r * w2 + lane]);
    }
    __syncwarp();
  }
  for (int e = lane; e < nl * nl; e += 32) {
    const int r = e / nl, j = e - r * nl;
    P[e] = G[r * w2 + nl + j];
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Blocks per column of the grid-stride opacity kernel: all the points of a
// column when the batch is small, about 128 blocks per SM in total otherwise
// (only the columns in the launch's evaluation kind work, a fifth or so of a
// large batch in the base-type launch, and their blocks should still fill
// the GPU; the others' blocks return after two loads).
static dim3 opacity_grid(const Batch& b, int tb) {
  const long need = ((long)b.max_nq * b.max_nz + tb - 1) / tb;
  const long share = (128L * b.n_sm + b.ncols - 1) / b.ncols;
  return dim3((unsigned)std::max(1L, std::min(need, share)), b.ncols);
}

// k_opacity_tan32: blocks of 256 frequencies x a run of depths per thread
// (the batch's tuned run, else kOpTanDepths).
static void launch_op_tan(const Batch& b, cudaStream_t s, int depths = 0) {
  const int dr = depths > 0 ? depths : (b.optan_depths > 0 ? b.optan_depths : kOpTanDepths);
  const int nqb = (b.max_nq + 255) / 256, nkc = (b.max_nz + dr - 1) / dr;
  k_opacity_tan32<<<dim3(nqb * nkc, b.ncols), 256, 0, s>>>(b.d_cols, nqb, dr);
}

int launch_opacity_tan(const Batch& b, cudaStream_t s, int depths) {
  launch_op_tan(b, s, depths);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

int launch_opacity_mixed(const Batch& b, cudaStream_t s, int skip_tangent) {
  const int tb = 256;
  k_pop_pairs<<<dim3((b.max_N + tb - 1) / tb, b.ncols), tb, 0, s>>>(b.d_cols);
  k_opacity<float><<<opacity_grid(b, tb), tb, 0, s>>>(b.d_cols, 1);   // base and RH92 columns
  if (!skip_tangent) launch_op_tan(b, s);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

// The assembly: tangent evaluations thread per depth, the others warp per depth.
static void launch_assemble(const Batch& b, cudaStream_t s) {
  k_assemble_tan<<<dim3((b.max_nz + kAsmTanThreads - 1) / kAsmTanThreads, b.ncols, std::max(1, b.max_nl)),
                   kAsmTanThreads, 0, s>>>(b.d_cols);
  k_assemble<<<dim3((b.max_nz + kAsmWarps - 1) / kAsmWarps, b.ncols), 32 * kAsmWarps, 0, s>>>(b.d_cols);
}

static void launch_rates_tan32(const Batch& b, cudaStream_t s) {
  k_rates_tan32<<<dim3((b.max_nz + kRateTanWarps * kRateTanDepths - 1) / (kRateTanWarps * kRateTanDepths),
                       b.max_nt, b.ncols),
                  32 * kRateTanWarps, 0, s>>>(b.d_cols);
}

int launch_evaluation(const Batch& b, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t side,
                      cudaEvent_t ev2, cudaEvent_t ev3, const cudaEvent_t* stage) {
  const int nc = b.ncols;
  if (nc == 0) return JFNK_OK;
  auto mark = [&](int j) -> int {
    if (stage) JFNK_CUDA(cudaEventRecordWithFlags(stage[j], s, cudaEventRecordExternal));
    return JFNK_OK;
  };
  const int tb = 256;
  dim3 g_qk((b.max_nq * b.max_nz + tb - 1) / tb, nc);
  dim3 g_ray((b.max_nq * 2 * b.max_nmu + 63) / 64, nc);
  if (b.formal_kind == FORMAL_SWEEP && side) {
    // Two independent chains over disjoint columns (a column is in one
    // evaluation kind per tick): tangent evaluations (FP32, issue-bound) on the
    // side stream, base and RH92 ones (float-pair sums, latency-bound) on s;
    // joined before the assembly, which reads both.
    JFNK_CUDA(cudaEventRecord(b.fork_ev, s));
    JFNK_CUDA(cudaStreamWaitEvent(side, b.fork_ev, 0));
    k_dir32<<<dim3((b.max_N + tb - 1) / tb, nc), tb, 0, side>>>(b.d_cols);
    if (!sweep_fused(b)) launch_op_tan(b, side);
    if (ev2) JFNK_CUDA(cudaEventRecordWithFlags(ev2, side, cudaEventRecordExternal));
    int rc = launch_formal_sweep(b, side, 2);
    if (rc) return rc;
    if (ev3) JFNK_CUDA(cudaEventRecordWithFlags(ev3, side, cudaEventRecordExternal));
    launch_rates_tan32(b, side);
    JFNK_CUDA(cudaEventRecord(b.join_ev, side));
    k_pop_pairs<<<dim3((b.max_N + tb - 1) / tb, nc), tb, 0, s>>>(b.d_cols);
    k_opacity<float><<<opacity_grid(b, tb), tb, 0, s>>>(b.d_cols, 1);
    if (ev0) JFNK_CUDA(cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal));
    if ((rc = launch_formal_sweep(b, s, 1))) return rc;
    if (ev1) JFNK_CUDA(cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal));
    if ((rc = launch_rates(b, s))) return rc;
    launch_dJdn_update(b, s);
    JFNK_CUDA(cudaStreamWaitEvent(s, b.join_ev, 0));
    launch_assemble(b, s);
    JFNK_CUDA(cudaGetLastError());
    return JFNK_OK;
  }
  if (int rm = mark(0)) return rm;
  if (b.formal_kind == FORMAL_MOVING) {
    // per-ray opacity, formal solution and rate integrals (velocity.cu), then
    // the common assembly
    int rc = launch_moving_evaluation(b, s, ev0, ev1);
    if (rc || (rc = mark(1))) return rc;
    launch_assemble(b, s);
    JFNK_CUDA(cudaGetLastError());
    return mark(2);
  }
  if (b.formal_kind == FORMAL_SWEEP) {
    // (float tangent direction,) opacity, then the per-frequency sweeps; with
    // events (a profiled tick) the tangent sweep is bracketed by ev2/ev3 and
    // the base-type sweep by ev0/ev1, each timed alone on this one stream
    k_dir32<<<dim3((b.max_N + tb - 1) / tb, nc), tb, 0, s>>>(b.d_cols);
    int rc0 = launch_opacity_mixed(b, s, sweep_fused(b) ? 1 : 0);
    if (rc0) return rc0;
    int rc;
    if (ev2) {
      JFNK_CUDA(cudaEventRecordWithFlags(ev2, s, cudaEventRecordExternal));
      if ((rc = launch_formal_sweep(b, s, 2))) return rc;
      if (ev3) JFNK_CUDA(cudaEventRecordWithFlags(ev3, s, cudaEventRecordExternal));
      if (ev0) JFNK_CUDA(cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal));
      if ((rc = launch_formal_sweep(b, s, 1))) return rc;
    } else {
      if (ev0) JFNK_CUDA(cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal));
      if ((rc = launch_formal_sweep(b, s))) return rc;
    }
    if (ev1) JFNK_CUDA(cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal));
  } else if (b.formal_kind == FORMAL_FUSED) {
    // opacity, then the fused formal solution with in-block ray sums
    k_opacity<double><<<opacity_grid(b, tb), tb, 0, s>>>(b.d_cols, 0);
    if (ev0) JFNK_CUDA(cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal));
    int rc = launch_formal_fused(b, s);
    if (rc) return rc;
    if (ev1) JFNK_CUDA(cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal));
  } else {
    k_opacity<double><<<opacity_grid(b, tb), tb, 0, s>>>(b.d_cols, 0);
    k_source_diff<double><<<g_qk, tb, 0, s>>>(b.d_cols);
    if (ev0) JFNK_CUDA(cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal));
    k_formal<double><<<g_ray, 64, 0, s>>>(b.d_cols);
    if (ev1) JFNK_CUDA(cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal));
    k_ray_sum<double><<<g_qk, tb, 0, s>>>(b.d_cols);
  }
  {
    int rc = launch_rates(b, s);
    if (rc) return rc;
    launch_dJdn_update(b, s);
    if (b.mixed) launch_rates_tan32(b, s);
    if ((rc = mark(1))) return rc;
  }
  launch_assemble(b, s);
  JFNK_CUDA(cudaGetLastError());
  return mark(2);
}


}  // namespace jfnk
