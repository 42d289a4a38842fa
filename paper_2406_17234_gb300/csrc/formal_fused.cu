// Fused formal solution + ray sums (steps a2 and the angle integral of a3),
// one block per (block of Qb frequencies, column).
//
// Everything transcendental in the piecewise-linear recurrence (App. A.1:
// exp(-dtau), w, a, b/dtau, and the tangent and preconditioner coefficients of
// App. A.2) depends on the opacities only, never on the intensity. So the
// block first computes those coefficients for every (depth, ray) pair in
// parallel into shared memory (phase A); one thread per ray then runs the
// sequential recurrence, which is a fused multiply-add per step (phase B);
// finally the rays are summed per (frequency, depth) in shared memory into
// J, dJ, Lambda_chi and Lambda_eta (phase C). No per-ray array reaches
// global memory.
//
// The recurrences (exactly those of Eqs. Iplus/Iminus, rewritten):
//   D = I - S:  D^k = D^u e + w (S^u - S^k)                   (all modes)
//   tangent:    dD^k = dD^u e - ddtau (e D^u + bq (S^u - S^k)) + w (dS^u - dS^k)
//   base:       I^k = I^u e + a S^k + b S^u ;  dI^k/dchi^k = hw-scaled a_chi
//               with S^u - I^u = -D^u ; dI^k/deta^k = a / chi^k
// where u is the upstream depth (k+1 for mu > 0, k-1 for mu < 0).
#include "formal_coef.cuh"

namespace jfnk {

constexpr int kFusedThreads = 256;
constexpr int kFusedSlots = 5;   // E, X(D), P1(dD coef | I), P2(dD | LX), LE
constexpr int kFusedStage = 7;   // chi, S, dS, dchi, ddS, two layer factors per (q, k)

__host__ __device__ inline size_t round16(size_t bytes) { return (bytes + 15) / 16 * 16; }

// Slot row stride: the rays of the block, padded to an odd count so that
// threads walking depths (phase C) hit distinct shared-memory banks.
__host__ __device__ inline int slot_stride(int qb, int nmu) {
  const int r = qb * 2 * nmu;
  return r | 1;
}

size_t fused_smem_bytes(int qb, int nz, int nmu, bool mixed) {
  const size_t rs = mixed ? 4 : 8;
  const size_t stage = round16(rs * ((size_t)kFusedStage * qb * nz + qb + 2 * nz + 4 * kMaxMu));
  const size_t slots = rs * (size_t)kFusedSlots * nz * slot_stride(qb, nmu);
  return stage + slots;
}

template <typename real>
__global__ void __launch_bounds__(kFusedThreads) k_formal_fused(const ColDesc* __restrict__ cols, int Qb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode_f(cd);
  if (mode == EV_SKIP) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq, nmu = T.nmu, nr = 2 * nmu;
  const int qb0 = blockIdx.x * Qb;
  if (qb0 >= nq) return;
  const int nqb = min(Qb, nq - qb0);
  const int R = slot_stride(Qb, nmu);
  const int nray = nqb * nr;
  const bool tan = (mode == EV_TANGENT);
  const bool der = (mode == EV_BASE || mode == EV_RH92);
  real* st = reinterpret_cast<real*>(smem_raw);
  real* s_chi = st;
  real* s_S = s_chi + Qb * nz;
  real* s_dS = s_S + Qb * nz;
  real* s_dchi = s_dS + Qb * nz;
  real* s_ddS = s_dchi + Qb * nz;
  real* s_rs = s_ddS + Qb * nz;   // layer k: 1/(|dz| (chi^k + chi^{k+1}))
  real* s_tz = s_rs + Qb * nz;    // layer k: |dz| (chi^k + chi^{k+1})
  real* s_Bb = s_tz + Qb * nz;
  real* s_dz = s_Bb + Qb + nz;    // |z_k - z_{k+1}| (one spare row of nz before it)
  real* s_mu = s_dz + nz;         // per angle: 1/(2 mu), 1/2 w_mu, 2 mu
  real* slot = reinterpret_cast<real*>(smem_raw + round16(sizeof(real) * ((size_t)kFusedStage * Qb * nz + Qb + 2 * nz + 4 * kMaxMu)));
  const size_t plane = (size_t)nz * R;
  real* E = slot;
  real* X = E + plane;
  real* P1 = X + plane;    // tangent: -ddtau e        | base: a S^k + b S^u, then hw I
  real* P2 = P1 + plane;   // tangent: coefficient, then hw dD | base: LX constant, then hw dI/dchi
  real* LE = P2 + plane;   // base: hw dI/deta
  const real* chi_g = reinterpret_cast<const real*>(cd.w.chi);
  const real* dchi_g = reinterpret_cast<const real*>(cd.w.dchi);
  const double* S64 = cd.w.S;
  const double* dS64 = cd.w.dS;

  // phase 0: stage the block's opacities and source-function differences
  for (int i = threadIdx.x; i < nqb * nz; i += blockDim.x) {
    const int ql = i / nz, k = i - ql * nz;
    const size_t o = (size_t)(qb0 + ql) * nz + k;
    s_chi[i] = chi_g[o];
    if (k < nz - 1) {   // layer factors shared by the 2 n_mu rays of the layer
      const real t = (real)T.dz[k] * (chi_g[o] + chi_g[o + 1]);
      s_tz[i] = t;
      s_rs[i] = (real)1 / t;
    }
    s_S[i] = (real)S64[o];
    s_dS[i] = (k < nz - 1) ? (real)(S64[o + 1] - S64[o]) : (real)0;   // formed in FP64
    if (tan) {
      // layer k: |dz| (dchi^k + dchi^{k+1}), so that ddtau = this / (2 mu)
      s_dchi[i] = (k < nz - 1) ? (real)T.dz[k] * (dchi_g[o] + dchi_g[o + 1]) : (real)0;
      s_ddS[i] = (k < nz - 1) ? (real)(dS64[o + 1] - dS64[o]) : (real)0;
    } else {
      s_dchi[i] = (real)1 / chi_g[o];   // base evaluations: 1/chi^k, shared by the 2 n_mu rays
    }
  }
  for (int ql = threadIdx.x; ql < nqb; ql += blockDim.x) {
    const int q = qb0 + ql;
    s_Bb[ql] = (real)(T.Bn[(size_t)q * nz + nz - 1] / T.c2[q]);
  }
  for (int k = threadIdx.x; k < nz - 1; k += blockDim.x) {
    s_dz[k] = (real)T.dz[k];
  }
  for (int m = threadIdx.x; m < nmu; m += blockDim.x) {
    s_mu[3 * m] = (real)(0.5 / T.mu[m]);
    s_mu[3 * m + 1] = (real)(0.5 * T.wmu[m]);
    s_mu[3 * m + 2] = (real)(2.0 * T.mu[m]);
  }
  __syncthreads();

  // phase A: coefficients of every (depth, ray) step, in parallel; each
  // thread keeps one ray and strides over depths (no index division in the loop)
  const int klanes = blockDim.x / nray;
  if ((int)threadIdx.x < klanes * nray) {
    const int ray = threadIdx.x % nray;
    const int kl = threadIdx.x / nray;
    const int ql = ray / nr, rr = ray - ql * nr;
    const bool up = rr < nmu;
    const int m = up ? rr : rr - nmu;
    const real inv2mu = s_mu[3 * m];
    const real hw = s_mu[3 * m + 1];
    const real two_mu = s_mu[3 * m + 2];
    const real* ch = s_chi + ql * nz;
    const real* rs = s_rs + ql * nz;
    const real* tz = s_tz + ql * nz;
    const real* dSq = s_dS + ql * nz;
    const int kbeg = up ? 0 : 1, kend = up ? nz - 1 : nz;   // steps into depth k
    for (int k = kbeg + kl; k < kend; k += klanes) {
      const int ku = up ? k + 1 : k - 1;
      const int kd = up ? k : k - 1;
      const real c0 = ch[k];
      const real h = s_dz[kd] * inv2mu;
      // dtau = |dz| (chi^k + chi^u) / (2 mu), 1/dtau = 2 mu / (|dz| (chi^k + chi^u)):
      // the layer's factors are staged once for its 2 n_mu rays
      const real dtau = tz[kd] * inv2mu;
      const real rdt = rs[kd] * two_mu;
      real e, w, a, bq;
      pl_coef_f(dtau, rdt, e, w, a, bq);
      const real dSin = up ? dSq[k] : -dSq[k - 1];
      const size_t si = (size_t)k * R + ray;
      E[si] = e;
      X[si] = w * dSin;
      if (tan) {
        const real ddtau = s_dchi[ql * nz + kd] * inv2mu;
        const real ddSin = up ? s_ddS[ql * nz + k] : -s_ddS[ql * nz + k - 1];
        P1[si] = -ddtau * e;
        P2[si] = -ddtau * bq * dSin + w * ddSin;
      } else if (der) {
        const real S0 = s_S[ql * nz + k], Su = s_S[ql * nz + ku];
        P1[si] = a * S0 + bq * dtau * Su;
        const real rc0 = s_dchi[ql * nz + k];   // 1/chi^k (base evaluations)
        P2[si] = hw * (-(S0 * rc0) * a - h * dSin * bq);
        LE[si] = hw * (a * rc0);
      }
    }
  }
  __syncthreads();

  // phase B: the sequential recurrence, one thread per ray
  for (int ray = threadIdx.x; ray < nray; ray += blockDim.x) {
    const int ql = ray / nr, rr = ray - ql * nr;
    const bool up = rr < nmu;
    const int m = up ? rr : rr - nmu;
    const int q = qb0 + ql;
    const real hw = s_mu[3 * m + 1];
    const int k0 = up ? nz - 1 : 0;
    const int step = up ? -1 : 1;
    const size_t o0 = (size_t)q * nz + k0;
    real D = up ? (real)(T.Bn[(size_t)q * nz + nz - 1] / T.c2[q] - S64[o0]) : (real)(-S64[o0]);
    real dD = tan ? (real)(-dS64[o0]) : (real)0;
    real I = up ? s_Bb[ql] : (real)0;
    size_t si = (size_t)k0 * R + ray;
    X[si] = hw * D;
    if (tan) P2[si] = hw * dD;
    if (der) { P1[si] = hw * I; P2[si] = 0; LE[si] = 0; }
    // In base evaluations D is re-anchored on I - S whenever that is the
    // better-conditioned value: D carries an absolute error of the order of
    // the largest |D| met upstream (attenuated along the ray), I - S one of
    // the order of |I| + |S|.
    real M = D < (real)0 ? -D : D;
#pragma unroll 4
    for (int s = 1; s < nz; ++s) {
      const int k = k0 + step * s;
      si = (size_t)k * R + ray;
      const real e = E[si];
      real Dn = D * e + X[si];
      if (tan) {
        const real dDn = dD * e + P1[si] * D + P2[si];
        P2[si] = hw * dDn;
        dD = dDn;
      } else if (der) {
        I = I * e + P1[si];
        P1[si] = hw * I;
        // dI^k/dchi^k: its slope on the upstream D is -hw h e (App. A.2)
        const int kd = up ? k : k - 1;
        P2[si] = P2[si] - hw * (s_dz[kd] * s_mu[3 * m]) * e * D;
        const real Sk = s_S[ql * nz + k];
        const real aD = Dn < (real)0 ? -Dn : Dn;
        M = fmax(M * e, aD);
        const real anchor = (I < (real)0 ? -I : I) + (Sk < (real)0 ? -Sk : Sk);
        if (anchor < M) {
          Dn = I - Sk;
          M = anchor;
        }
      }
      D = Dn;
      X[si] = hw * D;
    }
    if (up && der) cd.w.Iem[(size_t)q * nmu + m] = (double)I * T.c2[q];
  }
  __syncthreads();

  // phase C: sums over the rays of each (frequency, depth)
  double* Jout = cd.w.J;
  for (int i = threadIdx.x; i < nqb * nz; i += blockDim.x) {
    const int ql = i / nz, k = i - ql * nz;
    const int q = qb0 + ql;
    const size_t o = (size_t)q * nz + k;
    const size_t b0 = (size_t)k * R + ql * nr;
    const double c2 = T.c2[q];
    // ray sums in the working precision; only J = S + sum carries FP64
    real sD = 0, sa = 0;
    for (int rr = 0; rr < nr; ++rr) {
      const real v = X[b0 + rr];
      sD += v;
      sa += (v < (real)0 ? -v : v);
    }
    double J = (S64[o] + (double)sD) * c2;
    if (tan) {
      real sd = 0;
      for (int rr = 0; rr < nr; ++rr) sd += P2[b0 + rr];
      cd.w.dJ[o] = (dS64[o] + (double)sd) * c2;
    } else if (der) {
      real sI = 0, sx = 0, se = 0;
      for (int rr = 0; rr < nr; ++rr) {
        sI += P1[b0 + rr];
        sx += P2[b0 + rr];
        se += LE[b0 + rr];
      }
      // the representation with the smaller rounding error (intensities are >= 0)
      if ((sI < (real)0 ? -sI : sI) < sa) J = (double)sI * c2;
      jnew_ptr(cd)[o] = J;   // base and RH92 rates read J here
      cd.w.Lchi[o] = (double)sx * c2;
      cd.w.Leta[o] = (double)se;
    } else {
      Jout[o] = J;           // finite-difference evaluation
    }
  }
}

int fused_prepare(Batch* b) {
  if (b->formal_qb <= 0) return JFNK_OK;
  if (b->formal_threads <= 0) b->formal_threads = kFusedThreads;
  const size_t bytes = fused_smem_bytes(b->formal_qb, b->max_nz, b->max_nmu, b->mixed != 0);
  JFNK_CUDA(cudaFuncSetAttribute(k_formal_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return JFNK_OK;
}

static int launch_fused_cfg(const Batch& b, cudaStream_t s, int qb, int threads) {
  const size_t bytes = fused_smem_bytes(qb, b.max_nz, b.max_nmu, b.mixed != 0);
  dim3 g((b.max_nq + qb - 1) / qb, b.ncols);
  k_formal_fused<double><<<g, threads, bytes, s>>>(b.d_cols, qb);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

int launch_formal_fused(const Batch& b, cudaStream_t s) {
  return launch_fused_cfg(b, s, b.formal_qb, b.formal_threads);
}

// Autotuner: times the fused kernel in tangent mode (the bulk of a solve) on
// the batch's own columns for every (frequencies per block, threads per block)
// pair that fits, and keeps the fastest. Requires the columns' base evaluation
// buffers to be filled (chi, S) and a direction in w.v.
int fused_autotune(Batch* b, cudaStream_t s) {
  if (b->formal_qb <= 0) return JFNK_OK;
  const size_t cap = 227 * 1024;
  cudaEvent_t e0, e1;
  JFNK_CUDA(cudaEventCreate(&e0));
  JFNK_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bq = b->formal_qb, bt = b->formal_threads;
  for (int qb : {1, 2, 4, 8}) {
    const size_t bytes = fused_smem_bytes(qb, b->max_nz, b->max_nmu, b->mixed != 0);
    if (bytes > cap) continue;
    const int nray = qb * 2 * b->max_nmu;
    for (int threads : {64, 128, 256}) {
      if (threads < nray) continue;
      JFNK_CUDA(cudaFuncSetAttribute(k_formal_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      int rc = launch_fused_cfg(*b, s, qb, threads);   // warm-up
      if (rc) return rc;
      JFNK_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r)
        if ((rc = launch_fused_cfg(*b, s, qb, threads))) return rc;
      JFNK_CUDA(cudaEventRecord(e1, s));
      JFNK_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      JFNK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; bq = qb; bt = threads; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->formal_qb = bq;
  b->formal_threads = bt;
  return fused_prepare(b);
}

// Largest frequency block whose shared memory still lets two blocks share an SM
// (0 when even one frequency does not fit: the unfused kernels are used).
int fused_default_qb(int max_nz, int max_nmu, bool mixed) {
  const size_t cap = 227 * 1024;
  for (int qb : {8, 4, 2, 1})
    if (2 * fused_smem_bytes(qb, max_nz, max_nmu, mixed) <= cap) return qb;
  if (fused_smem_bytes(1, max_nz, max_nmu, mixed) <= cap) return 1;
  return 0;
}

}  // namespace jfnk
