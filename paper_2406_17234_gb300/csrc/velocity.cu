// Moving columns (a line-of-sight velocity field, Sect. 3.4): each direction
// of propagation sees its own Doppler-shifted line profile, so opacity and
// source function are per direction rather than shared by the rays of a
// frequency, the formal solution runs per ray with them, and the rate
// integrals weight every ray's intensity with the profile that ray sees:
//
//   chi_d = chi_c + chi_sca + sum_t V_t,d (n_lo - g n_up),
//   eta_d = eta_c + chi_sca J^dagger + sum_t (2 h nu^3/c^2) g V_t,d n_up,
//   R_ij = sum_nu W sum_d h_d V_t,d I_d,  R_ji = sum_nu W g sum_d h_d V_t,d (2 h nu^3/c^2 + I_d),
//   J = sum_d h_d I_d (for the background scattering), h_d = w_mu/2,
//
// with W = omega_t(nu) 4 pi/(h nu). The block-Jacobi blocks (first solution
// of Sect. 2.5.2) take per ray the local derivatives dI^k/dchi^k and
// dI^k/deta^k of App. A.2 with that ray's beta and gamma. FP64 throughout; the
// per-ray intensities, their tangents and local derivatives are stored
// ([2 n_mu][nq][nz] each), the assembly and the Krylov/Newton step are the
// static path's.
#include <cooperative_groups.h>

#include "formal_coef.cuh"

namespace jfnk {

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ int mv_mode(const ColDesc& cd) {
  if (cd.forced_mode >= 0) return cd.forced_mode;
  switch (cd.w.st->phase) {
    case PH_BASE: return EV_BASE;
    case PH_JVP:
    case PH_RESTART: return cd.w.st->fd_scheme ? EV_FD : EV_TANGENT;
    default: return EV_SKIP;   // RH92 is not defined here (rejected at the API)
  }
}

__device__ __forceinline__ const double* mv_dir(const ColDesc& cd) {
  if (cd.forced_mode >= 0) return cd.w.v;
  const int N = cd.t.nz * cd.t.nl;
  return cd.w.st->phase == PH_RESTART ? cd.w.x : cd.w.Vb + (size_t)cd.w.st->j * N;
}

// h_d = w_mu/2 of direction d (outgoing mu_1..mu_n, then ingoing)
__device__ __forceinline__ double mv_h(const ColTables& T, int d) {
  return 0.5 * T.wmu[d < T.nmu ? d : d - T.nmu];
}

}  // namespace

// Opacity and source function (or their tangents) of every (direction, nu, depth).
__global__ void k_mv_opacity(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = mv_mode(cd);
  if (mode == EV_SKIP) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq, nl = T.nl, nd = 2 * T.nmu;
  const size_t per = (size_t)nq * nz;
  const double* n = eval_pops(cd, mode);
  const double* v = mode == EV_TANGENT ? mv_dir(cd) : nullptr;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd * per; i += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / per);
    const size_t qk = i - (size_t)d * per;
    const int q = (int)(qk / nz), k = (int)(qk - (size_t)q * nz);
    const double* Vd = T.Vd + (size_t)d * T.nwin * nz;
    double a = 0.0, e = 0.0;   // sum V (x_lo - g x_up), sum (2 h nu^3/c^2) g V x_up
    const double* x = (mode == EV_TANGENT ? v : n) + (size_t)k * nl;
    for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
      const int t = T.q_t[s];
      const size_t pk = (size_t)(T.t_base[t] + q - T.t_q0[t]) * nz + k;
      const double V = Vd[pk], gV = T.G[pk] * V;
      a += V * x[T.t_lo[t]] - gV * x[T.t_up[t]];
      e += gV * x[T.t_up[t]];
    }
    e *= T.c2[q];
    if (mode == EV_TANGENT) {
      // tangent at the base point (J^dagger is not perturbed)
      const double chi = cd.w.mchi[i], S = cd.w.mS[i];
      cd.w.mdchi[i] = a;
      cd.w.mdS[i] = (e - S * a) / chi;
    } else {
      const double chi = T.chi_c[qk] + T.chi_sca[k] + a;
      const double eta = T.eta_c[qk] + T.chi_sca[k] * jdag_ptr(cd)[qk] + e;
      cd.w.mchi[i] = chi;
      cd.w.mS[i] = eta / chi;
    }
  }
}

// Formal solution of every ray (Eqs. Iplus/Iminus with the App. A.1
// coefficients; I = B_nu(T_bottom) entering at the bottom, 0 at the top), one
// thread per (direction, nu): the intensity form of the recurrence,
//   I^k = I^u e + a S^k + b S^u,  dtau = h (chi^k + chi^u), h = |dz|/(2 mu),
// and in base evaluations the local derivatives of App. A.2,
//   dI^k/dchi^k = -(S^k/chi^k) a + h (e (S^u - I^u) - (S^u - S^k) b/dtau),  dI^k/deta^k = a/chi^k,
// or in tangent evaluations the differentiated recurrence (de = -e ddtau,
// da = (b/dtau) ddtau, db = (e - b/dtau) ddtau, ddtau = h (dchi^k + dchi^u)).
__global__ void k_mv_formal(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = mv_mode(cd);
  if (mode == EV_SKIP) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq, nmu = T.nmu;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 2 * nmu * nq) return;
  const int d = r / nq, q = r - d * nq;
  const bool up = d < nmu;
  const double mu = T.mu[up ? d : d - nmu];
  const size_t row = ((size_t)d * nq + q) * nz;
  const double* chi = cd.w.mchi + row;
  const double* S = cd.w.mS + row;
  const bool tan = (mode == EV_TANGENT), base = (mode == EV_BASE);
  const double* dchi = tan ? cd.w.mdchi + row : nullptr;
  const double* dS = tan ? cd.w.mdS + row : nullptr;
  const double* Ib = cd.w.mI + row;   // the base point's intensities (tangent evaluations)
  double* Iout = tan ? cd.w.mdI + row : cd.w.mI + row;
  const int k0 = up ? nz - 1 : 0, step = up ? -1 : 1;
  double I = up ? T.Bn[(size_t)q * nz + nz - 1] : 0.0;   // boundary values (dI = 0 there)
  if (tan) I = 0.0;
  Iout[k0] = I;
  if (base) {
    cd.w.mLX[row + k0] = 0.0;
    cd.w.mLE[row + k0] = 0.0;
  }
  for (int k = k0 + step; k >= 0 && k < nz; k += step) {
    const int u = k - step;
    const double h = T.dz[up ? k : k - 1] / (2.0 * mu);
    const double dtau = h * (chi[k] + chi[u]);
    double e, w, a, bq;
    pl_coef_f(dtau, 1.0 / dtau, e, w, a, bq);
    const double b = bq * dtau;
    if (tan) {
      const double ddtau = h * (dchi[k] + dchi[u]);
      I = I * e - Ib[u] * e * ddtau + a * dS[k] + bq * ddtau * S[k] + b * dS[u] + (e - bq) * ddtau * S[u];
    } else {
      const double Iu = I;
      I = Iu * e + a * S[k] + b * S[u];
      if (base) {
        cd.w.mLX[row + k] = -(S[k] / chi[k]) * a + h * (e * (S[u] - Iu) - (S[u] - S[k]) * bq);
        cd.w.mLE[row + k] = a / chi[k];
      }
    }
    Iout[k] = I;
  }
  if (base && up) cd.w.Iem[(size_t)q * nmu + d] = I;   // the outgoing intensity at the top
}

// J = sum_d h_d I_d of a base evaluation, written into J_new.
__global__ void k_mv_moments(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  if (mv_mode(cd) != EV_BASE) return;
  const ColTables& T = cd.t;
  const size_t per = (size_t)T.nq * T.nz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per) return;
  double J = 0.0;
  for (int d = 0; d < 2 * T.nmu; ++d) J += mv_h(T, d) * cd.w.mI[(size_t)d * per + i];
  jnew_ptr(cd)[i] = J;
}

// Rate integrals of transition t at depth k: R_ij, R_ji from the rays'
// intensities (their tangents in tangent evaluations) and, in base
// evaluations, the block-Jacobi sums A_tj = sum_nu W sum_d h_d chi_t,d
// (beta_j,d dI_d/dchi_d + gamma_j,d dI_d/deta_d). A cluster of kMvRateSplit
// blocks takes one transition and 32 depths (lanes: coalesced rows of the
// tables and of the ray arrays); its blocks split the frequency window into
// chunks and their warps stride through a chunk, so that even one column
// spreads its FP64 sums over the GPU; the partial sums are added in warp
// order, then in rank order through distributed shared memory.
constexpr int kMvRateWarps = 4;
constexpr int kMvRateSplit = 8;   // blocks of a cluster splitting the frequency window

__global__ void __launch_bounds__(32 * kMvRateWarps) k_mv_rates(const ColDesc* __restrict__ cols) {
  cg::cluster_group cluster = cg::this_cluster();
  const int split = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int tile = blockIdx.x / split;
  const ColDesc& cd = cols[blockIdx.z];
  const int mode = mv_mode(cd);
  const ColTables& T = cd.t;
  const int t = blockIdx.y;
  const int nz = T.nz, nq = T.nq, nl = T.nl, nd = 2 * T.nmu;
  // uniform over the cluster (its blocks differ only in their frequency chunk)
  if (mode == EV_SKIP || t >= T.nt || tile * 32 >= nz) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int k = min(tile * 32 + lane, nz - 1);
  const bool tan = (mode == EV_TANGENT), base = (mode == EV_BASE);
  const int q0 = T.t_q0[t], q1 = T.t_q1[t], wb = T.t_base[t];
  const int nw = q1 - q0 + 1;
  const int qa = q0 + (int)(((long)nw * rank) / split), qb = q0 + (int)(((long)nw * (rank + 1)) / split) - 1;
  const double* n = eval_pops(cd, mode) + (size_t)k * nl;
  const double nlo = n[T.t_lo[t]], nup = n[T.t_up[t]];
  const size_t per = (size_t)nq * nz, vper = (size_t)T.nwin * nz;
  const double* Iray = tan ? cd.w.mdI : cd.w.mI;
  // per-lane sums: [0] R_up, [1] R_dn, [2 + j] the preconditioner's A_j (base)
  __shared__ double s_part[kMvRateWarps][2 + kMaxL][32];
  if (base)
    for (int j = 0; j < nl; ++j) s_part[wid][2 + j][lane] = 0.0;
  double ru = 0.0, rd = 0.0;
  for (int q = qa + wid; q <= qb; q += kMvRateWarps) {
    const int p = wb + q - q0;
    const size_t pk = (size_t)p * nz + k, qk = (size_t)q * nz + k;
    const double W = T.t_w[p] * T.rw[q], g = T.G[pk], c2 = T.c2[q];
    double su = 0.0, sd = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double hv = mv_h(T, d) * T.Vd[(size_t)d * vper + pk];
      const double Id = Iray[(size_t)d * per + qk];
      su += hv * Id;
      sd += hv * (tan ? Id : c2 + Id);
      if (base) {
        // chi_t,d W h_d times beta_j,d dI/dchi + gamma_j,d dI/deta over the
        // transitions active at nu
        const double c = W * hv * (nlo - g * nup);
        const double lx = cd.w.mLX[(size_t)d * per + qk], le = cd.w.mLE[(size_t)d * per + qk];
        for (int s = T.q_off[q]; s < T.q_off[q + 1]; ++s) {
          const int ts = T.q_t[s];
          const size_t ps = (size_t)(T.t_base[ts] + q - T.t_q0[ts]) * nz + k;
          const double Vs = T.Vd[(size_t)d * vper + ps], gVs = T.G[ps] * Vs;
          s_part[wid][2 + T.t_lo[ts]][lane] += c * (Vs * lx);
          s_part[wid][2 + T.t_up[ts]][lane] += c * (-gVs * lx + c2 * gVs * le);
        }
      }
    }
    ru += W * su;
    rd += W * g * sd;
  }
  s_part[wid][0][lane] = ru;
  s_part[wid][1][lane] = rd;
  __syncthreads();
  // the block's warps in warp order, then the cluster's blocks in rank order
  const int nacc = base ? 2 + nl : 2;
  if (wid == 0)
    for (int j = 0; j < nacc; ++j) {
      double v = s_part[0][j][lane];
      for (int w = 1; w < kMvRateWarps; ++w) v += s_part[w][j][lane];
      s_part[0][j][lane] = v;
    }
  cluster.sync();
  if (rank == 0 && wid == 0 && tile * 32 + lane < nz) {
    double acc[2 + kMaxL];
    for (int j = 0; j < nacc; ++j) acc[j] = s_part[0][j][lane];
    for (int r = 1; r < split; ++r) {
      const double* peer = cluster.map_shared_rank(&s_part[0][0][0], r);
      for (int j = 0; j < nacc; ++j) acc[j] += peer[j * 32 + lane];
    }
    const size_t o = (size_t)t * nz + k;
    if (tan) {
      cd.w.dRup[o] = acc[0];
      cd.w.dRdn[o] = acc[1];
    } else {
      cd.w.Rup[o] = acc[0];
      cd.w.Rdn[o] = acc[1];
      if (base)
        for (int j = 0; j < nl; ++j) cd.w.Apart[o * nl + j] = acc[2 + j];
    }
  }
  cluster.sync();   // peers keep their shared memory until rank 0 has read it
}

int launch_moving_evaluation(const Batch& b, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  const int nc = b.ncols;
  const long pts = 2L * b.max_nmu * b.max_nq * b.max_nz;
  const int tb = 256;
  k_mv_opacity<<<dim3((unsigned)std::min<long>((pts + tb - 1) / tb, 4096), nc), tb, 0, s>>>(b.d_cols);
  if (ev0) JFNK_CUDA(cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal));
  k_mv_formal<<<dim3((2 * b.max_nmu * b.max_nq + 127) / 128, nc), 128, 0, s>>>(b.d_cols);
  if (ev1) JFNK_CUDA(cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal));
  k_mv_moments<<<dim3((b.max_nq * b.max_nz + tb - 1) / tb, nc), tb, 0, s>>>(b.d_cols);
  {
    // clusters of kMvRateSplit blocks along x split each transition's window
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(((b.max_nz + 31) / 32) * kMvRateSplit, b.max_nt, nc);
    cfg.blockDim = dim3(32 * kMvRateWarps);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kMvRateSplit;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    JFNK_CUDA(cudaLaunchKernelEx(&cfg, k_mv_rates, (const ColDesc*)b.d_cols));
  }
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

}  // namespace jfnk
