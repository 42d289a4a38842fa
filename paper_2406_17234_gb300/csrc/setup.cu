// Setup of atoms and columns (Sect. 2.1.1; step a0 of the hot path): the
// union frequency grid with per-transition windows and quadrature weights
// (host), and the depth-dependent tables (device kernels): LTE populations,
// Voigt profiles, bound-free cross-sections and g_ij, Planck functions,
// background continuum and collision rates.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace jfnk {

// ---------------------------------------------------------------------------
// Voigt function H(a, v) = Re w(v + i a), w the Faddeeva function, by the
// rational expansion of Weideman (1994, SIAM J. Numer. Anal. 31, 1497):
// with t = L tan(theta/2), exp(-t^2)(L^2 + t^2) = sum_n c_n e^{i n theta}, and
// w(z) = 2/(L - iz)^2 sum_{n=0}^{N-1} c_{n+1} Z^n + 1/(sqrt(pi)(L - iz)),
// Z = (L + iz)/(L - iz), valid for Im z >= 0. The c_n are Fourier coefficients
// of a smooth periodic function, computed here on the host by the trapezoid
// rule (spectrally accurate) and uploaded once.
// ---------------------------------------------------------------------------
constexpr int kVoigtN = 40;
__constant__ double c_voigt[kVoigtN + 1];
__constant__ double c_voigt_L;

static void voigt_coefficients(double* coef, double* Lout) {
  const int N = kVoigtN;
  const double L = std::sqrt(N / std::sqrt(2.0));
  const int M = 8 * N;   // trapezoid points on [-pi, pi)
  for (int n = 0; n <= N; ++n) {
    double s = 0.0;
    for (int k = -M / 2 + 1; k < M / 2; ++k) {   // theta = +-pi contributes 0
      double th = 2.0 * kPi * k / M;
      double t = L * std::tan(0.5 * th);
      double f = std::exp(-t * t) * (L * L + t * t);
      s += f * std::cos(n * th);
    }
    coef[n] = s / M;
  }
  *Lout = L;
}

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

__device__ double voigt_H(double a, double v) {
  if (a == 0.0) return exp(-v * v);
  const double L = c_voigt_L;
  // z = v + i a; L - i z = (L + a) - i v; L + i z = (L - a) + i v
  cplx lm = {L + a, -v};
  cplx lp = {L - a, v};
  cplx Z = cdiv(lp, lm);
  cplx p = {c_voigt[kVoigtN], 0.0};
  for (int n = kVoigtN - 1; n >= 1; --n) {   // sum_{n=0}^{N-1} c_{n+1} Z^n by Horner
    p = cmul(p, Z);
    p.re += c_voigt[n];
  }
  cplx lm2 = cmul(lm, lm);
  cplx t1 = cdiv(p, lm2);
  cplx t2 = cdiv({1.0 / 1.7724538509055160273, 0.0}, lm);
  return 2.0 * t1.re + t2.re;
}

// ---------------------------------------------------------------------------
// Host: atom grids
// ---------------------------------------------------------------------------
static std::vector<double> line_offsets(int n, double q_core, double q_wing) {
  std::vector<double> x(n);
  for (int s = 0; s < n; ++s) {
    double u = 2.0 * s / (n - 1) - 1.0;
    if (q_wing <= 2.0 * q_core) {
      x[s] = q_wing * u;
    } else {
      double beta = 2.0 * std::acosh(q_wing / (2.0 * q_core));
      x[s] = q_wing * std::sinh(beta * u) / std::sinh(beta);
    }
  }
  return x;
}

int build_atom(const jfnk_atom_desc* d, AtomData* A) {
  if (!d) return fail(JFNK_E_INVALID, "atom descriptor is NULL");
  const int nl = d->n_levels;
  if (nl < 2 || nl > kMaxL) return fail(JFNK_E_INVALID, "n_levels must be in [2, 16]");
  if (!d->E_eV || !d->g || !d->stage) return fail(JFNK_E_INVALID, "level arrays are NULL");
  if (d->n_bb < 0 || d->n_bf < 0 || d->n_bb + d->n_bf < 1)
    return fail(JFNK_E_INVALID, "an atom needs at least one transition");
  if ((d->n_bb > 0 && !d->bb) || (d->n_bf > 0 && !d->bf))
    return fail(JFNK_E_INVALID, "transition arrays are NULL");
  if (!(d->mass_amu > 0.0) || !(d->vchar > 0.0))
    return fail(JFNK_E_INVALID, "mass_amu and vchar must be positive");
  A->nl = nl;
  A->E.assign(d->E_eV, d->E_eV + nl);
  A->g.assign(d->g, d->g + nl);
  A->stage.assign(d->stage, d->stage + nl);
  for (int l = 0; l < nl; ++l)
    if (!(A->g[l] > 0.0) || !std::isfinite(A->E[l]))
      return fail(JFNK_E_INVALID, "level weights must be positive and energies finite");
  A->mass = d->mass_amu;
  A->vchar = d->vchar;
  A->bb.assign(d->bb, d->bb + d->n_bb);
  A->bf.assign(d->bf, d->bf + d->n_bf);
  std::vector<std::vector<double>> grids;
  A->t_lo.clear(); A->t_up.clear(); A->t_kind.clear(); A->t_nu0.clear(); A->t_idx.clear();
  for (int b = 0; b < d->n_bb; ++b) {
    const jfnk_bb_desc& L = d->bb[b];
    if (L.i < 0 || L.j >= nl || L.i >= L.j) return fail(JFNK_E_INVALID, "bb levels must satisfy 0 <= i < j < n_levels");
    if (!(A->E[L.j] > A->E[L.i])) return fail(JFNK_E_INVALID, "bb upper level must lie above the lower");
    if (A->stage[L.j] != A->stage[L.i]) return fail(JFNK_E_INVALID, "bb levels must share a stage");
    if (L.n_nu < 3 || L.n_nu % 2 == 0) return fail(JFNK_E_INVALID, "bb n_nu must be odd and >= 3");
    if (!(L.q_core > 0.0) || !(L.q_wing > 0.0)) return fail(JFNK_E_INVALID, "bb q_core, q_wing must be positive");
    if (!(L.f >= 0.0) || !(L.damping >= 0.0) || !(L.upsilon >= 0.0) || !(L.eps >= 0.0 && L.eps < 1.0))
      return fail(JFNK_E_INVALID, "bb f, damping, upsilon must be >= 0 and eps in [0, 1)");
    double nu0 = (A->E[L.j] - A->E[L.i]) * kEV / kH;
    std::vector<double> x = line_offsets(L.n_nu, L.q_core, L.q_wing);
    std::vector<double> g(L.n_nu);
    for (int s = 0; s < L.n_nu; ++s) g[s] = nu0 * (1.0 + x[s] * A->vchar / kC);
    grids.push_back(g);
    A->t_lo.push_back(L.i); A->t_up.push_back(L.j); A->t_kind.push_back(0);
    A->t_nu0.push_back(nu0); A->t_idx.push_back(b);
  }
  for (int b = 0; b < d->n_bf; ++b) {
    const jfnk_bf_desc& F = d->bf[b];
    if (F.i < 0 || F.j >= nl || F.i >= F.j) return fail(JFNK_E_INVALID, "bf levels must satisfy 0 <= i < j < n_levels");
    if (A->stage[F.j] != A->stage[F.i] + 1) return fail(JFNK_E_INVALID, "bf continuum must be one stage above");
    if (!(A->E[F.j] > A->E[F.i])) return fail(JFNK_E_INVALID, "bf continuum must lie above the bound level");
    if (F.n_nu < 2 || !(F.y_max > 1.0)) return fail(JFNK_E_INVALID, "bf needs n_nu >= 2 and y_max > 1");
    if (!(F.alpha0 >= 0.0) || !(F.q0 >= 0.0)) return fail(JFNK_E_INVALID, "bf alpha0, q0 must be >= 0");
    double nue = (A->E[F.j] - A->E[F.i]) * kEV / kH;
    std::vector<double> g(F.n_nu);
    for (int s = 0; s < F.n_nu; ++s) g[s] = nue * std::pow(F.y_max, (double)s / (F.n_nu - 1));
    grids.push_back(g);
    A->t_lo.push_back(F.i); A->t_up.push_back(F.j); A->t_kind.push_back(1);
    A->t_nu0.push_back(nue); A->t_idx.push_back(b);
  }
  const int nt = (int)grids.size();
  if (nt > kMaxT) return fail(JFNK_E_INVALID, "at most 32 transitions per atom");
  A->nt = nt;
  std::vector<double> all;
  for (auto& g : grids) all.insert(all.end(), g.begin(), g.end());
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  A->nu = all;
  const int nq = (int)all.size();
  A->nq = nq;
  A->t_q0.resize(nt); A->t_q1.resize(nt); A->t_base.resize(nt);
  A->t_w.clear();
  int base = 0;
  for (int t = 0; t < nt; ++t) {
    double lo = *std::min_element(grids[t].begin(), grids[t].end());
    double hi = *std::max_element(grids[t].begin(), grids[t].end());
    int q0 = (int)(std::lower_bound(all.begin(), all.end(), lo) - all.begin());
    int q1 = (int)(std::lower_bound(all.begin(), all.end(), hi) - all.begin());
    A->t_q0[t] = q0; A->t_q1[t] = q1; A->t_base[t] = base;
    int nw = q1 - q0 + 1;
    std::vector<double> w(nw, 0.0);
    for (int p = 0; p + 1 < nw; ++p) {
      double dnu = all[q0 + p + 1] - all[q0 + p];
      w[p] += 0.5 * dnu;
      w[p + 1] += 0.5 * dnu;
    }
    A->t_w.insert(A->t_w.end(), w.begin(), w.end());
    base += nw;
  }
  A->nwin = base;
  // CSR of the transitions active at each frequency
  A->q_off.assign(nq + 1, 0);
  for (int t = 0; t < nt; ++t)
    for (int q = A->t_q0[t]; q <= A->t_q1[t]; ++q) A->q_off[q + 1]++;
  for (int q = 0; q < nq; ++q) A->q_off[q + 1] += A->q_off[q];
  A->q_t.assign(A->q_off[nq], 0);
  std::vector<int> fill(A->q_off.begin(), A->q_off.end() - 1);
  for (int t = 0; t < nt; ++t)
    for (int q = A->t_q0[t]; q <= A->t_q1[t]; ++q) A->q_t[fill[q]++] = t;
  return JFNK_OK;
}

static void gauss_legendre_01(int n, double* mu, double* w) {
  // Newton iteration on P_n from the Chebyshev-like initial guesses
  for (int i = 0; i < n; ++i) {
    double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      double pn = (n == 1) ? x : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (x * pn - pnm1) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    // recompute the derivative at the converged node
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1; p1 = p2;
    }
    double pn = (n == 1) ? x : p1, pnm1 = (n == 1) ? 1.0 : p0;
    dp = n * (x * pn - pnm1) / (x * x - 1.0);
    double wi = 2.0 / ((1.0 - x * x) * dp * dp);
    mu[n - 1 - i] = 0.5 * (x + 1.0);   // ascending on ]0,1[
    w[n - 1 - i] = 0.5 * wi;
  }
}

// ---------------------------------------------------------------------------
// Device kernels for the column tables
// ---------------------------------------------------------------------------
struct AtomDev {
  int nl, nt;
  double E[kMaxL], g[kMaxL];
  int stage[kMaxL];
  double mass;
};

__global__ void k_lte(AtomDev at, int nz, const double* T, const double* ne, const double* ntot,
                      double* nstar) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nz) return;
  double kT = kKB * T[k];
  int smin = at.stage[0];
  for (int l = 1; l < at.nl; ++l) smin = min(smin, at.stage[l]);
  double lsaha = log(2.0 * pow(2.0 * kPi * kME * kKB * T[k] / (kH * kH), 1.5) / ne[k]);
  double lw[kMaxL];
  double mx = -1e300;
  for (int l = 0; l < at.nl; ++l) {
    lw[l] = log(at.g[l]) - at.E[l] * kEV / kT + (at.stage[l] - smin) * lsaha;
    mx = fmax(mx, lw[l]);
  }
  double s = 0.0;
  for (int l = 0; l < at.nl; ++l) { lw[l] = exp(lw[l] - mx); s += lw[l]; }
  for (int l = 0; l < at.nl; ++l) nstar[k * at.nl + l] = ntot[k] * lw[l] / s;
}

__global__ void k_planck_background(int nq, int nz, const double* nu, const double* T,
                                    const double* rho, const double* ne, double kappa,
                                    double kappa_nu_ref, double kappa_power, double kappa_max,
                                    int thomson, double* Bn, double* chi_c, double* eta_c,
                                    double* chi_sca) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nz) return;
  int q = i / nz, k = i % nz;
  double v = nu[q];
  double B = (2.0 * kH * v * v * v / (kC * kC)) / expm1(kH * v / (kKB * T[k]));
  double kap = kappa;
  if (kappa_power != 0.0) kap = kappa * fmin(kappa_max, fmax(1.0, pow(v / kappa_nu_ref, kappa_power)));
  double cc = (kappa != 0.0) ? kap * rho[k] : 0.0;
  Bn[i] = B;
  chi_c[i] = cc;
  eta_c[i] = cc * B;
  if (q == 0) chi_sca[k] = thomson ? kSigmaT * ne[k] : 0.0;
}

struct TransDev {
  int kind, lo, up;
  double nu0, f, damping, alpha0;
};

// V and g on every window point of every transition (Eqs. Vij, Vij2, gij);
// line profiles unnormalised here.
__global__ void k_window_tables(int nt, const TransDev* tr, const int* t_q0, const int* t_base,
                                const int* win_t, int nwin, int nz, const double* nu,
                                const double* T, const double* ne, const double* vturb,
                                AtomDev at, double* V, double* G) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nwin * nz) return;
  int p = i / nz, k = i % nz;
  int t = win_t[p];
  const TransDev d = tr[t];
  int q = t_q0[t] + (p - t_base[t]);
  double v = nu[q];
  double kT = kKB * T[k];
  if (d.kind == 0) {
    double vt = vturb ? vturb[k] : 0.0;
    double dnud = d.nu0 / kC * sqrt(2.0 * kKB * T[k] / (at.mass * kAMU) + vt * vt);
    double x = (v - d.nu0) / dnud;
    double phi = voigt_H(d.damping, x) / (1.7724538509055160273 * dnud);
    V[i] = (kPi * kQE * kQE / (kME * kC)) * d.f * phi;
    G[i] = at.g[d.lo] / at.g[d.up];
  } else {
    double r = d.nu0 / v;
    V[i] = d.alpha0 * r * r * r;
    double phi_saha = (at.g[d.lo] / (2.0 * at.g[d.up])) *
                      pow(kH * kH / (2.0 * kPi * kME * kKB * T[k]), 1.5);
    G[i] = ne[k] * phi_saha * exp(((at.E[d.up] - at.E[d.lo]) * kEV - kH * v) / kT);
  }
}

// A moving column: the line profile seen along each direction d (signed
// cosine mu_d: +mu for the outgoing rays, -mu for the ingoing ones) is centred
// at nu_0 (1 + mu_d v/c) (Sect. 3.4); continua are not shifted. Unnormalised.
__global__ void k_window_tables_dir(int nt, const TransDev* tr, const int* t_q0, const int* t_base,
                                    const int* win_t, int nwin, int nz, int nmu, const double* nu,
                                    const double* T, const double* vturb, const double* vlos,
                                    const double* mu, AtomDev at, const double* V, double* Vd) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)nwin * nz;
  if (i >= 2 * (size_t)nmu * per) return;
  const int dd = (int)(i / per);
  const size_t pk = i - (size_t)dd * per;
  const int p = (int)(pk / nz), k = (int)(pk % nz);
  const int t = win_t[p];
  const TransDev d = tr[t];
  if (d.kind != 0) {
    Vd[i] = V[pk];
    return;
  }
  const double mud = dd < nmu ? mu[dd] : -mu[dd - nmu];
  const int q = t_q0[t] + (p - t_base[t]);
  const double vt = vturb ? vturb[k] : 0.0;
  const double dnud = d.nu0 / kC * sqrt(2.0 * kKB * T[k] / (at.mass * kAMU) + vt * vt);
  const double x = (nu[q] - d.nu0 * (1.0 + mud * vlos[k] / kC)) / dnud;
  Vd[i] = (kPi * kQE * kQE / (kME * kC)) * d.f * voigt_H(d.damping, x) / (1.7724538509055160273 * dnud);
}

// Float copies of the (normalised) window tables for mixed-mode tangents.
__global__ void k_float_copy(int nwin, int nz, const double* V, const double* G, float* V32, float* G32,
                             float2* VG32T) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nwin * nz) return;
  const size_t p = i / nz, k = i % nz;
  const float v = (float)V[i], g = (float)G[i];
  V32[i] = v;
  G32[i] = g;
  VG32T[k * nwin + p] = make_float2(v, g);
}

// Renormalise each line profile so that sum_q omega_t(q) phi(q, k) = 1 (for
// every direction's copy when ndir > 1: the tables follow one another).
__global__ void k_normalise_lines(int nt, const TransDev* tr, const int* t_q0, const int* t_q1,
                                  const int* t_base, const double* t_w, int nz, double* V, int ndir = 1,
                                  size_t dir_stride = 0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt * nz * ndir) return;
  const int dd = i / (nt * nz);
  i -= dd * nt * nz;
  V += (size_t)dd * dir_stride;
  int t = i / nz, k = i % nz;
  const TransDev d = tr[t];
  if (d.kind != 0) return;
  int nw = t_q1[t] - t_q0[t] + 1;
  double* Vt = V + (size_t)t_base[t] * nz;
  const double* w = t_w + t_base[t];
  double s = 0.0;
  const double scale = (kPi * kQE * kQE / (kME * kC)) * d.f;
  for (int p = 0; p < nw; ++p) s += w[p] * (Vt[(size_t)p * nz + k] / scale);
  if (s > 0.0)
    for (int p = 0; p < nw; ++p) Vt[(size_t)p * nz + k] /= s;
}

// Products of the window tables per (window point, depth): g V (stimulated
// emission and emissivity, Eqs. chi, eta) and the rate-integral weights W V and
// W g V with W = omega_t(nu_q) 4 pi/(h nu_q) (Eqs. Rij, Rji), so that each term
// of those sums takes one product.
__global__ void k_rate_weights(int nwin, int nz, const int* winT, const int* t_q0, const int* t_base,
                               const double* t_w, const double* rw, const double* V, const double* G,
                               double* gV, double* WV, double* WgV) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nwin * nz) return;
  const int p = (int)(i / nz);
  const int t = winT[p];
  const double W = t_w[p] * rw[t_q0[t] + p - t_base[t]];
  const double wv = W * V[i];
  gV[i] = G[i] * V[i];
  WV[i] = wv;
  WgV[i] = wv * G[i];
}

// The population-independent part of R_ji (Eq. Rji): sum over the window of
// W g V 2 h nu^3/c^2, in window order.
__global__ void k_spontaneous(int nt, int nz, const int* t_q0, const int* t_q1, const int* t_base,
                              const double* c2, const double* WgV, double* Rsp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt * nz) return;
  const int t = i / nz, k = i % nz;
  const int nw = t_q1[t] - t_q0[t] + 1;
  const double* w = WgV + (size_t)t_base[t] * nz + k;
  double s = 0.0;
  for (int p = 0; p < nw; ++p) s += w[(size_t)p * nz] * c2[t_q0[t] + p];
  Rsp[i] = s;
}

// Float-pair copies of FP64 tables (the mixed mode's base evaluations).
__global__ void k_pairs(const double* src, float2* dst, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const df p = df_from_double(src[i]);
    dst[i] = make_float2(p.hi, p.lo);
  }
}
// chi_c + chi_sca per (nu, depth), summed in FP64, as pairs
__global__ void k_chibg_pairs(int nq, int nz, const double* chi_c, const double* chi_sca, float2* dst) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (size_t)nq * nz) {
    const df p = df_from_double(chi_c[i] + chi_sca[i % nz]);
    dst[i] = make_float2(p.hi, p.lo);
  }
}

struct CollDev {
  int kind, lo, up;
  double nu0, f, upsilon, eps, q0;
};

__global__ void k_collisions(int nt, const CollDev* cd, AtomDev at, int nz, const double* T,
                             const double* ne, double* C) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nz) return;
  const int nl = at.nl;
  double* Ck = C + (size_t)k * nl * nl;
  for (int i = 0; i < nl * nl; ++i) Ck[i] = 0.0;
  double Tk = T[k], kT = kKB * Tk;
  for (int t = 0; t < nt; ++t) {
    const CollDev d = cd[t];
    double gi = at.g[d.lo], gj = at.g[d.up];
    if (d.kind == 0) {
      double hnu_kt = kH * d.nu0 / kT;
      double down;
      if (d.eps > 0.0) {
        double Aji = 8.0 * kPi * kPi * kQE * kQE * d.nu0 * d.nu0 / (kME * kC * kC * kC) * (gi / gj) * d.f;
        down = d.eps * Aji / ((1.0 - d.eps) * (-expm1(-hnu_kt)));
      } else {
        down = 8.63e-6 * ne[k] * d.upsilon / (gj * sqrt(Tk));
      }
      Ck[d.up * nl + d.lo] += down;
      Ck[d.lo * nl + d.up] += down * (gj / gi) * exp(-hnu_kt);
    } else {
      double dE = (at.E[d.up] - at.E[d.lo]) * kEV;
      double up = ne[k] * d.q0 * sqrt(Tk) * exp(-dE / kT);
      double ratio = ne[k] * (gi / (2.0 * gj)) * pow(kH * kH / (2.0 * kPi * kME * kT), 1.5) * exp(dE / kT);
      Ck[d.lo * nl + d.up] += up;
      Ck[d.up * nl + d.lo] += up * ratio;
    }
  }
}

// ---------------------------------------------------------------------------
// Host: column construction
// ---------------------------------------------------------------------------
static bool g_voigt_ready[64] = {false};

int build_atmosphere(jfnk_ctx* ctx, int lane, const AtomData& A, const jfnk_atmos_desc* d, AtmosData* M) {
  if (!d) return fail(JFNK_E_INVALID, "atmosphere descriptor is NULL");
  const int nz = d->n_depth;
  if (nz < 2 || nz > JFNK_MAX_DEPTH) return fail(JFNK_E_INVALID, "n_depth must be in [2, 1024]");
  if (d->n_mu < 1 || d->n_mu > kMaxMu) return fail(JFNK_E_INVALID, "n_mu must be in [1, 8]");
  if (!d->z || !d->T || !d->ne || !d->ntot) return fail(JFNK_E_INVALID, "z, T, ne, ntot are required");
  if (d->kappa != 0.0 && !d->rho) return fail(JFNK_E_INVALID, "rho is required when kappa != 0");
  if (d->kappa_power != 0.0 && !(d->kappa_nu_ref > 0.0)) return fail(JFNK_E_INVALID, "kappa_nu_ref must be positive");
  for (int k = 0; k < nz; ++k) {
    if (!(d->T[k] > 0.0) || !(d->ne[k] > 0.0) || !(d->ntot[k] > 0.0))
      return fail(JFNK_E_INVALID, "T, ne and ntot must be positive");
    if (k > 0 && !(std::fabs(d->z[k] - d->z[k - 1]) > 0.0))
      return fail(JFNK_E_INVALID, "z must be strictly monotonic");
    if (k > 1 && ((d->z[k] - d->z[k - 1]) > 0.0) != ((d->z[1] - d->z[0]) > 0.0))
      return fail(JFNK_E_INVALID, "z must be strictly monotonic");
  }
  int dev = ctx->device;
  if (!g_voigt_ready[dev]) {
    double coef[kVoigtN + 1], L;
    voigt_coefficients(coef, &L);
    JFNK_CUDA(cudaMemcpyToSymbol(c_voigt, coef, sizeof(coef)));
    JFNK_CUDA(cudaMemcpyToSymbol(c_voigt_L, &L, sizeof(double)));
    g_voigt_ready[dev] = true;
  }
  const int nq = A.nq, nl = A.nl, nt = A.nt, nwin = A.nwin, nmu = d->n_mu;
  M->nz = nz; M->nq = nq; M->nl = nl; M->nt = nt; M->nmu = nmu; M->nwin = nwin;
  M->moving = false;
  if (d->vlos)
    for (int k = 0; k < nz; ++k) {
      if (!std::isfinite(d->vlos[k]) || std::fabs(d->vlos[k]) >= 0.1 * kC)
        return fail(JFNK_E_INVALID, "vlos must be finite and below c/10");
      if (d->vlos[k] != 0.0) M->moving = true;
    }
  M->ray_points = (double)nq * 2.0 * nmu * nz;
  // one device arena for every table
  DeviceArena& ar = M->arena;
  ar.reset();
  ar.stream = ctx->setup_stream[lane];   // stream-ordered pool: dropping an atmosphere does not stall the device
  // host-computed tables first (one contiguous prefix, uploaded by one copy
  // from pinned staging), then the tables the setup kernels compute
  size_t o_nu = ar.take<double>(nq), o_c2 = ar.take<double>(nq), o_rw = ar.take<double>(nq),
         o_rc2 = ar.take<double>(nq);
  size_t o_qoff = ar.take<int>(nq + 1), o_qt = ar.take<int>(A.q_t.size() + 1);
  size_t o_tlo = ar.take<int>(nt), o_tup = ar.take<int>(nt), o_tq0 = ar.take<int>(nt),
         o_tq1 = ar.take<int>(nt), o_tbase = ar.take<int>(nt), o_winT = ar.take<int>(nwin);
  size_t o_tw = ar.take<double>(nwin);
  size_t o_dz = ar.take<double>(nz - 1), o_mu = ar.take<double>(nmu), o_wmu = ar.take<double>(nmu);
  size_t o_ntot = ar.take<double>(nz);
  size_t o_T = ar.take<double>(nz), o_ne = ar.take<double>(nz), o_rho = ar.take<double>(nz),
         o_vt = ar.take<double>(nz);
  size_t o_tr = ar.take<TransDev>(nt), o_cd = ar.take<CollDev>(nt);
  size_t o_W32 = ar.take<float>(nwin), o_Wr32 = ar.take<float>(nwin), o_c2f = ar.take<float>(nq);
  size_t o_qmeta = ar.take<int>((size_t)kQMetaT * nq), o_qtr = ar.take<int>((size_t)kQMetaT * nq);
  size_t o_W2 = ar.take<float2>(nwin), o_c2p = ar.take<float2>(nq), o_rc2p = ar.take<float2>(nq);
  size_t o_linc = ar.take<int>((size_t)nl * (nt + 1));
  size_t o_ang32 = ar.take<float4>(nmu), o_dz32 = ar.take<float2>(nz - 1);
  size_t o_vlos = ar.take<double>(M->moving ? nz : 0);
  const size_t host_prefix = ar.cursor;
  size_t o_V = ar.take<double>((size_t)nwin * nz), o_G = ar.take<double>((size_t)nwin * nz);
  size_t o_chic = ar.take<double>((size_t)nq * nz), o_etac = ar.take<double>((size_t)nq * nz);
  size_t o_sca = ar.take<double>(nz), o_B = ar.take<double>((size_t)nq * nz);
  size_t o_C = ar.take<double>((size_t)nz * nl * nl), o_nstar = ar.take<double>((size_t)nz * nl);
  size_t o_V32 = ar.take<float>((size_t)nwin * nz), o_G32 = ar.take<float>((size_t)nwin * nz);
  size_t o_VG32T = ar.take<float2>((size_t)nwin * nz);
  size_t o_WV = ar.take<double>((size_t)nwin * nz), o_WgV = ar.take<double>((size_t)nwin * nz),
         o_Rsp = ar.take<double>((size_t)nt * nz), o_gV = ar.take<double>((size_t)nwin * nz);
  size_t o_V2 = ar.take<float2>((size_t)nwin * nz), o_gV2 = ar.take<float2>((size_t)nwin * nz),
         o_chibg2 = ar.take<float2>((size_t)nq * nz), o_etac2 = ar.take<float2>((size_t)nq * nz),
         o_chisca2 = ar.take<float2>(nz);
  size_t o_Vd = ar.take<double>(M->moving ? 2 * (size_t)nmu * nwin * nz : 0);
  int rc = ar.allocate();
  if (rc) return rc;
  // host-side staging
  std::vector<double> c2(nq), rc2(nq), rw(nq), dzv(nz - 1), mu(nmu), wmu(nmu);
  for (int q = 0; q < nq; ++q) {
    c2[q] = 2.0 * kH * A.nu[q] * A.nu[q] * A.nu[q] / (kC * kC);
    rc2[q] = 1.0 / c2[q];
    rw[q] = 4.0 * kPi / (kH * A.nu[q]);
  }
  for (int k = 0; k + 1 < nz; ++k) dzv[k] = std::fabs(d->z[k] - d->z[k + 1]);
  gauss_legendre_01(nmu, mu.data(), wmu.data());
  std::vector<int> winT(nwin);
  std::vector<float> w32(nwin), wr32(nwin), c2f(nq);
  std::vector<float2> w2(nwin), c2p(nq), rc2p(nq);
  for (int q = 0; q < nq; ++q) {
    const df a = df_from_double(c2[q]), b = df_from_double(rc2[q]);
    c2p[q] = make_float2(a.hi, a.lo);
    rc2p[q] = make_float2(b.hi, b.lo);
  }
  for (int q = 0; q < nq; ++q) c2f[q] = (float)c2[q];
  for (int t = 0; t < nt; ++t)
    for (int p = 0; p <= A.t_q1[t] - A.t_q0[t]; ++p) {
      const int q = A.t_q0[t] + p;
      winT[A.t_base[t] + p] = t;
      w32[A.t_base[t] + p] = (float)(A.t_w[A.t_base[t] + p] * rw[q] * c2[q]);
      wr32[A.t_base[t] + p] = (float)(A.t_w[A.t_base[t] + p] * rw[q]);
      const df wp = df_from_double(A.t_w[A.t_base[t] + p] * rw[q]);
      w2[A.t_base[t] + p] = make_float2(wp.hi, wp.lo);
    }
  std::vector<TransDev> tr(nt);
  std::vector<CollDev> cd(nt);
  for (int t = 0; t < nt; ++t) {
    TransDev& x = tr[t];
    CollDev& c = cd[t];
    x.kind = c.kind = A.t_kind[t];
    x.lo = c.lo = A.t_lo[t];
    x.up = c.up = A.t_up[t];
    x.nu0 = c.nu0 = A.t_nu0[t];
    if (A.t_kind[t] == 0) {
      const jfnk_bb_desc& L = A.bb[A.t_idx[t]];
      x.f = c.f = L.f; x.damping = L.damping; x.alpha0 = 0.0;
      c.upsilon = L.upsilon; c.eps = L.eps; c.q0 = 0.0;
    } else {
      const jfnk_bf_desc& F = A.bf[A.t_idx[t]];
      x.f = c.f = 0.0; x.damping = 0.0; x.alpha0 = F.alpha0;
      c.upsilon = 0.0; c.eps = 0.0; c.q0 = F.q0;
    }
  }
  std::vector<double> zeros(nz, 0.0);
  cudaStream_t s = ctx->setup_stream[lane];
  char*& stage = ctx->stage[lane];
  if (ctx->stage_bytes[lane] < host_prefix) {
    if (stage) cudaFreeHost(stage);
    stage = nullptr;
    ctx->stage_bytes[lane] = 0;
    JFNK_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&stage), host_prefix, cudaHostAllocDefault));
    ctx->stage_bytes[lane] = host_prefix;
  }
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (off + bytes > host_prefix) return cudaErrorInvalidValue;   // only the host-computed prefix
    std::memcpy(stage + off, src, bytes);   // copied below at once
    return cudaSuccess;
  };
  JFNK_CUDA(up(o_nu, A.nu.data(), nq * 8));
  JFNK_CUDA(up(o_c2, c2.data(), nq * 8));
  JFNK_CUDA(up(o_rw, rw.data(), nq * 8));
  JFNK_CUDA(up(o_rc2, rc2.data(), nq * 8));
  JFNK_CUDA(up(o_qoff, A.q_off.data(), (nq + 1) * 4));
  JFNK_CUDA(up(o_qt, A.q_t.data(), A.q_t.size() * 4));
  JFNK_CUDA(up(o_tlo, A.t_lo.data(), nt * 4));
  JFNK_CUDA(up(o_tup, A.t_up.data(), nt * 4));
  JFNK_CUDA(up(o_tq0, A.t_q0.data(), nt * 4));
  JFNK_CUDA(up(o_tq1, A.t_q1.data(), nt * 4));
  JFNK_CUDA(up(o_tbase, A.t_base.data(), nt * 4));
  JFNK_CUDA(up(o_winT, winT.data(), nwin * 4));
  JFNK_CUDA(up(o_tw, A.t_w.data(), nwin * 8));
  JFNK_CUDA(up(o_W32, w32.data(), nwin * 4));
  JFNK_CUDA(up(o_Wr32, wr32.data(), nwin * 4));
  JFNK_CUDA(up(o_c2f, c2f.data(), nq * 4));
  JFNK_CUDA(up(o_W2, w2.data(), nwin * sizeof(float2)));
  JFNK_CUDA(up(o_c2p, c2p.data(), nq * sizeof(float2)));
  JFNK_CUDA(up(o_rc2p, rc2p.data(), nq * sizeof(float2)));
  std::vector<int> qmeta((size_t)kQMetaT * nq, -1), qtr((size_t)kQMetaT * nq, -1);
  for (int q = 0; q < nq; ++q)
    for (int s = A.q_off[q], j = 0; s < A.q_off[q + 1] && j < kQMetaT; ++s, ++j) {
      const int t = A.q_t[s];
      qmeta[(size_t)j * nq + q] = ((A.t_base[t] + q - A.t_q0[t]) << 8) | (A.t_lo[t] << 4) | A.t_up[t];
      qtr[(size_t)j * nq + q] = t;
    }
  JFNK_CUDA(up(o_qmeta, qmeta.data(), qmeta.size() * 4));
  JFNK_CUDA(up(o_qtr, qtr.data(), qtr.size() * 4));
  // per level, its transitions in index order (lower level: +, upper: -)
  std::vector<int> linc((size_t)nl * (nt + 1), -1);
  for (int l = 0; l < nl; ++l) {
    int j = 0;
    for (int t = 0; t < nt; ++t) {
      if (A.t_lo[t] == l) linc[(size_t)l * (nt + 1) + j++] = t << 1;
      else if (A.t_up[t] == l) linc[(size_t)l * (nt + 1) + j++] = (t << 1) | 1;
    }
  }
  JFNK_CUDA(up(o_linc, linc.data(), linc.size() * 4));
  // the sweep kernels' per-angle and per-layer constants, rounded once from FP64
  std::vector<float4> ang32(nmu);
  for (int m = 0; m < nmu; ++m)
    ang32[m] = make_float4((float)(0.5 / mu[m]), (float)(0.5 * wmu[m]), (float)(2.0 * mu[m]), 0.f);
  std::vector<float2> dz32(nz - 1);
  for (int k = 0; k + 1 < nz; ++k) dz32[k] = make_float2((float)dzv[k], (float)(1.0 / dzv[k]));
  JFNK_CUDA(up(o_ang32, ang32.data(), nmu * sizeof(float4)));
  if (M->moving) JFNK_CUDA(up(o_vlos, d->vlos, nz * 8));
  JFNK_CUDA(up(o_dz32, dz32.data(), (nz - 1) * sizeof(float2)));
  JFNK_CUDA(up(o_dz, dzv.data(), (nz - 1) * 8));
  JFNK_CUDA(up(o_mu, mu.data(), nmu * 8));
  JFNK_CUDA(up(o_wmu, wmu.data(), nmu * 8));
  JFNK_CUDA(up(o_ntot, d->ntot, nz * 8));
  JFNK_CUDA(up(o_T, d->T, nz * 8));
  JFNK_CUDA(up(o_ne, d->ne, nz * 8));
  JFNK_CUDA(up(o_rho, d->rho ? d->rho : zeros.data(), nz * 8));
  JFNK_CUDA(up(o_vt, d->vturb ? d->vturb : zeros.data(), nz * 8));
  JFNK_CUDA(up(o_tr, tr.data(), nt * sizeof(TransDev)));
  JFNK_CUDA(up(o_cd, cd.data(), nt * sizeof(CollDev)));
  JFNK_CUDA(cudaMemcpyAsync(ar.base, stage, host_prefix, cudaMemcpyHostToDevice, s));
  AtomDev at{};
  at.nl = nl; at.nt = nt; at.mass = A.mass;
  for (int l = 0; l < nl; ++l) { at.E[l] = A.E[l]; at.g[l] = A.g[l]; at.stage[l] = A.stage[l]; }
  double* T = ar.ptr<double>(o_T);
  double* ne = ar.ptr<double>(o_ne);
  const int tb = 256;
  k_lte<<<(nz + tb - 1) / tb, tb, 0, s>>>(at, nz, T, ne, ar.ptr<double>(o_ntot), ar.ptr<double>(o_nstar));
  k_planck_background<<<(nq * nz + tb - 1) / tb, tb, 0, s>>>(
      nq, nz, ar.ptr<double>(o_nu), T, ar.ptr<double>(o_rho), ne, d->kappa, d->kappa_nu_ref,
      d->kappa_power, d->kappa_max, d->thomson, ar.ptr<double>(o_B), ar.ptr<double>(o_chic),
      ar.ptr<double>(o_etac), ar.ptr<double>(o_sca));
  k_window_tables<<<(int)(((size_t)nwin * nz + tb - 1) / tb), tb, 0, s>>>(
      nt, ar.ptr<TransDev>(o_tr), ar.ptr<int>(o_tq0), ar.ptr<int>(o_tbase), ar.ptr<int>(o_winT),
      nwin, nz, ar.ptr<double>(o_nu), T, ne, d->vturb ? ar.ptr<double>(o_vt) : nullptr, at,
      ar.ptr<double>(o_V), ar.ptr<double>(o_G));
  k_normalise_lines<<<(nt * nz + tb - 1) / tb, tb, 0, s>>>(
      nt, ar.ptr<TransDev>(o_tr), ar.ptr<int>(o_tq0), ar.ptr<int>(o_tq1), ar.ptr<int>(o_tbase),
      ar.ptr<double>(o_tw), nz, ar.ptr<double>(o_V));
  if (M->moving) {
    const size_t nd = 2 * (size_t)nmu, per = (size_t)nwin * nz;
    k_window_tables_dir<<<(int)((nd * per + tb - 1) / tb), tb, 0, s>>>(
        nt, ar.ptr<TransDev>(o_tr), ar.ptr<int>(o_tq0), ar.ptr<int>(o_tbase), ar.ptr<int>(o_winT), nwin, nz, nmu,
        ar.ptr<double>(o_nu), T, d->vturb ? ar.ptr<double>(o_vt) : nullptr, ar.ptr<double>(o_vlos),
        ar.ptr<double>(o_mu), at, ar.ptr<double>(o_V), ar.ptr<double>(o_Vd));
    k_normalise_lines<<<(int)((nd * nt * nz + tb - 1) / tb), tb, 0, s>>>(
        nt, ar.ptr<TransDev>(o_tr), ar.ptr<int>(o_tq0), ar.ptr<int>(o_tq1), ar.ptr<int>(o_tbase),
        ar.ptr<double>(o_tw), nz, ar.ptr<double>(o_Vd), (int)nd, per);
  }
  k_rate_weights<<<(int)(((size_t)nwin * nz + tb - 1) / tb), tb, 0, s>>>(
      nwin, nz, ar.ptr<int>(o_winT), ar.ptr<int>(o_tq0), ar.ptr<int>(o_tbase), ar.ptr<double>(o_tw),
      ar.ptr<double>(o_rw), ar.ptr<double>(o_V), ar.ptr<double>(o_G), ar.ptr<double>(o_gV),
      ar.ptr<double>(o_WV), ar.ptr<double>(o_WgV));
  k_spontaneous<<<(nt * nz + tb - 1) / tb, tb, 0, s>>>(nt, nz, ar.ptr<int>(o_tq0), ar.ptr<int>(o_tq1),
                                                        ar.ptr<int>(o_tbase), ar.ptr<double>(o_c2),
                                                        ar.ptr<double>(o_WgV), ar.ptr<double>(o_Rsp));
  {
    const size_t nwz = (size_t)nwin * nz, nqz = (size_t)nq * nz;
    k_pairs<<<(int)((nwz + tb - 1) / tb), tb, 0, s>>>(ar.ptr<double>(o_V), ar.ptr<float2>(o_V2), nwz);
    k_pairs<<<(int)((nwz + tb - 1) / tb), tb, 0, s>>>(ar.ptr<double>(o_gV), ar.ptr<float2>(o_gV2), nwz);
    k_pairs<<<(int)((nqz + tb - 1) / tb), tb, 0, s>>>(ar.ptr<double>(o_etac), ar.ptr<float2>(o_etac2), nqz);
    k_pairs<<<(nz + tb - 1) / tb, tb, 0, s>>>(ar.ptr<double>(o_sca), ar.ptr<float2>(o_chisca2), (size_t)nz);
    k_chibg_pairs<<<(int)((nqz + tb - 1) / tb), tb, 0, s>>>(nq, nz, ar.ptr<double>(o_chic), ar.ptr<double>(o_sca),
                                                            ar.ptr<float2>(o_chibg2));
  }
  k_collisions<<<(nz + tb - 1) / tb, tb, 0, s>>>(nt, ar.ptr<CollDev>(o_cd), at, nz, T, ne,
                                                  ar.ptr<double>(o_C));
  k_float_copy<<<(int)(((size_t)nwin * nz + tb - 1) / tb), tb, 0, s>>>(
      nwin, nz, ar.ptr<double>(o_V), ar.ptr<double>(o_G), ar.ptr<float>(o_V32), ar.ptr<float>(o_G32),
      ar.ptr<float2>(o_VG32T));
  JFNK_CUDA(cudaGetLastError());
  JFNK_CUDA(cudaEventRecord(ctx->setup_done[lane], s));
  ColTables& tb_ = M->tables;
  tb_.nz = nz; tb_.nq = nq; tb_.nl = nl; tb_.nt = nt; tb_.nmu = nmu; tb_.nwin = nwin;
  tb_.max_overlap = 0;
  for (int q = 0; q < nq; ++q) tb_.max_overlap = std::max(tb_.max_overlap, A.q_off[q + 1] - A.q_off[q]);
  tb_.nu = ar.ptr<double>(o_nu); tb_.c2 = ar.ptr<double>(o_c2); tb_.rw = ar.ptr<double>(o_rw);
  tb_.q_off = ar.ptr<int>(o_qoff); tb_.q_t = ar.ptr<int>(o_qt);
  tb_.t_lo = ar.ptr<int>(o_tlo); tb_.t_up = ar.ptr<int>(o_tup); tb_.t_q0 = ar.ptr<int>(o_tq0);
  tb_.t_q1 = ar.ptr<int>(o_tq1); tb_.t_base = ar.ptr<int>(o_tbase); tb_.t_w = ar.ptr<double>(o_tw);
  tb_.V = ar.ptr<double>(o_V); tb_.G = ar.ptr<double>(o_G); tb_.dz = ar.ptr<double>(o_dz);
  tb_.gV = ar.ptr<double>(o_gV); tb_.rc2 = ar.ptr<double>(o_rc2);
  tb_.V2 = ar.ptr<float2>(o_V2); tb_.gV2 = ar.ptr<float2>(o_gV2); tb_.W2 = ar.ptr<float2>(o_W2);
  tb_.chibg2 = ar.ptr<float2>(o_chibg2); tb_.etac2 = ar.ptr<float2>(o_etac2);
  tb_.chisca2 = ar.ptr<float2>(o_chisca2); tb_.c2p = ar.ptr<float2>(o_c2p); tb_.rc2p = ar.ptr<float2>(o_rc2p);
  tb_.WV = ar.ptr<double>(o_WV); tb_.WgV = ar.ptr<double>(o_WgV); tb_.Rsp = ar.ptr<double>(o_Rsp);
  tb_.V32 = ar.ptr<float>(o_V32); tb_.G32 = ar.ptr<float>(o_G32); tb_.W32 = ar.ptr<float>(o_W32);
  tb_.VG32T = ar.ptr<float2>(o_VG32T);
  tb_.Wr32 = ar.ptr<float>(o_Wr32); tb_.c2f = ar.ptr<float>(o_c2f);
  tb_.qmeta = ar.ptr<int>(o_qmeta);
  tb_.qtr = ar.ptr<int>(o_qtr);
  tb_.lvl_inc = ar.ptr<int>(o_linc);
  tb_.mu = ar.ptr<double>(o_mu); tb_.wmu = ar.ptr<double>(o_wmu);
  tb_.ang32 = ar.ptr<float4>(o_ang32); tb_.dz32 = ar.ptr<float2>(o_dz32);
  tb_.Vd = M->moving ? ar.ptr<double>(o_Vd) : nullptr;
  tb_.chi_c = ar.ptr<double>(o_chic); tb_.eta_c = ar.ptr<double>(o_etac);
  tb_.chi_sca = ar.ptr<double>(o_sca); tb_.Bn = ar.ptr<double>(o_B); tb_.C = ar.ptr<double>(o_C);
  tb_.ntot = ar.ptr<double>(o_ntot); tb_.nstar = ar.ptr<double>(o_nstar);
  M->host_t_w = A.t_w;
  return JFNK_OK;
}

}  // namespace jfnk
