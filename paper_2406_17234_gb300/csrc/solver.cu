// On-device JFNK driver (Algorithm 2) and RH92 warm start, as a per-column
// state machine: every tick performs one F-class evaluation per in-flight
// column (a base evaluation, a Jacobian-vector product, a GMRES restart
// product or an RH92 formal solution) followed by one Krylov/Newton step,
// so that columns at different stages of their solves share each launch.
// A tick sequence is captured once in a CUDA graph and replayed until every
// column has finished; the host only polls a status word per column.
#include <algorithm>
#include <cmath>

#include "formal_coef.cuh"

namespace jfnk {

int DeviceArena::allocate() {
  release();
  bytes = cursor;
  if (bytes == 0) return JFNK_OK;
  cudaError_t e = stream ? cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, stream) : cudaMalloc(&base, bytes);
  if (e != cudaSuccess) {
    base = nullptr;
    return fail(JFNK_E_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
  }
  return JFNK_OK;
}

void DeviceArena::release() {
  if (base) {
    if (stream) cudaFreeAsync(base, stream);
    else cudaFree(base);
  }
  base = nullptr;
  bytes = 0;
}

// Offsets of one column's work buffers, relative to the start of its block.
struct ColLayout {
  size_t n, v, v32, chiT, S32T, dSkT, dchiT, dS32T, dJ32T, Jdag, Jnew, istar, chi, S, dSk, dchi, dS, ddSk, H, HI, dH,
      LX, LE, part, J, dJ, Lchi, Leta, Lchi32, Leta32, Rup, Rdn, dRup, dRdn, Apart, rh, F, dF, P, piv, Iem, Vb, Hh, cs, sn, gv, x,
      w, nprev, np, fdp, eta, etab32, n2, mchi, mS, mdchi, mdS, mI, mdI, mLX, mLE;
};

size_t column_bytes(const AtmosData& M, int kind, int mixed, int kmax, ColLayout* out) {
  DeviceArena ar;   // used as a cursor only
  ColLayout o{};
  const size_t rs = mixed ? sizeof(float) : sizeof(double);
  const size_t nz = M.nz, nq = M.nq, nl = M.nl, nt = M.nt, nmu = M.nmu, N = nz * nl;
  const bool per_ray = (kind == FORMAL_UNFUSED);   // unfused kernels need per-ray buffers
  const bool sweep = (kind == FORMAL_SWEEP);
  o.n = ar.take<double>(N); o.v = ar.take<double>(N);
  o.Jdag = ar.take<double>(nq * nz); o.Jnew = ar.take<double>(nq * nz);
  o.istar = ar.take<int>(nz);
  o.chi = ar.take<char>(rs * nq * nz); o.S = ar.take<double>(nq * nz);
  o.dSk = ar.take<char>(per_ray ? rs * nq * nz : 0);
  o.dchi = ar.take<char>(sweep ? 0 : rs * nq * nz); o.dS = ar.take<double>(sweep ? 0 : nq * nz);
  const size_t TQ = sweep ? (size_t)nz * col_pitch((int)nq) : 0;
  o.v32 = ar.take<float>(sweep ? N : 0);
  o.chiT = ar.take<float>(TQ); o.S32T = ar.take<float>(TQ); o.dSkT = ar.take<float>(TQ);
  o.dchiT = ar.take<float>(TQ); o.dS32T = ar.take<float>(TQ); o.dJ32T = ar.take<float>(TQ);
  o.ddSk = ar.take<char>(per_ray ? rs * nq * nz : 0);
  const size_t pr = per_ray ? rs * 2 * nmu * nq * nz : 0;
  o.H = ar.take<char>(pr); o.dH = ar.take<char>(pr); o.HI = ar.take<char>(pr);
  o.LX = ar.take<char>(pr); o.LE = ar.take<char>(pr);
  o.part = ar.take<char>(sweep ? sweep_scratch_bytes((int)nq, (int)nz) : 0);
  o.J = ar.take<double>(nq * nz); o.dJ = ar.take<double>(sweep ? 0 : nq * nz);
  o.Lchi = ar.take<double>(sweep ? 0 : nq * nz); o.Leta = ar.take<double>(sweep ? 0 : nq * nz);
  o.Lchi32 = ar.take<float>(sweep ? nq * nz : 0); o.Leta32 = ar.take<float>(sweep ? nq * nz : 0);
  o.Rup = ar.take<double>(nt * nz); o.Rdn = ar.take<double>(nt * nz);
  o.dRup = ar.take<double>(nt * nz); o.dRdn = ar.take<double>(nt * nz);
  o.Apart = ar.take<double>(nt * nz * nl);
  o.rh = ar.take<double>(nt * nz * kRhStride);
  o.F = ar.take<double>(N); o.dF = ar.take<double>(N);
  o.P = ar.take<double>(nz * nl * nl); o.piv = ar.take<int>(nz * nl);
  o.Iem = ar.take<double>(nq * nmu);
  o.Vb = ar.take<double>((size_t)(kmax + 1) * N); o.Hh = ar.take<double>((size_t)(kmax + 1) * kmax);
  o.cs = ar.take<double>(kmax); o.sn = ar.take<double>(kmax); o.gv = ar.take<double>(kmax + 1);
  o.x = ar.take<double>(N); o.w = ar.take<double>(N); o.nprev = ar.take<double>(N);
  o.np = ar.take<double>(N); o.fdp = ar.take<double>(N);
  o.eta = ar.take<double>(nq * nz); o.etab32 = ar.take<float>(mixed ? nq * nz : 0);
  o.n2 = ar.take<float2>(mixed ? N : 0);
  // moving columns: per-ray opacity, source function, intensity, tangents and local derivatives
  const size_t MR = kind == FORMAL_MOVING ? 2 * nmu * nq * nz : 0;
  o.mchi = ar.take<double>(MR); o.mS = ar.take<double>(MR); o.mdchi = ar.take<double>(MR);
  o.mdS = ar.take<double>(MR); o.mI = ar.take<double>(MR); o.mdI = ar.take<double>(MR);
  o.mLX = ar.take<double>(MR); o.mLE = ar.take<double>(MR);
  if (out) *out = o;
  return ar.cursor;
}

void column_bind(char* base, const AtmosData& M, int kind, int mixed, int kmax, SolverState* st, ColDesc* d) {
  ColLayout o;
  column_bytes(M, kind, mixed, kmax, &o);
  auto P = [&](size_t off) { return static_cast<void*>(base + off); };
  const bool sweep = (kind == FORMAL_SWEEP);
  d->t = M.tables;
  d->forced_mode = -1;
  d->mixed = mixed;
  d->opts = nullptr;
  ColWork& w = d->w;
  w = ColWork{};
  w.n = (double*)P(o.n); w.v = (double*)P(o.v);
  w.Jdag = (double*)P(o.Jdag); w.Jnew = (double*)P(o.Jnew);
  w.istar = (int*)P(o.istar);
  w.chi = P(o.chi); w.S = (double*)P(o.S); w.dSk = P(o.dSk);
  w.dchi = sweep ? nullptr : P(o.dchi); w.ddSk = P(o.ddSk);
  // the mixed tangent path is FP32 throughout: no FP64 tangent buffers
  w.dS = sweep ? nullptr : (double*)P(o.dS);
  if (sweep) {
    w.v32 = (float*)P(o.v32);
    w.chiT = (float*)P(o.chiT); w.S32T = (float*)P(o.S32T); w.dSkT = (float*)P(o.dSkT);
    w.dchiT = (float*)P(o.dchiT); w.dS32T = (float*)P(o.dS32T); w.dJ32T = (float*)P(o.dJ32T);
  }
  w.H = P(o.H); w.dH = P(o.dH); w.HI = P(o.HI); w.LX = P(o.LX); w.LE = P(o.LE);
  w.part = P(o.part);
  w.J = (double*)P(o.J); w.dJ = sweep ? nullptr : (double*)P(o.dJ);
  w.Lchi = sweep ? nullptr : (double*)P(o.Lchi); w.Leta = sweep ? nullptr : (double*)P(o.Leta);
  w.Lchi32 = sweep ? (float*)P(o.Lchi32) : nullptr; w.Leta32 = sweep ? (float*)P(o.Leta32) : nullptr;
  w.zeta = nullptr;
  w.Rup = (double*)P(o.Rup); w.Rdn = (double*)P(o.Rdn);
  w.dRup = (double*)P(o.dRup); w.dRdn = (double*)P(o.dRdn);
  w.Apart = (double*)P(o.Apart); w.rh = (double*)P(o.rh);
  w.F = (double*)P(o.F); w.dF = (double*)P(o.dF);
  w.P = (double*)P(o.P); w.piv = (int*)P(o.piv); w.Iem = (double*)P(o.Iem);
  w.Vb = (double*)P(o.Vb); w.Hh = (double*)P(o.Hh);
  w.cs = (double*)P(o.cs); w.sn = (double*)P(o.sn); w.gv = (double*)P(o.gv);
  w.x = (double*)P(o.x); w.w = (double*)P(o.w); w.nprev = (double*)P(o.nprev);
  w.np = (double*)P(o.np); w.fdp = (double*)P(o.fdp);
  w.eta = (double*)P(o.eta); w.etab32 = mixed ? (float*)P(o.etab32) : nullptr;
  w.n2 = mixed ? (float2*)P(o.n2) : nullptr;
  if (kind == FORMAL_MOVING) {
    w.mchi = (double*)P(o.mchi); w.mS = (double*)P(o.mS); w.mdchi = (double*)P(o.mdchi);
    w.mdS = (double*)P(o.mdS); w.mI = (double*)P(o.mI); w.mdI = (double*)P(o.mdI);
    w.mLX = (double*)P(o.mLX); w.mLE = (double*)P(o.mLE);
  }
  w.st = st;
}

int batch_create(Batch* b, const std::vector<const AtmosData*>& cols, int mixed, int kmax) {
  const int nc = (int)cols.size();
  b->ncols = nc;
  b->mixed = mixed;
  b->kmax = kmax;
  b->max_nz = b->max_nq = b->max_nt = b->max_N = b->max_nmu = b->max_nl = 0;
  DeviceArena& ar = b->arena;
  ar.reset();
  int mov = 0;
  for (auto* c : cols) {
    mov = std::max(mov, c->tables.max_overlap);
    b->max_nz = std::max(b->max_nz, c->nz);
    b->max_nq = std::max(b->max_nq, c->nq);
    b->max_nt = std::max(b->max_nt, c->nt);
    b->max_N = std::max(b->max_N, c->nz * c->nl);
    b->max_nmu = std::max(b->max_nmu, c->nmu);
    b->max_nl = std::max(b->max_nl, c->nl);
  }
  b->max_overlap = mov;
  bool moving = false;
  for (auto* c : cols) moving = moving || c->moving;
  if (moving && mixed)
    return fail(JFNK_E_INVALID, "moving columns (a velocity field) are solved in JFNK_FP64 only");
  {
    int dev = 0;
    JFNK_CUDA(cudaGetDevice(&dev));
    JFNK_CUDA(cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  b->formal_qb = mixed || moving ? 0 : fused_default_qb(b->max_nz, b->max_nmu, false);
  b->formal_kind = moving ? FORMAL_MOVING
                          : (mixed ? FORMAL_SWEEP : (b->formal_qb > 0 ? FORMAL_FUSED : FORMAL_UNFUSED));
  std::vector<size_t> off(nc);
  for (int c = 0; c < nc; ++c)
    off[c] = ar.take<char>(column_bytes(*cols[c], b->formal_kind, mixed, kmax, nullptr));
  size_t o_cols = ar.take<ColDesc>(nc);
  size_t o_state = ar.take<SolverState>(nc);
  size_t o_status = ar.take<int>(nc);
  size_t o_opts = ar.take<SolverOpts>(1);
  size_t o_view = ar.take<ColDesc>(nc);
  int rc = ar.allocate();
  if (rc) return rc;
  b->h_cols.resize(nc);
  b->d_cols = ar.ptr<ColDesc>(o_cols);
  b->d_state = ar.ptr<SolverState>(o_state);
  b->d_status = ar.ptr<int>(o_status);
  b->d_opts = ar.ptr<SolverOpts>(o_opts);
  b->d_view = ar.ptr<ColDesc>(o_view);
  for (int c = 0; c < nc; ++c)
    column_bind(ar.base + off[c], *cols[c], b->formal_kind, mixed, kmax, b->d_state + c, &b->h_cols[c]);
  JFNK_CUDA(cudaMemcpy(b->d_cols, b->h_cols.data(), nc * sizeof(ColDesc), cudaMemcpyHostToDevice));
  JFNK_CUDA(cudaMemset(b->d_state, 0, nc * sizeof(SolverState)));
  if (b->formal_kind == FORMAL_SWEEP) return sweep_prepare(b);
  if (b->formal_kind == FORMAL_MOVING) return JFNK_OK;
  return fused_prepare(b);
}

__global__ void k_set_forced(ColDesc* cols, int mode) { cols[blockIdx.x].forced_mode = mode; }

int batch_set_forced_mode(Batch* b, int mode, cudaStream_t s) {
  for (auto& c : b->h_cols) c.forced_mode = mode;
  k_set_forced<<<b->ncols, 1, 0, s>>>(b->d_cols, mode);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < nw; ++i) r += sh[i];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = sh[0];
  for (int i = 1; i < nw; ++i) r = fmax(r, sh[i]);
  __syncthreads();
  return r;
}

// Dense solve with partial pivoting of one small system (RH92 per depth).
__device__ bool small_solve(double* A, double* b, int nl) {
  for (int c = 0; c < nl; ++c) {
    int pr = c;
    double best = fabs(A[c * nl + c]);
    for (int r = c + 1; r < nl; ++r)
      if (fabs(A[r * nl + c]) > best) { best = fabs(A[r * nl + c]); pr = r; }
    if (!(best > 0.0)) return false;
    if (pr != c) {
      for (int j = 0; j < nl; ++j) { double t = A[c * nl + j]; A[c * nl + j] = A[pr * nl + j]; A[pr * nl + j] = t; }
      double t = b[c]; b[c] = b[pr]; b[pr] = t;
    }
    for (int r = c + 1; r < nl; ++r) {
      double f = A[r * nl + c] / A[c * nl + c];
      for (int j = c; j < nl; ++j) A[r * nl + j] -= f * A[c * nl + j];
      b[r] -= f * b[c];
    }
  }
  for (int r = nl - 1; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < nl; ++j) s -= A[r * nl + j] * b[j];
    b[r] = s / A[r * nl + r];
  }
  return true;
}

// RH92 update of depth k from the sums of an EV_RH92 evaluation; returns the
// population change measure of the depth (or NaN on a singular system). With
// clamp the correction is limited like a Newton correction (Sect. 2.2.2), so
// that no population of the depth falls below a tenth of its old value.
//
// The preconditioned rate equations M n' + c0 = 0 (plus the conservation row)
// are affine in n' and equal the residual F at n' = n, so n' = n + d with
// M d = -F(n) and sum d = n_tot - sum n, the same update. With ``correction``
// (mixed mode, once the iteration has settled) the correction d is solved
// from the residual the evaluation assembled in float-pair and FP64
// arithmetic, so that the FP32 sums in M (Psi*, the cross-coupling terms)
// affect the speed of convergence only and not the fixed point, which is then
// F(n) = 0 to the residual's accuracy (in optically thick lines the net rates
// cancel far below FP32 resolution of the gross rates). Far from the
// solution the direct form is the more robust one (M and c0 carry the same
// rounding), so the mixed mode starts with it.
__device__ double rh92_depth(const ColDesc& cd, int k, bool clamp, bool correction, double damp, double* out) {
  const ColTables& T = cd.t;
  const int nl = T.nl, nt = T.nt, nz = T.nz;
  double M[kMaxL * kMaxL], c0[kMaxL];
  for (int i = 0; i < nl * nl; ++i) M[i] = 0.0;
  for (int i = 0; i < nl; ++i) c0[i] = 0.0;
  const double* C = T.C + (size_t)k * nl * nl;
  for (int t = 0; t < nt; ++t) {
    const int lo = T.t_lo[t], up = T.t_up[t];
    const double* r = cd.w.rh + ((size_t)t * nz + k) * kRhStride;
    double coef[kMaxL];
    for (int j = 0; j < nl; ++j) coef[j] = 0.0;
    coef[lo] += r[0] + C[lo * nl + up];
    coef[up] -= r[1] + r[2] + C[up * nl + lo];
    for (int s = 0; s < nt; ++s) coef[T.t_up[s]] += r[kRhFixed + s];
    for (int j = 0; j < nl; ++j) {
      M[lo * nl + j] += coef[j];
      M[up * nl + j] -= coef[j];
    }
    c0[lo] += r[3];
    c0[up] -= r[3];
  }
  const int is = cd.w.istar[k];
  double* n = cd.w.n + k * nl;
  double rhs[kMaxL];
  if (correction) {
    const double* F = cd.w.F + (size_t)k * nl;   // F[is] = n_tot - sum n
    for (int i = 0; i < nl; ++i) rhs[i] = -F[i];
    rhs[is] = F[is];
  } else {
    for (int i = 0; i < nl; ++i) rhs[i] = -c0[i];
    rhs[is] = T.ntot[k];
  }
  for (int j = 0; j < nl; ++j) M[is * nl + j] = 1.0;
  if (!small_solve(M, rhs, nl)) return nan("");
  if (correction)
    for (int l = 0; l < nl; ++l) rhs[l] += n[l];   // n' = n + d
  double alpha = 1.0;
  if (clamp)
    for (int l = 0; l < nl; ++l) {
      const double d = rhs[l] - n[l];
      if (d < 0.0) alpha = fmin(alpha, 0.9 * n[l] / (-d));
    }
  double err = 0.0;
  double* o = out + (size_t)k * nl;
  for (int l = 0; l < nl; ++l) {
    double nn = clamp ? n[l] + alpha * (rhs[l] - n[l]) : rhs[l];
    if (damp < 1.0) nn = n[l] + damp * (nn - n[l]);
    err = fmax(err, 0.5 * fabs((nn - n[l]) / (nn + n[l])));
    o[l] = nn;
  }
  return err;
}

// ---------------------------------------------------------------------------
// Krylov / Newton step: one CTA per column
// ---------------------------------------------------------------------------
__device__ void apply_pinv(const ColDesc& cd, const double* in, double sign_in, const double* in2,
                           double sign_in2, double* out, bool precond = true) {
  // out = P^{-1} (sign_in in + sign_in2 in2): w.P holds the explicit block
  // inverses after a solver base evaluation; one thread per (depth, row)
  const int nz = cd.t.nz, nl = cd.t.nl;
  if (!precond) {   // no preconditioning: out = sign_in in + sign_in2 in2
    for (int idx = threadIdx.x; idx < nz * nl; idx += blockDim.x)
      out[idx] = sign_in * in[idx] + (in2 ? sign_in2 * in2[idx] : 0.0);
    return;
  }
  for (int idx = threadIdx.x; idx < nz * nl; idx += blockDim.x) {
    const int k = idx / nl, i = idx - k * nl;
    const double* Pi = cd.w.P + ((size_t)k * nl + i) * nl;
    const double* a = in + k * nl;
    const double* b2 = in2 ? in2 + k * nl : nullptr;
    double acc = 0.0;
    for (int j = 0; j < nl; ++j) {
      double xj = sign_in * a[j];
      if (b2) xj += sign_in2 * b2[j];
      acc += Pi[j] * xj;
    }
    out[idx] = acc;
  }
}

// Finite-difference JVPs (Sect. 2.4, Fig. 2): the step for direction u and
// the populations n + side eps u of the next evaluation. Called by every
// thread of the column's block.
__device__ void fd_prepare(const ColDesc& cd, SolverState* st, int scheme, const double* u, int side,
                           double* sh) {
  const int N = cd.t.nz * cd.t.nl;
  const double* n = cd.w.n;
  double su = 0.0, sn = 0.0, sa = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    su += u[i] * u[i];
    sn += n[i] * n[i];
    sa += fabs(n[i]);
  }
  su = block_sum(su, sh);
  sn = block_sum(sn, sh);
  sa = block_sum(sa, sh);
  const double un = sqrt(su);
  double eps = 1.0;
  if (un > 0.0) {
    if (scheme == 1) {
      const double b = 1e-6;
      eps = b * sa / ((double)N * un) + b;                 // eps_1
    } else {
      // eps_2: eps_mach^(1/r) sqrt(1 + ||n||)/||u||, r = 2 (forward) or 3 (central)
      const double root = scheme == 3 ? 6.0554544523933395e-06    // 2^(-52/3)
                                      : 1.4901161193847656e-08;   // 2^(-26)
      eps = root * sqrt(1.0 + sqrt(sn)) / un;
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) cd.w.np[i] = n[i] + side * eps * u[i];
  if (threadIdx.x == 0) {
    st->fd_eps = eps;
    st->fd_side = side;
  }
}

// <a, b> over the N entries of a column, summed by the whole block.
__device__ double block_dot(const double* a, const double* b, int N, double* sh) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) acc += a[i] * b[i];
  return block_sum(acc, sh);
}

// BiCGSTAB (van der Vorst 1992) on the left-preconditioned Newton system
// P^{-1} J x = -P^{-1} F with x_0 = 0 and the shadow residual r^ = r_0: each
// iteration is two state-machine steps, one per Jacobian-vector product
// (v = A p, then t = A s). Opening an iteration: rho' = <r^, r>,
// beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v). Returns false
// on a breakdown (rho' = 0), after which the Newton step takes the current x.
__device__ bool bicg_open(const ColDesc& cd, SolverState* st, double* sh) {
  const int N = cd.t.nz * cd.t.nl;
  double* Vb = cd.w.Vb;
  const double* r = Vb + (size_t)BS_R * N;
  const double* rh = Vb + (size_t)BS_RHAT * N;
  double* p = Vb + (size_t)BS_P * N;
  const double* v = Vb + (size_t)BS_V * N;
  const double rho = st->rho, alpha = st->alpha, omega = st->omega;
  const double rn = block_dot(rh, r, N, sh);
  if (!(rn != 0.0) || !(rn == rn)) return false;
  const double beta = (rn / rho) * (alpha / omega);
  for (int i = threadIdx.x; i < N; i += blockDim.x) p[i] = r[i] + beta * (p[i] - omega * v[i]);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->rho = rn;
    st->bstage = 0;
    st->j = BS_P;
  }
  return true;
}

// n = n_prev + alpha_k (step x^k) per depth, with the per-depth limiting of
// Sect. 2.2.2 when clamp is set (alpha_k = min(1, 0.9 min n_prev/|step dx|) over
// the negative entries), from the base populations saved in w.nprev; returns
// the population change 1/2 ||(n - n_prev)/(n + n_prev)||_inf of the column.
__device__ double newton_apply(const ColDesc& cd, bool clamp, double step, double* sh) {
  const int nz = cd.t.nz, nl = cd.t.nl;
  const double* x = cd.w.x;
  const double* np0 = cd.w.nprev;
  double* n = cd.w.n;
  double err = 0.0;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    double alpha = 1.0;
    if (clamp)
      for (int l = 0; l < nl; ++l) {
        const double dx = step * x[k * nl + l];
        if (dx < 0.0) alpha = fmin(alpha, 0.9 * np0[k * nl + l] / (-dx));
      }
    for (int l = 0; l < nl; ++l) {
      const double np = np0[k * nl + l];
      const double nn = np + alpha * (step * x[k * nl + l]);
      n[k * nl + l] = nn;
      err = fmax(err, 0.5 * fabs((nn - np) / (nn + np)));
    }
  }
  return block_max(err, sh);
}

constexpr int kKrylovThreads = 512;

__global__ void __launch_bounds__(kKrylovThreads) k_krylov(const ColDesc* __restrict__ cols,
                                                const SolverOpts* __restrict__ opts,
                                                int* status_out) {
  const ColDesc& cd = cols[blockIdx.x];
  const SolverOpts o = cd.opts ? *cd.opts : *opts;
  SolverState* st = cd.w.st;
  __shared__ double sh[32];
  __shared__ double s_h[kMaxKrylov + 1];
  __shared__ double s_y[kMaxKrylov];
  __shared__ double s_cs[kMaxKrylov], s_sn[kMaxKrylov];   // Givens state of the step
  __shared__ double s_H[(kMaxKrylov + 1) * kMaxKrylov];   // H and g for the least-squares solve
  __shared__ int s_next;      // decision broadcast
  __shared__ int s_solve;
  __shared__ double s_val;
  const int phase = st->phase;
  if (phase == PH_DONE) return;
  if ((phase == PH_JVP || phase == PH_RESTART) && st->ticks + 1 >= o.max_ticks) {
    // the tick budget runs out inside a Krylov solve: this product was the last
    if (threadIdx.x == 0) {
      st->F_calls++;
      st->jvp_calls++;
      st->ticks++;
      st->status = JFNK_E_TIMEOUT;
      st->phase = PH_DONE;
      status_out[blockIdx.x] = st->status;
    }
    return;
  }
  const int nz = cd.t.nz, nl = cd.t.nl, N = nz * nl;
  const int kmax = o.krylov_max;
  double* w = cd.w.w;
  double* x = cd.w.x;
  double* Vb = cd.w.Vb;
  enum { NX_NONE, NX_NEWTON, NX_START_GMRES, NX_DONE };
  int next = NX_NONE;
  double start_beta = 0.0;

  if (phase == PH_RH92) {
    // mixed mode: the correction form once the change has fallen below 1e-2
    const bool corr = cd.mixed && st->rh92_iter > 0 && st->err < 1e-2;
    const double damp = st->rh_damp > 0.0 ? st->rh_damp : 1.0;
    const int it0 = st->rh92_iter;
    __syncthreads();
    // the new populations are staged in w.x and committed only when every
    // depth's update is finite
    double err = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
      double e = rh92_depth(cd, k, o.clamp != 0, corr, damp, cd.w.x);
      err = (e == e) ? fmax(err, e) : INFINITY;
    }
    err = block_max(err, sh);
    if (!(err < INFINITY) && it0 > 0 && damp > 1.0 / 64.0) {
      // a non-finite evaluation or update (a marginal column driven into an
      // unphysical state by the previous step): back to the populations of the
      // last iteration that evaluated finitely, and half the RH92 step from
      // there; J^dagger is still that evaluation's mean intensity
      for (int i = threadIdx.x; i < N; i += blockDim.x) cd.w.n[i] = cd.w.nprev[i];
      if (threadIdx.x == 0) {
        st->F_calls++;
        st->ticks++;
        st->rh_damp = 0.5 * damp;
        if (st->ticks >= o.max_ticks) { st->status = JFNK_E_TIMEOUT; st->phase = PH_DONE; }
        status_out[blockIdx.x] = st->status;
      }
      return;
    }
    if (err < INFINITY) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        cd.w.nprev[i] = cd.w.n[i];
        cd.w.n[i] = cd.w.x[i];
      }
    }
    if (threadIdx.x == 0) st->rh_damp = fmin(1.0, 2.0 * damp);
    // ||F||_inf of the evaluation the update was formed from (reported by
    // RH92-only solves)
    double fm = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) fm = fmax(fm, fabs(cd.w.F[i]));
    fm = block_max(fm, sh);
    if (threadIdx.x == 0) {
      st->jsel ^= 1;   // J(n) becomes the lagged J^dagger
      st->F_calls++;
      st->ticks++;
      st->rh92_iter++;
      st->err = err;
      if (o.solver == JFNK_SOLVER_RH92) {
        st->Fnorm = fm;
        if (st->rh92_iter == 1) st->F0norm = fm;
      }
      if (!(err < INFINITY)) { st->status = JFNK_E_NAN; st->phase = PH_DONE; }
      else if (o.solver == JFNK_SOLVER_RH92) {
        // the reference method alone: converged on the population change
        if (err < o.ftol) { st->status = JFNK_OK; st->phase = PH_DONE; }
        else if (st->rh92_iter >= o.maxiter) { st->status = JFNK_E_MAXITER; st->phase = PH_DONE; }
        else if (st->ticks >= o.max_ticks) { st->status = JFNK_E_TIMEOUT; st->phase = PH_DONE; }
      }
      else if (err < o.rh92_switch || st->rh92_iter >= o.rh92_warmup) st->phase = PH_BASE;
      else if (st->ticks >= o.max_ticks) { st->status = JFNK_E_TIMEOUT; st->phase = PH_DONE; }
      status_out[blockIdx.x] = st->status;
    }
    return;
  }

  if (phase == PH_BASE) {
    double fm = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      double f = cd.w.F[i];
      if (!(fabs(f) < INFINITY)) bad = true;
      fm = fmax(fm, fabs(f));
    }
    fm = block_max(bad ? INFINITY : fm, sh);
    if (o.line_search > 0 && st->ls_pending) {
      // this base evaluation is a trial point of the line search (Sect. 2.2.2):
      // accepted when ||F||_inf fell below its value at the previous base point,
      // else the correction is halved from the previous populations and tried
      // again (the lagged J^dagger stays that of the previous base point); the
      // last allowed trial is kept either way
      const bool better = (fm < INFINITY) && fm < st->ls_Fprev;
      const int left = st->ls_left;
      const double step = st->ls_step;
      __syncthreads();
      if (!better && left > 0) {
        const double e = newton_apply(cd, o.clamp != 0, 0.5 * step, sh);
        if (threadIdx.x == 0) {
          st->F_calls++;
          st->ticks++;
          st->ls_step = 0.5 * step;
          st->ls_left = left - 1;
          st->err = e;
          if (st->ticks >= o.max_ticks) { st->status = JFNK_E_TIMEOUT; st->phase = PH_DONE; }
          status_out[blockIdx.x] = st->status;
        }
        return;
      }
      if (threadIdx.x == 0) st->ls_pending = 0;
    }
    if (threadIdx.x == 0) {
      st->F_calls++;
      st->ticks++;
      st->Fnorm = fm;
      st->fd_scheme = o.jvp;   // the kind of this Newton step's JVP evaluations
      int nx = NX_START_GMRES;
      if (!(fm < INFINITY)) { st->status = JFNK_E_NAN; nx = NX_DONE; }
      else if (st->newton_iter == 0) st->F0norm = fm;
      else if (st->err <= o.ftol && fm <= o.fdrop * st->F0norm) { st->status = JFNK_OK; nx = NX_DONE; }
      if (nx != NX_DONE && st->newton_iter >= o.maxiter) { st->status = JFNK_E_MAXITER; nx = NX_DONE; }
      if (nx != NX_DONE && st->ticks >= o.max_ticks) { st->status = JFNK_E_TIMEOUT; nx = NX_DONE; }
      s_next = nx;
    }
    __syncthreads();
    next = s_next;
    if (next == NX_DONE) {
      if (threadIdx.x == 0) { st->phase = PH_DONE; status_out[blockIdx.x] = st->status; }
      return;
    }
    // r0 = -P^{-1} F (x0 = 0)
    apply_pinv(cd, cd.w.F, -1.0, nullptr, 0.0, w, o.precond != 0);
    for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = 0.0;
    __syncthreads();
    double ss = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) ss += w[i] * w[i];
    double beta = sqrt(block_sum(ss, sh));
    if (threadIdx.x == 0) {
      st->r0norm = beta;
      st->restarts = 0;
    }
    next = NX_START_GMRES;
    if (!(beta > 0.0)) {
      // F is exactly zero: nothing to correct
      if (threadIdx.x == 0) { st->status = (beta == 0.0) ? JFNK_OK : JFNK_E_NAN; st->phase = PH_DONE; status_out[blockIdx.x] = st->status; }
      return;
    }
    start_beta = beta;
    if (o.krylov == JFNK_KRYLOV_BICGSTAB) {
      // r = r^ = P^{-1}(-F), p = v = 0, rho = alpha = omega = 1
      double* Vr = Vb + (size_t)BS_R * N;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        Vr[i] = w[i];
        Vb[(size_t)BS_RHAT * N + i] = w[i];
        Vb[(size_t)BS_P * N + i] = 0.0;
        Vb[(size_t)BS_V * N + i] = 0.0;
      }
      if (threadIdx.x == 0) {
        st->rho = st->alpha = st->omega = 1.0;
        st->bit = 0;
      }
      __syncthreads();
      if (bicg_open(cd, st, sh)) {
        if (o.jvp) fd_prepare(cd, st, o.jvp, Vb + (size_t)BS_P * N, +1, sh);
        if (threadIdx.x == 0) { st->phase = PH_JVP; status_out[blockIdx.x] = st->status; }
        return;
      }
      next = NX_NEWTON;   // breakdown at the start: the Newton step keeps x = 0
    }
  } else if (o.krylov == JFNK_KRYLOV_BICGSTAB) {
    // a Jacobian-vector product of BiCGSTAB (A p or A s) is in dF
    const int scheme = st->fd_scheme;
    if (scheme) {
      const int side = st->fd_side;
      const double eps = st->fd_eps;
      const double* u = Vb + (size_t)st->j * N;
      __syncthreads();   // every thread has read the state before it changes
      if (scheme == 3 && side > 0) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
          cd.w.fdp[i] = cd.w.dF[i];
          cd.w.np[i] = cd.w.n[i] - eps * u[i];
        }
        if (threadIdx.x == 0) {
          st->fd_side = -1;
          st->F_calls++;
          st->ticks++;
          status_out[blockIdx.x] = st->status;
        }
        return;
      }
      for (int i = threadIdx.x; i < N; i += blockDim.x)
        cd.w.dF[i] = scheme == 3 ? (cd.w.fdp[i] - cd.w.dF[i]) / (2.0 * eps) : (cd.w.dF[i] - cd.w.F[i]) / eps;
      __syncthreads();
    }
    const int stage = st->bstage;
    const double r0n = st->r0norm;
    __syncthreads();
    if (threadIdx.x == 0) { st->F_calls++; st->jvp_calls++; st->ticks++; }
    double* r = Vb + (size_t)BS_R * N;
    const double* rh = Vb + (size_t)BS_RHAT * N;
    const double* p = Vb + (size_t)BS_P * N;
    double* v = Vb + (size_t)BS_V * N;
    double* sv = Vb + (size_t)BS_S * N;
    double* t = Vb + (size_t)BS_T * N;
    bool fin = false, bad = false;
    if (stage == 0) {
      // v = P^{-1} J p, alpha = rho/<r^, v>, s = r - alpha v
      apply_pinv(cd, cd.w.dF, 1.0, nullptr, 0.0, v, o.precond != 0);
      __syncthreads();
      const double alpha = st->rho / block_dot(rh, v, N, sh);
      for (int i = threadIdx.x; i < N; i += blockDim.x) sv[i] = r[i] - alpha * v[i];
      __syncthreads();
      const double sn = sqrt(block_dot(sv, sv, N, sh));
      bad = !(alpha == alpha) || !(sn == sn);
      if (!bad && sn < o.rtol * r0n) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] += alpha * p[i];
        fin = true;
      } else if (!bad) {
        if (threadIdx.x == 0) {
          st->alpha = alpha;
          st->bstage = 1;
          st->j = BS_S;
        }
        if (o.jvp) fd_prepare(cd, st, o.jvp, sv, +1, sh);
        if (threadIdx.x == 0) { st->phase = PH_JVP; status_out[blockIdx.x] = st->status; }
        return;
      }
    } else {
      // t = P^{-1} J s, omega = <t, s>/<t, t>, x += alpha p + omega s, r = s - omega t
      apply_pinv(cd, cd.w.dF, 1.0, nullptr, 0.0, t, o.precond != 0);
      __syncthreads();
      const double ts = block_dot(t, sv, N, sh), tt = block_dot(t, t, N, sh);
      const double omega = tt > 0.0 ? ts / tt : 0.0;
      const double alpha = st->alpha;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        x[i] += alpha * p[i] + omega * sv[i];
        r[i] = sv[i] - omega * t[i];
      }
      __syncthreads();
      const double rn = sqrt(block_dot(r, r, N, sh));
      const int it = st->bit + 1;
      bad = !(omega == omega) || !(rn == rn);
      __syncthreads();
      if (threadIdx.x == 0) {
        st->omega = omega;
        st->bit = it;
      }
      __syncthreads();
      fin = bad || rn < o.rtol * r0n || omega == 0.0 || it >= kBicgMaxIter;
      if (!fin) {
        if (bicg_open(cd, st, sh)) {
          if (o.jvp) fd_prepare(cd, st, o.jvp, Vb + (size_t)BS_P * N, +1, sh);
          if (threadIdx.x == 0) { st->phase = PH_JVP; status_out[blockIdx.x] = st->status; }
          return;
        }
        fin = true;   // breakdown: the Newton step takes the current x
      }
    }
    if (bad) {
      if (threadIdx.x == 0) { st->status = JFNK_E_NAN; st->phase = PH_DONE; status_out[blockIdx.x] = st->status; }
      return;
    }
    __syncthreads();
    next = NX_NEWTON;
  } else {
    // a Jacobian-vector product J u is in dF (u = V_j or u = x); with a
    // difference scheme dF holds F(n + side eps u) and the quotient is formed here
    const int scheme = st->fd_scheme;
    if (scheme) {
      const int side = st->fd_side;
      const double eps = st->fd_eps;
      const double* u = (phase == PH_RESTART) ? x : Vb + (size_t)st->j * N;
      __syncthreads();   // every thread has read the state before it changes
      if (scheme == 3 && side > 0) {
        // central difference, first half: keep F(n + eps u), evaluate F(n - eps u) next
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
          cd.w.fdp[i] = cd.w.dF[i];
          cd.w.np[i] = cd.w.n[i] - eps * u[i];
        }
        if (threadIdx.x == 0) {
          st->fd_side = -1;
          st->F_calls++;
          st->ticks++;
          status_out[blockIdx.x] = st->status;
        }
        return;
      }
      for (int i = threadIdx.x; i < N; i += blockDim.x)
        cd.w.dF[i] = scheme == 3 ? (cd.w.fdp[i] - cd.w.dF[i]) / (2.0 * eps) : (cd.w.dF[i] - cd.w.F[i]) / eps;
      __syncthreads();
    }
    if (threadIdx.x == 0) { st->F_calls++; st->jvp_calls++; st->ticks++; }
    if (phase == PH_RESTART) {
      apply_pinv(cd, cd.w.F, -1.0, cd.w.dF, -1.0, w, o.precond != 0);   // r = P^{-1}(-F - J x)
      __syncthreads();
      double ss = 0.0;
      for (int i = threadIdx.x; i < N; i += blockDim.x) ss += w[i] * w[i];
      double beta = sqrt(block_sum(ss, sh));
      if (threadIdx.x == 0) {
        if (!(beta == beta)) { st->status = JFNK_E_NAN; s_next = NX_DONE; }
        else if (beta < o.rtol * st->r0norm) s_next = NX_NEWTON;
        else { st->restarts++; s_next = NX_START_GMRES; }
        s_val = beta;
      }
      __syncthreads();
      next = s_next;
      start_beta = s_val;
      if (next == NX_DONE) {
        if (threadIdx.x == 0) { st->phase = PH_DONE; status_out[blockIdx.x] = st->status; }
        return;
      }
    } else {
      const int j = st->j;
      apply_pinv(cd, cd.w.dF, 1.0, nullptr, 0.0, w, o.precond != 0);
      __syncthreads();
      // classical Gram-Schmidt, twice (CGS2)
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
      for (int i = threadIdx.x; i <= j; i += blockDim.x) s_h[i] = 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = wid; i <= j; i += nwarp) {
          const double* vi = Vb + (size_t)i * N;
          double s = 0.0;
          for (int e = lane; e < N; e += 32) s += vi[e] * w[e];
          s = warp_sum(s);
          if (lane == 0) s_y[i] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < N; e += blockDim.x) {
          double acc = w[e];
          for (int i = 0; i <= j; ++i) acc -= s_y[i] * Vb[(size_t)i * N + e];
          w[e] = acc;
        }
        for (int i = threadIdx.x; i <= j; i += blockDim.x) s_h[i] += s_y[i];
        __syncthreads();
      }
      double ss = 0.0;
      for (int i = threadIdx.x; i < N; i += blockDim.x) ss += w[i] * w[i];
      const double hnext = sqrt(block_sum(ss, sh));
      // the Givens state staged in shared memory by every thread, so that the
      // serial update below touches no global memory on its dependent chain
      for (int i = threadIdx.x; i < j; i += blockDim.x) {
        s_cs[i] = cd.w.cs[i];
        s_sn[i] = cd.w.sn[i];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double* Hh = cd.w.Hh;
        double* gv = cd.w.gv;
        s_h[j + 1] = hnext;
        for (int i = 0; i < j; ++i) {   // previous Givens rotations
          const double a = s_h[i], bb = s_h[i + 1];
          s_h[i] = s_cs[i] * a + s_sn[i] * bb;
          s_h[i + 1] = -s_sn[i] * a + s_cs[i] * bb;
        }
        const double a = s_h[j], bb = s_h[j + 1];
        const double rr = hypot(a, bb);
        const double cj = rr == 0.0 ? 1.0 : a / rr, sj = rr == 0.0 ? 0.0 : bb / rr;
        cd.w.cs[j] = cj;
        cd.w.sn[j] = sj;
        s_h[j] = rr;
        s_h[j + 1] = 0.0;
        for (int i = 0; i <= j + 1; ++i) Hh[i * kmax + j] = s_h[i];   // column j of the rotated H
        const double gj = gv[j];
        gv[j + 1] = -sj * gj;
        gv[j] = cj * gj;
        const double resid = fabs(sj * gj);
        const bool conv = resid < o.rtol * st->r0norm || !(hnext > 1e-300 * st->r0norm);
        const bool full = (j + 1 >= kmax);
        int nx, solve = 0;
        if (!(resid == resid) || !(rr == rr)) { st->status = JFNK_E_NAN; nx = NX_DONE; }
        else if (!conv && !full) nx = NX_NONE;       // continue Arnoldi
        else {
          solve = 1;                                  // y = H^{-1} g below
          nx = (conv || st->restarts >= o.max_restarts) ? NX_NEWTON : 100;   // 100: restart
        }
        s_next = nx;
        s_solve = solve;
        s_val = hnext;
      }
      __syncthreads();
      if (s_solve) {
        // y = H^{-1} g (upper triangular, j+1): H and g gathered into shared
        // memory by every thread, then one back substitution
        const int m1 = j + 1;
        for (int e = threadIdx.x; e < m1 * m1; e += blockDim.x) {
          const int r = e / m1, c = e - r * m1;
          s_H[r * kMaxKrylov + c] = c >= r ? cd.w.Hh[r * kmax + c] : 0.0;
        }
        for (int r = threadIdx.x; r < m1; r += blockDim.x) s_y[r] = cd.w.gv[r];
        __syncthreads();
        if (threadIdx.x == 0)
          for (int r = j; r >= 0; --r) {
            double sv = s_y[r];
            for (int c = r + 1; c <= j; ++c) sv -= s_H[r * kMaxKrylov + c] * s_y[c];
            s_y[r] = sv / s_H[r * kMaxKrylov + r];
          }
        __syncthreads();
      }
      next = s_next;
      if (next == NX_DONE) {
        if (threadIdx.x == 0) { st->phase = PH_DONE; status_out[blockIdx.x] = st->status; }
        return;
      }
      if (next == NX_NONE) {
        const double hn = s_val;
        double* vn = Vb + (size_t)(j + 1) * N;
        for (int e = threadIdx.x; e < N; e += blockDim.x) vn[e] = w[e] / hn;
        if (o.jvp) {
          __syncthreads();
          fd_prepare(cd, st, o.jvp, vn, +1, sh);
        }
        if (threadIdx.x == 0) { st->j = j + 1; st->phase = PH_JVP; status_out[blockIdx.x] = st->status; }
        return;
      }
      // x += V y
      for (int e = threadIdx.x; e < N; e += blockDim.x) {
        double acc = x[e];
        for (int i = 0; i <= j; ++i) acc += s_y[i] * Vb[(size_t)i * N + e];
        x[e] = acc;
      }
      __syncthreads();
      if (next == 100) {
        if (o.jvp) fd_prepare(cd, st, o.jvp, x, +1, sh);   // the restart residual needs J x
        if (threadIdx.x == 0) { st->phase = PH_RESTART; status_out[blockIdx.x] = st->status; }
        return;
      }
    }
  }

  if (next == NX_START_GMRES) {
    const double beta = start_beta;
    for (int e = threadIdx.x; e < N; e += blockDim.x) Vb[e] = w[e] / beta;
    if (o.jvp) {
      __syncthreads();
      fd_prepare(cd, st, o.jvp, Vb, +1, sh);
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i <= kmax; ++i) cd.w.gv[i] = 0.0;
      cd.w.gv[0] = beta;
      st->j = 0;
      st->phase = PH_JVP;
      status_out[blockIdx.x] = st->status;
    }
    return;
  }

  // Newton update with per-depth limiting (Sect. 2.2.2): n += alpha_k x^k,
  // from the base populations kept in w.nprev (a line search may halve it)
  for (int i = threadIdx.x; i < N; i += blockDim.x) cd.w.nprev[i] = cd.w.n[i];
  __syncthreads();
  const double err = newton_apply(cd, o.clamp != 0, 1.0, sh);
  if (threadIdx.x == 0) {
    st->jsel ^= 1;   // J(n^p) becomes J^dagger_{p+1}
    st->err = err;
    st->newton_iter++;
    st->phase = PH_BASE;
    st->ls_pending = o.line_search > 0;
    st->ls_left = o.line_search;
    st->ls_step = 1.0;
    st->ls_Fprev = st->Fnorm;   // ||F||_inf at the base point n^p
    status_out[blockIdx.x] = st->status;
  }
}

int launch_krylov_step(const Batch& b, cudaStream_t s) {
  k_krylov<<<b.ncols, kKrylovThreads, 0, s>>>(b.d_cols, b.d_opts, b.d_status);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

__global__ void k_rh92_apply(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cd.t.nz) return;
  rh92_depth(cd, k, false, false, 1.0, cd.w.n);   // the plain update: jfnk_rh92_update applies no limiting
}

// Zero-radiation initial guess (Sect. 2.2.1): the rate equations with I = 0,
// i.e. collisions plus spontaneous radiative rates R_ji = sum_nu W g V
// 2 h nu^3/c^2 (the J = 0 limit of Eqs. Rij/Rji), with the conservation row on
// the most populated LTE level; one thread per depth. Expects n = LTE.
__global__ void k_zero_radiation(const ColDesc* __restrict__ cols) {
  const ColDesc& cd = cols[blockIdx.y];
  const ColTables& T = cd.t;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.nz) return;
  const int nl = T.nl, nt = T.nt, nz = T.nz;
  double M[kMaxL * kMaxL], rhs[kMaxL];
  for (int i = 0; i < nl * nl; ++i) M[i] = 0.0;
  const double* C = T.C + (size_t)k * nl * nl;
  for (int t = 0; t < nt; ++t) {
    const int lo = T.t_lo[t], up = T.t_up[t], q0 = T.t_q0[t], q1 = T.t_q1[t], base = T.t_base[t];
    double rdn = 0.0;
    for (int q = q0; q <= q1; ++q) {
      const size_t p = (size_t)(base + q - q0);
      rdn += T.t_w[p] * T.rw[q] * T.G[p * nz + k] * T.V[p * nz + k] * T.c2[q];
    }
    const double ur = C[lo * nl + up], dr = C[up * nl + lo] + rdn;
    // d n_lo/dt = -n_lo ur + n_up dr, d n_up/dt = +n_lo ur - n_up dr
    M[lo * nl + lo] += ur;
    M[lo * nl + up] -= dr;
    M[up * nl + lo] -= ur;
    M[up * nl + up] += dr;
  }
  double* n = cd.w.n + (size_t)k * nl;
  int is = 0;
  for (int l = 1; l < nl; ++l)
    if (n[l] > n[is]) is = l;
  for (int l = 0; l < nl; ++l) rhs[l] = 0.0;
  for (int j = 0; j < nl; ++j) M[is * nl + j] = 1.0;
  rhs[is] = T.ntot[k];
  if (!small_solve(M, rhs, nl)) return;   // singular: the LTE start stays
  for (int l = 0; l < nl; ++l) n[l] = rhs[l];
}

int launch_zero_radiation(const Batch& b, cudaStream_t s) {
  dim3 g((b.max_nz + 63) / 64, b.ncols);
  k_zero_radiation<<<g, 64, 0, s>>>(b.d_cols);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

int launch_rh92_update(const Batch& b, cudaStream_t s) {
  dim3 g((b.max_nz + 63) / 64, b.ncols);
  k_rh92_apply<<<g, 64, 0, s>>>(b.d_cols);
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

}  // namespace jfnk
