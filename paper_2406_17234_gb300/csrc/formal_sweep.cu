// Mixed-precision formal solution + ray sums, one thread per (frequency,
// column): the thread carries every angle of a hemisphere at once (n_mu
// independent recurrences, the instruction-level parallelism of the sweep)
// and walks the column twice.
//
//   down sweep (mu < 0 rays, top to bottom): the per-depth sums of the
//     hemisphere over its angles go to a scratch array laid out [k][q], so
//     that the threads of a warp (consecutive frequencies) write one
//     contiguous segment per depth;
//   up sweep (mu > 0 rays, bottom to top): the hemisphere's own sums are added
//     to the stored ones and the depth's outputs are written (J, J_new,
//     Lambda_chi, Lambda_eta in base evaluations, dJ in tangent ones).
//
// No per-ray value is stored anywhere: the coefficients of a step (App. A.1,
// App. A.2) are formed in registers right where the recurrence needs them,
// and the optical-depth reciprocal of a layer is shared by the angles.
//
// The recurrences are those of the fused kernel (Eqs. Iplus/Iminus in the
// difference form D = I - S, the tangent dD, and in base evaluations the
// intensity form I with the re-anchoring of D on I - S); only the order of
// the ray sums differs: each hemisphere is summed over its angles first and
// the two hemisphere sums are then added.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "formal_coef.cuh"

namespace jfnk {

constexpr int kSweepParts = 5;   // base: sum D, sum |D|, sum I, sum dI/dchi, sum dI/deta (x 1/2 w)

// Scratch of the down sweep: [kSweepParts][nz][col_pitch(nq)] floats.
__host__ __device__ inline int sweep_pitch(int nq) { return col_pitch(nq); }

size_t sweep_scratch_bytes(int nq, int nz) {
  return sizeof(float) * (size_t)kSweepParts * nz * sweep_pitch(nq);
}

// App. A.1 coefficients of a step of optical depth x (r = 1/x): e = exp(-x),
// w = (1 - e)/x, a = 1 - w, bq = (w - e)/x; below x = 0.1 each comes from its
// Taylor series (truncated after x^5, below 3e-10 relative).
// e^(-x) on the MUFU as 2^(-x log2 e) (flush-to-zero: e below 2^-126 is 0).
__device__ __forceinline__ float exp_neg(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(mul(x, -1.4426950408889634f)));
  return y;
}

// Asynchronous 4-byte copies global -> shared (each thread copies and later
// reads back only its own words, so waiting on its own copy groups suffices).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Fused tangent sweep: the line-table entries of each depth are copied into a
// shared-memory ring kRing - 1 depths ahead of the recurrence; a stage holds
// per thread V, G, v_lo, v_up of the first two transitions and S.
constexpr int kRing = 4;
constexpr int kRingSlots = 9;
__host__ __device__ inline size_t ring_floats(int threads) { return (size_t)kRing * kRingSlots * threads; }

// Which form of the coefficients a step takes: chosen per step (CM_EITHER),
// or known for every angle of the depth (CM_SERIES: all steps below 0.1;
// CM_DIRECT: none), the same choice as CM_EITHER makes for each step.
enum CoefMode { CM_EITHER = 0, CM_SERIES = 1, CM_DIRECT = 2 };

template <int CM = CM_EITHER>
__device__ __forceinline__ void pl_coef_rn(float x, float r, float& e, float& w, float& a, float& bq) {
  e = exp_neg(x);
  if (CM == CM_SERIES || (CM == CM_EITHER && x < 0.1f)) {
    w = fma3(fma3(fma3(fma3(fma3(-1.0f / 720.0f, x, 1.0f / 120.0f), x, -1.0f / 24.0f), x, 1.0f / 6.0f), x, -0.5f), x, 1.0f);
    a = mul(x, fma3(fma3(fma3(fma3(fma3(-1.0f / 5040.0f, x, 1.0f / 720.0f), x, -1.0f / 120.0f), x, 1.0f / 24.0f), x, -1.0f / 6.0f), x, 0.5f));
    bq = fma3(fma3(fma3(fma3(1.0f / 144.0f, x, -1.0f / 30.0f), x, 1.0f / 8.0f), x, -1.0f / 3.0f), x, 0.5f);
  } else {
    w = mul(sub(1.0f, e), r);
    a = sub(1.0f, w);
    bq = mul(sub(w, e), r);
  }
}

// Quantities of one depth step shared by all angles of a hemisphere.
struct StepIn {
  float csum;    // chi^k + chi^u
  float rs;      // 1/(chi^k + chi^u)
  float dzk;     // |z_k - z_u|
  float idzk;    // 1/|z_k - z_u|
  float tz;      // |dz| (chi^k + chi^u):   dtau = tz / (2 mu)
  float rz;      // 1/(|dz| (chi^k + chi^u)): 1/dtau = rz 2 mu
  float dtz;     // |dz| (dchi^k + dchi^u): ddtau = dtz / (2 mu)
  float dSin;    // S^u - S^k (formed from the S pairs, then rounded)
  float S0, Su;  // S^k, S^u
  float rc0;     // 1/chi^k
  float dcs;     // dchi^k + dchi^u
  float ddSin;   // dS^u - dS^k
};

// Contributions of one ray to the sums of its depth, each already x 1/2 w_mu.
struct RayOut {
  float xD, xI, xx, xe, xd;
};

// One step of one ray into depth k from its upstream neighbour u:
//   D^k  = D^u e + w (S^u - S^k)                                  (D = I - S)
//   dD^k = dD^u e - ddtau (e D^u + bq (S^u - S^k)) + w (dS^u - dS^k)
//   I^k  = I^u e + a S^k + b S^u,  b = bq dtau                      (base)
//   dI^k/dchi^k = -(S^k/chi^k) a - h (S^u - S^k) bq - h e D^u,      (App. A.2)
//   dI^k/deta^k = a/chi^k,  h = |dz|/(2 mu), dtau = h (chi^k + chi^u)
// In base evaluations D is re-anchored on I - S whenever that is the
// better-conditioned value: D carries an absolute error of the order of the
// largest |D| met upstream (attenuated along the ray), I - S one of the order
// of |I| + |S|.
template <bool TAN, int CM = CM_EITHER>
__device__ __forceinline__ RayOut ray_step(const StepIn& in, float inv2mu, float two_mu, float hw, float& D,
                                           float& I, float& M, float& dD) {
  RayOut o;
  // the depth's factors are formed once per depth (StepIn), one multiply per angle here
  const float dtau = mul(in.tz, inv2mu);
  const float rdt = mul(in.rz, two_mu);
  float e, w, a, bq;
  pl_coef_rn<CM>(dtau, rdt, e, w, a, bq);
  const float Du = D;
  float Dn = fma3(Du, e, mul(w, in.dSin));
  if (TAN) {
    const float ddtau = mul(in.dtz, inv2mu);
    const float dDn = fma3(dD, e, fma3(-ddtau, fma3(e, Du, mul(bq, in.dSin)), mul(w, in.ddSin)));
    dD = dDn;
    o.xd = mul(hw, dDn);
    o.xD = o.xI = o.xx = o.xe = 0.f;
  } else {
    const float h = mul(in.dzk, inv2mu);
    const float In = fma3(I, e, fma3(a, in.S0, mul(mul(bq, dtau), in.Su)));
    const float lx = -fma3(mul(in.S0, in.rc0), a, mul(h, fma3(in.dSin, bq, mul(e, Du))));
    o.xI = mul(hw, In);
    o.xx = mul(hw, lx);
    o.xe = mul(hw, mul(a, in.rc0));
    M = fmaxf(mul(M, e), fabsf(Dn));
    const float anchor = add(fabsf(In), fabsf(in.S0));
    if (anchor < M) {
      Dn = sub(In, in.S0);
      M = anchor;
    }
    I = In;
    o.xD = mul(hw, Dn);
    o.xd = 0.f;
  }
  D = Dn;
  return o;
}

// Sum of the angle contributions in the fixed tree of a 3-level xor butterfly
// over 8 lanes, (x0 + x4) + (x2 + x6) and (x1 + x5) + (x3 + x7), with the terms
// of angles m >= MU (zero by construction, known at compile time) left out:
// x + 0 = x, so the sum has the butterfly's value.
struct Part {
  float v;
  bool on;
};
__device__ __forceinline__ Part padd(Part a, Part b) {
  if (a.on && b.on) return Part{add(a.v, b.v), true};
  return a.on ? a : b;
}
template <int MU>
__device__ __forceinline__ float tree_mu(const float* x) {
  Part p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = Part{i < MU ? x[i] : 0.f, i < MU};
  const Part s = padd(padd(padd(p[0], p[4]), padd(p[2], p[6])), padd(padd(p[1], p[5]), padd(p[3], p[7])));
  return s.on ? s.v : 0.f;
}
__device__ __forceinline__ float butterfly8(float v) {
  v = add(v, __shfl_xor_sync(0xffffffffu, v, 4));
  v = add(v, __shfl_xor_sync(0xffffffffu, v, 2));
  v = add(v, __shfl_xor_sync(0xffffffffu, v, 1));
  return v;
}

// Output of one depth from the two hemisphere sums (base: D, |D|, I, Lchi, Leta).
// J = (S + sum D) c2, or (sum I) c2 where that representation carries the
// smaller rounding error (intensities are >= 0), is formed in pair arithmetic
// and written once, into J_new (the rates read it there); the Lambda
// diagonals are FP32 sums and stay float. The sweeps serve the mixed mode
// only, whose Jacobian-vector products are exact tangents (no difference
// evaluations).
struct BaseOut {
  df J;
  float lx, le;
};
__device__ __forceinline__ BaseOut base_out(df Sk, df c2, float c2f, float fD, float fa, float fI, float fx, float fe) {
  BaseOut r;
  r.J = fabsf(fI) < fa ? df_mul_f(c2, fI) : df_mul(df_add_f(Sk, fD), c2);
  r.lx = mul(fx, c2f);
  r.le = fe;
  return r;
}
__device__ __forceinline__ void write_base(const ColDesc& cd, size_t o, df Sk, df c2, float c2f, float fD, float fa,
                                           float fI, float fx, float fe) {
  const BaseOut r = base_out(Sk, c2, c2f, fD, fa, fI, fx, fe);
  df_store(as_pairs(jnew_ptr(cd)), o, r.J);
  cd.w.Lchi32[o] = r.lx;
  cd.w.Leta32[o] = r.le;
}

// Outward pass of a base-type sweep: the per-frequency output rows ([q][k]:
// J pair, Lchi, Leta) are staged per warp for kStageD depths in shared memory
// ([plane][lane][depth], row stride kStageD + 1: the 32 lanes' words of one
// depth fall in 32 banks) and then written row by row, consecutive lanes on
// consecutive depths of a row, instead of one scattered word per lane.
// (Staging the input rows the same way, through a double buffer of
// asynchronous copies, was slower: 1.02 against 0.94 ms per tick; the larger
// shared memory leaves less L1, where those rows are mostly hits.)
constexpr int kStageD = 8;
constexpr int kStagePlane = 32 * (kStageD + 1);
constexpr int kWarpStage = 4 * kStagePlane;
__host__ __device__ inline size_t stage_floats(int threads) { return (size_t)(threads / 32) * kWarpStage; }
// Tangent output: dJ (normalised by 2 h nu^3/c^2) in float, depth-major, read
// by the FP32 tangent rate integrals; o indexes the depth-major arrays.
__device__ __forceinline__ void write_tan(const ColDesc& cd, size_t o, float dS, float fd) {
  cd.w.dJ32T[o] = add(dS, fd);
}

// Stages |dz| and 1/|dz| of the block's column in shared memory.
__device__ __forceinline__ void stage_dz(const ColTables& T, float* s_dz, float* s_idz) {
  for (int k = threadIdx.x; k < T.nz - 1; k += blockDim.x) {
    const float2 d = T.dz32[k];
    s_dz[k] = d.x;
    s_idz[k] = d.y;
  }
}

// ---------------------------------------------------------------------------
// Variant 1: one thread per frequency, all angles of a hemisphere in registers.
// ---------------------------------------------------------------------------
// Base evaluations read chi and S per frequency row ([q][k], S as a float
// pair), form S^u - S^k in pair arithmetic, and leave depth-major float
// copies of chi, S and the rounded differences for the tangent evaluations
// of the same Newton step;
// those then read depth-major float arrays only (one 128-byte line per warp
// and depth) and run entirely in FP32.
// EXACT: the column has exactly MU angles (no per-angle guards). FUSE
// (tangent, inward pass): the opacity tangent dchi, dS of each depth is formed
// here from the line tables, with the arithmetic of the separate opacity
// kernel (tan_acc, tan_dS: the same bits), and stored for the outward pass.
template <int MU, bool TAN, bool UP, bool EXACT, bool FUSE = false>
__device__ __forceinline__ void sweep_thread(const ColDesc& cd, int q, const float* __restrict__ s_dz,
                                             const float* __restrict__ s_idz, float* __restrict__ s_ring = nullptr,
                                             float* __restrict__ s_stage = nullptr, unsigned amask = 0u,
                                             int na = 0) {
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq, nmu = T.nmu, nl = T.nl;
  const size_t pitch = (size_t)col_pitch(nq);
  const size_t pstride = (size_t)nz * pitch;
  const size_t row = (size_t)q * nz;
  const float* __restrict__ chi = reinterpret_cast<const float*>(cd.w.chi) + row;
  const float2* __restrict__ S2 = as_pairs(cd.w.S) + row;   // S as float pairs
  float* __restrict__ chiT = cd.w.chiT + q;
  float* __restrict__ S32T = cd.w.S32T + q;
  float* __restrict__ dSkT = cd.w.dSkT + q;
  const float* __restrict__ dchiT = cd.w.dchiT + q;
  const float* __restrict__ dS32T = cd.w.dS32T + q;
  float* __restrict__ part = reinterpret_cast<float*>(cd.w.part) + q;
  const double c2 = T.c2[q];
  const float c2f = T.c2f[q];
  const df c2p = df_load(T.c2p, q);

  float inv2mu[MU], hw[MU], two_mu[MU];
#pragma unroll
  for (int m = 0; m < MU; ++m) {
    const bool on = EXACT || m < nmu;
    const float4 a = on ? T.ang32[m] : make_float4(0.f, 0.f, 0.f, 0.f);
    inv2mu[m] = a.x;
    hw[m] = a.y;
    two_mu[m] = a.z;
  }
  // the transitions active at nu (packed window point << 8 | lo << 4 | up),
  // constant along the column: the first two held, the others read when used
  constexpr bool FT = FUSE && TAN && !UP;
  int pm0 = -1, pm1 = -1;
  if (FT) {
    pm0 = __ldg(T.qmeta + q);
    pm1 = __ldg(T.qmeta + (size_t)nq + q);
  }
  // FUSE: the asynchronous copies of depth kk's table entries into ring stage
  // kk % kRing (one commit group per depth, empty past the column's end)
  const int bd = blockDim.x;
  auto tan_issue = [&](int kk) {
    if (kk < nz) {
      float* r = s_ring + (size_t)(kk % kRing) * kRingSlots * bd + threadIdx.x;
      const float* __restrict__ VGk = reinterpret_cast<const float*>(T.VG32T + (size_t)kk * T.nwin);
      const float* __restrict__ vk = cd.w.v32 + (size_t)kk * nl;
      if (pm0 >= 0) {
        cp_async4(r, VGk + 2 * (pm0 >> 8));
        cp_async4(r + bd, VGk + 2 * (pm0 >> 8) + 1);
        cp_async4(r + 2 * bd, vk + ((pm0 >> 4) & 15));
        cp_async4(r + 3 * bd, vk + (pm0 & 15));
      }
      if (pm1 >= 0) {
        cp_async4(r + 4 * bd, VGk + 2 * (pm1 >> 8));
        cp_async4(r + 5 * bd, VGk + 2 * (pm1 >> 8) + 1);
        cp_async4(r + 6 * bd, vk + ((pm1 >> 4) & 15));
        cp_async4(r + 7 * bd, vk + (pm1 & 15));
      }
      cp_async4(r + 8 * bd, S32T + (size_t)kk * pitch);
    }
    cp_async_commit();
  };
  // ... and the opacity tangent of depth kk formed from its stage (and the
  // rest of the depth's transitions, read directly; the order of the
  // separate opacity kernel; chi_k: the float opacity of that depth), stored
  // for the outward pass. Every copy but those of the kRing - 2 most recent
  // depths has landed after the wait.
  auto tan_finish = [&](int kk, float chik, float& dc, float& dS) {
    cp_async_wait<kRing - 2>();
    const float* r = s_ring + (size_t)(kk % kRing) * kRingSlots * bd + threadIdx.x;
    TanAcc ta;
    if (pm0 >= 0) tan_acc(ta, r[0], r[bd], r[2 * bd], r[3 * bd]);
    if (pm1 >= 0) {
      tan_acc(ta, r[4 * bd], r[5 * bd], r[6 * bd], r[7 * bd]);
      const float2* __restrict__ VGk = T.VG32T + (size_t)kk * T.nwin;
      const float* __restrict__ vk = cd.w.v32 + (size_t)kk * nl;
#pragma unroll
      for (int j = 2; j < kQMetaT; ++j) {
        const int m = __ldg(T.qmeta + (size_t)j * nq + q);
        if (m < 0) break;
        const float2 a = __ldg(VGk + (m >> 8));
        tan_acc(ta, a.x, a.y, __ldg(vk + ((m >> 4) & 15)), __ldg(vk + (m & 15)));
      }
    }
    dc = ta.dchi;
    dS = tan_dS(ta, r[8 * bd], chik);
    const size_t o = (size_t)kk * pitch + q;
    cd.w.dchiT[o] = dc;
    cd.w.dS32T[o] = dS;
  };
  // tangent opacity of depth kk, left by the opacity kernel or (outward pass
  // of a fused sweep) by the inward pass
  auto tan_in = [&](int kk, float& dc, float& dS) {
    const size_t o = (size_t)kk * pitch;
    dc = dchiT[o];
    dS = dS32T[o];
  };

  // boundary depth: I = 0 at the top, I = B at the bottom (Sect. 2.1)
  const int k0 = UP ? nz - 1 : 0;
  df Sp = df_load(S2, k0);
  float cp = TAN ? chiT[k0 * pitch] : chi[k0];
  float dSp = 0.f, dcp = 0.f;
  if (FT) {
#pragma unroll
    for (int j = 0; j < kRing - 1; ++j) tan_issue(k0 + j);
    tan_finish(k0, cp, dcp, dSp);
    tan_issue(k0 + kRing - 1);
  } else if (TAN) {
    tan_in(k0, dcp, dSp);
  }
  float Su = Sp.hi;
  if (!TAN && !UP) {
    chiT[0] = cp;
    S32T[0] = Su;
  }
  const double Ib64 = UP ? T.Bn[row + nz - 1] / c2 : 0.0;
  const float D0 = df_to_float(df_sub(df_from_double(Ib64), Sp));
  const float I0 = __double2float_rn(Ib64);
  const float dD0 = -dSp;
  float D[MU], I[MU], M[MU], dD[MU];
  float xD[8], xa[8], xI[8], xx[8], xe[8], xd[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) xD[m] = xa[m] = xI[m] = xx[m] = xe[m] = xd[m] = 0.f;
#pragma unroll
  for (int m = 0; m < MU; ++m) {
    D[m] = D0;
    I[m] = I0;
    M[m] = fabsf(D0);
    dD[m] = dD0;
    if (EXACT || m < nmu) {
      xD[m] = mul(hw[m], D0);
      xa[m] = fabsf(xD[m]);
      xI[m] = mul(hw[m], I0);
      xd[m] = mul(hw[m], dD0);
    }
  }
  // the inward pass leaves its hemisphere sums of each depth in part; the
  // outward pass adds its own to them (pt: those of depth k, loaded ahead)
  constexpr int NP = TAN ? 1 : kSweepParts;
  auto emit = [&](int k, df Sk, float dS, const float* pt) {
    float* pp = part + (size_t)k * pitch;
    if (TAN) {
      const float td = tree_mu<MU>(xd);
      if (!UP) pp[0] = td;
      else write_tan(cd, (size_t)k * pitch + q, dS, add(td, pt[0]));
      return;
    }
    const float tD = tree_mu<MU>(xD), ta = tree_mu<MU>(xa), tI = tree_mu<MU>(xI), tx = tree_mu<MU>(xx),
                te = tree_mu<MU>(xe);
    if (!UP) {
      pp[0] = tD;
      pp[pstride] = ta;
      pp[2 * pstride] = tI;
      pp[3 * pstride] = tx;
      pp[4 * pstride] = te;
    } else {
      const BaseOut r = base_out(Sk, c2p, c2f, add(tD, pt[0]), add(ta, pt[1]), add(tI, pt[2]), add(tx, pt[3]),
                                 add(te, pt[4]));
      const int lane = threadIdx.x & 31;
      float* w = s_stage + lane * (kStageD + 1) + (k % kStageD);
      w[0] = r.J.hi;
      w[kStagePlane] = r.J.lo;
      w[2 * kStagePlane] = r.lx;
      w[3 * kStagePlane] = r.le;
      if (k % kStageD == 0) {
        // the depths k .. k + kStageD - 1 of the warp's rows are complete
        __syncwarp(amask);
        const int nk = min(kStageD, nz - k);
        const int q0w = q - lane;
        float2* __restrict__ J2 = as_pairs(jnew_ptr(cd));
        if (na == 32 && nk == kStageD) {
          // full warp, full block: lane -> (row lane / 8 + 4 i, depth lane % 8)
          static_assert(kStageD == 8, "the full-block flush maps 4 rows x 8 depths per pass");
          const int kk = lane & 7;
          const size_t o0 = (size_t)(q0w + (lane >> 3)) * nz + k + kk;
          const float* s0 = s_stage + (lane >> 3) * (kStageD + 1) + kk;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float* sr = s0 + 4 * i * (kStageD + 1);
            const size_t o = o0 + (size_t)(4 * i) * nz;
            J2[o] = make_float2(sr[0], sr[kStagePlane]);
            cd.w.Lchi32[o] = sr[2 * kStagePlane];
            cd.w.Leta32[o] = sr[3 * kStagePlane];
          }
        } else {
          for (int e = lane; e < na * nk; e += na) {
            const int rr = e / nk, kk = e - rr * nk;
            const float* sr = s_stage + rr * (kStageD + 1) + kk;
            const size_t o = (size_t)(q0w + rr) * nz + k + kk;
            J2[o] = make_float2(sr[0], sr[kStagePlane]);
            cd.w.Lchi32[o] = sr[2 * kStagePlane];
            cd.w.Leta32[o] = sr[3 * kStagePlane];
          }
        }
        __syncwarp(amask);
      }
    }
  };
  float pt_n[NP];
  auto load_parts = [&](int kk) {
    if (UP) {
#pragma unroll
      for (int j = 0; j < NP; ++j) pt_n[j] = part[(size_t)kk * pitch + j * pstride];
    }
  };
  load_parts(k0);
  emit(k0, Sp, dSp, pt_n);

  // the next depth's inputs are prepared one step ahead
  int kn = UP ? nz - 2 : 1;
  float c_n = 0.f, dc_n = 0.f, dS_n = 0.f, dSl_n = 0.f, Sf_n = 0.f;
  df S_n = df_make(0.f, 0.f);
  auto load = [&](int kk) {
    load_parts(kk);
    if (TAN) {
      c_n = chiT[(size_t)kk * pitch];
      dSl_n = dSkT[(size_t)(UP ? kk : kk - 1) * pitch];
      if (!FT) tan_in(kk, dc_n, dS_n);
    } else if (UP) {
      // the outward sweep of a base evaluation reads the float copies its own
      // inward sweep left (coalesced; the same values, no pair difference)
      // and the S pair for J only
      c_n = chiT[(size_t)kk * pitch];
      Sf_n = S32T[(size_t)kk * pitch];
      dSl_n = dSkT[(size_t)kk * pitch];
      S_n = df_load(S2, kk);
    } else {
      c_n = chi[kk];
      S_n = df_load(S2, kk);
    }
  };
  if (nz > 1) load(kn);
  for (int s = 1; s < nz; ++s) {
    const int k = kn;
    const int kd = UP ? k : k - 1;   // layer between k and its upstream neighbour
    const float c0 = c_n, dSl = dSl_n, Sf = Sf_n;
    float dc0 = dc_n, dS0 = dS_n;
    if (FT) {
      tan_finish(k, c0, dc0, dS0);
      tan_issue(k + kRing - 1);
    }
    const df Sk = S_n;
    float pt[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) pt[j] = pt_n[j];
    if (s + 1 < nz) {
      kn = UP ? k - 1 : k + 1;
      load(kn);
    }
    StepIn in;
    in.csum = add(c0, cp);
    in.rs = rcp_approx(in.csum);
    in.dzk = s_dz[kd];
    in.idzk = s_idz[kd];
    in.tz = mul(in.dzk, in.csum);
    in.rz = mul(in.rs, in.idzk);
    in.dtz = 0.f;
    if (TAN) {
      in.dSin = UP ? dSl : -dSl;
      in.S0 = in.Su = in.rc0 = 0.f;
      in.dcs = add(dc0, dcp);
      in.dtz = mul(in.dzk, in.dcs);
      in.ddSin = sub(dSp, dS0);
    } else {
      // S^u - S^k formed from the pairs, then rounded
      in.dSin = UP ? dSl : df_to_float(df_sub(Sp, Sk));
      in.S0 = UP ? Sf : Sk.hi;
      if (!UP) {
        // depth-major copies for the tangent evaluations
        chiT[(size_t)k * pitch] = c0;
        S32T[(size_t)k * pitch] = in.S0;
        dSkT[(size_t)kd * pitch] = -in.dSin;   // S^{k} - S^{k-1}
      }
      in.Su = Su;
      in.rc0 = rcp_approx(c0);
      in.dcs = in.ddSin = 0.f;
    }
    auto angles = [&](auto cm) {
      constexpr int CM = decltype(cm)::value;
#pragma unroll
      for (int m = 0; m < MU; ++m) {
        if (EXACT || m < nmu) {
          const RayOut r = ray_step<TAN, CM>(in, inv2mu[m], two_mu[m], hw[m], D[m], I[m], M[m], dD[m]);
          xD[m] = r.xD;
          xa[m] = fabsf(r.xD);
          xI[m] = r.xI;
          xx[m] = r.xx;
          xe[m] = r.xe;
          xd[m] = r.xd;
        }
      }
    };
    if (EXACT) {
      // the angles' optical depths tz/(2 mu) fall with m (mu ascending): one
      // test on the first and last angle settles the form for all of them
      if (!(mul(in.tz, inv2mu[MU - 1]) < 0.1f)) angles(std::integral_constant<int, CM_DIRECT>());
      else if (mul(in.tz, inv2mu[0]) < 0.1f) angles(std::integral_constant<int, CM_SERIES>());
      else angles(std::integral_constant<int, CM_EITHER>());
    } else {
      angles(std::integral_constant<int, CM_EITHER>());
    }
    emit(k, Sk, dS0, pt);
    Sp = Sk;
    Su = in.S0;
    cp = c0;
    dSp = dS0;
    dcp = dc0;
  }
  if (UP && !TAN) {
#pragma unroll
    for (int m = 0; m < MU; ++m)
      if (EXACT || m < nmu) cd.w.Iem[(size_t)q * nmu + m] = __dmul_rn((double)I[m], c2);
  }
}

// One kernel per evaluation kind (its own register allocation): blocks of
// columns in the other kind return at once. FUSE: the tangent kernel forms
// the opacity tangent itself (no separate opacity-tangent launch).
template <int MU, bool TAN, bool FUSE>
__device__ __forceinline__ void formal_sweep_block(const ColDesc* __restrict__ cols) {
  extern __shared__ float s_tab[];   // FUSE: the copy ring; then [nz] |dz|, [nz] 1/|dz|
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode_f(cd);
  if (mode == EV_SKIP || (mode == EV_TANGENT) != TAN) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq;
  if ((int)(blockIdx.x * blockDim.x) >= nq) return;   // uniform over the block
  // FUSE: the copy ring; base-type sweeps: the output stage; then the |dz| tables
  float* s_ring = FUSE ? s_tab : nullptr;
  float* s_stage = TAN ? nullptr : s_tab + (size_t)(threadIdx.x >> 5) * kWarpStage;
  float* s_dz = s_tab + (FUSE ? ring_floats(blockDim.x) : 0) + (TAN ? 0 : stage_floats(blockDim.x));
  float* s_idz = s_dz + nz;
  stage_dz(T, s_dz, s_idz);
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  // the lanes of a warp with a frequency form a prefix of it
  const unsigned amask = __ballot_sync(0xffffffffu, q < nq);
  if (q >= nq) return;
  const int na = __popc(amask);
  if (T.nmu == MU) {   // uniform over the block: every angle slot is in use
    sweep_thread<MU, TAN, false, true, FUSE>(cd, q, s_dz, s_idz, s_ring, s_stage, amask, na);
    sweep_thread<MU, TAN, true, true>(cd, q, s_dz, s_idz, nullptr, s_stage, amask, na);
  } else {
    sweep_thread<MU, TAN, false, false, FUSE>(cd, q, s_dz, s_idz, s_ring, s_stage, amask, na);
    sweep_thread<MU, TAN, true, false>(cd, q, s_dz, s_idz, nullptr, s_stage, amask, na);
  }
}

template <int MU, bool TAN>
__global__ void __launch_bounds__(256) k_formal_sweep(const ColDesc* __restrict__ cols) {
  formal_sweep_block<MU, TAN, false>(cols);
}

// The tangent sweep that forms the opacity tangent itself (forced variant):
// 128-thread blocks, at most 72 registers (seven blocks per SM). Measured on
// the 1,216-column batch against the separate opacity-tangent kernel
// (per tick, all on one stream): opacity stage 1.67 -> 0.63 ms, tangent sweep
// 1.54 -> 2.91 ms; whole solve 529 -> 554 ms. At 64 registers (spills) the
// sweep took 3.51 ms, unbounded (100 registers) 3.69 ms.
constexpr int kFusedThreads = 128;
template <int MU>
__global__ void __launch_bounds__(kFusedThreads, 7) k_formal_sweep_fused(const ColDesc* __restrict__ cols) {
  formal_sweep_block<MU, true, true>(cols);
}

// ---------------------------------------------------------------------------
// Variant 2 (small launches): one warp per two frequencies; lane = (frequency
// of the pair, hemisphere, angle), so both hemispheres advance together and
// every lane runs one ray. A hemisphere's sums come from an xor butterfly
// over its 8 angle lanes (the tree of tree8), land in shared memory per
// depth, and the 16 lanes of a frequency then combine the two hemispheres
// depth by depth (coalesced output rows).
// ---------------------------------------------------------------------------
constexpr int kWarpParts = kSweepParts;

__host__ __device__ inline size_t warp_variant_smem(int nz, int warps) {
  return sizeof(float) * (2 * (size_t)nz + (size_t)warps * 2 * 2 * kWarpParts * nz);
}

template <bool TAN>
__device__ __forceinline__ void sweep_warp(const ColDesc& cd, int q, float* __restrict__ wp,
                                           const float* __restrict__ s_dz, const float* __restrict__ s_idz) {
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq, nmu = T.nmu;
  const int lane = threadIdx.x & 31;
  const int qi = lane >> 4, hemi = (lane >> 3) & 1, m = lane & 7;
  const int leader = lane & ~7;
  const bool up = hemi == 1;
  const bool valid = q < nq;
  const int qq = valid ? q : nq - 1;
  const size_t row = (size_t)qq * nz;
  const size_t pitch = (size_t)col_pitch(nq);
  const float* __restrict__ chi = reinterpret_cast<const float*>(cd.w.chi) + row;
  const float2* __restrict__ S2 = as_pairs(cd.w.S) + row;   // S as float pairs
  float* __restrict__ chiT = cd.w.chiT + qq;
  float* __restrict__ S32T = cd.w.S32T + qq;
  float* __restrict__ dSkT = cd.w.dSkT + qq;
  const float* __restrict__ dchiT = cd.w.dchiT + qq;
  const float* __restrict__ dS32T = cd.w.dS32T + qq;
  const double c2 = T.c2[qq];
  const float c2f = T.c2f[qq];
  const df c2p = df_load(T.c2p, qq);
  const bool on = m < nmu;
  const float4 ang = on ? T.ang32[m] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float inv2mu = ang.x;
  const float hw = ang.y;
  const float two_mu = ang.z;
  float* hp = wp + (size_t)(qi * 2 + hemi) * kWarpParts * nz;   // this hemisphere's sums [v][k]
  const bool writer = !TAN && !up && m == 0 && valid;           // depth-major copies
  auto tan_in = [&](int kk, float& dc, float& dS) {
    const size_t o = (size_t)kk * pitch;
    dc = dchiT[o];
    dS = dS32T[o];
  };

  const int k0 = up ? nz - 1 : 0;
  df Sp = df_load(S2, k0);
  float cp = TAN ? chiT[k0 * pitch] : chi[k0];
  float dSp = 0.f, dcp = 0.f;
  if (TAN) tan_in(k0, dcp, dSp);
  float Su = Sp.hi;
  if (writer) {
    chiT[0] = cp;
    S32T[0] = Su;
  }
  const double Ib64 = up ? T.Bn[row + nz - 1] / c2 : 0.0;
  const float D0 = df_to_float(df_sub(df_from_double(Ib64), Sp));
  const float I0 = __double2float_rn(Ib64);
  const float dD0 = -dSp;
  float D = D0, I = I0, M = fabsf(D0), dD = dD0;
  RayOut r;
  r.xD = on ? mul(hw, D0) : 0.f;
  r.xI = on ? mul(hw, I0) : 0.f;
  r.xx = r.xe = 0.f;
  r.xd = on ? mul(hw, dD0) : 0.f;
  auto store = [&](int k) {
    if (TAN) {
      const float td = butterfly8(r.xd);
      if (m == 0) hp[k] = td;
    } else {
      const float tD = butterfly8(r.xD), ta = butterfly8(fabsf(r.xD)), tI = butterfly8(r.xI);
      const float tx = butterfly8(r.xx), te = butterfly8(r.xe);
      if (m == 0) {
        hp[k] = tD;
        hp[nz + k] = ta;
        hp[2 * nz + k] = tI;
        hp[3 * nz + k] = tx;
        hp[4 * nz + k] = te;
      }
    }
  };
  store(k0);
  // the next depth's inputs are loaded one step ahead (latency off the chain)
  float c_n = 0.f, dc_n = 0.f, dS_n = 0.f, dSl_n = 0.f;
  df S_n = df_make(0.f, 0.f);
  auto load = [&](int s) {
    const int k = up ? nz - 1 - s : s;
    const int kd = up ? k : k - 1;
    if (TAN) {
      c_n = chiT[(size_t)k * pitch];
      tan_in(k, dc_n, dS_n);
      dSl_n = dSkT[(size_t)kd * pitch];
    } else {
      c_n = chi[k];
      if (m == 0) S_n = df_load(S2, k);
    }
  };
  if (nz > 1) load(1);
  for (int s = 1; s < nz; ++s) {
    const int k = up ? nz - 1 - s : s;
    const int kd = up ? k : k - 1;
    StepIn in;
    const float c0 = c_n;
    float dc0 = 0.f, dS0 = 0.f;
    const float dSl = dSl_n;
    const df Sk = S_n;
    if (TAN) {
      dc0 = dc_n;
      dS0 = dS_n;
    }
    if (s + 1 < nz) load(s + 1);
    if (TAN) {
      in.dSin = up ? dSl : -dSl;
      in.S0 = in.Su = in.rc0 = 0.f;
      in.dcs = add(dc0, dcp);
      in.ddSin = sub(dSp, dS0);
    } else {
      // the pair difference is formed once per hemisphere (angle lane 0)
      float dSin = 0.f, S0 = 0.f;
      if (m == 0) {
        dSin = df_to_float(df_sub(Sp, Sk));
        S0 = Sk.hi;
        Sp = Sk;
        if (writer) {
          chiT[(size_t)k * pitch] = c0;
          S32T[(size_t)k * pitch] = S0;
          dSkT[(size_t)kd * pitch] = -dSin;   // S^{k} - S^{k-1}
        }
      }
      in.dSin = __shfl_sync(0xffffffffu, dSin, leader);
      in.S0 = __shfl_sync(0xffffffffu, S0, leader);
      in.Su = Su;
      in.rc0 = rcp_approx(c0);
      in.dcs = in.ddSin = 0.f;
    }
    in.csum = add(c0, cp);
    in.rs = rcp_approx(in.csum);
    in.dzk = s_dz[kd];
    in.idzk = s_idz[kd];
    in.tz = mul(in.dzk, in.csum);
    in.rz = mul(in.rs, in.idzk);
    in.dtz = TAN ? mul(in.dzk, in.dcs) : 0.f;
    if (on) {
      r = ray_step<TAN>(in, inv2mu, two_mu, hw, D, I, M, dD);
    } else {
      r.xD = r.xI = r.xx = r.xe = r.xd = 0.f;
    }
    store(k);
    Su = in.S0;
    cp = c0;
    dcp = dc0;
    dSp = dS0;
  }
  if (up && on && valid && !TAN) cd.w.Iem[(size_t)q * nmu + m] = __dmul_rn((double)I, c2);
  __syncwarp();
  if (!valid) return;
  // combine the hemispheres of frequency q, depths strided over its 16 lanes
  const float* dn = wp + (size_t)(qi * 2 + 0) * kWarpParts * nz;
  const float* upp = wp + (size_t)(qi * 2 + 1) * kWarpParts * nz;
  for (int k = lane & 15; k < nz; k += 16) {
    if (TAN) {
      const size_t o = (size_t)k * pitch + q;
      write_tan(cd, o, cd.w.dS32T[o], add(upp[k], dn[k]));
    } else {
      write_base(cd, row + k, df_load(S2, k), c2p, c2f, add(upp[k], dn[k]), add(upp[nz + k], dn[nz + k]),
                 add(upp[2 * nz + k], dn[2 * nz + k]), add(upp[3 * nz + k], dn[3 * nz + k]),
                 add(upp[4 * nz + k], dn[4 * nz + k]));
    }
  }
}

__global__ void __launch_bounds__(256) k_formal_sweep_warp(const ColDesc* __restrict__ cols, int which) {
  extern __shared__ float s_tab[];   // [nz] |dz|, [nz] 1/|dz|, per warp [2][2][parts][nz]
  const ColDesc& cd = cols[blockIdx.y];
  const int mode = eval_mode_f(cd);
  if (mode == EV_SKIP || (which == 1 && mode == EV_TANGENT) || (which == 2 && mode != EV_TANGENT)) return;
  const ColTables& T = cd.t;
  const int nz = T.nz, nq = T.nq;
  const int warps = blockDim.x >> 5;
  if ((int)blockIdx.x * warps * 2 >= nq) return;   // uniform over the block
  float* s_dz = s_tab;
  float* s_idz = s_tab + nz;
  stage_dz(T, s_dz, s_idz);
  __syncthreads();
  const int wid = threadIdx.x >> 5;
  float* wp = s_tab + 2 * nz + (size_t)wid * 2 * 2 * kWarpParts * nz;
  const int q = ((int)blockIdx.x * warps + wid) * 2 + ((threadIdx.x & 31) >> 4);
  if (mode == EV_TANGENT) sweep_warp<true>(cd, q, wp, s_dz, s_idz);
  else sweep_warp<false>(cd, q, wp, s_dz, s_idz);
}

// Angle counts with their own instantiation; a launch uses the smallest one
// that covers every column of the batch (columns with fewer angles predicate
// the rest off).
static int sweep_mu_class(int nmu) {
  if (nmu <= 2) return 2;
  if (nmu <= 3) return 3;
  if (nmu <= 4) return 4;
  if (nmu <= 5) return 5;
  return 8;
}

// Dynamic shared memory of a sweep block: its |dz| tables, padded so that at
// most ``occ`` blocks fit on a multiprocessor when occ > 0. Fewer resident
// columns keep the outward pass's re-reads of the inward pass's inputs in L2.
static size_t sweep_smem(int max_nz, int occ, int threads, bool tan, bool fuse = false) {
  const size_t need =
      sizeof(float) * (2 * (size_t)max_nz + (fuse ? ring_floats(threads) : 0) + (tan ? 0 : stage_floats(threads)));
  if (occ <= 0) return need;
  const size_t cap = (size_t)227 * 1024;
  const size_t pad = (size_t)228 * 1024 / occ - 1024;
  return std::min(cap, std::max(need, pad));
}

template <int MU>
static void launch_mu(const Batch& b, cudaStream_t s, int threads, int which, int occ_tan, int occ_base, int fuse) {
  dim3 g((b.max_nq + threads - 1) / threads, b.ncols);
  if (which != 1) {
    const size_t sm = sweep_smem(b.max_nz, occ_tan, threads, true, fuse != 0);
    if (fuse) k_formal_sweep_fused<MU><<<g, threads, sm, s>>>(b.d_cols);
    else k_formal_sweep<MU, true><<<g, threads, sm, s>>>(b.d_cols);
  }
  if (which != 2)
    k_formal_sweep<MU, false><<<g, threads, sweep_smem(b.max_nz, occ_base, threads, false), s>>>(b.d_cols);
}

template <int MU>
static int allow_smem_mu() {
  JFNK_CUDA(cudaFuncSetAttribute(k_formal_sweep<MU, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  JFNK_CUDA(cudaFuncSetAttribute(k_formal_sweep_fused<MU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024));
  JFNK_CUDA(cudaFuncSetAttribute(k_formal_sweep<MU, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  return JFNK_OK;
}

// variant 1: ``size`` threads per block, at most occ_tan / occ_base blocks per
// SM (0: no cap); variant 2: ``size`` warps per block; which: 0 every column,
// 1 base-type evaluations, 2 tangent ones
static int launch_sweep_cfg(const Batch& b, cudaStream_t s, int variant, int size, int which = 0, int occ_tan = 0,
                            int occ_base = 0, int fuse = 0) {
  if (fuse && (variant != 1 || size != kFusedThreads))
    return fail(JFNK_E_INVALID, "fused tangent sweep: thread variant with 128-thread blocks only");
  if (variant == 2) {
    const int fpb = 2 * size;   // frequencies per block
    dim3 g((b.max_nq + fpb - 1) / fpb, b.ncols);
    k_formal_sweep_warp<<<g, 32 * size, warp_variant_smem(b.max_nz, size), s>>>(b.d_cols, which);
  } else {
    switch (sweep_mu_class(b.max_nmu)) {
      case 2: launch_mu<2>(b, s, size, which, occ_tan, occ_base, fuse); break;
      case 3: launch_mu<3>(b, s, size, which, occ_tan, occ_base, fuse); break;
      case 4: launch_mu<4>(b, s, size, which, occ_tan, occ_base, fuse); break;
      case 5: launch_mu<5>(b, s, size, which, occ_tan, occ_base, fuse); break;
      default: launch_mu<8>(b, s, size, which, occ_tan, occ_base, fuse); break;
    }
  }
  JFNK_CUDA(cudaGetLastError());
  return JFNK_OK;
}

static bool warp_variant_fits(int nz, int warps) {
  return warp_variant_smem(nz, warps) <= (size_t)227 * 1024;
}

int sweep_prepare(Batch* b) {
  const size_t bytes = warp_variant_smem(b->max_nz, 8);
  JFNK_CUDA(cudaFuncSetAttribute(k_formal_sweep_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::min(bytes, (size_t)227 * 1024)));
  int rc;
  if ((rc = allow_smem_mu<2>()) || (rc = allow_smem_mu<3>()) || (rc = allow_smem_mu<4>()) ||
      (rc = allow_smem_mu<5>()) || (rc = allow_smem_mu<8>()))
    return rc;
  if (b->sweep_variant == 0) {
    b->sweep_variant = 1;
    b->formal_threads = 128;
  }
  return JFNK_OK;
}

bool sweep_fused(const Batch& b) { return b.sweep_fuse > 0 && b.sweep_variant != 2 && b.max_overlap <= kQMetaT; }

int launch_formal_sweep(const Batch& b, cudaStream_t s, int which) {
  return launch_sweep_cfg(b, s, b.sweep_variant == 2 ? 2 : 1, b.formal_threads > 0 ? b.formal_threads : 128,
                          which, b.sweep_occ, b.sweep_occ_base, sweep_fused(b) ? b.sweep_fuse : 0);
}

int sweep_warp_size(int nz) {
  for (int w : {4, 2, 1})
    if (warp_variant_fits(nz, w)) return w;
  return 0;
}

// Autotuner of the sweep kernels, timed on the batch's own columns: the
// tangent sweep (the columns in tangent mode) over variant 1 with 32..256
// threads per block and a cap of 2..8 resident blocks per SM or none, and
// variant 2 with 1..8 warps per block (where its shared memory fits); then,
// for variant 1, the base-type sweep's cap (columns in base mode). First the
// opacity tangent's run of depths per thread. Every choice gives bit-identical
// results, so it changes the speed only.
int sweep_autotune(Batch* b, cudaStream_t s) {
  cudaEvent_t e0, e1;
  JFNK_CUDA(cudaEventCreate(&e0));
  JFNK_CUDA(cudaEventCreate(&e1));
  int rc = JFNK_OK;
  // a tangent candidate without fusion is timed with the separate opacity-tangent launch it needs
  auto once = [&](int variant, int size, int which, int ot, int ob, int fuse) -> int {
    if (which == 2 && !fuse) {
      int r = launch_opacity_tan(*b, s);
      if (r) return r;
    }
    return launch_sweep_cfg(*b, s, variant, size, which, ot, ob, fuse);
  };
  // a candidate's time: the fastest of five launches timed one by one, after a
  // warm-up (single launches differ by a few per cent; the minimum is stable)
  auto timed = [&](int variant, int size, int which, int ot, int ob, float* ms, int fuse = 0) -> int {
    int r = once(variant, size, which, ot, ob, fuse);   // warm-up
    if (r) return r;
    float best = 1e30f;
    for (int i = 0; i < 5; ++i) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return fail(JFNK_E_CUDA, "autotune event");
      if ((r = once(variant, size, which, ot, ob, fuse))) return r;
      float t = 0.f;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        return fail(JFNK_E_CUDA, "autotune timing");
      best = std::min(best, t);
    }
    *ms = best;
    return JFNK_OK;
  };
  // the opacity tangent's run of depths per thread (the depth tile of its
  // grid): the default of 16 unless another run gains 2 %
  {
    auto time_optan = [&](int dr, float* ms) -> int {
      int r = launch_opacity_tan(*b, s, dr);   // warm-up
      if (r) return r;
      float best = 1e30f;
      for (int i = 0; i < 5; ++i) {
        if (cudaEventRecord(e0, s) != cudaSuccess) return fail(JFNK_E_CUDA, "autotune event");
        if ((r = launch_opacity_tan(*b, s, dr))) return r;
        float t = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
          return fail(JFNK_E_CUDA, "autotune timing");
        best = std::min(best, t);
      }
      *ms = best;
      return JFNK_OK;
    };
    float bo = 0.f;
    int bd = 16;
    if (!(rc = time_optan(16, &bo))) {
      bo *= 0.98f;
      for (int dr : {4, 8, 32}) {
        float ms = 0.f;
        if ((rc = time_optan(dr, &ms))) break;
        if (ms < bo) { bo = ms; bd = dr; }
      }
    }
    b->optan_depths = bd;
  }
  // The fused opacity tangent (forced variant only) is not a candidate: timed
  // alone it can win, but inside a tick the separate opacity-tangent kernel
  // overlaps the base-type chain on the other stream, and the fused sweep
  // made the whole solve about 11 % slower.
  struct Cand { int variant, size, occ, fuse; };
  std::vector<Cand> cands;
  for (int t : {32, 64, 128, 256})
    for (int occ : {0, 2, 4, 8}) cands.push_back({1, t, occ, 0});
  for (int w : {1, 2, 4, 8}) cands.push_back({2, w, 0, 0});
  // the default (128 threads, no cap) stays unless a candidate beats it by 2 %:
  // closer than that, single measurements flip between runs
  float best = 1e30f;
  Cand bc{1, 128, 0, 0};
  if ((rc = timed(1, 128, 2, 0, 0, &best))) best = 1e30f;
  best *= 0.98f;
  for (const auto& c : cands) {
    if (rc) break;
    if (c.variant == 2 && !warp_variant_fits(b->max_nz, c.size)) continue;
    if (c.variant == 1 && c.occ > 0 && c.size * c.occ > 2048) continue;
    if (c.variant == 1 && c.size == 128 && c.occ == 0) continue;
    float ms = 0.f;
    if ((rc = timed(c.variant, c.size, 2, c.occ, 0, &ms, c.fuse))) break;
    if (ms < best) { best = ms; bc = c; }
  }
  int best_base = 0;
  if (!rc && bc.variant == 1) {
    // the base-type sweep's cap, on the same columns in base mode
    if (!(rc = batch_set_forced_mode(b, EV_BASE, s))) {
      float bb = 1e30f;
      for (int occ : {0, 2, 3, 4, 6, 8}) {
        if (occ > 0 && bc.size * occ > 2048) continue;
        float ms = 0.f;
        if ((rc = timed(1, bc.size, 1, bc.occ, occ, &ms))) break;
        if (occ == 0) ms *= 0.98f;   // no cap unless a cap gains 2 %
        if (ms < bb) { bb = ms; best_base = occ; }
      }
      if (!rc) rc = batch_set_forced_mode(b, EV_TANGENT, s);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->sweep_variant = bc.variant;
  b->formal_threads = bc.size;
  b->sweep_occ = bc.variant == 1 ? bc.occ : 0;
  b->sweep_occ_base = bc.variant == 1 ? best_base : 0;
  b->sweep_fuse = bc.variant == 1 ? bc.fuse : 0;
  return JFNK_OK;
}

}  // namespace jfnk
