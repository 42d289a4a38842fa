// Shared definitions of the JFNK NLTE library (device structures, constants,
// error handling). Internal header; the public interface is include/jfnk.h.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "jfnk.h"

namespace jfnk {

// cgs constants (CODATA 2018)
constexpr double kH = 6.62607015e-27;
constexpr double kC = 2.99792458e10;
constexpr double kKB = 1.380649e-16;
constexpr double kME = 9.1093837015e-28;
constexpr double kQE = 4.80320471e-10;
constexpr double kEV = 1.602176634e-12;
constexpr double kAMU = 1.66053906660e-24;
constexpr double kSigmaT = 6.6524587321e-25;
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxL = JFNK_MAX_LEVELS;
constexpr int kMaxMu = JFNK_MAX_MU;
constexpr int kMaxKrylov = 64;
constexpr int kMaxT = 32;      // transitions per atom

// Evaluation modes of one F-class pass over a column.
enum EvalMode : int {
  EV_SKIP = 0,      // column finished: kernels return immediately
  EV_BASE = 1,      // F(n), new J, preconditioner coefficients
  EV_TANGENT = 2,   // J_F(n) v (tangent of every step)
  EV_RH92 = 3,      // F(n), new J, Lambda_eta (RH92 update afterwards)
  EV_FD = 4,        // F(n + s eps u) for a finite-difference JVP: J^dagger and the
                    // conservation rows of the base point, F into dF, no new J or P
};

// Solver phases of the per-column state machine (one evaluation per tick).
enum Phase : int {
  PH_BASE = 0,      // next evaluation: base point of a Newton step
  PH_JVP = 1,       // next evaluation: J v_j (Arnoldi direction)
  PH_RESTART = 2,   // next evaluation: J x (GMRES restart residual)
  PH_RH92 = 3,      // next evaluation: RH92 formal solution
  PH_DONE = 4,
};

// Immutable tables of one column (device pointers), built at atmosphere creation.
struct ColTables {
  int nz, nq, nl, nt, nmu, nwin;  // nwin = sum over transitions of window points
  int max_overlap;                // most transitions active at one frequency
  const double* nu;       // [nq]
  const double* c2;       // [nq] 2 h nu^3 / c^2
  const double* rw;       // [nq] 4 pi / (h nu)
  const int* q_off;       // [nq+1] CSR: transitions active at q
  const int* q_t;         // [q_off[nq]]
  const int* t_lo;        // [nt]
  const int* t_up;
  const int* t_q0;        // first union index of the window
  const int* t_q1;        // last union index (inclusive)
  const int* t_base;      // offset of transition t in window-point arrays
  const double* t_w;      // [nwin] trapezoid weight omega_t(nu_q)
  const double* V;        // [nwin][nz]
  const double* G;        // [nwin][nz]
  const double* gV;       // [nwin][nz] g V
  // float pairs (hi + lo, about 48 bits) of the tables the mixed mode's
  // base evaluations need beyond FP32, for arithmetic on the FP32 pipe
  const float2* V2;       // [nwin][nz] V
  const float2* gV2;      // [nwin][nz] g V
  const float2* W2;       // [nwin] W = omega_t(nu_q) 4 pi/(h nu_q)
  const float2* chibg2;   // [nq][nz] chi_c + chi_sca
  const float2* etac2;    // [nq][nz] eta_c
  const float2* chisca2;  // [nz] chi_sca
  const float2* c2p;      // [nq] 2 h nu^3/c^2
  const float2* rc2p;     // [nq] c^2/(2 h nu^3)
  const double* rc2;      // [nq] c^2 / (2 h nu^3)
  const double* WV;       // [nwin][nz] W V with W = omega_t(nu_q) 4 pi/(h nu_q): rate-integral weights
  const double* WgV;      // [nwin][nz] W g V
  const double* Rsp;      // [nt][nz] sum_q W g V 2 h nu^3/c^2: the spontaneous part of R_ji
  const float* V32;       // [nwin][nz] float copies (mixed-mode tangent evaluations)
  const float* G32;       // [nwin][nz]
  const float2* VG32T;    // [nz][nwin] the same pairs (V, G), depth-major
  const float* W32;       // [nwin] omega_t(nu_q) 4 pi/(h nu_q) 2 h nu_q^3/c^2 in float
  const float* Wr32;      // [nwin] omega_t(nu_q) 4 pi/(h nu_q) in float
  const float* c2f;       // [nq] 2 h nu^3/c^2 in float
  const int* lvl_inc;     // [nl][nt + 1] transitions of each level in order, packed as
                          // t << 1 | (1 if the level is the upper one), -1 after the last
  const int* qmeta;       // [kQMetaT][nq] transitions active at nu_q, packed as
                          // window point << 8 | lo << 4 | up; -1 past the last
  const int* qtr;         // [kQMetaT][nq] the same transitions' indices t
  const double* dz;       // [nz-1] |z_k - z_{k+1}|
  const double* mu;       // [nmu]
  const double* wmu;      // [nmu]
  const double* Vd;       // [2 nmu][nwin][nz] V_ij seen along each direction (outgoing
                          // mu_1..mu_n, then ingoing): a moving column; null when static
  const float4* ang32;    // [nmu] (1/(2 mu), w_mu/2, 2 mu, 0), each the FP64 value rounded once
  const float2* dz32;     // [nz-1] (|dz|, 1/|dz|) likewise
  const double* chi_c;    // [nq][nz]
  const double* eta_c;    // [nq][nz]
  const double* chi_sca;  // [nz]
  const double* Bn;       // [nq][nz] Planck function
  const double* C;        // [nz][nl][nl] collision rate i -> j
  const double* ntot;     // [nz]
  const double* nstar;    // [nz][nl]
};

struct SolverOpts {
  double ftol, fdrop, rtol, rh92_switch;
  int maxiter, krylov_max, max_restarts, clamp, rh92_warmup, max_ticks;
  int precond;   // 1: apply P^{-1} (block Jacobi); 0: no preconditioning
  int jvp;       // 0 exact tangent; 1 forward eps_1; 2 forward eps_2; 3 central eps_2
  int krylov;    // 0 GMRES; 1 BiCGSTAB
  int solver;    // 0 Algorithm 2 (after an optional RH92 start); 1 RH92 iterations only
  int line_search;   // 0 off; k > 0 at most k halvings of a Newton correction
};

// Preconditioner variant (solution of Sect. 2.5.2) a base evaluation builds for
// column cd: its own options, else the batch's, else the first solution.
struct ColDesc;

// BiCGSTAB vectors of a column in the Krylov basis buffer (slots of N doubles).
enum BicgSlot : int { BS_R = 0, BS_RHAT = 1, BS_P = 2, BS_V = 3, BS_S = 4, BS_T = 5 };
constexpr int kBicgMaxIter = 200;   // iterations per Newton step

// Per-column solver state (device memory, written by the Krylov kernel only).
struct SolverState {
  int phase;
  int status;          // 1 running, 0 converged, < 0 error code
  int newton_iter;
  int rh92_iter;
  int j;               // current Arnoldi index
  int restarts;
  int F_calls;
  int jvp_calls;
  int ticks;
  int jsel;            // 1: the roles of the two mean-intensity buffers are swapped
  double beta;         // norm of the current restart residual
  double r0norm;       // norm of the Newton step's initial Krylov residual
  double F0norm;
  double Fnorm;
  double err;
  int fd_scheme;       // JVPs: 0 exact tangent, 1/2 forward difference, 3 central difference
  int fd_side;         // central difference: +1 before F(n + eps u), -1 before F(n - eps u)
  double fd_eps;       // difference step of the current JVP
  int bstage;          // BiCGSTAB: 0 the pending product is A p, 1 it is A s
  int bit;             // BiCGSTAB iterations of this Newton step
  double rho, alpha, omega;   // BiCGSTAB scalars
  int ls_pending;      // line search: the next base evaluation is a trial point
  int ls_left;         // halvings left
  double ls_step;      // fraction of the Newton correction taken
  double ls_Fprev;     // ||F||_inf at the base point the correction came from
  double rh_damp;      // RH92 step fraction (0 = full), halved after a non-finite iteration
};

// Work buffers of one column (device pointers). ``real`` buffers hold float in
// the mixed mode and double in the FP64 mode.
struct ColWork {
  double* n;        // [nz][nl] base populations
  double* v;        // [nz][nl] tangent direction for explicit JVPs
  double* Jdag;     // [nq][nz]
  double* Jnew;     // [nq][nz]
  int* istar;       // [nz]
  void* chi;        // [nq][nz] real
  double* S;        // [nq][nz] source function normalised by 2 h nu^3/c^2
  void* dSk;        // [nq][nz] real: S^{k+1} - S^k formed in FP64 (0 at the bottom)
  void* dchi;       // [nq][nz] real
  double* dS;       // [nq][nz] tangent of S (normalised)
  void* ddSk;       // [nq][nz] real: dS^{k+1} - dS^k
  void* H;          // [2 nmu][nz][nq] real: per-ray 1/2 w (I - S)  (value)
  void* HI;         // [2 nmu][nz][nq] real: per-ray 1/2 w I (base evaluations)
  void* dH;         // tangent
  void* LX;         // per-ray 1/2 w dI^k/dchi^k
  void* LE;         // per-ray 1/2 w dI^k/deta^k
  void* part;       // [5][nz][pitch] float: down-sweep ray sums of the sweep kernel
  // mixed mode, FP32 tangent path; depth-major [nz][col_pitch(nq)] arrays
  float* v32;       // [N] float copy of the tangent direction
  float* chiT;      // chi at the base point
  float* S32T;      // S at the base point (normalised)
  float* dSkT;      // row k: S^{k+1} - S^k, formed in FP64 and rounded
  float* dchiT;     // tangent of chi
  float* dS32T;     // tangent of S (normalised)
  float* dJ32T;     // tangent of J (normalised)
  double* J;        // [nq][nz]
  double* dJ;
  double* Lchi;     // [nq][nz] Lambda diagonals dJ/dchi, dJ/deta (FP64 mode)
  double* Leta;
  float* Lchi32;    // [nq][nz] the same in float (mixed mode, where they are FP32 sums)
  float* Leta32;
  double* zeta;     // [nq][nz][nl] beta_j Lchi + gamma_j Leta (preconditioner)
  double* Rup;      // [nt][nz]
  double* Rdn;
  double* dRup;
  double* dRdn;
  double* Apart;    // [nt][nz][nl]
  double* rh;       // [nt][nz][RH_STRIDE] RH92 sums
  double* F;        // [nz][nl]
  double* dF;       // [nz][nl]
  double* P;        // [nz][nl][nl] (LU factors after a base evaluation)
  int* piv;         // [nz][nl]
  double* Iem;      // [nq][nmu] emergent intensity
  // Krylov
  double* Vb;       // [(kmax+1)][N]
  double* Hh;       // [(kmax+1)][kmax]
  double* cs;       // [kmax]
  double* sn;       // [kmax]
  double* gv;       // [kmax+1]
  double* x;        // [N]
  double* w;        // [N]
  double* nprev;    // [N]
  double* eta;      // [nq][nz] emissivity of an RH92 evaluation, for Jeff = J - Psi* eta
  float2* n2;       // [N] populations as float pairs (mixed-mode base evaluations)
  float* etab32;    // [nq][nz] its background part eta_c + chi_sca J^dagger (mixed mode)
  double* np;       // [N] populations of a finite-difference evaluation (n + s eps u)
  double* fdp;      // [N] F(n + eps u) of a central difference
  // moving column (per-ray path, FP64): [2 nmu][nq][nz] each
  double* mchi;     // opacity of each direction
  double* mS;       // source function of each direction
  double* mdchi;    // their tangents
  double* mdS;
  double* mI;       // intensity of each ray
  double* mdI;      // its tangent
  double* mLX;      // dI^k/dchi^k of each ray (base evaluations)
  double* mLE;      // dI^k/deta^k
  double* dJdn;     // [nq][nz][nl] lagged d J/d n_j of the second preconditioner
                    // solution (null until a solve asks for it)
  SolverState* st;
};

// Transitions per frequency held in ColTables::qmeta (more go through q_off/q_t).
constexpr int kQMetaT = 8;

// Row pitch of the depth-major float arrays: frequencies rounded up to 32.
__host__ __device__ inline int col_pitch(int nq) { return (nq + 31) & ~31; }

struct ColDesc {
  ColTables t;
  ColWork w;
  int forced_mode;   // >= 0: evaluation mode for explicit API calls; < 0: from st->phase
  int mixed;         // 1: FP32 formal solution (buffers are float)
  const SolverOpts* opts;   // this column's solver options (null: the batch's)
};

__device__ __forceinline__ int precond_variant(const ColDesc& cd, const SolverOpts* bopts) {
  const SolverOpts* o = cd.opts ? cd.opts : bopts;
  const int v = o ? o->precond : 1;
  return (v == 2 && !cd.w.dJdn) ? 1 : (v < 1 ? 1 : v);
}

// Mixed mode: S, J^dagger, J_new and the RH92 emissivity hold float pairs
// (hi, lo) in the bytes of their FP64 arrays.
__host__ __device__ __forceinline__ float2* as_pairs(double* p) { return reinterpret_cast<float2*>(p); }
__host__ __device__ __forceinline__ const float2* as_pairs(const double* p) {
  return reinterpret_cast<const float2*>(p);
}

// The lagged mean intensity J^dagger and the newly computed J live in two
// buffers whose roles swap after every Newton update (no copy); explicit
// evaluations always read w.Jdag and write w.Jnew.
__device__ __forceinline__ const double* jdag_ptr(const ColDesc& cd) {
  return (cd.forced_mode < 0 && cd.w.st->jsel) ? cd.w.Jnew : cd.w.Jdag;
}
__device__ __forceinline__ double* jnew_ptr(const ColDesc& cd) {
  return (cd.forced_mode < 0 && cd.w.st->jsel) ? cd.w.Jdag : cd.w.Jnew;
}

// Populations an evaluation of kind ``mode`` reads (perturbed ones for a
// finite-difference JVP).
__device__ __forceinline__ const double* eval_pops(const ColDesc& cd, int mode) {
  return mode == EV_FD ? cd.w.np : cd.w.n;
}

// RH92 per-transition sums: [0] sum W V Jeff, [1] sum W g V Jeff, [2] sum W U,
// [3] sum W chi_t Psi eta_bg, [4 + s] sum W chi_t Psi U_s.
constexpr int kRhFixed = 4;
constexpr int kRhStride = kRhFixed + kMaxT;

// ---- error handling --------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define JFNK_CUDA(expr)                                                        \
  do {                                                                         \
    cudaError_t _e = (expr);                                                   \
    if (_e != cudaSuccess)                                                     \
      return ::jfnk::fail(JFNK_E_CUDA, std::string(#expr) + ": " +             \
                                           cudaGetErrorString(_e));            \
  } while (0)

// ---- device helpers --------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace jfnk
