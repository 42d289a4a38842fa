/*
 * jfnk.h -- C ABI of the GB300 JFNK NLTE library.
 *
 * The library evaluates the residual F(n) of the statistical-equilibrium
 * equations of one model atom on plane-parallel columns (Arramy, de la Cruz
 * Rodriguez & Leenaarts 2024, Sect. 2.1, Algorithm 1), its Jacobian-vector
 * products (Sect. 2.4), the block-Jacobi preconditioner (Sect. 2.5.2), and
 * solves F(n) = 0 with the Jacobian-free Newton-Krylov method of Algorithm 2,
 * optionally started by RH92 iterations (Sect. 3.5). Every step of the
 * computation runs in CUDA kernels built for sm_103a.
 *
 * Conventions
 *   - Every function returns an int status: JFNK_OK (0) or a negative error
 *     code; jfnk_last_error() returns a thread-local message for the last
 *     failure on the calling thread.
 *   - Handles are opaque and owned by the library; free them with the
 *     matching jfnk_destroy_* call. Descriptor arrays are copied at creation
 *     time and stay owned by the caller.
 *   - Population vectors follow the paper's ordering (Sect. 2.1.1):
 *     n[k * n_levels + l], depth index k = 0 at the top of the column.
 *     Residuals F, directions v and products J v use the same layout.
 *   - Mean intensities J[q * n_depth + k] use the atom's union frequency grid
 *     (ascending, jfnk_atom_frequencies) and the column's depth index.
 *   - Arrays passed with JFNK_MEM_HOST are host pointers (pageable or pinned)
 *     and are copied in/out on ``stream``; with JFNK_MEM_DEVICE they are
 *     device pointers on the context's device, read and written on
 *     ``stream``. ``stream`` is a cudaStream_t (NULL = legacy default stream).
 *     Host-memory calls synchronise the stream before returning; device-memory
 *     calls return after enqueuing unless stated otherwise.
 *   - cgs units throughout.
 */
#ifndef JFNK_H
#define JFNK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define JFNK_OK            0
#define JFNK_E_INVALID    -1   /* bad argument or descriptor                  */
#define JFNK_E_NOMEM      -2   /* device or host allocation failed            */
#define JFNK_E_CUDA       -3   /* a CUDA runtime call failed                  */
#define JFNK_E_DIVERGED   -4   /* solver left the domain (negative opacity)   */
#define JFNK_E_NAN        -5   /* non-finite residual or Krylov quantity      */
#define JFNK_E_TIMEOUT    -6   /* tick budget exhausted before convergence    */
#define JFNK_E_MAXITER    -7   /* Newton iteration limit reached              */

#define JFNK_MAX_LEVELS   16   /* N_l limit (levels including continua)       */
#define JFNK_MAX_MU        8   /* Gauss-Legendre points per hemisphere        */
#define JFNK_MAX_DEPTH  1024

typedef enum { JFNK_MEM_HOST = 0, JFNK_MEM_DEVICE = 1 } jfnk_mem;
/* JFNK_FP64: every step in FP64. JFNK_MIXED: formal solution, tangents and
 * the preconditioner and RH92 sums in FP32; the source function, the mean
 * intensity, the base opacity and rate sums in float pairs (hi + lo, about 48
 * bits, on the FP32 pipe); rate-equation assembly, block inverses, GMRES and
 * the Newton update in FP64. Arrays crossing the API are FP64 in both. */
typedef enum { JFNK_FP64 = 0, JFNK_MIXED = 1 } jfnk_precision;
typedef enum {
  JFNK_INIT_LTE = 0,             /* Saha-Boltzmann populations (Sect. 2.2.1)     */
  JFNK_INIT_USER = 1,            /* n_inout holds the initial guess              */
  JFNK_INIT_ZERO_RADIATION = 2   /* rate equations with I = 0 (Sect. 2.2.1)      */
} jfnk_init_kind;

typedef struct jfnk_ctx jfnk_ctx;
typedef struct jfnk_atom jfnk_atom;
typedef struct jfnk_atmos jfnk_atmos;

/* Bound-bound transition i -> j (0-based, i < j), Sect. 2.1.1 Eq. Vij.
 * V_ij = (pi e^2 / m_e c) f phi(nu), phi a Voigt profile of damping a with the
 * Doppler width of the local temperature and micro-turbulence, renormalised so
 * that its quadrature sums to one. Collisions: C_ji = 8.63e-6 n_e Upsilon /
 * (g_j sqrt(T)), or, if eps > 0, C_ji = eps A_ji / ((1 - eps)(1 - exp(-h nu/kT)))
 * (two-level thermalisation parameter); C_ij by detailed balance.
 * Frequency grid: n_nu (odd) points, offsets x in reference Doppler widths
 * dnu_ref = nu_0 vchar / c: x = q_wing u for q_wing <= 2 q_core, otherwise
 * x = q_wing sinh(beta u)/sinh(beta) with beta = 2 acosh(q_wing/(2 q_core)),
 * u uniform on [-1, 1]. */
typedef struct {
  int i, j;
  double f;          /* absorption oscillator strength                       */
  double damping;    /* Voigt damping parameter a                            */
  double upsilon;    /* effective collision strength                         */
  double eps;        /* > 0 overrides upsilon (two-level eps law)            */
  int n_nu;
  double q_core, q_wing;
} jfnk_bb_desc;

/* Bound-free transition from bound level i to continuum level j, Eq. Vij2 and
 * Eq. gij. alpha(nu) = alpha0 (nu_edge / nu)^3 on nu = nu_edge y_max^(s/(n_nu-1)).
 * Collisional ionisation C_ij = n_e q0 sqrt(T) exp(-(E_j - E_i)/kT),
 * recombination by detailed balance. */
typedef struct {
  int i, j;
  double alpha0;     /* cross-section at the edge [cm^2]                      */
  double q0;         /* [cm^3 s^-1 K^-1/2]                                    */
  int n_nu;
  double y_max;      /* nu_max / nu_edge                                      */
} jfnk_bf_desc;

typedef struct {
  int n_levels;                 /* N_l <= JFNK_MAX_LEVELS                     */
  const double* E_eV;           /* [n_levels] energies above the ground level */
  const double* g;              /* [n_levels] statistical weights             */
  const int* stage;             /* [n_levels] ionisation stage                */
  int n_bb;
  const jfnk_bb_desc* bb;
  int n_bf;
  const jfnk_bf_desc* bf;
  double mass_amu;
  double vchar;                 /* reference velocity of line grids [cm/s]    */
} jfnk_atom_desc;

/* One column. Background continuum (Sect. 2.1.1, Eqs. chi/eta):
 * chi_c = kappa(nu) rho, kappa(nu) = kappa min(kappa_max, max(1, (nu/kappa_nu_ref)^kappa_power))
 * (kappa_power = 0: grey), eta_c = chi_c B_nu(T), chi_sca = sigma_T n_e if
 * thomson != 0, with the lagged mean intensity J^dagger in the scattering
 * emissivity. Boundary conditions (Sect. 2.1.2): I = B_nu(T_bottom) entering
 * at the bottom, I = 0 entering at the top. */
typedef struct {
  int n_depth;                  /* 2 <= N_z <= JFNK_MAX_DEPTH                 */
  const double* z;              /* [n_depth] height, strictly monotonic       */
  const double* T;
  const double* ne;
  const double* ntot;           /* total density of the active atom           */
  const double* rho;            /* may be NULL when kappa == 0                */
  const double* vturb;          /* may be NULL (no micro-turbulence) [cm/s]   */
  double kappa, kappa_nu_ref, kappa_power, kappa_max;
  int thomson;
  int n_mu;                     /* Gauss-Legendre points on ]0,1[, 1..JFNK_MAX_MU */
  const double* vlos;           /* [n_depth] line-of-sight velocity [cm/s], > 0 towards
                                   the top (Sect. 3.4); NULL or all zero: static. A
                                   moving column's lines are Doppler-shifted per
                                   direction: every ray has its own profile, opacity
                                   and source function (FP64 evaluations and
                                   Algorithm 2 with GMRES or BiCGSTAB, exact or
                                   difference JVPs, the first preconditioner
                                   solution; no RH92 and no mixed precision)     */
} jfnk_atmos_desc;

/* Formal-solution kernel of a batch (all give the solution of Eqs. Iplus/
 * Iminus; the two sweep kernels of the mixed mode are bit-identical). */
typedef enum {
  JFNK_FORMAL_PER_RAY = 0,       /* per-ray buffers, separate ray-sum kernel      */
  JFNK_FORMAL_FUSED = 1,         /* FP64: block per frequency group, shared memory */
  JFNK_FORMAL_SWEEP_THREAD = 2,  /* mixed: thread per frequency, all angles        */
  JFNK_FORMAL_SWEEP_WARP = 3,    /* mixed: warp per frequency pair, lane per ray   */
  JFNK_FORMAL_MOVING = 4,        /* moving columns: thread per ray, per-ray opacity */
  JFNK_FORMAL_SWEEP_THREAD_FUSED = 5 /* mixed: thread per frequency, the tangent sweep
                                    forming the JVP evaluations' opacity tangent itself
                                    (at most 8 transitions overlap at any frequency) */
} jfnk_formal_kernel;

/* Jacobian-vector products inside GMRES (Sect. 2.4, Fig. 2). The default is
 * the exact tangent of every step, the eps -> 0 limit of the complex step
 * (Eq. complex); the difference schemes evaluate F at n +- eps u with J^dagger
 * and the conservation rows of the base point: forward with eps_1 = b
 * sum|n|/(N ||u||) + b (b = 1e-6) or eps_2 = eps_mach^(1/2) sqrt(1 + ||n||)/||u||,
 * central with eps_mach^(1/3) sqrt(1 + ||n||)/||u||. The difference schemes
 * run in JFNK_FP64 only (a difference of FP32 residuals at these steps would
 * be rounding noise); other precisions return JFNK_E_INVALID. */
typedef enum {
  JFNK_JVP_TANGENT = 0,
  JFNK_JVP_FORWARD_EPS1 = 1,
  JFNK_JVP_FORWARD_EPS2 = 2,
  JFNK_JVP_CENTRAL = 3
} jfnk_jvp_scheme;

/* Krylov solver of the Newton steps (Sect. 2.3): GMRES (Arnoldi with CGS2,
 * Givens rotations, restart after krylov_max vectors, one JVP per iteration)
 * or BiCGSTAB (van der Vorst 1992: two JVPs per iteration, at most 200
 * iterations per Newton step; needs krylov_max >= 5, its six vectors live in
 * the GMRES basis buffer). Both left-preconditioned, x_0 = 0, stopping when
 * the preconditioned residual falls below rtol times its initial norm. */
typedef enum { JFNK_KRYLOV_GMRES = 0, JFNK_KRYLOV_BICGSTAB = 1 } jfnk_krylov;

/* The nonlinear solver: Algorithm 2 (after the optional RH92 start), or the
 * paper's reference method alone, RH92 iterations (Rybicki & Hummer 1992, full
 * preconditioning) until the population change 1/2 ||(n' - n)/(n' + n)||_inf
 * falls below ftol, at most maxiter iterations (limited per depth like the
 * Newton corrections when clamp is set). */
typedef enum { JFNK_SOLVER_JFNK = 0, JFNK_SOLVER_RH92 = 1 } jfnk_solver_kind;

/* Solver options (Algorithm 2; defaults from jfnk_default_options). */
typedef struct {
  double ftol;          /* 1/2 ||(n - n_prev)/(n + n_prev)||_inf threshold (1e-4)  */
  double fdrop;         /* required ||F||_inf drop factor (1e-2)                   */
  double rtol;          /* Krylov relative tolerance (1e-2)                        */
  int maxiter;          /* Newton iterations (100)                                 */
  int krylov_max;       /* GMRES basis size before restart (50, <= 64)             */
  int max_restarts;     /* GMRES restarts per Newton step (20)                     */
  int precision;        /* jfnk_precision                                          */
  int init;             /* jfnk_init_kind                                          */
  int clamp;            /* per-depth limiting of negative corrections (1), applied
                           to Newton and to hybrid-start RH92 corrections         */
  int rh92_warmup;      /* > 0: hybrid start, at most this many RH92 iterations    */
  double rh92_switch;   /* switch to JFNK when the RH92 change is below (1e-2)     */
  int max_ticks;        /* F-class evaluations allowed per column (20000)          */
  int profile;          /* 1: time the formal-solution kernel of every active tick
                           (mixed mode: the tangent and base-type sweeps then run
                           one after the other instead of side by side, so that
                           each is timed alone; the results are the same)       */
  int formal_variant;   /* mixed mode: 0 autotuned, JFNK_FORMAL_SWEEP_THREAD,
                           JFNK_FORMAL_SWEEP_WARP or JFNK_FORMAL_SWEEP_THREAD_FUSED
                           forced (identical results)                             */
  int precond;          /* block-Jacobi preconditioner after the solutions of
                           Sect. 2.5.2: 1 first (background-scattering derivative
                           neglected; default), 2 second (chi_sca dJ/dn lagged from
                           the previous preconditioner build, zero at the start),
                           3 third (local self-consistent scattering term);
                           0: none (the Krylov solver works on J x = -F)          */
  int jvp;              /* Jacobian-vector products: JFNK_JVP_TANGENT (default) or a
                           finite difference of Fig. 2 (jfnk_jvp_scheme)          */
  int krylov;           /* jfnk_krylov: JFNK_KRYLOV_GMRES (default) or BICGSTAB    */
  int solver;           /* jfnk_solver_kind: JFNK_SOLVER_JFNK (default) or RH92    */
  int line_search;      /* 0: off (default); k > 0: backtracking on ||F||_inf after
                           each Newton update (Sect. 2.2.2), step 1, 1/2, 1/4, ...
                           until ||F||_inf falls below its value at the previous
                           base point, at most k halvings (each one F evaluation) */
} jfnk_options;

typedef struct {
  int status;           /* JFNK_OK when converged, else an error code               */
  int newton_iters;
  int rh92_iters;
  int F_calls;          /* F-class evaluations: base F, JVPs and RH92 solutions    */
  int jvp_calls;
  double F_norm;        /* final ||F||_inf                                          */
  double F_norm0;       /* ||F||_inf at the first JFNK base point                   */
  double dn_norm;       /* last population change                                  */
  double ray_points;    /* formal-solution ray-points evaluated (F_calls x rays)   */
  double formal_ms;     /* profile: summed duration of the formal-solution kernel
                           (mixed mode: of the base-type sweep launches)           */
  int formal_launches;  /* profile: number of timed launches (active ticks)        */
  int kernel_launches;  /* CUDA kernels launched by the solve (graph nodes included) */
  int formal_qb;        /* fused kernel: frequencies per block (0 for the others)   */
  int formal_threads;   /* threads per block (warps per block: JFNK_FORMAL_SWEEP_WARP) */
  int formal_kernel;    /* jfnk_formal_kernel that ran the formal solution          */
  double formal_tan_ms; /* profile, mixed mode: summed duration of the tangent-sweep
                           launches (the JVP evaluations' formal solutions)       */
  int formal_occ;       /* thread-per-frequency sweep: resident blocks per SM allowed
                           to the tangent sweep (0: no cap; chosen by the autotuner) */
  int formal_occ_base;  /* the same for the base-type sweep                        */
  int formal_fuse;      /* thread-per-frequency sweep: 0 when a separate kernel forms
                           the opacity tangent of the JVP evaluations, 1 when the
                           tangent sweep's inward pass forms it
                           (JFNK_FORMAL_SWEEP_THREAD_FUSED)                       */
  double stage_ms[6];   /* profile: summed durations over the active ticks of each
                           stage of a tick, all on one stream: [0] opacity (up to
                           the first formal kernel), [1] tangent sweep (mixed
                           mode), [2] base-type formal solution, [3] rate
                           integrals (and, moving columns, moments), [4] assembly
                           and preconditioner factorisation, [5] Krylov step      */
  int opacity_depths;   /* mixed mode: depths per thread of the opacity-tangent kernel
                           (its depth tile, chosen by the autotuner; 0: not tuned) */
} jfnk_stats;

/* ---- context ------------------------------------------------------------ */
const char* jfnk_last_error(void);
void jfnk_default_options(jfnk_options* o);
/* Creates a context on CUDA device ``device``. */
int jfnk_init(int device, jfnk_ctx** ctx);
int jfnk_destroy_ctx(jfnk_ctx* ctx);

/* ---- setup (Sect. 2.1, step a0) ------------------------------------------ */
/* Validates the descriptor and builds the union frequency grid, the transition
 * windows and their trapezoid quadrature weights. */
int jfnk_create_atom(jfnk_ctx* ctx, const jfnk_atom_desc* d, jfnk_atom** out);
int jfnk_destroy_atom(jfnk_atom* a);
int jfnk_atom_info(const jfnk_atom* a, int* n_levels, int* n_transitions, int* n_nu);
/* Copies the union frequency grid [n_nu] (Hz) to host memory. */
int jfnk_atom_frequencies(const jfnk_atom* a, double* nu);

/* Builds the depth-dependent tables of one column on the device: LTE
 * populations, Voigt profiles, bound-free g_ij, Planck functions, background
 * and collision rates. Enqueued on the context's internal stream and
 * synchronised before returning. */
int jfnk_create_atmosphere(jfnk_ctx* ctx, const jfnk_atom* atom, const jfnk_atmos_desc* d,
                           jfnk_atmos** out);
/* Returns the column's tables to the device's stream-ordered pool (on the
 * context's internal stream: no device-wide synchronisation, so a serving loop
 * can drop finished columns while others run). The caller must not destroy an
 * atmosphere that a launched solve still uses, nor after its context. */
int jfnk_destroy_atmosphere(jfnk_atmos* a);
/* n_depth, n_nu, n_levels, n_transitions, and ray-points per evaluation. */
int jfnk_atmos_info(const jfnk_atmos* a, int* n_depth, int* n_nu, int* n_levels,
                    int* n_transitions, double* ray_points);
/* Table export for tests: which = 0 LTE populations [nz*nl], 1 Planck B [nq*nz],
 * 2 collision rates C[k][i][j] [nz*nl*nl], 3 V_t on its window [sum_t w_t * nz]
 * (transition-major, window-point-major, depth fastest), 4 g_t likewise,
 * 5 quadrature weights omega_t on the window [sum_t w_t], 6 chi_c [nq*nz],
 * 7 eta_c [nq*nz], 8 (moving columns) V_t seen along each direction
 * [2 n_mu][sum_t w_t][nz] (outgoing mu_1..mu_n, then ingoing). ``count`` is
 * the capacity of ``out`` in doubles. */
int jfnk_atmos_table(const jfnk_atmos* a, int which, double* out, size_t count);

/* ---- the hot path --------------------------------------------------------- */
/* Residual F(n) (Algorithm 1, Eqs. residuals_1/2) with the lagged mean
 * intensity J_dagger in the background-scattering emissivity. The conservation
 * row of each depth is the most populated level of n (lowest index on ties).
 * J_new (nullable) receives the new mean intensity; I_emergent (nullable) the
 * outgoing intensity at the top [nq * n_mu] (q-major). */
int jfnk_residual(jfnk_ctx* ctx, const jfnk_atmos* a, int precision,
                  const double* n, const double* J_dagger, double* F, double* J_new,
                  double* I_emergent, jfnk_mem where, void* stream);

/* Jacobian-vector product J_F(n) v (Sect. 2.4): exact first-order tangent
 * propagation through every step of Algorithm 1, the value the complex-step
 * scheme of Eq. complex converges to as eps -> 0. J_dagger and the
 * conservation rows are taken at n and not perturbed. */
int jfnk_jvp(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, const double* n,
             const double* J_dagger, const double* v, double* Jv, jfnk_mem where, void* stream);

/* Block-Jacobi preconditioner P^k = Gamma^k + A^kk with the conservation row
 * set to -1 (Sect. 2.5.1-2.5.2, first solution), unfactored, P[k][i][j]. */
int jfnk_block_jacobi(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, const double* n,
                      const double* J_dagger, double* P, jfnk_mem where, void* stream);

/* The preconditioner blocks of any of the three solutions of Sect. 2.5.2
 * (variant 1, 2 or 3), unfactored, P[k][i][j], for tests of the variants.
 * dJdn_prev [nq*nz*nl] (q-major, then depth, then level; nullable = zero) is
 * the lagged estimate d J_nu^k/d n_j^k that variant 2 uses; dJdn_out (same
 * layout, nullable) receives variant 2's renewed estimate. Other arguments as
 * jfnk_block_jacobi. JFNK_E_INVALID for another variant. */
int jfnk_block_jacobi_variant(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, int variant,
                              const double* n, const double* J_dagger, const double* dJdn_prev,
                              double* P, double* dJdn_out, jfnk_mem where, void* stream);

/* One RH92 population update (Rybicki & Hummer 1992 with full preconditioning,
 * the paper's reference method): n_out from the formal solution at n. The
 * update is returned as solved, without the per-depth limiting that
 * jfnk_solve applies to the RH92 corrections of a hybrid start. */
int jfnk_rh92_update(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, const double* n,
                     const double* J_dagger, double* n_out, double* J_new, jfnk_mem where,
                     void* stream);

/* Solve F(n) = 0 with Algorithm 2 on the device. n_inout: initial guess when
 * o->init == JFNK_INIT_USER, solution on return [nz*nl]. J_inout (nullable):
 * initial J^dagger on input if non-NULL (else B_nu(T)), final mean intensity
 * on return. Synchronises ``stream`` before returning. */
int jfnk_solve(jfnk_ctx* ctx, const jfnk_atmos* a, const jfnk_options* o, double* n_inout,
               double* J_inout, jfnk_stats* stats, jfnk_mem where, void* stream);

/* Solves n_cols independent columns together: every residual of one JFNK
 * tick (one F-class evaluation per in-flight column) runs in one launch
 * sequence captured in a CUDA graph. n_inout[c] / J_inout[c] as above (the
 * J_inout array itself may be NULL). */
int jfnk_batch_solve(jfnk_ctx* ctx, int n_cols, const jfnk_atmos* const* cols,
                     const jfnk_options* o, double* const* n_inout, double* const* J_inout,
                     jfnk_stats* stats, jfnk_mem where, void* stream);

/* ---- persistent batches -------------------------------------------------------- */
/* A batch plan owns the device work buffers of n_cols columns (precision and
 * Krylov size fixed at creation) and its tick graph, so that repeated solves
 * pay for allocation, autotuning and graph capture once. The atmospheres must
 * outlive the plan. jfnk_batch_run solves every column like jfnk_batch_solve
 * (o->precision must equal the plan's, o->krylov_max <= its krylov_max). */
typedef struct jfnk_batch jfnk_batch;
int jfnk_batch_create(jfnk_ctx* ctx, int n_cols, const jfnk_atmos* const* cols, int precision,
                      int krylov_max, jfnk_batch** out);
int jfnk_batch_run(jfnk_batch* b, const jfnk_options* o, double* const* n_inout,
                   double* const* J_inout, jfnk_stats* stats, jfnk_mem where, void* stream);
int jfnk_batch_destroy(jfnk_batch* b);

/* ---- residual without device allocation -------------------------------------- */
/* The paper has no counterpart to this entry point: it is a deployment aid.
 * Same result as jfnk_residual(ctx, a, JFNK_FP64, n, J_dagger, F, J_new, NULL,
 * JFNK_MEM_DEVICE, stream), but every work buffer comes from one fixed device
 * array of JFNK_STATIC_SCRATCH_BYTES built into the library (held on every GPU
 * that loads it until the process exits), so the call never allocates device
 * memory. For callers that cannot allocate: code running under a memory budget
 * owned by another allocator, or latency-critical loops that must not pay for
 * cudaMalloc (which can synchronise the device and fail mid-run).
 *   n [nz*nl], J_dagger [nq*nz] (nullable: B_nu(T)), F [nz*nl], J_new [nq*nz]
 *   (nullable): device pointers on the context's device; the work is enqueued
 *   on ``stream`` and the call returns without synchronising.
 * The formal solution runs in the fused kernel of jfnk_residual, whose buffers
 * take roughly nq * nz * 6 * 8 bytes; a column too deep for it (a frequency's
 * rays over all depths beyond one block's shared memory) takes the per-ray
 * kernels, about nq * nz * (8 n_mu + 9) * 8 bytes. A column whose buffers
 * exceed the array is rejected with JFNK_E_INVALID and a message giving the
 * size needed.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture (a first call on a
 * stream that is being captured returns JFNK_E_INVALID). Every call shares
 * the array: calls that overlap on the GPU race and must be serialised by the
 * caller. The enqueued kernels read the atmosphere's tables: synchronise
 * ``stream`` before destroying the atmosphere (jfnk_destroy_atmosphere returns
 * the tables to a pool on another stream, not ordered after this one). */
#define JFNK_STATIC_SCRATCH_BYTES (32u << 20)
int jfnk_residual_static(jfnk_ctx* ctx, const jfnk_atmos* a, const double* n,
                         const double* J_dagger, double* F, double* J_new, void* stream);

/* ---- serving: continuous batching of column solves ------------------------ */
/* A server solves independent columns (Algorithm 2 per column) as they
 * arrive. It holds max_slots columns on the device at once; every step
 * advances all of them by one captured tick graph (8 F-class evaluations
 * each) and, between steps, retires finished columns and admits queued ones
 * in arrival order. A queued column is admitted when a slot is free AND its
 * own work buffers (jfnk_server_bytes) fit in the server's device memory pool,
 * which is carved by a first-fit allocator: large and small columns share the
 * pool as memory frees up. Populations, Krylov bases, opacities and
 * intensities stay resident on the device for the whole solve. A column's
 * result does not depend on the other columns in flight. */
typedef struct jfnk_server jfnk_server;

typedef struct {
  int max_slots;        /* columns in flight at once (>= 1)                        */
  int max_depth;        /* slot shape: the largest n_depth a request may have      */
  int max_freq;         /* largest union frequency grid                            */
  int max_levels;       /* largest level count (<= JFNK_MAX_LEVELS)                */
  int max_trans;        /* largest transition count (<= 32)                        */
  int max_mu;           /* largest angle count per hemisphere (<= JFNK_MAX_MU)     */
  size_t mem_bytes;     /* device memory pool for work buffers; 0: half the free memory */
  jfnk_options opts;    /* default options of a request (init must be LTE)         */
} jfnk_server_desc;

typedef struct {
  long long id;         /* the id given to jfnk_server_submit                      */
  int status;           /* JFNK_OK when converged                                  */
  jfnk_stats stats;
  double t_submit;      /* jfnk_server_clock at submission, admission and retirement */
  double t_admit;
  double t_done;
} jfnk_result;

/* Creates a server on ctx (its own stream). Errors: JFNK_E_INVALID for a bad
 * shape or options, JFNK_E_NOMEM when the pool cannot be allocated. */
int jfnk_server_create(jfnk_ctx* ctx, const jfnk_server_desc* d, jfnk_server** out);
/* Device bytes of the work buffers of column ``a`` in this server. */
int jfnk_server_bytes(jfnk_server* sv, const jfnk_atmos* a, size_t* bytes);
/* Enqueues a solve of column ``a`` from LTE populations. ``a`` (and its atom)
 * must stay alive until the result has been polled. n_out (host, nz*nl
 * doubles, nullable) receives the populations before the result is reported.
 * opts (nullable: the server's) sets this column's tolerances, limits and
 * hybrid start; its precision must be the server's, its krylov_max at most
 * the server's, and its precond not 2 (the server keeps no lagged estimate). JFNK_E_INVALID when ``a`` exceeds the slot shape or the pool,
 * or for such options. May be called from another thread than
 * jfnk_server_step. */
int jfnk_server_submit(jfnk_server* sv, const jfnk_atmos* a, long long id, double* n_out,
                       const jfnk_options* opts);
/* Admits, runs one tick graph over the columns in flight, retires the finished
 * ones. n_active / n_queued (nullable): columns in flight / waiting after it. */
int jfnk_server_step(jfnk_server* sv, int* n_active, int* n_queued);
/* Moves up to ``max`` finished results to ``out``; *n gets their number. */
int jfnk_server_poll(jfnk_server* sv, jfnk_result* out, int max, int* n);
/* Seconds since the server was created (steady clock). */
double jfnk_server_clock(jfnk_server* sv);
int jfnk_server_destroy(jfnk_server* sv);

/* ---- measurement ----------------------------------------------------------- */
/* Throughput probe of one arithmetic pipe on the context's device, for roofline
 * denominators: kind 0 = FP64 fused multiply-add, 1 = FP32 fused multiply-add,
 * 2 = FP64 exp(), 3 = MUFU base-2 exponential (ex2.approx.ftz.f32). Runs a fixed dependent-chain workload
 * over every SM and returns operations per second (an FMA counts as 2 flops;
 * an exp as 1 operation). */
int jfnk_probe_alu(jfnk_ctx* ctx, int kind, double* ops_per_s);

/* Accuracy check of the float-pair arithmetic (hi + lo, about 48 bits, on the
 * FP32 pipe) that the mixed mode's base evaluations use for S, J, the opacity
 * sums (Eqs. chi, eta) and the rate sums (Eqs. Rij, Rji): each a[i], b[i] is
 * rounded to a pair, combined by op (0 sum, 1 difference, 2 product,
 * 3 quotient, 4 same-sign accumulation) and returned as hi + lo in FP64.
 * Host arrays of n values, caller-owned; JFNK_E_INVALID for an unknown op,
 * n < 0 or NULL pointers. */
int jfnk_check_arith(jfnk_ctx* ctx, int op, const double* a, const double* b, double* out, int n);

#ifdef __cplusplus
}
#endif
#endif /* JFNK_H */
