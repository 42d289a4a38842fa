// Host-side objects of the library and the interfaces between its units.
#pragma once

#include <memory>
#include <mutex>

#include "common.cuh"

namespace jfnk {

// Bump allocator over one device allocation: callers reserve typed blocks,
// then allocate once; every block is 256-byte aligned. With a stream the
// block comes from the device's stream-ordered pool (cudaMallocAsync /
// cudaFreeAsync on that stream), so that releasing it does not wait for the
// whole device, as cudaFree does: a serving loop creates and drops one
// atmosphere per request while other columns run.
struct DeviceArena {
  char* base = nullptr;
  size_t bytes = 0;
  size_t cursor = 0;
  cudaStream_t stream = nullptr;
  void reset() { cursor = 0; }
  template <typename T>
  size_t take(size_t count) {
    size_t off = cursor;
    cursor += ((count * sizeof(T) + 255) / 256) * 256;
    if (cursor == off) cursor += 256;
    return off;
  }
  int allocate();
  void release();
  template <typename T>
  T* ptr(size_t off) const {
    return reinterpret_cast<T*>(base + off);
  }
  ~DeviceArena() { release(); }
};

struct AtomData {
  int nl = 0, nt = 0, nq = 0, nwin = 0;
  std::vector<double> E, g;
  std::vector<int> stage;
  double mass = 0, vchar = 0;
  std::vector<jfnk_bb_desc> bb;
  std::vector<jfnk_bf_desc> bf;
  std::vector<double> nu;
  std::vector<int> t_lo, t_up, t_kind, t_idx, t_q0, t_q1, t_base;
  std::vector<double> t_nu0, t_w;
  std::vector<int> q_off, q_t;
};

struct AtmosData {
  int nz = 0, nq = 0, nl = 0, nt = 0, nmu = 0, nwin = 0;
  bool moving = false;                // a line-of-sight velocity field (per-direction profiles)
  double ray_points = 0;
  DeviceArena arena;
  ColTables tables{};
  std::vector<double> host_t_w;
};

}  // namespace jfnk

struct jfnk_ctx {
  int device = 0;
  int n_sm = 0;
  // atmosphere set-up lanes: a stream (highest priority), its pinned staging
  // buffer and the event of its last set-up; callers take lanes in turn and
  // wait for their own set-up outside the context lock
  static constexpr int kSetupLanes = 4;
  cudaStream_t setup_stream[kSetupLanes] = {};
  cudaEvent_t setup_done[kSetupLanes] = {};
  char* stage[kSetupLanes] = {};
  size_t stage_bytes[kSetupLanes] = {};
  int next_lane = 0;
  cudaStream_t stream = nullptr;      // stream of the evaluations and solves
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::mutex mu;
};

struct jfnk_atom {
  jfnk_ctx* ctx;
  jfnk::AtomData d;
};

struct jfnk_atmos {
  jfnk_ctx* ctx;
  const jfnk_atom* atom;
  jfnk::AtmosData d;
  void* work = nullptr;               // cached single-column work buffers
};

namespace jfnk {

int build_atom(const jfnk_atom_desc* d, AtomData* A);
// Enqueues the set-up of one column on set-up lane ``lane`` (its stream and
// staging buffer, which must be idle) and records the lane's event; the
// tables are ready once that event has completed.
int build_atmosphere(jfnk_ctx* ctx, int lane, const AtomData& A, const jfnk_atmos_desc* d, AtmosData* M);

// Formal-solution kernels: per-ray buffers + ray-sum kernel (any size),
// in-block fused kernel (FP64), per-frequency sweep kernel (mixed precision).
enum FormalKind { FORMAL_UNFUSED = 0, FORMAL_FUSED = 1, FORMAL_SWEEP = 2, FORMAL_MOVING = 3 };

// A batch of columns with their work buffers, resident on the device.
struct Batch {
  int ncols = 0;
  int mixed = 0;
  int kmax = 0;
  int max_nz = 0, max_nq = 0, max_nt = 0, max_N = 0, max_nmu = 0;
  int max_nl = 0;   // largest level count (compacted views keep the full batch's)
  int optan_depths = 0;   // opacity tangent: depths per thread (autotuned; 0: the default)
  DeviceArena arena;
  ColDesc* d_cols = nullptr;          // device array [ncols]
  std::vector<ColDesc> h_cols;        // host mirror
  SolverState* d_state = nullptr;     // [ncols]
  int* d_status = nullptr;            // [ncols] copy of st.status for polling
  SolverOpts* d_opts = nullptr;       // solver options read by the Krylov kernel
  cudaGraphExec_t graph = nullptr;    // captured tick sequence
  int graph_ticks = 0;
  bool graph_profiled = false;
  int formal_kind = 0;                // FORMAL_UNFUSED, FORMAL_FUSED or FORMAL_SWEEP
  int formal_qb = 0;                  // frequencies per block of the fused formal kernel
  int formal_threads = 0;             // fused: threads per block; sweep: threads (variant 1) or warps (2)
  int sweep_variant = 0;              // sweep kernel: 1 thread per frequency, 2 warp per frequency pair
  int sweep_fuse = 0;                 // thread variant: the tangent sweep forms the opacity tangent itself
                                      // (1, forced variant only), 0: a separate kernel does
  int sweep_occ = 0, sweep_occ_base = 0;   // thread variant: blocks per SM allowed (0: no cap) for the
                                           // tangent and base-type sweeps (shared-memory padding)
  int tuned_variant = 0, tuned_size = 0, tuned_fuse = 0;   // autotuner's choice (a forced variant may
                                                          // replace it for a solve)
  int max_overlap = 0;                // most transitions active at one frequency over the batch
  int n_sm = 1;                       // multiprocessors of the batch's device
  bool tuned = false;                 // autotuner has run on this batch
  int graph_kernels = 0;              // kernel nodes in the captured tick graph
  long replays = 0;                   // graph replays of the last solve
  std::vector<cudaEvent_t> tick_ev;   // event pairs around the formal kernel(s) of each tick
  // mixed mode: the tangent kernels of a tick run on a side stream, beside the
  // base kernels of the other columns, and join before the assembly
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  std::vector<float> tick_ms;         // per-tick formal-kernel durations of the last solve (base-type sweep)
  std::vector<float> tick_tan_ms;     // per-tick tangent-sweep durations (mixed mode)
  std::vector<float> tick_stage_ms;   // per tick, kStages durations (jfnk_stats.stage_ms order)
  int* h_status = nullptr;            // pinned host mirror of d_status
  // launch view over the columns still running (straggler compaction)
  ColDesc* d_view = nullptr;          // device array [ncols] of the view's descriptors
  cudaGraphExec_t graph_view = nullptr;
  int compactions = 0;                // view rebuilds in the last solve
  // lagged d J/d n of the second preconditioner solution, allocated on the
  // first solve that asks for it ([nq][nz][nl] per column, in one arena)
  DeviceArena dJ_arena;
  bool has_dJdn = false;
  ~Batch();
};

// Work buffers of one column: bytes of its block (256-byte aligned parts), and
// the descriptor of a column whose block starts at ``base``.
struct ColLayout;
size_t column_bytes(const AtmosData& M, int kind, int mixed, int kmax, ColLayout* out);
void column_bind(char* base, const AtmosData& M, int kind, int mixed, int kmax, SolverState* st, ColDesc* d);

// Allocates work buffers for columns ``tabs`` (precision: mixed or FP64).
int batch_create(Batch* b, const std::vector<const AtmosData*>& cols, int mixed, int kmax);
// Launch sequence of one F-class evaluation for every column of the batch.
// ev0/ev1 (optional) are recorded around the formal-solution kernel. With a
// side stream (mixed mode) the tangent kernels go there, forked from and joined
// back into s, and ev2/ev3 bracket the tangent sweep (ev0/ev1 the base one).
// stage (optional, without a side stream): three events recorded at the start
// of the evaluation, after the rate integrals and after the assembly.
int launch_evaluation(const Batch& b, cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                      cudaStream_t side = nullptr, cudaEvent_t ev2 = nullptr, cudaEvent_t ev3 = nullptr,
                      const cudaEvent_t* stage = nullptr);
// Creates the side stream and the fork/join events of a mixed-mode batch.
int ensure_side_stream(Batch* b);
// Allocates and binds the lagged d J/d n buffers of every column (once).
int ensure_dJdn(Batch* b, cudaStream_t s);
// Launch of the Krylov/Newton state machine step.
int launch_krylov_step(const Batch& b, cudaStream_t s);
// Fused formal solution + ray sums (formal_fused.cu).
size_t fused_smem_bytes(int qb, int nz, int nmu, bool mixed);
int fused_default_qb(int max_nz, int max_nmu, bool mixed);
int fused_prepare(Batch* b);
int launch_formal_fused(const Batch& b, cudaStream_t s);
int fused_autotune(Batch* b, cudaStream_t s);
// Per-frequency sweep kernel of the mixed mode (formal_sweep.cu).
size_t sweep_scratch_bytes(int nq, int nz);
int sweep_prepare(Batch* b);
// which: 0 every column, 1 base-type evaluations only, 2 tangent ones only
int launch_formal_sweep(const Batch& b, cudaStream_t s, int which = 0);
// The tangent sweep of this batch forms the opacity tangent itself (so the
// separate opacity-tangent kernel is not launched).
bool sweep_fused(const Batch& b);
// The separate mixed-mode opacity-tangent kernel (residual.cu).
// depths: the run of depths per thread (0: the batch's tuned run).
int launch_opacity_tan(const Batch& b, cudaStream_t s, int depths = 0);
// Warps per block of the warp variant whose shared memory fits depth nz (0: none).
int sweep_warp_size(int nz);
int sweep_autotune(Batch* b, cudaStream_t s);
// Mixed mode: converts the J^dagger of columns d_cols[0, ncols) (FP64, as
// filled by the host or the tables) to float pairs in place (to_pairs), or
// their J_new back to FP64; FP64 columns are left alone.
int launch_j_pairs(const ColDesc* d_cols, int ncols, size_t max_qz, cudaStream_t s, bool to_pairs);
// Moving columns (velocity.cu): one F-class evaluation of every column of a
// batch whose formal kind is FORMAL_MOVING (opacity per direction, formal
// solution per ray, moments, rate integrals; then the common assembly).
int launch_moving_evaluation(const Batch& b, cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// Kernel attributes of the current device, set once per context (residual.cu).
int prepare_kernels();
// Opacity kernel of the mixed mode (tangent columns skipped when the sweeps form it).
int launch_opacity_mixed(const Batch& b, cudaStream_t s, int skip_tangent);
// Solver options: checks, device copy (api.cu).
int validate_options(const jfnk_options* o);
void options_to_device(const jfnk_options* o, SolverOpts* so);
// Captures kTicksPerGraph ticks (evaluation + Krylov step) of the batch's launch view.
constexpr int kTicksPerGraph = 8;
int capture_ticks(Batch* b, cudaStream_t s, bool profile, cudaGraphExec_t* out);
// Sets every column's forced evaluation mode (explicit API calls) or -1.
int batch_set_forced_mode(Batch* b, int mode, cudaStream_t s);
// Conservation rows from the current populations.
int launch_istar(const Batch& b, cudaStream_t s);
// Zero-radiation initial guess (rate equations with I = 0) in every column's n;
// reads n = LTE populations for the conservation rows.
int launch_zero_radiation(const Batch& b, cudaStream_t s);
// RH92 per-depth update from an EV_RH92 evaluation (explicit API path).
int launch_rh92_update(const Batch& b, cudaStream_t s);

}  // namespace jfnk
