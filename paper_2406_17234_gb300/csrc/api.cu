// C ABI of the library (include/jfnk.h): contexts, atoms, columns, explicit
// residual / JVP / preconditioner / RH92 evaluations, and the solvers.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace jfnk {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

Batch::~Batch() {
  if (graph) cudaGraphExecDestroy(graph);
  if (graph_view) cudaGraphExecDestroy(graph_view);
  if (h_status) cudaFreeHost(h_status);
  for (cudaEvent_t e : tick_ev) cudaEventDestroy(e);
  if (fork_ev) cudaEventDestroy(fork_ev);
  if (join_ev) cudaEventDestroy(join_ev);
  if (side) cudaStreamDestroy(side);
}

int ensure_side_stream(Batch* b) {
  if (b->side) return JFNK_OK;
  JFNK_CUDA(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
  JFNK_CUDA(cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming));
  JFNK_CUDA(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
  return JFNK_OK;
}

// Events per tick of a profiled graph: ev0/ev1 around the (base-type) formal
// kernel, ev2/ev3 around the tangent sweep (mixed mode), then the tick's start,
// the end of its rate integrals, of its assembly and of its Krylov step.
constexpr int kTickEvents = 8;
constexpr int kStages = 6;
static int tick_events(const Batch&) { return kTickEvents; }

// Work buffers and the tick graph of one column, cached in its handle.
struct SingleWork {
  std::unique_ptr<Batch> b[2];
};

static SingleWork* single_work(const jfnk_atmos* a) {
  return reinterpret_cast<SingleWork*>(a->work);
}

static int get_single(const jfnk_atmos* a, int mixed, Batch** out) {
  SingleWork* sw = single_work(a);
  if (!sw->b[mixed]) {
    std::unique_ptr<Batch> b(new Batch());
    std::vector<const AtmosData*> cols{&a->d};
    int rc = batch_create(b.get(), cols, mixed, kMaxKrylov);
    if (rc) return rc;
    sw->b[mixed] = std::move(b);
  }
  *out = sw->b[mixed].get();
  return JFNK_OK;
}

static int copy_in(void* dst, const void* src, size_t bytes, jfnk_mem where, cudaStream_t s) {
  JFNK_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            where == JFNK_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  return JFNK_OK;
}

static int copy_out(void* dst, const void* src, size_t bytes, jfnk_mem where, cudaStream_t s) {
  JFNK_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            where == JFNK_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  return JFNK_OK;
}

static int check_common(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, jfnk_mem where) {
  if (!ctx || !a) return fail(JFNK_E_INVALID, "context and atmosphere are required");
  if (a->ctx != ctx) return fail(JFNK_E_INVALID, "atmosphere belongs to another context");
  if (precision != JFNK_FP64 && precision != JFNK_MIXED) return fail(JFNK_E_INVALID, "unknown precision");
  if (where != JFNK_MEM_HOST && where != JFNK_MEM_DEVICE) return fail(JFNK_E_INVALID, "unknown memory kind");
  JFNK_CUDA(cudaSetDevice(ctx->device));
  return JFNK_OK;
}

// One explicit evaluation of the single-column batch in mode ``mode``; a base
// evaluation builds the preconditioner blocks of solution ``variant``.
static int explicit_eval(jfnk_ctx* ctx, const jfnk_atmos* a, Batch* b, int mode, const double* n,
                         const double* Jdag, jfnk_mem where, cudaStream_t s, int variant = 1) {
  const ColDesc& c = b->h_cols[0];
  const AtmosData& M = a->d;
  const size_t N = (size_t)M.nz * M.nl, QZ = (size_t)M.nq * M.nz;
  int rc;
  {
    jfnk_options o;
    jfnk_default_options(&o);
    o.precond = variant;
    SolverOpts so;
    options_to_device(&o, &so);
    JFNK_CUDA(cudaMemcpyAsync(b->d_opts, &so, sizeof(so), cudaMemcpyHostToDevice, s));
  }
  if (n && (rc = copy_in(c.w.n, n, N * 8, where, s))) return rc;
  if (Jdag) {
    if ((rc = copy_in(c.w.Jdag, Jdag, QZ * 8, where, s))) return rc;
  } else {
    JFNK_CUDA(cudaMemcpyAsync(c.w.Jdag, M.tables.Bn, QZ * 8, cudaMemcpyDeviceToDevice, s));
  }
  if ((rc = batch_set_forced_mode(b, mode, s))) return rc;
  if (b->mixed && (rc = launch_j_pairs(b->d_cols, 1, QZ, s, true))) return rc;
  return launch_evaluation(*b, s);
}

void options_to_device(const jfnk_options* o, SolverOpts* so) {
  so->ftol = o->ftol;
  so->fdrop = o->fdrop;
  so->rtol = o->rtol;
  so->rh92_switch = o->rh92_switch;
  so->maxiter = o->maxiter;
  so->krylov_max = o->krylov_max;
  so->max_restarts = o->max_restarts;
  so->clamp = o->clamp;
  so->rh92_warmup = o->rh92_warmup;
  so->max_ticks = o->max_ticks;
  so->precond = o->precond;
  so->jvp = o->jvp;
  so->krylov = o->krylov;
  so->solver = o->solver;
  so->line_search = o->line_search;
}

int validate_options(const jfnk_options* o) {
  if (!o) return fail(JFNK_E_INVALID, "options are NULL");
  if (!(o->rtol > 0.0 && o->rtol < 1.0)) return fail(JFNK_E_INVALID, "rtol must be in (0, 1)");
  if (!(o->ftol >= 0.0) || !(o->fdrop >= 0.0)) return fail(JFNK_E_INVALID, "ftol, fdrop must be >= 0");
  if (o->krylov_max < 1 || o->krylov_max > kMaxKrylov) return fail(JFNK_E_INVALID, "krylov_max must be in [1, 64]");
  if (o->maxiter < 1 || o->max_restarts < 0 || o->max_ticks < 1) return fail(JFNK_E_INVALID, "iteration limits must be positive");
  if (o->precision != JFNK_FP64 && o->precision != JFNK_MIXED) return fail(JFNK_E_INVALID, "unknown precision");
  if (o->init != JFNK_INIT_LTE && o->init != JFNK_INIT_USER && o->init != JFNK_INIT_ZERO_RADIATION)
    return fail(JFNK_E_INVALID, "init must be JFNK_INIT_LTE, JFNK_INIT_USER or JFNK_INIT_ZERO_RADIATION");
  if (o->precond < 0 || o->precond > 3) return fail(JFNK_E_INVALID, "precond must be 0, 1, 2 or 3");
  if (o->line_search < 0 || o->line_search > 60) return fail(JFNK_E_INVALID, "line_search must be in [0, 60]");
  if (o->jvp < JFNK_JVP_TANGENT || o->jvp > JFNK_JVP_CENTRAL) return fail(JFNK_E_INVALID, "unknown jvp scheme");
  if (o->jvp != JFNK_JVP_TANGENT && o->precision != JFNK_FP64)
    return fail(JFNK_E_INVALID, "difference JVPs need precision JFNK_FP64");
  if (o->rh92_warmup < 0) return fail(JFNK_E_INVALID, "rh92_warmup must be >= 0");
  if (o->krylov != JFNK_KRYLOV_GMRES && o->krylov != JFNK_KRYLOV_BICGSTAB)
    return fail(JFNK_E_INVALID, "krylov must be JFNK_KRYLOV_GMRES or JFNK_KRYLOV_BICGSTAB");
  if (o->krylov == JFNK_KRYLOV_BICGSTAB && o->krylov_max < 5)
    return fail(JFNK_E_INVALID, "BiCGSTAB keeps its six vectors in the Krylov basis: krylov_max must be >= 5");
  if (o->solver != JFNK_SOLVER_JFNK && o->solver != JFNK_SOLVER_RH92)
    return fail(JFNK_E_INVALID, "solver must be JFNK_SOLVER_JFNK or JFNK_SOLVER_RH92");
  if (o->formal_variant != 0 && o->formal_variant != JFNK_FORMAL_SWEEP_THREAD &&
      o->formal_variant != JFNK_FORMAL_SWEEP_WARP && o->formal_variant != JFNK_FORMAL_SWEEP_THREAD_FUSED)
    return fail(JFNK_E_INVALID,
                "formal_variant must be 0, JFNK_FORMAL_SWEEP_THREAD, JFNK_FORMAL_SWEEP_WARP or "
                "JFNK_FORMAL_SWEEP_THREAD_FUSED");
  return JFNK_OK;
}

__global__ void k_init_state(SolverState* st, int n, int phase) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  SolverState s{};
  s.phase = phase;
  s.status = 1;
  st[c] = s;
}


// Captures kTicksPerGraph ticks (evaluation + Krylov step) of the batch's
// current launch view into an executable graph.
int capture_ticks(Batch* b, cudaStream_t s, bool profile, cudaGraphExec_t* out) {
  const int ne = tick_events(*b);
  if (profile && (int)b->tick_ev.size() < ne * kTicksPerGraph) {
    for (cudaEvent_t e : b->tick_ev) cudaEventDestroy(e);
    b->tick_ev.assign(ne * kTicksPerGraph, nullptr);
    for (auto& e : b->tick_ev) JFNK_CUDA(cudaEventCreate(&e));
  }
  if (b->formal_kind == FORMAL_SWEEP) {
    int rs = ensure_side_stream(b);
    if (rs) return rs;
  }
  cudaGraph_t g;
  JFNK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = JFNK_OK;
  for (int t = 0; t < kTicksPerGraph && !rc; ++t) {
    cudaEvent_t* ev = profile ? &b->tick_ev[(size_t)ne * t] : nullptr;
    // a profiled tick runs the tangent and base-type chains one after the
    // other on s (no side stream), so that each sweep's events time it alone
    const bool sweep = b->formal_kind == FORMAL_SWEEP;
    rc = launch_evaluation(*b, s, ev ? ev[0] : nullptr, ev ? ev[1] : nullptr, profile ? nullptr : b->side,
                           ev && sweep ? ev[2] : nullptr, ev && sweep ? ev[3] : nullptr, ev ? ev + 4 : nullptr);
    if (!rc) rc = launch_krylov_step(*b, s);   // P^k was factorised by the assembly
    if (!rc && ev && cudaEventRecordWithFlags(ev[7], s, cudaEventRecordExternal) != cudaSuccess)
      rc = fail(JFNK_E_CUDA, "tick event record");
  }
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(JFNK_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  size_t nnodes = 0;
  cudaGraphGetNodes(g, nullptr, &nnodes);
  std::vector<cudaGraphNode_t> nodes(nnodes);
  cudaGraphGetNodes(g, nodes.data(), &nnodes);
  b->graph_kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) b->graph_kernels++;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(JFNK_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  b->graph_ticks = kTicksPerGraph;
  return JFNK_OK;
}

static int ensure_graph(Batch* b, cudaStream_t s, bool profile) {
  if (b->graph && b->graph_profiled == profile) return JFNK_OK;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  int rc = capture_ticks(b, s, profile, &b->graph);
  if (rc) return rc;
  b->graph_profiled = profile;
  if (!b->h_status) JFNK_CUDA(cudaMallocHost(&b->h_status, sizeof(int) * std::max(1, b->ncols)));
  return JFNK_OK;
}

// Runs the tick graph until every column has left the running state. When at
// most half of the columns of the current launch view are still running, the
// view is rebuilt over those columns only (their descriptors are gathered
// into d_view, the launch extents shrink) and its tick graph recaptured, so
// that finished columns stop costing launched blocks.
static int run_to_completion(Batch* b, const jfnk_options* o, cudaStream_t s) {
  const bool profile = o->profile != 0;
  int rc = ensure_graph(b, s, profile);
  if (rc) return rc;
  b->tick_ms.clear();
  b->tick_tan_ms.clear();
  b->tick_stage_ms.clear();
  b->replays = 0;
  b->compactions = 0;
  // the full view, restored before returning
  const int nfull = b->ncols;
  ColDesc* dfull = b->d_cols;
  const int fz = b->max_nz, fq = b->max_nq, ft = b->max_nt, fN = b->max_N, fm = b->max_nmu;
  const int fvariant = b->sweep_variant, fthreads = b->formal_threads;
  std::vector<int> view(nfull);
  for (int c = 0; c < nfull; ++c) view[c] = c;
  cudaGraphExec_t cur = b->graph;
  const long max_replays = (long)o->max_ticks / b->graph_ticks + 2;
  rc = JFNK_OK;
  for (long r = 0; r < max_replays && !rc; ++r) {
    if (cudaGraphLaunch(cur, s) != cudaSuccess) { rc = fail(JFNK_E_CUDA, "cudaGraphLaunch failed"); break; }
    b->replays++;
    if (cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int) * b->ncols, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { rc = fail(JFNK_E_CUDA, "status poll failed"); break; }
    if (profile) {
      // the formal kernels' own durations (base-type and tangent sweeps apart)
      const int ne = tick_events(*b);
      const bool sweep = b->formal_kind == FORMAL_SWEEP;
      for (int t = 0; t < b->graph_ticks; ++t) {
        const cudaEvent_t* e = &b->tick_ev[(size_t)ne * t];
        auto span = [&](int i, int j) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e[i], e[j]);
          return ms;
        };
        const float base = span(0, 1), tan = sweep ? span(2, 3) : 0.f;
        b->tick_ms.push_back(base);
        b->tick_tan_ms.push_back(tan);
        // opacity (up to the first formal kernel), tangent sweep, base-type
        // formal solution, rate integrals, assembly, Krylov step
        const float st[kStages] = {span(4, sweep ? 2 : 0), tan, base, span(1, 5), span(5, 6), span(6, 7)};
        b->tick_stage_ms.insert(b->tick_stage_ms.end(), st, st + kStages);
      }
    }
    std::vector<int> running;
    for (int c = 0; c < b->ncols; ++c)
      if (b->h_status[c] == 1) running.push_back(view[c]);
    if (running.empty()) break;
    if (b->ncols > 1 && (int)running.size() * 2 <= b->ncols) {
      std::vector<ColDesc> hv;
      int mz = 0, mq = 0, mt = 0, mN = 0, mm = 0;
      for (int c : running) {
        const ColDesc& d = b->h_cols[c];
        hv.push_back(d);
        mz = std::max(mz, d.t.nz); mq = std::max(mq, d.t.nq); mt = std::max(mt, d.t.nt);
        mN = std::max(mN, d.t.nz * d.t.nl); mm = std::max(mm, d.t.nmu);
      }
      std::vector<int> ones(running.size(), 1);
      if (cudaMemcpyAsync(b->d_view, hv.data(), sizeof(ColDesc) * hv.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(b->d_status, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { rc = fail(JFNK_E_CUDA, "view rebuild failed"); break; }
      b->d_cols = b->d_view;
      b->ncols = (int)running.size();
      b->max_nz = mz; b->max_nq = mq; b->max_nt = mt; b->max_N = mN; b->max_nmu = mm;
      // a few columns: one thread per frequency leaves most SMs idle, and the
      // warp-per-frequency-pair sweep (same results) finishes each tick sooner
      if (b->formal_kind == FORMAL_SWEEP && b->sweep_variant == 1 &&
          (long)b->ncols * b->max_nq < 256L * b->n_sm && sweep_warp_size(b->max_nz) > 0) {
        b->sweep_variant = 2;
        b->formal_threads = sweep_warp_size(b->max_nz);
      }
      if (b->graph_view) { cudaGraphExecDestroy(b->graph_view); b->graph_view = nullptr; }
      if ((rc = capture_ticks(b, s, profile, &b->graph_view))) break;
      cur = b->graph_view;
      view = running;
      b->compactions++;
    }
  }
  b->d_cols = dfull;
  b->ncols = nfull;
  b->max_nz = fz; b->max_nq = fq; b->max_nt = ft; b->max_N = fN; b->max_nmu = fm;
  b->sweep_variant = fvariant;
  b->formal_threads = fthreads;
  return rc;
}

static void drop_graphs(Batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (b->graph_view) {
    cudaGraphExecDestroy(b->graph_view);
    b->graph_view = nullptr;
  }
}

// Selects a sweep variant, block size and opacity-tangent placement; captured
// graphs with other shapes are dropped.
static int set_sweep_config(Batch* b, int variant, int size, int fuse) {
  if (b->sweep_variant == variant && b->formal_threads == size && b->sweep_fuse == fuse) return JFNK_OK;
  b->sweep_variant = variant;
  b->formal_threads = size;
  b->sweep_fuse = fuse;
  drop_graphs(b);
  return JFNK_OK;
}

int ensure_dJdn(Batch* b, cudaStream_t s) {
  if (b->has_dJdn) return JFNK_OK;
  DeviceArena& ar = b->dJ_arena;
  ar.reset();
  std::vector<size_t> off(b->ncols);
  for (int c = 0; c < b->ncols; ++c) {
    const ColTables& T = b->h_cols[c].t;
    off[c] = ar.take<double>((size_t)T.nq * T.nz * T.nl);
  }
  int rc = ar.allocate();
  if (rc) return rc;
  for (int c = 0; c < b->ncols; ++c) b->h_cols[c].w.dJdn = ar.ptr<double>(off[c]);
  JFNK_CUDA(cudaMemcpyAsync(b->d_cols, b->h_cols.data(), sizeof(ColDesc) * b->ncols, cudaMemcpyHostToDevice, s));
  b->has_dJdn = true;
  drop_graphs(b);   // the tick graph gains the estimate's renewal kernel
  return JFNK_OK;
}

static int prepare_solve(Batch* b, const std::vector<const jfnk_atmos*>& cols,
                         const jfnk_options* o, double* const* n_in, double* const* J_in,
                         jfnk_mem where, cudaStream_t s) {
  if (b->formal_kind == FORMAL_MOVING &&
      (o->rh92_warmup > 0 || o->solver != JFNK_SOLVER_JFNK || o->precond > 1))
    return fail(JFNK_E_INVALID,
                "moving columns: Algorithm 2 without an RH92 start, with the first preconditioner solution or none");
  SolverOpts so;
  options_to_device(o, &so);
  JFNK_CUDA(cudaMemcpyAsync(b->d_opts, &so, sizeof(so), cudaMemcpyHostToDevice, s));
  int rc = batch_set_forced_mode(b, -1, s);
  if (rc) return rc;
  if (o->precond == 2) {
    // the lagged estimate starts at zero in every solve
    if ((rc = ensure_dJdn(b, s))) return rc;
    JFNK_CUDA(cudaMemsetAsync(b->dJ_arena.base, 0, b->dJ_arena.bytes, s));
  }
  const int phase = (o->rh92_warmup > 0 || o->solver == JFNK_SOLVER_RH92) ? PH_RH92 : PH_BASE;
  k_init_state<<<(b->ncols + 127) / 128, 128, 0, s>>>(b->d_state, b->ncols, phase);
  JFNK_CUDA(cudaGetLastError());
  JFNK_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int) * b->ncols, s));
  for (int c = 0; c < b->ncols; ++c) {
    const ColDesc& cd = b->h_cols[c];
    const AtmosData& M = cols[c]->d;
    const size_t N = (size_t)M.nz * M.nl, QZ = (size_t)M.nq * M.nz;
    if (o->init == JFNK_INIT_USER) {
      if (!n_in || !n_in[c]) return fail(JFNK_E_INVALID, "JFNK_INIT_USER needs n_inout");
      if ((rc = copy_in(cd.w.n, n_in[c], N * 8, where, s))) return rc;
    } else {   // LTE, also the conservation rows of the zero-radiation guess
      JFNK_CUDA(cudaMemcpyAsync(cd.w.n, M.tables.nstar, N * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (J_in && J_in[c]) {
      if ((rc = copy_in(cd.w.Jdag, J_in[c], QZ * 8, where, s))) return rc;
    } else {
      JFNK_CUDA(cudaMemcpyAsync(cd.w.Jdag, M.tables.Bn, QZ * 8, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (b->mixed && (rc = launch_j_pairs(b->d_cols, b->ncols, (size_t)b->max_nq * b->max_nz, s, true))) return rc;
  if (o->init == JFNK_INIT_ZERO_RADIATION && (rc = launch_zero_radiation(*b, s))) return rc;
  if (b->formal_kind == FORMAL_SWEEP && o->formal_variant != 0) {
    // a forced sweep variant (results are the same as with the tuned one)
    const int v = o->formal_variant == JFNK_FORMAL_SWEEP_WARP ? 2 : 1;
    const int size = v == 2 ? sweep_warp_size(b->max_nz) : 128;
    if (size == 0) return fail(JFNK_E_INVALID, "JFNK_FORMAL_SWEEP_WARP: the column is too deep for its shared memory");
    const int fuse = o->formal_variant == JFNK_FORMAL_SWEEP_THREAD_FUSED ? 1 : 0;
    if (fuse && b->max_overlap > kQMetaT)
      return fail(JFNK_E_INVALID, "JFNK_FORMAL_SWEEP_THREAD_FUSED: more than 8 transitions overlap at a frequency");
    if ((rc = set_sweep_config(b, v, size, fuse))) return rc;
  } else if (!b->tuned && b->formal_kind != FORMAL_UNFUSED) {
    // tune the formal kernel once per batch, on its own columns: a base
    // evaluation at the initial state, then tangent data along v = n
    if ((rc = batch_set_forced_mode(b, EV_BASE, s))) return rc;
    if ((rc = launch_evaluation(*b, s))) return rc;
    for (int c = 0; c < b->ncols; ++c) {
      const AtmosData& M = cols[c]->d;
      JFNK_CUDA(cudaMemcpyAsync(b->h_cols[c].w.v, b->h_cols[c].w.n, (size_t)M.nz * M.nl * 8,
                                cudaMemcpyDeviceToDevice, s));
    }
    if ((rc = batch_set_forced_mode(b, EV_TANGENT, s))) return rc;
    if ((rc = launch_evaluation(*b, s))) return rc;
    if ((rc = b->formal_kind == FORMAL_SWEEP ? sweep_autotune(b, s) : fused_autotune(b, s))) return rc;
    b->tuned = true;
    b->tuned_variant = b->sweep_variant;
    b->tuned_size = b->formal_threads;
    b->tuned_fuse = b->sweep_fuse;
    drop_graphs(b);   // graphs captured with other launch shapes are stale
    if ((rc = batch_set_forced_mode(b, -1, s))) return rc;
  } else if (b->tuned && b->formal_kind == FORMAL_SWEEP) {
    if ((rc = set_sweep_config(b, b->tuned_variant, b->tuned_size, b->tuned_fuse))) return rc;
  }
  // mark every column as running for the host poll
  std::vector<int> ones(b->ncols, 1);
  JFNK_CUDA(cudaMemcpyAsync(b->d_status, ones.data(), sizeof(int) * b->ncols, cudaMemcpyHostToDevice, s));
  JFNK_CUDA(cudaStreamSynchronize(s));
  return JFNK_OK;
}

static int finish_solve(Batch* b, const std::vector<const jfnk_atmos*>& cols, double* const* n_out,
                        double* const* J_out, jfnk_stats* stats, jfnk_mem where, cudaStream_t s,
                        int* worst) {
  std::vector<SolverState> st(b->ncols);
  JFNK_CUDA(cudaMemcpyAsync(st.data(), b->d_state, sizeof(SolverState) * b->ncols, cudaMemcpyDeviceToHost, s));
  JFNK_CUDA(cudaStreamSynchronize(s));
  int rc;
  if (b->mixed && J_out && (rc = launch_j_pairs(b->d_cols, b->ncols, (size_t)b->max_nq * b->max_nz, s, false)))
    return rc;
  for (int c = 0; c < b->ncols; ++c) {
    const ColDesc& cd = b->h_cols[c];
    const AtmosData& M = cols[c]->d;
    const size_t N = (size_t)M.nz * M.nl, QZ = (size_t)M.nq * M.nz;
    if (n_out && n_out[c] && (rc = copy_out(n_out[c], cd.w.n, N * 8, where, s))) return rc;
    // after the last base evaluation the new J sits in the buffer opposite to J^dagger
    const double* Jfinal = st[c].jsel ? cd.w.Jdag : cd.w.Jnew;   // FP64 again in mixed mode
    if (J_out && J_out[c] && (rc = copy_out(J_out[c], Jfinal, QZ * 8, where, s))) return rc;
  }
  JFNK_CUDA(cudaStreamSynchronize(s));
  *worst = JFNK_OK;
  int active = 0;
  for (int c = 0; c < b->ncols; ++c) active = std::max(active, st[c].ticks);
  active = std::min(active, (int)b->tick_ms.size());
  double kernel_ms = 0.0, tan_ms = 0.0, stage_ms[kStages] = {};
  for (int t = 0; t < active; ++t) kernel_ms += b->tick_ms[t];
  for (int t = 0; t < active && t < (int)b->tick_tan_ms.size(); ++t) tan_ms += b->tick_tan_ms[t];
  for (int t = 0; t < active && (size_t)(t + 1) * kStages <= b->tick_stage_ms.size(); ++t)
    for (int j = 0; j < kStages; ++j) stage_ms[j] += b->tick_stage_ms[(size_t)t * kStages + j];
  for (int c = 0; c < b->ncols; ++c) {
    const SolverState& x = st[c];
    int status = x.status == 1 ? JFNK_E_TIMEOUT : x.status;
    if (stats) {
      jfnk_stats& S = stats[c];
      S.status = status;
      S.newton_iters = x.newton_iter;
      S.rh92_iters = x.rh92_iter;
      S.F_calls = x.F_calls;
      S.jvp_calls = x.jvp_calls;
      S.F_norm = x.Fnorm;
      S.F_norm0 = x.F0norm;
      S.dn_norm = x.err;
      S.ray_points = (double)x.F_calls * cols[c]->d.ray_points;
      S.formal_ms = kernel_ms;
      S.formal_tan_ms = tan_ms;
      for (int j = 0; j < kStages; ++j) S.stage_ms[j] = stage_ms[j];
      S.opacity_depths = b->formal_kind == FORMAL_SWEEP ? b->optan_depths : 0;
      S.formal_occ = b->formal_kind == FORMAL_SWEEP && b->sweep_variant != 2 ? b->sweep_occ : 0;
      S.formal_occ_base = b->formal_kind == FORMAL_SWEEP && b->sweep_variant != 2 ? b->sweep_occ_base : 0;
      S.formal_fuse = b->formal_kind == FORMAL_SWEEP && sweep_fused(*b) ? b->sweep_fuse : 0;
      S.formal_launches = active;
      S.kernel_launches = (int)(b->replays * b->graph_kernels) + 2;   // + state init, mode reset
      S.formal_qb = b->formal_kind == FORMAL_FUSED ? b->formal_qb : 0;
      S.formal_threads = b->formal_threads;
      S.formal_kernel = b->formal_kind == FORMAL_SWEEP
                            ? (b->sweep_variant == 2 ? JFNK_FORMAL_SWEEP_WARP
                               : (sweep_fused(*b) ? JFNK_FORMAL_SWEEP_THREAD_FUSED : JFNK_FORMAL_SWEEP_THREAD))
                            : (b->formal_kind == FORMAL_FUSED ? JFNK_FORMAL_FUSED
                               : (b->formal_kind == FORMAL_MOVING ? JFNK_FORMAL_MOVING : JFNK_FORMAL_PER_RAY));
    }
    if (status != JFNK_OK && *worst == JFNK_OK) *worst = status;
  }
  return JFNK_OK;
}

// Runs ``body`` on the context's stream ordered after ``user``; the user stream
// waits for the result. Host-memory calls are synchronised.
template <typename F>
int on_ctx_stream(jfnk_ctx* ctx, void* user, jfnk_mem where, F body) {
  cudaStream_t us = reinterpret_cast<cudaStream_t>(user);
  JFNK_CUDA(cudaEventRecord(ctx->ev_in, us));
  JFNK_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  int rc = body(ctx->stream);
  JFNK_CUDA(cudaEventRecord(ctx->ev_out, ctx->stream));
  JFNK_CUDA(cudaStreamWaitEvent(us, ctx->ev_out, 0));
  if (rc) return rc;
  if (where == JFNK_MEM_HOST) JFNK_CUDA(cudaStreamSynchronize(ctx->stream));
  return JFNK_OK;
}

}  // namespace jfnk

using namespace jfnk;

extern "C" {

const char* jfnk_last_error(void) { return g_last_error.c_str(); }

void jfnk_default_options(jfnk_options* o) {
  if (!o) return;
  o->ftol = 1e-4;
  o->fdrop = 1e-2;
  o->rtol = 1e-2;
  o->maxiter = 100;
  o->krylov_max = 50;
  o->max_restarts = 20;
  o->precision = JFNK_FP64;
  o->init = JFNK_INIT_LTE;
  o->clamp = 1;
  o->rh92_warmup = 0;
  o->rh92_switch = 1e-2;
  o->max_ticks = 20000;
  o->profile = 0;
  o->formal_variant = 0;
  o->precond = 1;
  o->jvp = JFNK_JVP_TANGENT;
  o->krylov = JFNK_KRYLOV_GMRES;
  o->solver = JFNK_SOLVER_JFNK;
  o->line_search = 0;
}

int jfnk_init(int device, jfnk_ctx** out) {
  if (!out) return fail(JFNK_E_INVALID, "out is NULL");
  *out = nullptr;
  int count = 0;
  JFNK_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(JFNK_E_INVALID, "no such CUDA device");
  JFNK_CUDA(cudaSetDevice(device));
  jfnk_ctx* c = new jfnk_ctx();
  c->device = device;
  cudaDeviceProp p;
  cudaError_t e = cudaGetDeviceProperties(&p, device);
  if (e != cudaSuccess) { delete c; return fail(JFNK_E_CUDA, cudaGetErrorString(e)); }
  c->n_sm = p.multiProcessorCount;
  if (int rc = prepare_kernels()) { delete c; return rc; }
  {
    // the stream-ordered pool keeps freed atmosphere tables for reuse
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  // atmosphere set-up runs at the highest stream priority: its small kernels
  // are scheduled ahead of queued blocks of running solves, so that a request
  // being built does not wait behind a served batch's long launches
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  e = cudaSuccess;
  for (int i = 0; i < jfnk_ctx::kSetupLanes && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithPriority(&c->setup_stream[i], cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->setup_done[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) { delete c; return fail(JFNK_E_CUDA, cudaGetErrorString(e)); }
  *out = c;
  return JFNK_OK;
}

int jfnk_destroy_ctx(jfnk_ctx* c) {
  if (!c) return JFNK_OK;
  cudaSetDevice(c->device);
  for (int i = 0; i < jfnk_ctx::kSetupLanes; ++i) {
    if (c->setup_done[i]) cudaEventSynchronize(c->setup_done[i]);
    if (c->setup_stream[i]) cudaStreamDestroy(c->setup_stream[i]);
    if (c->setup_done[i]) cudaEventDestroy(c->setup_done[i]);
    if (c->stage[i]) cudaFreeHost(c->stage[i]);
  }
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  delete c;
  cudaGetLastError();   // a teardown failure must not surface in a later call
  return JFNK_OK;
}

int jfnk_create_atom(jfnk_ctx* ctx, const jfnk_atom_desc* d, jfnk_atom** out) {
  if (!ctx || !out) return fail(JFNK_E_INVALID, "context and out are required");
  *out = nullptr;
  jfnk_atom* a = new jfnk_atom();
  a->ctx = ctx;
  int rc = build_atom(d, &a->d);
  if (rc) { delete a; return rc; }
  *out = a;
  return JFNK_OK;
}

int jfnk_destroy_atom(jfnk_atom* a) {
  delete a;
  return JFNK_OK;
}

int jfnk_atom_info(const jfnk_atom* a, int* n_levels, int* n_transitions, int* n_nu) {
  if (!a) return fail(JFNK_E_INVALID, "atom is NULL");
  if (n_levels) *n_levels = a->d.nl;
  if (n_transitions) *n_transitions = a->d.nt;
  if (n_nu) *n_nu = a->d.nq;
  return JFNK_OK;
}

int jfnk_atom_frequencies(const jfnk_atom* a, double* nu) {
  if (!a || !nu) return fail(JFNK_E_INVALID, "atom and nu are required");
  std::memcpy(nu, a->d.nu.data(), sizeof(double) * a->d.nq);
  return JFNK_OK;
}

int jfnk_create_atmosphere(jfnk_ctx* ctx, const jfnk_atom* atom, const jfnk_atmos_desc* d,
                           jfnk_atmos** out) {
  if (!ctx || !atom || !out) return fail(JFNK_E_INVALID, "context, atom and out are required");
  if (atom->ctx != ctx) return fail(JFNK_E_INVALID, "atom belongs to another context");
  *out = nullptr;
  // the set-up is enqueued under the context lock on the next set-up lane,
  // whose previous set-up (and so its staging buffer) must be finished; the
  // wait for this one happens outside the lock, so that several callers
  // (the producer threads of a server) overlap their set-ups on the device
  std::unique_lock<std::mutex> lk(ctx->mu);
  JFNK_CUDA(cudaSetDevice(ctx->device));
  const int lane = ctx->next_lane;
  ctx->next_lane = (lane + 1) % jfnk_ctx::kSetupLanes;
  JFNK_CUDA(cudaEventSynchronize(ctx->setup_done[lane]));
  jfnk_atmos* a = new jfnk_atmos();
  a->ctx = ctx;
  a->atom = atom;
  int rc = build_atmosphere(ctx, lane, atom->d, d, &a->d);
  if (rc) {
    cudaStreamSynchronize(ctx->setup_stream[lane]);   // nothing left in flight on the lane
    delete a;
    return rc;
  }
  const cudaEvent_t done = ctx->setup_done[lane];
  lk.unlock();
  JFNK_CUDA(cudaEventSynchronize(done));   // the tables are ready for every stream
  a->work = new SingleWork();
  *out = a;
  return JFNK_OK;
}

int jfnk_destroy_atmosphere(jfnk_atmos* a) {
  if (!a) return JFNK_OK;
  cudaSetDevice(a->ctx->device);
  delete single_work(a);
  delete a;
  cudaGetLastError();   // a teardown failure must not surface in a later call
  return JFNK_OK;
}

int jfnk_atmos_info(const jfnk_atmos* a, int* n_depth, int* n_nu, int* n_levels, int* n_transitions,
                    double* ray_points) {
  if (!a) return fail(JFNK_E_INVALID, "atmosphere is NULL");
  if (n_depth) *n_depth = a->d.nz;
  if (n_nu) *n_nu = a->d.nq;
  if (n_levels) *n_levels = a->d.nl;
  if (n_transitions) *n_transitions = a->d.nt;
  if (ray_points) *ray_points = a->d.ray_points;
  return JFNK_OK;
}

int jfnk_atmos_table(const jfnk_atmos* a, int which, double* out, size_t count) {
  if (!a || !out) return fail(JFNK_E_INVALID, "atmosphere and out are required");
  const AtmosData& M = a->d;
  const ColTables& T = M.tables;
  const double* src = nullptr;
  size_t n = 0;
  switch (which) {
    case 0: src = T.nstar; n = (size_t)M.nz * M.nl; break;
    case 1: src = T.Bn; n = (size_t)M.nq * M.nz; break;
    case 2: src = T.C; n = (size_t)M.nz * M.nl * M.nl; break;
    case 3: src = T.V; n = (size_t)M.nwin * M.nz; break;
    case 4: src = T.G; n = (size_t)M.nwin * M.nz; break;
    case 5: src = T.t_w; n = (size_t)M.nwin; break;
    case 6: src = T.chi_c; n = (size_t)M.nq * M.nz; break;
    case 7: src = T.eta_c; n = (size_t)M.nq * M.nz; break;
    case 8:
      if (!T.Vd) return fail(JFNK_E_INVALID, "table 8 exists for moving columns only");
      src = T.Vd; n = 2 * (size_t)M.nmu * M.nwin * M.nz; break;
    default: return fail(JFNK_E_INVALID, "unknown table");
  }
  if (count < n) return fail(JFNK_E_INVALID, "output buffer too small");
  JFNK_CUDA(cudaSetDevice(a->ctx->device));
  JFNK_CUDA(cudaMemcpy(out, src, n * sizeof(double), cudaMemcpyDeviceToHost));
  return JFNK_OK;
}

int jfnk_residual(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, const double* n,
                  const double* J_dagger, double* F, double* J_new, double* I_emergent,
                  jfnk_mem where, void* stream) {
  int rc = check_common(ctx, a, precision, where);
  if (rc) return rc;
  if (!n || !F) return fail(JFNK_E_INVALID, "n and F are required");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Batch* b;
  if ((rc = get_single(a, precision == JFNK_MIXED, &b))) return rc;
  return on_ctx_stream(ctx, stream, where, [&](cudaStream_t s) {
    int r = explicit_eval(ctx, a, b, EV_BASE, n, J_dagger, where, s);
    if (r) return r;
    const ColDesc& c = b->h_cols[0];
    const AtmosData& M = a->d;
    if ((r = copy_out(F, c.w.F, (size_t)M.nz * M.nl * 8, where, s))) return r;
    if (J_new && b->mixed && (r = launch_j_pairs(b->d_cols, 1, (size_t)M.nq * M.nz, s, false))) return r;
    if (J_new && (r = copy_out(J_new, c.w.Jnew, (size_t)M.nq * M.nz * 8, where, s))) return r;
    if (I_emergent && (r = copy_out(I_emergent, c.w.Iem, (size_t)M.nq * M.nmu * 8, where, s))) return r;
    return 0;
  });
}

int jfnk_jvp(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, const double* n,
             const double* J_dagger, const double* v, double* Jv, jfnk_mem where, void* stream) {
  int rc = check_common(ctx, a, precision, where);
  if (rc) return rc;
  if (!n || !v || !Jv) return fail(JFNK_E_INVALID, "n, v and Jv are required");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Batch* b;
  if ((rc = get_single(a, precision == JFNK_MIXED, &b))) return rc;
  return on_ctx_stream(ctx, stream, where, [&](cudaStream_t s) {
    int r = explicit_eval(ctx, a, b, EV_BASE, n, J_dagger, where, s);   // rates and rows at n
    if (r) return r;
    const ColDesc& c = b->h_cols[0];
    const AtmosData& M = a->d;
    const size_t N = (size_t)M.nz * M.nl;
    if ((r = copy_in(c.w.v, v, N * 8, where, s))) return r;
    if ((r = batch_set_forced_mode(b, EV_TANGENT, s))) return r;
    if ((r = launch_evaluation(*b, s))) return r;
    return copy_out(Jv, c.w.dF, N * 8, where, s);
  });
}

int jfnk_block_jacobi(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, const double* n,
                      const double* J_dagger, double* P, jfnk_mem where, void* stream) {
  int rc = check_common(ctx, a, precision, where);
  if (rc) return rc;
  if (!n || !P) return fail(JFNK_E_INVALID, "n and P are required");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Batch* b;
  if ((rc = get_single(a, precision == JFNK_MIXED, &b))) return rc;
  return on_ctx_stream(ctx, stream, where, [&](cudaStream_t s) {
    int r = explicit_eval(ctx, a, b, EV_BASE, n, J_dagger, where, s);
    if (r) return r;
    const AtmosData& M = a->d;
    return copy_out(P, b->h_cols[0].w.P, (size_t)M.nz * M.nl * M.nl * 8, where, s);
  });
}

int jfnk_block_jacobi_variant(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, int variant,
                              const double* n, const double* J_dagger, const double* dJdn_prev,
                              double* P, double* dJdn_out, jfnk_mem where, void* stream) {
  int rc = check_common(ctx, a, precision, where);
  if (rc) return rc;
  if (!n || !P) return fail(JFNK_E_INVALID, "n and P are required");
  if (variant < 1 || variant > 3) return fail(JFNK_E_INVALID, "variant must be 1, 2 or 3");
  if (a->d.moving && variant != 1) return fail(JFNK_E_INVALID, "moving columns: the first solution only");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Batch* b;
  if ((rc = get_single(a, precision == JFNK_MIXED, &b))) return rc;
  return on_ctx_stream(ctx, stream, where, [&](cudaStream_t s) {
    const AtmosData& M = a->d;
    const size_t nD = (size_t)M.nq * M.nz * M.nl;
    int r;
    if (variant == 2) {
      if ((r = ensure_dJdn(b, s))) return r;
      if (dJdn_prev) {
        if ((r = copy_in(b->h_cols[0].w.dJdn, dJdn_prev, nD * 8, where, s))) return r;
      } else {
        JFNK_CUDA(cudaMemsetAsync(b->h_cols[0].w.dJdn, 0, nD * 8, s));
      }
    }
    if ((r = explicit_eval(ctx, a, b, EV_BASE, n, J_dagger, where, s, variant))) return r;
    if ((r = copy_out(P, b->h_cols[0].w.P, (size_t)M.nz * M.nl * M.nl * 8, where, s))) return r;
    if (variant == 2 && dJdn_out && (r = copy_out(dJdn_out, b->h_cols[0].w.dJdn, nD * 8, where, s))) return r;
    return 0;
  });
}

int jfnk_rh92_update(jfnk_ctx* ctx, const jfnk_atmos* a, int precision, const double* n,
                     const double* J_dagger, double* n_out, double* J_new, jfnk_mem where,
                     void* stream) {
  int rc = check_common(ctx, a, precision, where);
  if (rc) return rc;
  if (!n || !n_out) return fail(JFNK_E_INVALID, "n and n_out are required");
  if (a->d.moving) return fail(JFNK_E_INVALID, "RH92 is not available for moving columns");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Batch* b;
  if ((rc = get_single(a, precision == JFNK_MIXED, &b))) return rc;
  return on_ctx_stream(ctx, stream, where, [&](cudaStream_t s) {
    int r = explicit_eval(ctx, a, b, EV_RH92, n, J_dagger, where, s);
    if (r) return r;
    if ((r = launch_rh92_update(*b, s))) return r;
    const ColDesc& c = b->h_cols[0];
    const AtmosData& M = a->d;
    if ((r = copy_out(n_out, c.w.n, (size_t)M.nz * M.nl * 8, where, s))) return r;
    if (J_new && b->mixed && (r = launch_j_pairs(b->d_cols, 1, (size_t)M.nq * M.nz, s, false))) return r;
    if (J_new && (r = copy_out(J_new, c.w.Jnew, (size_t)M.nq * M.nz * 8, where, s))) return r;
    return 0;
  });
}

int jfnk_solve(jfnk_ctx* ctx, const jfnk_atmos* a, const jfnk_options* o, double* n_inout,
               double* J_inout, jfnk_stats* stats, jfnk_mem where, void* stream) {
  int rc = check_common(ctx, a, o ? o->precision : 0, where);
  if (rc) return rc;
  if ((rc = validate_options(o))) return rc;
  if (!n_inout) return fail(JFNK_E_INVALID, "n_inout is required");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Batch* b;
  if ((rc = get_single(a, o->precision == JFNK_MIXED, &b))) return rc;
  std::vector<const jfnk_atmos*> cols{a};
  int worst = JFNK_OK;
  rc = on_ctx_stream(ctx, stream, where, [&](cudaStream_t s) {
    int r = prepare_solve(b, cols, o, &n_inout, &J_inout, where, s);
    if (r) return r;
    if ((r = run_to_completion(b, o, s))) return r;
    return finish_solve(b, cols, &n_inout, &J_inout, stats, where, s, &worst);
  });
  if (rc) return rc;
  if (worst != JFNK_OK) return fail(worst, "column did not converge (see stats.status)");
  return JFNK_OK;
}

}  // extern "C"

struct jfnk_batch {
  jfnk_ctx* ctx;
  std::vector<const jfnk_atmos*> cols;
  jfnk::Batch b;
  int precision;
};

extern "C" {

int jfnk_batch_create(jfnk_ctx* ctx, int n_cols, const jfnk_atmos* const* cols_in, int precision,
                      int krylov_max, jfnk_batch** out) {
  if (!ctx || !out) return fail(JFNK_E_INVALID, "context and out are required");
  *out = nullptr;
  if (n_cols < 1 || !cols_in) return fail(JFNK_E_INVALID, "a batch needs at least one column");
  if (krylov_max < 1 || krylov_max > kMaxKrylov) return fail(JFNK_E_INVALID, "krylov_max must be in [1, 64]");
  std::unique_ptr<jfnk_batch> h(new jfnk_batch());
  h->ctx = ctx;
  h->precision = precision;
  h->cols.assign(cols_in, cols_in + n_cols);
  std::vector<const AtmosData*> data;
  int rc;
  for (auto* a : h->cols) {
    if ((rc = check_common(ctx, a, precision, JFNK_MEM_HOST))) return rc;
    data.push_back(&a->d);
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  if ((rc = batch_create(&h->b, data, precision == JFNK_MIXED, krylov_max))) return rc;
  *out = h.release();
  return JFNK_OK;
}

int jfnk_batch_destroy(jfnk_batch* b) {
  if (!b) return JFNK_OK;
  cudaSetDevice(b->ctx->device);
  delete b;
  cudaGetLastError();   // a teardown failure must not surface in a later call
  return JFNK_OK;
}

int jfnk_batch_run(jfnk_batch* h, const jfnk_options* o, double* const* n_inout,
                   double* const* J_inout, jfnk_stats* stats, jfnk_mem where, void* stream) {
  if (!h) return fail(JFNK_E_INVALID, "batch is NULL");
  int rc = validate_options(o);
  if (rc) return rc;
  if (o->precision != h->precision) return fail(JFNK_E_INVALID, "options precision differs from the batch's");
  if (o->krylov_max > h->b.kmax) return fail(JFNK_E_INVALID, "krylov_max exceeds the batch's");
  if (!n_inout) return fail(JFNK_E_INVALID, "n_inout is required");
  if (where != JFNK_MEM_HOST && where != JFNK_MEM_DEVICE) return fail(JFNK_E_INVALID, "unknown memory kind");
  jfnk_ctx* ctx = h->ctx;
  JFNK_CUDA(cudaSetDevice(ctx->device));
  std::lock_guard<std::mutex> lk(ctx->mu);
  int worst = JFNK_OK;
  Batch* b = &h->b;
  rc = on_ctx_stream(ctx, stream, where, [&](cudaStream_t s) {
    int r = prepare_solve(b, h->cols, o, n_inout, J_inout, where, s);
    if (r) return r;
    if ((r = run_to_completion(b, o, s))) return r;
    return finish_solve(b, h->cols, n_inout, J_inout, stats, where, s, &worst);
  });
  if (rc) return rc;
  if (worst != JFNK_OK) return fail(worst, "some columns did not converge (see stats[].status)");
  return JFNK_OK;
}

int jfnk_batch_solve(jfnk_ctx* ctx, int n_cols, const jfnk_atmos* const* cols_in,
                     const jfnk_options* o, double* const* n_inout, double* const* J_inout,
                     jfnk_stats* stats, jfnk_mem where, void* stream) {
  if (!ctx) return fail(JFNK_E_INVALID, "context is NULL");
  if (n_cols < 0 || (n_cols > 0 && (!cols_in || !n_inout))) return fail(JFNK_E_INVALID, "bad batch arguments");
  if (n_cols == 0) return JFNK_OK;
  int rc = validate_options(o);
  if (rc) return rc;
  jfnk_batch* h = nullptr;
  if ((rc = jfnk_batch_create(ctx, n_cols, cols_in, o->precision, std::max(o->krylov_max, 1), &h))) return rc;
  rc = jfnk_batch_run(h, o, n_inout, J_inout, stats, where, stream);
  jfnk_batch_destroy(h);
  return rc;
}

}  // extern "C"
