// Serving runtime: continuous batching of independent column solves.
//
// The server is a batch of S slots whose tick graph (kTicksPerGraph F-class
// evaluations + Krylov steps of every slot) is captured once, for the slot
// shape given at creation. The kernels read each slot's descriptor (and its
// solver options) from device memory at run time, so between two graph
// launches the host can retire a finished column and bind a new one to its
// slot by rewriting the slot's descriptor, options and solver state: nothing
// is recaptured. An empty slot is a column in the done state, which every
// kernel skips.
//
// Work buffers come from one device pool carved by a first-fit allocator with
// coalescing (host-side bookkeeping): a queued column is admitted, in arrival
// order, when a slot is free and its own buffers (column_bytes) fit, so that
// small and large columns share the memory as it frees up.
#include <chrono>
#include <deque>
#include <map>
#include <mutex>

#include "internal.cuh"

namespace jfnk {

// First-fit allocator over [0, bytes) with coalescing of freed neighbours.
class PoolAllocator {
 public:
  void init(size_t bytes) {
    free_.clear();
    if (bytes) free_[0] = bytes;
  }
  bool alloc(size_t len, size_t* off) {
    len = round(len);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < len) continue;
      *off = it->first;
      const size_t rest = it->second - len, next = it->first + len;
      free_.erase(it);
      if (rest) free_[next] = rest;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t len) {
    len = round(len);
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  static size_t round(size_t n) { return (n + 255) / 256 * 256; }
  std::map<size_t, size_t> free_;   // offset -> length
};

struct ServerReq {
  const jfnk_atmos* a = nullptr;
  long long id = 0;
  double* n_out = nullptr;
  SolverOpts o{};
  int rh92 = 0;                   // hybrid start: begin with RH92 iterations
  size_t off = 0, bytes = 0;
  double t_submit = 0, t_admit = 0;
};

}  // namespace jfnk

using namespace jfnk;

struct jfnk_server {
  jfnk_ctx* ctx = nullptr;
  jfnk_server_desc desc{};
  int mixed = 0, kind = 0, kmax = 0;
  Batch b;                        // slot descriptors, states, statuses and options
  SolverOpts* d_sopts = nullptr;  // [S] options of the column in each slot
  DeviceArena pool;               // work buffers of the columns in flight
  PoolAllocator alloc;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::chrono::steady_clock::time_point t0;
  std::mutex qmu;                 // queue (submit may run on another thread)
  std::deque<ServerReq> queue;
  std::mutex dmu;                 // finished results
  std::vector<jfnk_result> done;
  std::vector<ServerReq> slot;
  std::vector<char> busy;
  int* h_status = nullptr;        // pinned mirror of the slot statuses
  // pinned staging per slot for admissions and retirements: a step enqueues
  // all its copies and synchronises once (a slot's staging is not rewritten
  // before the step that used it has drained)
  ColDesc* hp_cols = nullptr;
  SolverState* hp_state = nullptr;
  SolverOpts* hp_opts = nullptr;

  double clock() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

int check_shape(const jfnk_server* sv, const jfnk_atmos* a) {
  const AtmosData& M = a->d;
  const jfnk_server_desc& d = sv->desc;
  if (M.nz > d.max_depth || M.nq > d.max_freq || M.nl > d.max_levels || M.nt > d.max_trans || M.nmu > d.max_mu)
    return fail(JFNK_E_INVALID, "column exceeds the server's slot shape");
  return JFNK_OK;
}

// Binds request r to slot i: descriptor, options, solver state, LTE
// populations and J^dagger = B_nu(T).
int admit(jfnk_server* sv, int i, ServerReq& r) {
  Batch& b = sv->b;
  const AtmosData& M = r.a->d;
  ColDesc& d = b.h_cols[i];
  column_bind(sv->pool.base + r.off, M, sv->kind, sv->mixed, sv->kmax, b.d_state + i, &d);
  d.opts = sv->d_sopts + i;
  SolverState& st = sv->hp_state[i];
  st = SolverState{};
  st.phase = r.rh92 ? PH_RH92 : PH_BASE;
  st.status = 1;
  sv->hp_cols[i] = d;
  sv->hp_opts[i] = r.o;
  const size_t N = (size_t)M.nz * M.nl, QZ = (size_t)M.nq * M.nz;
  JFNK_CUDA(cudaMemcpyAsync(b.d_cols + i, sv->hp_cols + i, sizeof(ColDesc), cudaMemcpyHostToDevice, sv->stream));
  JFNK_CUDA(cudaMemcpyAsync(b.d_state + i, sv->hp_state + i, sizeof(SolverState), cudaMemcpyHostToDevice,
                            sv->stream));
  JFNK_CUDA(cudaMemcpyAsync(sv->d_sopts + i, sv->hp_opts + i, sizeof(SolverOpts), cudaMemcpyHostToDevice,
                            sv->stream));
  JFNK_CUDA(cudaMemcpyAsync(d.w.n, M.tables.nstar, N * 8, cudaMemcpyDeviceToDevice, sv->stream));
  JFNK_CUDA(cudaMemcpyAsync(d.w.Jdag, M.tables.Bn, QZ * 8, cudaMemcpyDeviceToDevice, sv->stream));
  if (sv->mixed) {
    int rc = launch_j_pairs(b.d_cols + i, 1, QZ, sv->stream, true);
    if (rc) return rc;
  }
  sv->h_status[i] = 1;
  JFNK_CUDA(cudaMemcpyAsync(b.d_status + i, sv->h_status + i, sizeof(int), cudaMemcpyHostToDevice, sv->stream));
  r.t_admit = sv->clock();
  sv->slot[i] = r;
  sv->busy[i] = 1;
  return JFNK_OK;
}

// Enqueues the copies out of a finished slot (state and populations).
int retire_copy(jfnk_server* sv, int i) {
  Batch& b = sv->b;
  ServerReq& r = sv->slot[i];
  const AtmosData& M = r.a->d;
  JFNK_CUDA(cudaMemcpyAsync(sv->hp_state + i, b.d_state + i, sizeof(SolverState), cudaMemcpyDeviceToHost,
                            sv->stream));
  if (r.n_out)
    JFNK_CUDA(cudaMemcpyAsync(r.n_out, b.h_cols[i].w.n, (size_t)M.nz * M.nl * 8, cudaMemcpyDeviceToHost,
                              sv->stream));
  return JFNK_OK;
}

// After the step's copies have drained: the slot's result, its pool block freed.
int retire(jfnk_server* sv, int i) {
  Batch& b = sv->b;
  ServerReq& r = sv->slot[i];
  const AtmosData& M = r.a->d;
  const SolverState& x = sv->hp_state[i];
  jfnk_result res{};
  res.id = r.id;
  res.status = x.status == 1 ? JFNK_E_TIMEOUT : x.status;
  jfnk_stats& S = res.stats;
  S.status = res.status;
  S.newton_iters = x.newton_iter;
  S.rh92_iters = x.rh92_iter;
  S.F_calls = x.F_calls;
  S.jvp_calls = x.jvp_calls;
  S.F_norm = x.Fnorm;
  S.F_norm0 = x.F0norm;
  S.dn_norm = x.err;
  S.ray_points = (double)x.F_calls * M.ray_points;
  S.formal_threads = b.formal_threads;
  S.formal_kernel = sv->kind == FORMAL_SWEEP
                        ? (b.sweep_variant == 2 ? JFNK_FORMAL_SWEEP_WARP : JFNK_FORMAL_SWEEP_THREAD)
                        : (sv->kind == FORMAL_FUSED ? JFNK_FORMAL_FUSED : JFNK_FORMAL_PER_RAY);
  res.t_submit = r.t_submit;
  res.t_admit = r.t_admit;
  res.t_done = sv->clock();
  sv->alloc.release(r.off, r.bytes);
  sv->busy[i] = 0;
  {
    std::lock_guard<std::mutex> lk(sv->dmu);
    sv->done.push_back(res);
  }
  return JFNK_OK;
}

}  // namespace

extern "C" {

int jfnk_server_create(jfnk_ctx* ctx, const jfnk_server_desc* d, jfnk_server** out) {
  if (!ctx || !d || !out) return fail(JFNK_E_INVALID, "ctx, desc and out are required");
  *out = nullptr;
  int rc = validate_options(&d->opts);
  if (rc) return rc;
  if (d->opts.init != JFNK_INIT_LTE) return fail(JFNK_E_INVALID, "server requests start from LTE");
  if (d->opts.formal_variant != 0) return fail(JFNK_E_INVALID, "server chooses its formal kernel itself");
  if (d->opts.precond == 2)
    return fail(JFNK_E_INVALID, "the server does not keep the lagged estimate of preconditioner variant 2");
  if (d->max_slots < 1 || d->max_depth < 2 || d->max_depth > JFNK_MAX_DEPTH || d->max_freq < 1 ||
      d->max_levels < 2 || d->max_levels > JFNK_MAX_LEVELS || d->max_trans < 1 || d->max_trans > kMaxT ||
      d->max_mu < 1 || d->max_mu > JFNK_MAX_MU)
    return fail(JFNK_E_INVALID, "invalid server slot shape");
  JFNK_CUDA(cudaSetDevice(ctx->device));
  jfnk_server* sv = new jfnk_server();
  sv->ctx = ctx;
  sv->desc = *d;
  sv->mixed = d->opts.precision == JFNK_MIXED;
  sv->kmax = d->opts.krylov_max;
  sv->t0 = std::chrono::steady_clock::now();
  const int S = d->max_slots;
  Batch& b = sv->b;
  b.ncols = S;
  b.mixed = sv->mixed;
  b.kmax = sv->kmax;
  b.max_nz = d->max_depth;
  b.max_nq = d->max_freq;
  b.max_nt = d->max_trans;
  b.max_N = d->max_depth * d->max_levels;
  b.max_nmu = d->max_mu;
  b.max_nl = d->max_levels;
  b.max_overlap = d->max_trans;
  b.n_sm = ctx->n_sm;
  b.formal_qb = sv->mixed ? 0 : fused_default_qb(d->max_depth, d->max_mu, false);
  b.formal_kind = sv->mixed ? FORMAL_SWEEP : (b.formal_qb > 0 ? FORMAL_FUSED : FORMAL_UNFUSED);
  sv->kind = b.formal_kind;
  if (sv->kind == FORMAL_SWEEP) {
    // few frequencies in flight: the warp-per-frequency-pair sweep (same results)
    const int ws = sweep_warp_size(d->max_depth);
    if ((long)S * d->max_freq < 256L * ctx->n_sm && ws > 0) {
      b.sweep_variant = 2;
      b.formal_threads = ws;
    }
  }
  auto bail = [&](int code) {
    jfnk_server_destroy(sv);
    return code;
  };
  DeviceArena& ar = b.arena;
  const size_t o_cols = ar.take<ColDesc>(S), o_state = ar.take<SolverState>(S), o_status = ar.take<int>(S),
               o_opts = ar.take<SolverOpts>(1), o_view = ar.take<ColDesc>(S), o_sopts = ar.take<SolverOpts>(S);
  if ((rc = ar.allocate())) return bail(rc);
  b.d_cols = ar.ptr<ColDesc>(o_cols);
  b.d_state = ar.ptr<SolverState>(o_state);
  b.d_status = ar.ptr<int>(o_status);
  b.d_opts = ar.ptr<SolverOpts>(o_opts);
  b.d_view = ar.ptr<ColDesc>(o_view);
  sv->d_sopts = ar.ptr<SolverOpts>(o_sopts);
  b.h_cols.assign(S, ColDesc{});
  std::vector<SolverState> st(S);
  for (int i = 0; i < S; ++i) {
    b.h_cols[i].forced_mode = -1;
    b.h_cols[i].mixed = sv->mixed;
    b.h_cols[i].w.st = b.d_state + i;
    st[i] = SolverState{};
    st[i].phase = PH_DONE;
  }
  SolverOpts so;
  options_to_device(&d->opts, &so);
  if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&sv->h_status, sizeof(int) * S) != cudaSuccess ||
      cudaMallocHost(&sv->hp_cols, sizeof(ColDesc) * S) != cudaSuccess ||
      cudaMallocHost(&sv->hp_state, sizeof(SolverState) * S) != cudaSuccess ||
      cudaMallocHost(&sv->hp_opts, sizeof(SolverOpts) * S) != cudaSuccess)
    return bail(fail(JFNK_E_CUDA, "server stream or pinned status buffer"));
  for (int i = 0; i < S; ++i) sv->h_status[i] = 0;
  if (cudaMemcpy(b.d_cols, b.h_cols.data(), sizeof(ColDesc) * S, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b.d_state, st.data(), sizeof(SolverState) * S, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b.d_status, sv->h_status, sizeof(int) * S, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b.d_opts, &so, sizeof(so), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(JFNK_E_CUDA, "server descriptors"));
  if ((rc = sv->kind == FORMAL_SWEEP ? sweep_prepare(&b) : fused_prepare(&b))) return bail(rc);
  // the pool: half the free memory unless given, at most S columns of the slot shape
  size_t free_b = 0, total_b = 0;
  JFNK_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t pool_b = d->mem_bytes ? d->mem_bytes : free_b / 2;
  AtmosData shape;
  shape.nz = d->max_depth;
  shape.nq = d->max_freq;
  shape.nl = d->max_levels;
  shape.nt = d->max_trans;
  shape.nmu = d->max_mu;
  const size_t one = column_bytes(shape, sv->kind, sv->mixed, sv->kmax, nullptr);
  pool_b = std::min(pool_b, one * (size_t)S);
  if (pool_b > free_b) return bail(fail(JFNK_E_NOMEM, "server pool larger than the free device memory"));
  sv->pool.cursor = pool_b;
  if ((rc = sv->pool.allocate())) return bail(rc);
  sv->alloc.init(pool_b);
  sv->slot.assign(S, ServerReq{});
  sv->busy.assign(S, 0);
  if ((rc = capture_ticks(&b, sv->stream, false, &sv->graph))) return bail(rc);
  *out = sv;
  return JFNK_OK;
}

int jfnk_server_bytes(jfnk_server* sv, const jfnk_atmos* a, size_t* bytes) {
  if (!sv || !a || !bytes) return fail(JFNK_E_INVALID, "server, atmosphere and bytes are required");
  *bytes = column_bytes(a->d, sv->kind, sv->mixed, sv->kmax, nullptr);
  return JFNK_OK;
}

int jfnk_server_submit(jfnk_server* sv, const jfnk_atmos* a, long long id, double* n_out,
                       const jfnk_options* opts) {
  if (!sv || !a) return fail(JFNK_E_INVALID, "server and atmosphere are required");
  if (a->ctx != sv->ctx) return fail(JFNK_E_INVALID, "atmosphere belongs to another context");
  int rc = check_shape(sv, a);
  if (rc) return rc;
  if (a->d.moving) return fail(JFNK_E_INVALID, "the server solves static columns only");
  const jfnk_options* o = opts ? opts : &sv->desc.opts;
  if ((rc = validate_options(o))) return rc;
  if (o->precision != sv->desc.opts.precision || o->krylov_max > sv->kmax || o->init != JFNK_INIT_LTE ||
      o->formal_variant != 0 || o->precond == 2)
    return fail(JFNK_E_INVALID,
                "request options: precision, krylov_max, init, formal_variant or precond do not fit the server");
  ServerReq r;
  r.a = a;
  r.id = id;
  r.n_out = n_out;
  options_to_device(o, &r.o);
  r.rh92 = o->rh92_warmup > 0 || o->solver == JFNK_SOLVER_RH92;
  r.bytes = column_bytes(a->d, sv->kind, sv->mixed, sv->kmax, nullptr);
  if (r.bytes > sv->pool.bytes) return fail(JFNK_E_INVALID, "column larger than the server's memory pool");
  r.t_submit = sv->clock();
  std::lock_guard<std::mutex> lk(sv->qmu);
  sv->queue.push_back(r);
  return JFNK_OK;
}

int jfnk_server_step(jfnk_server* sv, int* n_active, int* n_queued) {
  if (!sv) return fail(JFNK_E_INVALID, "server is NULL");
  JFNK_CUDA(cudaSetDevice(sv->ctx->device));
  const int S = sv->b.ncols;
  int rc;
  // admission, in arrival order: a free slot and room in the pool
  for (int i = 0; i < S; ++i) {
    if (sv->busy[i]) continue;
    ServerReq r;
    {
      std::lock_guard<std::mutex> lk(sv->qmu);
      if (sv->queue.empty()) break;
      r = sv->queue.front();
      if (!sv->alloc.alloc(r.bytes, &r.off)) break;   // wait for memory to free up
      sv->queue.pop_front();
    }
    if ((rc = admit(sv, i, r))) return rc;
  }
  int active = 0;
  for (int i = 0; i < S; ++i) active += sv->busy[i];
  if (active) {
    if (cudaGraphLaunch(sv->graph, sv->stream) != cudaSuccess) return fail(JFNK_E_CUDA, "cudaGraphLaunch failed");
    JFNK_CUDA(cudaMemcpyAsync(sv->h_status, sv->b.d_status, sizeof(int) * S, cudaMemcpyDeviceToHost, sv->stream));
    JFNK_CUDA(cudaStreamSynchronize(sv->stream));
    // every finished slot's copies first, one synchronisation, then the results
    bool any = false;
    for (int i = 0; i < S; ++i)
      if (sv->busy[i] && sv->h_status[i] != 1) {
        if ((rc = retire_copy(sv, i))) return rc;
        any = true;
      }
    if (any) JFNK_CUDA(cudaStreamSynchronize(sv->stream));
    for (int i = 0; i < S; ++i)
      if (sv->busy[i] && sv->h_status[i] != 1 && (rc = retire(sv, i))) return rc;
  }
  if (n_active) {
    int a = 0;
    for (int i = 0; i < S; ++i) a += sv->busy[i];
    *n_active = a;
  }
  if (n_queued) {
    std::lock_guard<std::mutex> lk(sv->qmu);
    *n_queued = (int)sv->queue.size();
  }
  return JFNK_OK;
}

int jfnk_server_poll(jfnk_server* sv, jfnk_result* out, int max, int* n) {
  if (!sv || !n || (max > 0 && !out)) return fail(JFNK_E_INVALID, "server, out and n are required");
  std::lock_guard<std::mutex> lk(sv->dmu);
  const int k = std::max(0, std::min(max, (int)sv->done.size()));
  for (int i = 0; i < k; ++i) out[i] = sv->done[i];
  sv->done.erase(sv->done.begin(), sv->done.begin() + k);
  *n = k;
  return JFNK_OK;
}

double jfnk_server_clock(jfnk_server* sv) { return sv ? sv->clock() : 0.0; }

int jfnk_server_destroy(jfnk_server* sv) {
  if (!sv) return JFNK_OK;
  cudaSetDevice(sv->ctx->device);
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  if (sv->graph) cudaGraphExecDestroy(sv->graph);
  if (sv->h_status) cudaFreeHost(sv->h_status);
  if (sv->hp_cols) cudaFreeHost(sv->hp_cols);
  if (sv->hp_state) cudaFreeHost(sv->hp_state);
  if (sv->hp_opts) cudaFreeHost(sv->hp_opts);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  delete sv;
  cudaGetLastError();   // a teardown failure must not surface in a later call
  return JFNK_OK;
}

}  // extern "C"
