// jfnk_residual_static: the residual evaluation of jfnk_residual (FP64,
// device memory) for callers that cannot allocate device memory.
//
// Who needs it: code that runs under a device-memory budget owned by another
// allocator (for instance a framework's caching allocator that has reserved
// the pool), and latency-critical loops that must never pay for cudaMalloc,
// which may synchronise the device and can fail under memory pressure in the
// middle of a run. jfnk_residual allocates its work buffers on first use per
// column; this entry point instead takes them from one file-scope device
// array that every GPU loading the library holds until the process exits.
//
// The array is shared by every call on a device and keeps the previous
// call's contents. No buffer of the evaluation is read before it is written,
// so nothing needs clearing between calls; calls whose work overlaps on the
// GPU (different streams, or threads without ordering) race on the array and
// must be serialised by the caller.
#include <mutex>

#include "internal.cuh"

namespace jfnk {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // JFNK_STATIC_SCRATCH_BYTES

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device addresses of g_static_scratch, one per device, looked up once with
// that device current (the host-side symbol is only a stand-in).
static char* g_static_addr[256] = {nullptr};
static std::mutex g_static_mu;

static int static_scratch(int device, cudaStream_t s, char** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (device < 0 || device >= 256) return fail(JFNK_E_INVALID, "device index out of range");
  if (!g_static_addr[device]) {
    // the one-time lookup may load the module on this device: refuse it in
    // the middle of a stream capture rather than disturb the capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess)
      return fail(JFNK_E_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(JFNK_E_INVALID,
                  "the first jfnk_residual_static call on a device must not be made while its stream is "
                  "being captured (it looks up the static scratch's device address once)");
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail(JFNK_E_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_static_addr[device] = static_cast<char*>(p);
  }
  *out = g_static_addr[device];
  return JFNK_OK;
}

// 256-byte aligned bump layout inside the static array (offsets only).
struct StaticLayout {
  size_t cursor = 0;
  template <typename T>
  size_t take(size_t count) {
    size_t off = cursor;
    cursor += ((count * sizeof(T) + 255) / 256) * 256;
    if (cursor == off) cursor += 256;
    return off;
  }
};

// The column descriptor travels by value as a kernel parameter and is stored
// into the static array on the device (no host staging buffer).
__global__ void k_store_static_desc(ColDesc* dst, ColDesc src) { *dst = src; }

}  // namespace jfnk

using namespace jfnk;

extern "C" int jfnk_residual_static(jfnk_ctx* ctx, const jfnk_atmos* a, const double* n,
                                    const double* J_dagger, double* F, double* J_new,
                                    void* stream) {
  if (!ctx || !a || !n || !F) return fail(JFNK_E_INVALID, "ctx, atmosphere, n and F are required");
  if (a->ctx != ctx) return fail(JFNK_E_INVALID, "atmosphere belongs to another context");
  if (a->d.moving) return fail(JFNK_E_INVALID, "moving columns need jfnk_residual (per-ray buffers)");
  JFNK_CUDA(cudaSetDevice(ctx->device));
  const AtmosData& M = a->d;
  const size_t nz = M.nz, nq = M.nq, nl = M.nl, nt = M.nt, nmu = M.nmu;
  const size_t N = nz * nl, QZ = nq * nz;
  // the fused formal kernel (the one jfnk_residual runs) needs no per-ray
  // buffers; the per-ray path only when a frequency's rays exceed its shared memory
  const int qb = fused_default_qb((int)nz, (int)nmu, false);
  const bool fused = qb > 0;
  const size_t per_ray = fused ? 0 : 2 * nmu * QZ;
  StaticLayout L;
  const size_t o_desc = L.take<ColDesc>(1);
  const size_t o_n = L.take<double>(N), o_Jdag = L.take<double>(QZ), o_Jnew = L.take<double>(QZ);
  const size_t o_istar = L.take<int>(nz);
  const size_t o_chi = L.take<double>(QZ), o_S = L.take<double>(QZ), o_dSk = L.take<double>(fused ? 0 : QZ);
  const size_t o_H = L.take<double>(per_ray), o_LX = L.take<double>(per_ray), o_LE = L.take<double>(per_ray),
               o_HI = L.take<double>(per_ray);
  const size_t o_J = L.take<double>(fused ? 0 : QZ), o_Lchi = L.take<double>(QZ), o_Leta = L.take<double>(QZ);
  const size_t o_Rup = L.take<double>(nt * nz), o_Rdn = L.take<double>(nt * nz);
  const size_t o_Apart = L.take<double>(nt * nz * nl);
  const size_t o_F = L.take<double>(N), o_P = L.take<double>(nz * nl * nl);
  const size_t o_Iem = L.take<double>(nq * nmu);
  if (L.cursor > kStaticScratchBytes)
    return fail(JFNK_E_INVALID,
                "column too large for the static scratch of jfnk_residual_static (needs " +
                    std::to_string(L.cursor) + " bytes, limit " +
                    std::to_string(kStaticScratchBytes) + "); use jfnk_residual");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* base = nullptr;
  int rc = static_scratch(ctx->device, s, &base);
  if (rc) return rc;

  ColDesc cd{};
  cd.t = M.tables;
  cd.forced_mode = EV_BASE;
  cd.mixed = 0;
  ColWork& w = cd.w;
  w.n = reinterpret_cast<double*>(base + o_n);
  w.Jdag = reinterpret_cast<double*>(base + o_Jdag);
  w.Jnew = reinterpret_cast<double*>(base + o_Jnew);
  w.istar = reinterpret_cast<int*>(base + o_istar);
  w.chi = base + o_chi;
  w.S = reinterpret_cast<double*>(base + o_S);
  if (!fused) {
    w.dSk = base + o_dSk;
    w.H = base + o_H;
    w.HI = base + o_HI;
    w.LX = base + o_LX;
    w.LE = base + o_LE;
    w.J = reinterpret_cast<double*>(base + o_J);
  }
  w.Lchi = reinterpret_cast<double*>(base + o_Lchi);
  w.Leta = reinterpret_cast<double*>(base + o_Leta);
  w.Rup = reinterpret_cast<double*>(base + o_Rup);
  w.Rdn = reinterpret_cast<double*>(base + o_Rdn);
  w.Apart = reinterpret_cast<double*>(base + o_Apart);
  w.F = reinterpret_cast<double*>(base + o_F);
  w.P = reinterpret_cast<double*>(base + o_P);
  w.Iem = reinterpret_cast<double*>(base + o_Iem);
  // tangent, RH92 and Krylov buffers stay null: a base evaluation never touches them

  k_store_static_desc<<<1, 1, 0, s>>>(reinterpret_cast<ColDesc*>(base + o_desc), cd);
  JFNK_CUDA(cudaGetLastError());
  JFNK_CUDA(cudaMemcpyAsync(w.n, n, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  JFNK_CUDA(cudaMemcpyAsync(w.Jdag, J_dagger ? J_dagger : M.tables.Bn, QZ * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
  Batch b;   // launch geometry only; owns no memory here
  b.ncols = 1;
  b.mixed = 0;
  b.max_nz = (int)nz;
  b.max_nq = (int)nq;
  b.max_nt = (int)nt;
  b.max_N = (int)N;
  b.max_nmu = (int)nmu;
  b.max_nl = (int)nl;
  b.n_sm = ctx->n_sm;
  b.formal_kind = fused ? FORMAL_FUSED : FORMAL_UNFUSED;
  b.formal_qb = qb;
  if (fused && (rc = fused_prepare(&b))) return rc;
  b.d_cols = reinterpret_cast<ColDesc*>(base + o_desc);
  if ((rc = launch_evaluation(b, s))) {
    b.d_cols = nullptr;
    return rc;
  }
  b.d_cols = nullptr;
  JFNK_CUDA(cudaMemcpyAsync(F, w.F, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (J_new) JFNK_CUDA(cudaMemcpyAsync(J_new, w.Jnew, QZ * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return JFNK_OK;
}
