// Arithmetic-pipe throughput probe (roofline denominators for ALU-bound
// kernels): every thread runs independent dependent chains of one operation.
#include "formal_coef.cuh"

namespace jfnk {

constexpr int kChains = 8;
constexpr int kIters = 4096;
// FP32 and MUFU launches run 8x longer (about 2 ms), so that each launch is
// timed at the clock the SMs hold under load rather than during a ramp
constexpr int kIters32 = 8 * kIters;

template <typename T, int ITERS>
__global__ void k_probe_fma(T* out, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)12345.678) out[0] = s;   // keeps the chains alive
}

__global__ void k_probe_exp64(double* out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = -1e-3 * (threadIdx.x + c);
  for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -exp(x[c]) * 0.5;
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[0] = s;
}

// MUFU throughput: dependent chains of the hardware base-2 exponential, issued
// as inline PTX so that the compiler can neither fold nor merge them.
__device__ __forceinline__ float ex2_mufu(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void k_probe_exp32(float* out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int it = 0; it < kIters32; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = ex2_mufu(-x[c]);   // stays in [1/2, 1)
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[0] = s;
}

__global__ void k_check_arith(int op, const double* a, const double* b, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const df x = df_from_double(a[i]), y = df_from_double(b[i]);
  df r;
  switch (op) {
    case 0: r = df_add(x, y); break;
    case 1: r = df_sub(x, y); break;
    case 2: r = df_mul(x, y); break;
    case 3: r = df_div(x, y); break;
    default: r = df_acc(x, y); break;
  }
  out[i] = df_to_double(r);
}

}  // namespace jfnk

using namespace jfnk;

extern "C" int jfnk_check_arith(jfnk_ctx* ctx, int op, const double* a, const double* b, double* q, int n) {
  if (!ctx || op < 0 || op > 4 || n < 0 || (n > 0 && (!a || !b || !q)))
    return fail(JFNK_E_INVALID, "bad arithmetic-check arguments");
  if (n == 0) return JFNK_OK;
  JFNK_CUDA(cudaSetDevice(ctx->device));
  double* d = nullptr;
  JFNK_CUDA(cudaMalloc(&d, sizeof(double) * 3 * (size_t)n));
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d, a, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, b, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_check_arith<<<(n + 255) / 256, 256, 0, s>>>(op, d, d + n, d + 2 * (size_t)n, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(q, d + 2 * (size_t)n, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return fail(JFNK_E_CUDA, cudaGetErrorString(e));
  return JFNK_OK;
}

extern "C" int jfnk_probe_alu(jfnk_ctx* ctx, int kind, double* ops_per_s) {
  if (!ctx || !ops_per_s || kind < 0 || kind > 3) return fail(JFNK_E_INVALID, "bad probe arguments");
  JFNK_CUDA(cudaSetDevice(ctx->device));
  double* d;
  JFNK_CUDA(cudaMalloc(&d, 64));
  const int threads = 256, blocks = ctx->n_sm * 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t s = ctx->stream;
  float best = 1e30f;
  for (int rep = 0; rep < 10; ++rep) {
    cudaEventRecord(e0, s);
    switch (kind) {
      case 0: k_probe_fma<double, kIters><<<blocks, threads, 0, s>>>(d, 0.999999, 1e-7); break;
      case 1: k_probe_fma<float, kIters32><<<blocks, threads, 0, s>>>((float*)d, 0.999999f, 1e-7f); break;
      case 2: k_probe_exp64<<<blocks, threads, 0, s>>>(d); break;
      case 3: k_probe_exp32<<<blocks, threads, 0, s>>>((float*)d); break;
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 1 && ms < best) best = ms;   // the first two launches are warm-ups
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (err != cudaSuccess) return fail(JFNK_E_CUDA, cudaGetErrorString(err));
  const double threads_total = (double)threads * blocks;
  double ops;
  if (kind == 0) ops = threads_total * kChains * kIters * 2.0;
  else if (kind == 1) ops = threads_total * kChains * kIters32 * 2.0;
  else if (kind == 2) ops = threads_total * kChains * (kIters / 8);
  else ops = threads_total * kChains * kIters32;
  *ops_per_s = ops / (best * 1e-3);
  return JFNK_OK;
}
