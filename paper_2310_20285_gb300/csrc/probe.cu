// Throughput probes of the units that bound the small-D kernel product: the MUFU exp2
// (one per kernel value of RBF, the exponential of Matern) and FP32 FFMA.  Each thread
// runs 8 independent dependency chains so that latency is hidden; the result is
// operations per second over the whole GPU, timed with CUDA events on the stream.
#include <algorithm>

#include "internal.h"

namespace itergp {
namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// x <- 2^(-x) keeps every value in (0, 1] (no overflow, no denormals).
__global__ void probe_ex2_kernel(int iters, float seed, float* sink) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed * (threadIdx.x + 1 + c) * 1e-6f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = ex2_approx(-v[c]);
  }
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += v[c];
  if (acc == 12345.f) sink[blockIdx.x] = acc;   // keeps the chains live
}

// v <- v * a + b with |a| < 1 stays bounded.
__global__ void probe_ffma_kernel(int iters, float seed, float* sink) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed * (threadIdx.x + c);
  const float a = 0.999f, b = 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
  }
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += v[c];
  if (acc == 12345.f) sink[blockIdx.x] = acc;
}

}  // namespace

int probe_throughput(DeviceContext* ctx, int what, double* ops_per_s, cudaStream_t stream) {
  const int blocks = 8 * ctx->num_sms, threads = 256, iters = 4096;
  Scratch sink;
  ITERGP_CUDA_TRY(sink.alloc(ctx, sizeof(float) * blocks, stream));
  cudaEvent_t e0, e1;
  ITERGP_CUDA_TRY(cudaEventCreate(&e0));
  ITERGP_CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {   // first launch warms up
    err = cudaEventRecord(e0, stream);
    if (what == 0)
      probe_ex2_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5f, sink.as<float>()), ::itergp::note_launch();
    else
      probe_ffma_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5f, sink.as<float>()), ::itergp::note_launch();
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0) best_ms = std::min(best_ms, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ITERGP_CUDA_TRY(err);
  const double ops = static_cast<double>(blocks) * threads * iters * kChains * (what == 0 ? 1.0 : 2.0);
  *ops_per_s = ops / (best_ms * 1e-3);
  return ITERGP_OK;
}

}  // namespace itergp

extern "C" int itergp_probe_throughput(int32_t what, double* ops_per_s, itergp_stream stream) {
  if ((what != 0 && what != 1) || !ops_per_s) return ITERGP_EINVAL;
  itergp::DeviceContext* ctx = itergp::current_context();
  if (!ctx) return ITERGP_ECUDA;
  return itergp::probe_throughput(ctx, what, ops_per_s, static_cast<cudaStream_t>(stream));
}
