// Throughput probes of the units that bound the kernel product: the MUFU exp2 (one per
// kernel value of RBF, the exponential of Matern) and rsqrt (Matern's distance), FP32
// FFMA, FP64 DFMA, and the tcgen05 MMA in the shapes the product issues (SS M = 128 with
// N = 128 or 256, the same while other warps stream TMEM loads, the TS form of the
// weighted sum, and the SS form with TF32 operands).  Results are operations per second
// over the whole GPU, timed with CUDA events on the stream.
#include <algorithm>

#include "internal.h"
#include "tc_ptx.cuh"

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

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// x <- 1 / sqrt(x) stays in [min(x0, 1/sqrt(x0)), max(...)] and tends to 1.
__global__ void probe_rsqrt_kernel(int iters, float seed, float* sink) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = 0.5f + seed * (threadIdx.x + 1 + c) * 1e-4f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = rsqrt_approx(v[c]);
  }
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += v[c];
  if (acc == 12345.f) sink[blockIdx.x] = acc;
}

// The FFMA chain in FP64.
__global__ void probe_dfma_kernel(int iters, double seed, float* sink) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed * (threadIdx.x + c);
  const double a = 0.999, b = 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += v[c];
  if (acc == 12345.0) sink[blockIdx.x] = static_cast<float>(acc);
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

// One CTA per SM issues back-to-back tcgen05.mma kind::f16 (BF16 in, FP32 accumulate,
// K = 16 each) from one elected thread, 4 per 64-wide K slice, alternating between two
// TMEM accumulators as the product's double-buffered G does.
//   MODE 0: SS, A 128 x 64 and B N x 64 in shared memory (128-byte swizzle, K-major)
//   MODE 1: MODE 0 while warps 4-7 stream tcgen05.ld of 32 columns from a third region
//   MODE 2: TS, A (packed BF16 pairs) read from TMEM columns 256.., B N x 64 in shared memory
//   MODE 3: MODE 0 with kind::tf32 (the same 128-byte rows read as 32 FP32 values, K = 8)
// Operands are BF16 values in [0.5, 1) with random signs, which read as FP32 are also in
// [0.5, 1) (finite sums).  Every wait is bounded; on expiry ITERGP_ETIMEOUT goes to the
// status word.
constexpr uint64_t kProbeWaitNs = 2000000000ull;

template <int N, int MODE>
__global__ void __launch_bounds__(256, 1) probe_mma_kernel(int iters, int* status, float* sink) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  constexpr uint32_t A_BYTES = 128 * 64 * 2, B_BYTES = N * 64 * 2;
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s, finished_s;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint32_t* w = reinterpret_cast<uint32_t*>(smem);
  for (uint32_t i = threadIdx.x; i < (A_BYTES + B_BYTES) / 4; i += blockDim.x) {
    const uint32_t h = (i + 1u) * 2654435761u;
    const uint32_t lo = (h & 0x807Fu) | 0x3F00u, hi = ((h >> 16) & 0x807Fu) | 0x3F00u;
    w[i] = lo | (hi << 16);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    abort_s = 0;
    finished_s = 0;
    mbar_init(&done, 1);
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc(&tmem_base_s, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tmem_base_s;
  volatile int* ab = &abort_s;
  if (MODE == 2 && warp >= 4) {
    // A operand of the TS form: 128 lanes x 32 columns of packed BF16 pairs at column 256
    uint32_t r[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = 0x3F003F00u ^ ((lane * 16u + i) & 0x80008000u);
    const uint32_t lane_base = static_cast<uint32_t>(32 * (warp - 4)) << 16;
    tmem_st16(tb + lane_base + 256, r);
    tmem_st16(tb + lane_base + 272, r);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = MODE == 3 ? idesc_tf32_f32(128, N) : idesc_bf16_f32(128, N);
      const uint64_t dA = sdesc_kmajor_sw128(smem_u32(smem));
      const uint64_t dB = sdesc_kmajor_sw128(smem_u32(smem + A_BYTES));
      for (int it = 0; it < iters; ++it) {
        const uint32_t d = MODE == 2 ? 384u : (N == 128 ? static_cast<uint32_t>(it & 1) * 128u : 0u);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc = (it < 2 && kk == 0) ? 0u : 1u;
          if (MODE == 2)
            mma_ts(tb + d, tb + 256 + 8 * kk, dB + 2 * kk, idesc, acc);
          else if (MODE == 3)
            mma_ss_tf32(tb + d, dA + 2 * kk, dB + 2 * kk, idesc, acc);
          else
            mma_ss(tb + d, dA + 2 * kk, dB + 2 * kk, idesc, acc);
        }
      }
      mma_commit(&done);
      mbar_wait(&done, 0, ab, kProbeWaitNs);
      finished_s = 1;
    }
  } else if (MODE == 1 && warp >= 4) {
    // concurrent TMEM reads of columns 256..383 (not written by the MMAs)
    const uint32_t lane_base = static_cast<uint32_t>(32 * (warp - 4)) << 16;
    uint32_t acc = 0;
    volatile int* fin = &finished_s;
    for (int rep = 0; rep < (1 << 22) && !*fin && !*ab; ++rep) {
      uint32_t v[32];
      tmem_ld32(tb + lane_base + 256 + 32 * (rep & 3), v);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 32; ++i) acc ^= v[i];
    }
    if (acc == 0x12345678u) sink[blockIdx.x] = 1.f;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tb, 512);
  }
  if (threadIdx.x == 0 && abort_s) atomicExch(status, ITERGP_ETIMEOUT);
}

}  // namespace

// MMA-rate probe: what = 2 (SS, N = 128), 3 (SS, N = 256), 4 (SS, N = 128 with concurrent
// TMEM loads), 5 (TS, N = 80), 6 (SS TF32, N = 128); flops per second over the whole GPU.
int probe_mma(DeviceContext* ctx, int what, double* ops_per_s, cudaStream_t stream) {
  const int blocks = ctx->num_sms, iters = 20000;
  const size_t smem = 160 * 1024;   // one CTA per SM (the kernel allocates all of TMEM)
  int n = 128;
  void (*fn)(int, int*, float*) = nullptr;
  switch (what) {
    case 2: fn = probe_mma_kernel<128, 0>; break;
    case 3: fn = probe_mma_kernel<256, 0>; n = 256; break;
    case 4: fn = probe_mma_kernel<128, 1>; break;
    case 6: fn = probe_mma_kernel<128, 3>; break;
    default: fn = probe_mma_kernel<80, 2>; n = 80; break;
  }
  const int k_per_mma = what == 6 ? 8 : 16;
  Scratch sink;
  ITERGP_CUDA_TRY(sink.alloc(ctx, sizeof(float) * blocks, stream));
  ITERGP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  cudaEvent_t e0, e1;
  ITERGP_CUDA_TRY(cudaEventCreate(&e0));
  ITERGP_CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {   // first launch warms up
    err = cudaEventRecord(e0, stream);
    if (err == cudaSuccess) {
      fn<<<blocks, 256, smem, stream>>>(iters, ctx->status, sink.as<float>());
      ::itergp::note_launch();
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0) best_ms = std::min(best_ms, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ITERGP_CUDA_TRY(err);
  *ops_per_s = static_cast<double>(blocks) * iters * 4 * 2.0 * 128 * n * k_per_mma / (best_ms * 1e-3);
  return ITERGP_OK;
}

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
    else if (what == 1)
      probe_ffma_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5f, sink.as<float>()), ::itergp::note_launch();
    else if (what == 7)
      probe_dfma_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5, sink.as<float>()), ::itergp::note_launch();
    else
      probe_rsqrt_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5f, sink.as<float>()), ::itergp::note_launch();
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
  // flops for the fused multiply-adds (2 each), operations for the MUFU probes
  const double ops = static_cast<double>(blocks) * threads * iters * kChains * (what == 1 || what == 7 ? 2.0 : 1.0);
  *ops_per_s = ops / (best_ms * 1e-3);
  return ITERGP_OK;
}

}  // namespace itergp

extern "C" int itergp_probe_throughput(int32_t what, double* ops_per_s, itergp_stream stream) {
  if (what < 0 || what > 8 || !ops_per_s) return ITERGP_EINVAL;
  itergp::DeviceContext* ctx = itergp::current_context();
  if (!ctx) return ITERGP_ECUDA;
  if (what >= 2 && what <= 6) return itergp::probe_mma(ctx, what, ops_per_s, static_cast<cudaStream_t>(stream));
  return itergp::probe_throughput(ctx, what, ops_per_s, static_cast<cudaStream_t>(stream));
}
