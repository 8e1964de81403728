// Throughput probes of the units that bound the kernel product: the MUFU exp2 (one per
// kernel value of RBF, the exponential of Matern) and rsqrt (Matern's distance), FP32
// FFMA, FP64 DFMA, and the tcgen05 MMA in the shapes the product issues (SS M = 128 with
// N = 128 or 256, the same while other warps stream TMEM loads, the TS form of the
// weighted sum, the SS form with TF32 operands, and the CTA-pair forms of M = 256, with
// static operands or fed by a TMA ring like the product's distance GEMM).
// Results are operations per second over the whole GPU, timed with CUDA events on the
// stream.  Measurement tooling of the bench: built as its own library
// (libitergp_probe.so), not part of the product library.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/itergp_probe.h"
#include "../csrc/tc_ptx.cuh"
#include "../csrc/tma_host.h"

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

// The CTA-pair forms: clusters of two CTAs; the even CTA's thread issues cta_group::2
// tcgen05.mma of M = 256 back to back (4 per 64-wide K slice, alternating two TMEM
// accumulators for N = 128).  Each CTA holds A 128 x 64 and its half of B (N / 2 rows) in
// shared memory (SS), or A in its TMEM (TS).  Operand words as in probe_mma_kernel (read as
// FP16 they lie in [1.75, 1.88) with random signs: finite sums).  Both CTAs of a pair meet
// at every cluster barrier; the one wait is bounded.
template <int N, bool TS, bool F16>
__global__ void __launch_bounds__(256, 1) probe_mma_pair_kernel(int iters, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  constexpr uint32_t A_BYTES = 128 * 64 * 2, B_BYTES = (N / 2) * 64 * 2;
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const uint32_t h = cluster_rank();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint32_t* w = reinterpret_cast<uint32_t*>(smem);
  for (uint32_t i = threadIdx.x; i < (A_BYTES + B_BYTES) / 4; i += blockDim.x) {
    const uint32_t x = (i + 1u + 977u * h) * 2654435761u;
    const uint32_t lo = (x & 0x807Fu) | 0x3F00u, hi = ((x >> 16) & 0x807Fu) | 0x3F00u;
    w[i] = lo | (hi << 16);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    abort_s = 0;
    mbar_init(&done, 1);
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc_pair(&tmem_base_s, 512);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tb = tmem_base_s;
  volatile int* ab = &abort_s;
  if (TS && warp >= 4) {   // A operand of the TS form: packed pairs at column 256, both CTAs
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
  cluster_sync_all();
  tc_fence_after();
  if (warp == 1 && lane == 0 && h == 0) {
    const uint32_t idesc = F16 ? idesc_f16_f32(256, N) : idesc_bf16_f32(256, N);
    const uint64_t dA = sdesc_kmajor_sw128(smem_u32(smem));
    const uint64_t dB = sdesc_kmajor_sw128(smem_u32(smem + A_BYTES));
    for (int it = 0; it < iters; ++it) {
      const uint32_t d = TS ? 384u : (N == 128 ? static_cast<uint32_t>(it & 1) * 128u : 0u);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t acc = (it < 2 && kk == 0) ? 0u : 1u;
        if (TS)
          mma_ts_pair(tb + d, tb + 256 + 8 * kk, dB + 2 * kk, idesc, acc);
        else
          mma_ss_pair(tb + d, dA + 2 * kk, dB + 2 * kk, idesc, acc);
      }
    }
    mma_commit_pair_local(&done);
    mbar_wait(&done, 0, ab, kProbeWaitNs);
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc_pair(tb, 512);
  }
  if (threadIdx.x == 0 && abort_s) atomicExch(status, ITERGP_ETIMEOUT);
}

// Ring-fed pair-form MMAs: clusters of two CTAs stream stages of K = 64 (A hi and lo, 128
// rows per CTA; B hi and lo, N / 2 rows per CTA) from a 64 MB FP16 array through a ring of
// 3 stages (TMA loads on the even CTA's full barriers, MMA commits on both CTAs' empty
// barriers), and the even CTA issues the product's three-term order on every stage
// (A_hi B_lo, A_lo B_hi per K step, then A_hi B_hi): the distance GEMM of the pair form
// with its refills and without its epilogue.  Every wait is bounded.
template <int N>
__global__ void __launch_bounds__(128, 1)
probe_ring_pair_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                       int stages, int* status) {
  constexpr int NST = 3, NC = N / 2;
  constexpr uint32_t A_PART = 128 * 128, B_PART = NC * 128, SB = 2 * A_PART + 2 * B_PART;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[NST], empty[NST], drain;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t h = cluster_rank();
  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&drain, 1);
    abort_s = 0;
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc_pair(&tmem_base_s, 256);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tb = tmem_base_s;
  volatile int* ab = &abort_s;
  const int pair_id = blockIdx.x / 2;
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < stages; ++i) {
      const int s = i % NST;
      if (i >= NST && !mbar_wait_cluster(&empty[s], static_cast<uint32_t>((i / NST - 1) & 1), ab, kProbeWaitNs)) break;
      uint8_t* base = smem + s * SB;
      const int x = 64 * (i % 12);
      const int ya = (128 * (2 * pair_id + static_cast<int>(h)) + 384 * (i % 7)) % 30000;   // this CTA's A rows
      const int yb = (NC * (2 * (i % 50) + static_cast<int>(h))) % 30000;                 // the shared B chunk
      if (h == 0) mbar_arrive_expect_tx(&full[s], 2 * SB);
      const uint32_t fb = cluster_addr(smem_u32(&full[s]), 0u);
      tma_load_2d_pair(base, &mA, fb, x, ya);
      tma_load_2d_pair(base + A_PART, &mA, fb, x + 64, ya);
      tma_load_2d_pair(base + 2 * A_PART, &mB, fb, x, yb);
      tma_load_2d_pair(base + 2 * A_PART + B_PART, &mB, fb, x + 64, yb);
    }
  } else if (warp == 1 && lane == 0 && h == 0) {
    const uint32_t idesc = idesc_f16_f32(256, N);
    const uint64_t d0 = sdesc_kmajor_sw128(smem_u32(smem));
    for (int i = 0; i < stages; ++i) {
      const int s = i % NST;
      const uint32_t ph = static_cast<uint32_t>((i / NST) & 1);
      if (!mbar_try_wait(&full[s], ph) && !mbar_wait(&full[s], ph, ab, kProbeWaitNs)) break;
      tc_fence_after();
      const uint64_t dAh = d0 + static_cast<uint64_t>(s) * (SB >> 4);
      const uint64_t dAl = dAh + (A_PART >> 4), dBh = dAh + (2 * A_PART >> 4), dBl = dBh + (B_PART >> 4);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        mma_ss_pair(tb, dAh + 2 * kk, dBl + 2 * kk, idesc, (i | kk) ? 1u : 0u);
        mma_ss_pair(tb, dAl + 2 * kk, dBh + 2 * kk, idesc, 1u);
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_ss_pair(tb, dAh + 2 * kk, dBh + 2 * kk, idesc, 1u);
      mma_commit_pair_both(&empty[s]);
    }
    mma_commit_pair_local(&drain);
    mbar_wait_drain(&drain, 0, kProbeWaitNs);
  }
  tc_fence_before();
  __syncthreads();
  if (abort_s) {   // copies in flight land before the CTA can exit
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 1000000ull) {
    }
  }
  cluster_sync_all();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc_pair(tb, 256);
  }
  if (threadIdx.x == 0 && abort_s) atomicExch(status, ITERGP_ETIMEOUT);
}

// Device buffers of one probe call (the probe library has no pool of its own).
struct ProbeBufs {
  float* sink = nullptr;
  int* status = nullptr;
  ~ProbeBufs() {
    if (sink) cudaFree(sink);
    if (status) cudaFree(status);
  }
  cudaError_t alloc(int blocks) {
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * blocks);
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
    return e;
  }
};

int to_status(cudaError_t e) {
  if (e == cudaSuccess) return ITERGP_OK;
  return e == cudaErrorMemoryAllocation ? ITERGP_ENOMEM : ITERGP_ECUDA;
}

// Times `launch` (best of two after a warm-up); ms of the fastest launch.
template <class F>
cudaError_t time_best(F launch, cudaStream_t stream, float* best_ms) {
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  *best_ms = 1e30f;
  for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {   // first launch warms up
    err = cudaEventRecord(e0, stream);
    if (err == cudaSuccess) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0) *best_ms = std::min(*best_ms, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

int read_status(const ProbeBufs& b) {
  int st = 0;
  if (cudaMemcpy(&st, b.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ITERGP_ECUDA;
  return st;
}

// MMA-rate probe, one CTA per SM: what = 2 (SS, N = 128), 3 (SS, N = 256), 4 (SS, N = 128
// with concurrent TMEM loads), 5 (TS, N = 80), 6 (SS TF32, N = 128).
int probe_mma(int sms, int what, double* ops_per_s, cudaStream_t stream) {
  const int blocks = sms, iters = 20000;
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
  ProbeBufs b;
  cudaError_t err = b.alloc(blocks);
  if (err == cudaSuccess) err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  float ms = 0.f;
  if (err == cudaSuccess)
    err = time_best([&] {
      fn<<<blocks, 256, smem, stream>>>(iters, b.status, b.sink);
      return cudaGetLastError();
    }, stream, &ms);
  if (err != cudaSuccess) return to_status(err);
  if (const int st = read_status(b)) return st;
  *ops_per_s = static_cast<double>(blocks) * iters * 4 * 2.0 * 128 * n * k_per_mma / (ms * 1e-3);
  return ITERGP_OK;
}

// Pair-form MMA rate: what = 9 (SS FP16, N = 128), 10 (SS FP16, N = 256), 11 (TS BF16,
// N = 80), 12 (SS FP16, N = 192); as many clusters as can be resident at once.
int probe_mma_pair(int what, double* ops_per_s, cudaStream_t stream) {
  const int iters = 20000;
  const size_t smem = 160 * 1024;
  int n = 128;
  void (*fn)(int, int*) = nullptr;
  switch (what) {
    case 9: fn = probe_mma_pair_kernel<128, false, true>; break;
    case 10: fn = probe_mma_pair_kernel<256, false, true>; n = 256; break;
    case 12: fn = probe_mma_pair_kernel<192, false, true>; n = 192; break;
    default: fn = probe_mma_pair_kernel<80, true, false>; n = 80; break;
  }
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return to_status(err);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(2);
  int clusters = 0;
  err = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
  if (err != cudaSuccess) return to_status(err);
  if (clusters < 1) return ITERGP_EUNSUPPORTED;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * clusters));
  ProbeBufs b;
  err = b.alloc(1);
  float ms = 0.f;
  if (err == cudaSuccess)
    err = time_best([&] { return cudaLaunchKernelEx(&cfg, fn, iters, b.status); }, stream, &ms);
  if (err != cudaSuccess) return to_status(err);
  if (const int st = read_status(b)) return st;
  *ops_per_s = static_cast<double>(clusters) * iters * 4 * 2.0 * 256 * n * 16 / (ms * 1e-3);
  return ITERGP_OK;
}

// Ring-fed pair-form MMA rate: what = 13 (N = 128), 14 (N = 192); MMA flops per second of
// as many clusters as can be resident at once.
int probe_ring_pair(int what, double* ops_per_s, cudaStream_t stream) {
  const int n = what == 13 ? 128 : 192, stages = 4000;
  void (*fn)(const CUtensorMap, const CUtensorMap, int, int*) =
      what == 13 ? probe_ring_pair_kernel<128> : probe_ring_pair_kernel<192>;
  const size_t smem = 3 * (2 * 128 * 128 + 2 * (n / 2) * 128) + 1024;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return to_status(err);
  const uint64_t rows = 32768, cols = 1024;
  void* src = nullptr;
  err = cudaMalloc(&src, rows * cols * 2);
  if (err != cudaSuccess) return to_status(err);
  // FP16 0x3C3C (1.06) everywhere: finite sums
  err = cudaMemsetAsync(src, 0x3C, rows * cols * 2, stream);
  CUtensorMap maps[2];
  if (err == cudaSuccess &&
      !(encode_bf16_sw128(&maps[0], src, rows, cols, cols, 128, CU_TENSOR_MAP_DATA_TYPE_FLOAT16) &&
        encode_bf16_sw128(&maps[1], src, rows, cols, cols, static_cast<uint32_t>(n / 2), CU_TENSOR_MAP_DATA_TYPE_FLOAT16)))
    err = cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(2);
  int clusters = 0;
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
  ProbeBufs b;
  if (err == cudaSuccess) err = b.alloc(1);
  float ms = 0.f;
  if (err == cudaSuccess && clusters >= 1) {
    cfg.gridDim = dim3(static_cast<unsigned>(2 * clusters));
    err = time_best([&] { return cudaLaunchKernelEx(&cfg, fn, maps[0], maps[1], stages, b.status); }, stream, &ms);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  cudaFree(src);
  if (err != cudaSuccess) return to_status(err);
  if (clusters < 1) return ITERGP_EUNSUPPORTED;
  if (const int st = read_status(b)) return st;
  *ops_per_s = static_cast<double>(clusters) * stages * 12 * 2.0 * 256 * n * 16 / (ms * 1e-3);
  return ITERGP_OK;
}

int probe_units(int sms, int what, double* ops_per_s, cudaStream_t stream) {
  const int blocks = 8 * sms, threads = 256, iters = 4096;
  ProbeBufs b;
  cudaError_t err = b.alloc(blocks);
  float ms = 0.f;
  if (err == cudaSuccess)
    err = time_best([&] {
      if (what == 0)
        probe_ex2_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5f, b.sink);
      else if (what == 1)
        probe_ffma_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5f, b.sink);
      else if (what == 7)
        probe_dfma_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5, b.sink);
      else
        probe_rsqrt_kernel<<<blocks, threads, 0, stream>>>(iters, 0.5f, b.sink);
      return cudaGetLastError();
    }, stream, &ms);
  if (err != cudaSuccess) return to_status(err);
  // flops for the fused multiply-adds (2 each), operations for the MUFU probes
  const double ops = static_cast<double>(blocks) * threads * iters * kChains * (what == 1 || what == 7 ? 2.0 : 1.0);
  *ops_per_s = ops / (ms * 1e-3);
  return ITERGP_OK;
}

}  // namespace
}  // namespace itergp

extern "C" int itergp_probe_throughput(int32_t what, double* ops_per_s, itergp_stream stream) {
  if (what < 0 || what > 14 || !ops_per_s) return ITERGP_EINVAL;
  (void)cudaGetLastError();
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ITERGP_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (what >= 13) return itergp::probe_ring_pair(what, ops_per_s, s);
  if (what >= 9) return itergp::probe_mma_pair(what, ops_per_s, s);
  if (what >= 2 && what <= 6) return itergp::probe_mma(sms, what, ops_per_s, s);
  return itergp::probe_units(sms, what, ops_per_s, s);
}
