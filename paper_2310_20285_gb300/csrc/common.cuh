// Internal declarations shared by the translation units of libitergp.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../include/itergp.h"

namespace itergp {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kSqrt3 = 1.7320508075688772f;

// Kernel-function constants prepared on the host.
struct KParams {
  int kind;      // ITERGP_RBF / ITERGP_MATERN32
  float s;       // outputscale
  float c_exp;   // RBF: -log2(e) / (2 l^2)          Matern: unused
  float c_u;     // Matern: sqrt(3) / l               RBF: unused
  float log2s;   // log2(s): RBF values as 2^(c_exp r^2 + log2 s) in the tensor-core epilogue
};

inline KParams make_kparams(const itergp_kernel& k) {
  KParams p;
  p.kind = k.kind;
  p.s = k.outputscale;
  const double l = k.lengthscale;
  p.c_exp = static_cast<float>(-1.4426950408889634 / (2.0 * l * l));
  p.c_u = static_cast<float>(1.7320508075688772 / l);
  p.log2s = static_cast<float>(std::log2(static_cast<double>(k.outputscale)));
  return p;
}

// k(r^2) in FP32 with the accurate library exp2f / sqrtf (plain path).
template <int KIND>
__device__ __forceinline__ float kernel_eval_accurate(float r2, const KParams& kp) {
  if (KIND == ITERGP_RBF) {
    return kp.s * exp2f(r2 * kp.c_exp);
  } else {
    const float u = sqrtf(r2) * kp.c_u;
    return kp.s * (1.0f + u) * exp2f(-kLog2e * u);
  }
}

// Hardware approximations (MUFU): ex2.approx has a relative error of about 2^-22 and
// sqrt.approx about 2^-23, well inside the tensor-core paths' error budget.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 2^e for -126 <= e <= 127, built from its bit pattern (exact).
__device__ __forceinline__ float pow2i(int e) { return __int_as_float((e + 127) << 23); }

// The exponent e of a power-of-two scale 2^e that brings a block of values whose largest
// magnitude has the bit pattern `maxbits` (a non-negative float) into [128, 256): for
// m 2^k with m in [0.5, 1), e = 8 - k; 0 for zero or non-finite maxima; clamped to
// [-126, 126].
__device__ __forceinline__ int scale_exp_of_max(uint32_t maxbits) {
  const int bexp = static_cast<int>((maxbits >> 23) & 0xFFu);
  int e = 0;
  if (maxbits != 0u && bexp != 0xFF) e = 8 - (bexp == 0 ? -125 : bexp - 126);
  return max(-126, min(126, e));
}

template <int KIND>
__device__ __forceinline__ float kernel_eval_fast(float r2, const KParams& kp) {
  if (KIND == ITERGP_RBF) {
    return kp.s * ex2_approx(r2 * kp.c_exp);
  } else {
    const float u = sqrt_approx(r2) * kp.c_u;
    return kp.s * (1.0f + u) * ex2_approx(-kLog2e * u);
  }
}

// -------------------------------------------------------------------- host utilities

#define ITERGP_CUDA_TRY(expr)                                  \
  do {                                                         \
    cudaError_t err__ = (expr);                                \
    if (err__ != cudaSuccess) {                                \
      ::itergp::record_cuda_error(err__, #expr, __FILE__, __LINE__); \
      return (err__ == cudaErrorMemoryAllocation) ? ITERGP_ENOMEM : ITERGP_ECUDA; \
    }                                                          \
  } while (0)

void record_cuda_error(cudaError_t err, const char* expr, const char* file, int line);

// Per-device runtime state: status word written by kernels, a stream-ordered pool for
// scratch, and device properties.
struct DeviceContext {
  int device = -1;
  int num_sms = 0;
  int cc_major = 0, cc_minor = 0;
  size_t smem_optin = 0;
  int* status = nullptr;           // device int: 0 = OK, else itergp_status
  cudaMemPool_t pool = nullptr;
  cudaStream_t release = nullptr;  // non-blocking stream for stream-ordered frees
  bool tcgen05 = false;            // sm_100 family with tcgen05 / TMA
};

// Context of the current device (created on first use).  Returns nullptr on failure.
DeviceContext* current_context();

// Stream-ordered scratch allocation from the library pool.
cudaError_t scratch_alloc(DeviceContext* ctx, void** p, size_t bytes, cudaStream_t s);
void scratch_free(void* p, cudaStream_t s);

// A caller-provided block of device memory that scratch_alloc carves from (bump pointer,
// 256-byte aligned) instead of the pool while it is installed on the calling thread.
// Only the allocation-free entry point installs one; scratch_free ignores its blocks.
struct ScratchArena {
  char* base = nullptr;
  size_t size = 0;
  size_t used = 0;
};
void set_thread_arena(ScratchArena* arena);

// RAII scratch block freed (stream-ordered) at scope exit.
struct Scratch {
  void* ptr = nullptr;
  cudaStream_t stream = nullptr;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() {
    if (ptr) scratch_free(ptr, stream);
  }
  cudaError_t alloc(DeviceContext* ctx, size_t bytes, cudaStream_t s) {
    stream = s;
    return scratch_alloc(ctx, &ptr, bytes < 256 ? 256 : bytes, s);
  }
  template <class T>
  T* as(size_t byte_offset = 0) const {
    return reinterpret_cast<T*>(static_cast<char*>(ptr) + byte_offset);
  }
};

// Pool accounting of a fit: between begin and end, every scratch_alloc / scratch_free of
// the calling thread (and pool_track_add of other pool blocks) updates the live bytes;
// end returns their peak.
void pool_track_begin();
int64_t pool_track_end();
void pool_track_add(void* p, size_t bytes);
void pool_track_remove(void* p);

// Bound of every device-side wait of the tensor-core product launched by this thread
// (default 4 s); a fit installs its wait_limit_ns for its duration.
constexpr uint64_t kDefaultWaitNs = 4000000000ull;
uint64_t thread_wait_limit();
void set_thread_wait_limit(uint64_t ns);
struct WaitLimitGuard {
  uint64_t prev;
  explicit WaitLimitGuard(uint64_t ns) : prev(thread_wait_limit()) {
    if (ns != 0) set_thread_wait_limit(ns);
  }
  ~WaitLimitGuard() { set_thread_wait_limit(prev); }
  WaitLimitGuard(const WaitLimitGuard&) = delete;
  WaitLimitGuard& operator=(const WaitLimitGuard&) = delete;
};

// Launch accounting: every kernel launch site calls note_launch(); the fused product
// kernel's launches are optionally bracketed by events (timing_begin / timing_end).
void note_launch(int64_t n = 1);
void timing_begin(cudaStream_t s);
void timing_end(cudaStream_t s);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace itergp
