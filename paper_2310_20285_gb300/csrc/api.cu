// C-ABI entry points of libitergp: argument validation, per-device context, the model
// object and the predictive epilogue.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <memory>
#include <mutex>
#include <vector>

#include <unordered_map>

#include "internal.h"

namespace itergp {

int winv_apply_launch(DeviceContext* ctx, const float* f, int64_t n, int c, const float* x,
                      float* out, cudaStream_t s);
int pseudo_targets_launch(DeviceContext* ctx, const float* f, const int32_t* y, int64_t n, int c,
                          float* out, cudaStream_t s);
int sym_eig_launch(DeviceContext* ctx, const double* M, int b, double* lam, double* U,
                   cudaStream_t s);

namespace {
thread_local char t_last_error[512] = "";
}

void record_cuda_error(cudaError_t err, const char* expr, const char* file, int line) {
  static const bool verbose = std::getenv("ITERGP_DEBUG") != nullptr;
  const char* base = std::strrchr(file, '/');
  std::snprintf(t_last_error, sizeof(t_last_error), "%s: %s (%s:%d)", expr, cudaGetErrorString(err),
                base ? base + 1 : file, line);
  if (verbose) std::fprintf(stderr, "[itergp] %s\n", t_last_error);
}

namespace {
std::mutex g_ctx_mu;
DeviceContext* g_ctx[64] = {};

std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_timing{false};
std::mutex g_timing_mu;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_timed;   // recorded (begin, end) pairs
thread_local cudaEvent_t t_begin = nullptr;
}  // namespace

void note_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Kernel timing records plain events; inside a stream capture an event record only
// orders the capture, so captured launches are not timed.
bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

void timing_begin(cudaStream_t s) {
  if (!g_timing.load(std::memory_order_relaxed) || stream_capturing(s)) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, s);
  t_begin = e;
}

void timing_end(cudaStream_t s) {
  if (!t_begin) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, s);
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timed.emplace_back(t_begin, e);
  t_begin = nullptr;
}

DeviceContext* current_context() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  if (g_ctx[dev]) return g_ctx[dev];
  auto* c = new DeviceContext();
  c->device = dev;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  c->num_sms = prop.multiProcessorCount;
  c->cc_major = prop.major;
  c->cc_minor = prop.minor;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  c->tcgen05 = (prop.major == 10);   // sm_100 / sm_103 family: tcgen05, TMEM, TMA
  if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess || cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
    cudaFree(c->status);
    delete c;
    return nullptr;
  }
  uint64_t threshold = UINT64_MAX;
  cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  if (cudaStreamCreateWithFlags(&c->release, cudaStreamNonBlocking) != cudaSuccess) {
    cudaMemPoolDestroy(c->pool);
    cudaFree(c->status);
    delete c;
    return nullptr;
  }
  g_ctx[dev] = c;
  return c;
}

namespace {
thread_local ScratchArena* t_arena = nullptr;
}

void set_thread_arena(ScratchArena* arena) { t_arena = arena; }

namespace {
thread_local uint64_t t_wait_ns = kDefaultWaitNs;
}  // namespace
uint64_t thread_wait_limit() { return t_wait_ns; }
void set_thread_wait_limit(uint64_t ns) { t_wait_ns = ns; }

// Pool bytes this thread holds while a fit tracks them (host order of allocation and
// release, which is the order the stream reuses the memory in).
namespace {
struct PoolTrack {
  bool on = false;
  int64_t live = 0, peak = 0;
  std::unordered_map<void*, size_t> sizes;
};
thread_local PoolTrack t_track;
}  // namespace

void pool_track_begin() {
  t_track.on = true;
  t_track.live = t_track.peak = 0;
  t_track.sizes.clear();
}
int64_t pool_track_end() {
  t_track.on = false;
  t_track.sizes.clear();
  return t_track.peak;
}
void pool_track_add(void* p, size_t bytes) {
  if (!t_track.on || !p) return;
  t_track.sizes[p] = bytes;
  t_track.live += static_cast<int64_t>(bytes);
  t_track.peak = std::max(t_track.peak, t_track.live);
}
void pool_track_remove(void* p) {
  if (!t_track.on) return;
  auto it = t_track.sizes.find(p);
  if (it == t_track.sizes.end()) return;
  t_track.live -= static_cast<int64_t>(it->second);
  t_track.sizes.erase(it);
}

cudaError_t scratch_alloc(DeviceContext* ctx, void** p, size_t bytes, cudaStream_t s) {
  if (t_arena != nullptr) {
    const size_t off = align_up(t_arena->used, 256);
    if (off + bytes > t_arena->size) return cudaErrorMemoryAllocation;
    *p = t_arena->base + off;
    t_arena->used = off + bytes;
    return cudaSuccess;
  }
  const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, s);
  if (e == cudaSuccess) pool_track_add(*p, bytes);
  return e;
}

void scratch_free(void* p, cudaStream_t s) {
  if (t_arena != nullptr && static_cast<char*>(p) >= t_arena->base &&
      static_cast<char*>(p) < t_arena->base + t_arena->size)
    return;
  pool_track_remove(p);
  cudaFreeAsync(p, s);
}

namespace {

// mean = Y[:, :C]; var_c = s - sum_b Y[:, C + b C + c]^2; probs = softmax(mean / sqrt(1 + pi/8 var))
// probs: softmax -- probit-approximated class probabilities (App. C.3); Bernoulli --
// P(y = 1) by the same probit approximation; Poisson -- predictive mean count
// E[e^f] = e^(mean + var / 2); Gaussian -- the predictive mean of y.
// Prior variance per output: one outputscale per class, or the shared one (n == 0).
struct ClassScales {
  float s[64];
  int n;
};

__global__ void predict_epilogue_kernel(const float* __restrict__ Y, int64_t m, int C, int B,
                                        int64_t P, float s_shared, const ClassScales cs,
                                        float* __restrict__ mean, float* __restrict__ var,
                                        float* __restrict__ probs, int lik) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* yi = Y + i * P;
    float mx = -INFINITY;
    for (int c = 0; c < C; ++c) {
      mean[i * C + c] = yi[c];
      if (var || probs) {
        float acc = 0.f;
        for (int b = 0; b < B; ++b) {
          const float q = yi[C + b * C + c];
          acc = fmaf(q, q, acc);
        }
        const float vc = (cs.n ? cs.s[c] : s_shared) - acc;
        if (var) var[i * C + c] = vc;
        if (probs) {
          const float a = yi[c] / sqrtf(1.f + 0.39269908169872414f * vc);
          probs[i * C + c] = a;
          mx = fmaxf(mx, a);
        }
      }
    }
    if (probs && lik != ITERGP_LIK_SOFTMAX) {
      for (int c = 0; c < C; ++c) {
        float acc = 0.f;
        for (int b = 0; b < B; ++b) {
          const float q = yi[C + b * C + c];
          acc = fmaf(q, q, acc);
        }
        const float vc = (cs.n ? cs.s[c] : s_shared) - acc;
        if (lik == ITERGP_LIK_BERNOULLI)
          probs[i * C + c] = 1.f / (1.f + expf(-yi[c] / sqrtf(1.f + 0.39269908169872414f * vc)));
        else if (lik == ITERGP_LIK_POISSON)
          probs[i * C + c] = expf(yi[c] + 0.5f * vc);
        else
          probs[i * C + c] = yi[c];
      }
      continue;
    }
    if (probs) {
      float se = 0.f;
      for (int c = 0; c < C; ++c) {
        const float e = expf(probs[i * C + c] - mx);
        probs[i * C + c] = e;
        se += e;
      }
      for (int c = 0; c < C; ++c) probs[i * C + c] /= se;
    }
  }
}

// S_view[n][col]: col < C -> v[n][col]; col = C + b C + c -> Q[b][n][c]
// Deterministic pseudo-random fill (integer hash of the index; timing inputs only).
__global__ void fill_hash_kernel(float* __restrict__ x, int64_t n, uint32_t seed, float lo, float hi) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint32_t h = static_cast<uint32_t>(i) * 0x9E3779B1u ^ seed ^ static_cast<uint32_t>(i >> 32);
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    x[i] = lo + (hi - lo) * static_cast<float>(h >> 8) * (1.f / 16777216.f);
  }
}

__global__ void gather_vq_kernel(const float* __restrict__ v, const float* __restrict__ Q,
                                 int64_t n, int C, int B, float* __restrict__ out) {
  const int64_t P = static_cast<int64_t>(C) * (1 + B);
  const int64_t total = n * P;
  const int64_t nc = n * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / P, col = e % P;
    float x;
    if (col < C) {
      x = v[i * C + col];
    } else {
      const int64_t b = (col - C) / C, c = (col - C) % C;
      x = Q[b * nc + i * C + c];
    }
    out[e] = x;
  }
}

}  // namespace
}  // namespace itergp

using namespace itergp;

namespace itergp {

// An entry point reports only its own CUDA failures: a runtime error left on this thread
// by earlier, unrelated calls is cleared first (errors of the device are sticky and still
// surface through the next call that touches it).
void clear_stale_error() { (void)cudaGetLastError(); }

int validate_fit_params(const itergp_fit_params* prm) {
  if (!prm) return ITERGP_EINVAL;
  if (prm->n < 1 || prm->d < 1 || prm->d > 4096 || prm->c < 1 || prm->c > 64 || !prm->X)
    return ITERGP_EINVAL;
  switch (prm->likelihood) {
    case ITERGP_LIK_SOFTMAX:
      if (prm->c < 2 || !prm->y) return ITERGP_EINVAL;
      break;
    case ITERGP_LIK_BERNOULLI:
    case ITERGP_LIK_POISSON:
      if (prm->c != 1 || !prm->y) return ITERGP_EINVAL;
      break;
    case ITERGP_LIK_GAUSSIAN:
      if (!prm->y_real || !(prm->noise > 0.f) || !std::isfinite(prm->noise)) return ITERGP_EINVAL;
      break;
    default:
      return ITERGP_EINVAL;
  }
  if (!kernel_ok(&prm->kernel) || !precision_ok(prm->precision)) return ITERGP_EINVAL;
  if (prm->class_kernels)
    for (int c = 0; c < prm->c; ++c)
      if (!kernel_ok(&prm->class_kernels[c])) return ITERGP_EINVAL;
  if (prm->policy != ITERGP_POLICY_CG && prm->policy != ITERGP_POLICY_UNIT) return ITERGP_EINVAL;
  if (prm->max_newton < 1 || prm->max_iters < 0 || prm->max_newton > 100000) return ITERGP_EINVAL;
  if (!(prm->tol_abs >= 0) || !(prm->tol_rel >= 0)) return ITERGP_EINVAL;
  if (prm->wait_limit_ns != 0 && (prm->wait_limit_ns < 1000000ull || prm->wait_limit_ns > 60000000000ull))
    return ITERGP_EINVAL;
  return ITERGP_OK;
}

int64_t buffer_capacity(const itergp_fit_params& p) {
  const int64_t nc = p.n * p.c;
  int64_t bcap = static_cast<int64_t>(p.max_newton) * p.max_iters;
  if (p.recycle && p.rank >= 0) bcap = std::min<int64_t>(bcap, static_cast<int64_t>(p.rank) + p.max_iters);
  if (!p.recycle) bcap = std::min<int64_t>(bcap, p.max_iters);
  bcap = std::min<int64_t>(bcap, nc);
  return std::max<int64_t>(bcap, 1);
}

void model_release(itergp_model* m, cudaStream_t s) {
  if (!m) return;
  if (m->mem) cudaFreeAsync(m->mem, s);
  if (m->used) cudaEventDestroy(m->used);
  delete m;
}

void free_models(std::vector<itergp_model*>& ms, cudaStream_t s) {
  for (auto* m : ms) model_release(m, s);
  ms.clear();
}

// Fits params[0..count) with one schedule; on success fills models/reports.
int fit_many(const itergp_fit_params* params, int count, itergp_model** out,
             itergp_fit_report* reports, cudaStream_t s, bool batch) {
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  if (precision_is_tensor(params[0].precision) && !ctx->tcgen05) return ITERGP_EUNSUPPORTED;
  std::vector<itergp_model*> models(count, nullptr);
  std::vector<itergp_fit_report> reps(count);
  std::vector<int> finalB(count, 0);
  std::vector<int> status(count, ITERGP_OK);
  std::vector<FitProblem> probs(count);
  struct TrackGuard {   // the call's peak pool bytes: models, workspace and product scratch
    int64_t* peak;
    explicit TrackGuard(int64_t* p) : peak(p) { pool_track_begin(); }
    ~TrackGuard() { *peak = pool_track_end(); }
  };
  int64_t peak_bytes = 0;
  std::unique_ptr<TrackGuard> track(new TrackGuard(&peak_bytes));
  WaitLimitGuard wait_guard(params[0].wait_limit_ns);
  for (int i = 0; i < count; ++i) {
    const itergp_fit_params& prm = params[i];
    const int64_t n = prm.n, nc = n * prm.c;
    const int64_t bcap = buffer_capacity(prm);
    if (bcap > 512) {
      free_models(models, s);
      return ITERGP_EINVAL;
    }
    auto* mdl = new itergp_model();
    models[i] = mdl;
    mdl->device = ctx->device;
    mdl->n = n;
    mdl->d = prm.d;
    mdl->c = prm.c;
    mdl->bcap = static_cast<int>(bcap);
    mdl->kernel = prm.kernel;
    if (prm.class_kernels) mdl->class_kernels.assign(prm.class_kernels, prm.class_kernels + prm.c);
    mdl->precision = prm.precision;
    mdl->likelihood = prm.likelihood;
    if (cudaEventCreateWithFlags(&mdl->used, cudaEventDisableTiming) != cudaSuccess) mdl->used = nullptr;
    const size_t xb = align_up(sizeof(float) * n * prm.d, 256);
    const size_t rb = rows_workspace_bytes(prm.precision, n, static_cast<int>(prm.d));
    const size_t vb = align_up(sizeof(float) * nc, 256);
    const size_t qb = align_up(sizeof(float) * nc * bcap, 256);
    mdl->bytes = static_cast<int64_t>(xb + rb + 2 * vb + qb);
    if (cudaMallocFromPoolAsync(&mdl->mem, mdl->bytes, ctx->pool, s) != cudaSuccess) {
      mdl->mem = nullptr;
      free_models(models, s);
      return ITERGP_ENOMEM;
    }
    pool_track_add(mdl->mem, static_cast<size_t>(mdl->bytes));
    char* base = static_cast<char*>(mdl->mem);
    mdl->X = reinterpret_cast<float*>(base);
    mdl->v = reinterpret_cast<float*>(base + xb + rb);
    mdl->f = reinterpret_cast<float*>(base + xb + rb + vb);
    mdl->Q = reinterpret_cast<float*>(base + xb + rb + 2 * vb);
    int rc = ITERGP_OK;
    if (cudaMemcpyAsync(mdl->X, prm.X, sizeof(float) * n * prm.d, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      rc = ITERGP_ECUDA;
    if (rc == ITERGP_OK)
      rc = prepare_rows(prm.precision, mdl->X, n, static_cast<int>(prm.d), prm.d, base + xb, &mdl->xop, s);
    if (rc != ITERGP_OK) {
      free_models(models, s);
      return rc;
    }
    FitProblem& fp = probs[i];
    fp.prm = &prm;
    fp.kp = make_kparams(prm.kernel);
    for (const itergp_kernel& kc : mdl->class_kernels) fp.class_kp.push_back(make_kparams(kc));
    fp.xop = &mdl->xop;
    fp.v = mdl->v;
    fp.f = mdl->f;
    fp.Q = mdl->Q;
    fp.bcap = static_cast<int>(bcap);
    fp.rep = &reps[i];
    fp.final_B = &finalB[i];
    fp.status = &status[i];
  }
  // fit_run_batch waits for the stream and reports the fit's own errors (device errors of
  // single problems in `status`, wait limits in its return value)
  const int rc = fit_run_batch(ctx, probs, s, params[0].graph != 0);
  if (rc != ITERGP_OK) {
    cudaStreamSynchronize(s);
    free_models(models, s);
    return rc;
  }
  if (!batch && status[0] != ITERGP_OK) {
    free_models(models, s);
    return status[0];
  }
  track.reset();   // ends the tracking: peak_bytes holds the call's peak
  for (int i = 0; i < count; ++i) {
    reps[i].device_bytes = status[i] == ITERGP_OK ? models[i]->bytes : 0;
    reps[i].peak_bytes = peak_bytes;
    if (reports) reports[i] = reps[i];
    if (status[i] != ITERGP_OK) {   // this problem failed alone; the others stand
      model_release(models[i], s);
      out[i] = nullptr;
      continue;
    }
    models[i]->B = finalB[i];
    if (models[i]->used) cudaEventRecord(models[i]->used, s);
    out[i] = models[i];
  }
  return ITERGP_OK;
}


}  // namespace itergp


extern "C" {

const char* itergp_version(void) { return "0.1.0"; }

const char* itergp_last_error(void) { return t_last_error; }

int itergp_timing_enable(int enable) {
  g_timing.store(enable != 0);
  return ITERGP_OK;
}

int itergp_timing_read(double* kernel_ms, int64_t* launches) {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    ev.swap(g_timed);
  }
  double total = 0.0;
  int rc = ITERGP_OK;
  for (auto& pr : ev) {
    float ms = 0.f;
    if (cudaEventSynchronize(pr.second) != cudaSuccess ||
        cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess)
      rc = ITERGP_ECUDA;
    total += ms;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  if (kernel_ms) *kernel_ms = total;
  if (launches) *launches = static_cast<int64_t>(ev.size());
  return rc;
}

int64_t itergp_launch_count(void) { return g_launches.load(); }

const char* itergp_status_string(int status) {
  switch (status) {
    case ITERGP_OK: return "ok";
    case ITERGP_EINVAL: return "invalid argument";
    case ITERGP_ENOMEM: return "out of device memory";
    case ITERGP_ECUDA: return "CUDA runtime error";
    case ITERGP_ENUMERIC: return "non-finite value on the device";
    case ITERGP_ETIMEOUT: return "device-side wait exceeded its bound";
    case ITERGP_EUNSUPPORTED: return "unsupported device (needs sm_100 family / sm_103a)";
    case ITERGP_ESCRATCH: return "problem needs more scratch than the fixed static buffer holds";
    case ITERGP_EGONE: return "model not resident (evicted, released or failed)";
    default: return "unknown status";
  }
}

int itergp_sync_status(itergp_stream stream) {
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ITERGP_CUDA_TRY(cudaStreamSynchronize(s));
  int h = 0;
  ITERGP_CUDA_TRY(cudaMemcpy(&h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
  ITERGP_CUDA_TRY(cudaMemset(ctx->status, 0, sizeof(int)));
  return h;
}

int itergp_kmatvec(const itergp_kernel* kernel, int32_t precision, const float* A, int64_t m,
                   const float* B, int64_t n, int64_t d, const float* S, int64_t p, float* Y,
                   itergp_stream stream) {
  clear_stale_error();
  if (!kernel_ok(kernel) || !precision_ok(precision)) return ITERGP_EINVAL;
  if (m < 0 || n < 0 || p < 0 || d < 1 || d > 4096 || p > 65536) return ITERGP_EINVAL;
  if (m == 0 || p == 0) return ITERGP_OK;
  if (!Y || (n > 0 && (!A || !B || !S))) return ITERGP_EINVAL;
  if (n > 0 && m > 0 && !A) return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  if (precision_is_tensor(precision) && !ctx->tcgen05) return ITERGP_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const KParams kp = make_kparams(*kernel);
  const bool same = (A == B) && (m == n);
  const size_t ba = rows_workspace_bytes(precision, m, static_cast<int>(d));
  const size_t bb = same ? 0 : rows_workspace_bytes(precision, n, static_cast<int>(d));
  Scratch ws;
  ITERGP_CUDA_TRY(ws.alloc(ctx, ba + bb, s));
  RowOperand opA, opB;
  int rc = prepare_rows(precision, A, m, static_cast<int>(d), d, ws.as<void>(), &opA, s);
  if (rc != ITERGP_OK) return rc;
  if (same) {
    opB = opA;
  } else {
    rc = prepare_rows(precision, B, n, static_cast<int>(d), d, ws.as<char>(ba), &opB, s);
    if (rc != ITERGP_OK) return rc;
  }
  return kmv_execute(ctx, kp, opA, opB, S, p, p, Y, p, s, nullptr);
}

int itergp_kmatvec_classes(const itergp_kernel* kernels, int32_t c, int32_t precision, const float* A,
                           int64_t m, const float* B, int64_t n, int64_t d, const float* S, int64_t p,
                           float* Y, itergp_stream stream) {
  clear_stale_error();
  if (!kernels || c < 1 || c > 64 || !precision_ok(precision)) return ITERGP_EINVAL;
  for (int k = 0; k < c; ++k)
    if (!kernel_ok(&kernels[k])) return ITERGP_EINVAL;
  if (m < 0 || n < 0 || p < 0 || d < 1 || d > 4096 || p > 65536) return ITERGP_EINVAL;
  if (m == 0 || p == 0) return ITERGP_OK;
  if (!Y || !A || (n > 0 && (!B || !S))) return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  if (precision_is_tensor(precision) && !ctx->tcgen05) return ITERGP_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<KParams> kps;
  for (int k = 0; k < c; ++k) kps.push_back(make_kparams(kernels[k]));
  const bool same = (A == B) && (m == n);
  const size_t ba = rows_workspace_bytes(precision, m, static_cast<int>(d));
  const size_t bb = same ? 0 : rows_workspace_bytes(precision, n, static_cast<int>(d));
  Scratch ws;
  ITERGP_CUDA_TRY(ws.alloc(ctx, ba + bb, s));
  RowOperand opA, opB;
  int rc = prepare_rows(precision, A, m, static_cast<int>(d), d, ws.as<void>(), &opA, s);
  if (rc != ITERGP_OK) return rc;
  if (same) {
    opB = opA;
  } else {
    rc = prepare_rows(precision, B, n, static_cast<int>(d), d, ws.as<char>(ba), &opB, s);
    if (rc != ITERGP_OK) return rc;
  }
  return kmv_classes(ctx, kps.data(), c, opA, opB, S, p, p, Y, p, s, nullptr);
}

int itergp_winv_apply(const float* f, int64_t n, int32_t c, const float* x, float* out,
                      itergp_stream stream) {
  clear_stale_error();
  if (n < 0 || c < 2 || c > 64) return ITERGP_EINVAL;
  if (n > 0 && (!f || !x || !out)) return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  return winv_apply_launch(ctx, f, n, c, x, out, static_cast<cudaStream_t>(stream));
}

int itergp_pseudo_targets(const float* f, const int32_t* y, int64_t n, int32_t c, float* out,
                          itergp_stream stream) {
  clear_stale_error();
  if (n < 0 || c < 2 || c > 64) return ITERGP_EINVAL;
  if (n > 0 && (!f || !y || !out)) return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  return pseudo_targets_launch(ctx, f, y, n, c, out, static_cast<cudaStream_t>(stream));
}

int itergp_sym_eig(const double* M, int32_t b, double* lam, double* U, itergp_stream stream) {
  clear_stale_error();
  if (b < 1 || b > 512 || !M || !lam || !U) return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  return sym_eig_launch(ctx, M, b, lam, U, static_cast<cudaStream_t>(stream));
}


int itergp_fit(const itergp_fit_params* prm, itergp_model** out, itergp_fit_report* report,
               itergp_stream stream) {
  clear_stale_error();
  if (!prm || !out) return ITERGP_EINVAL;
  *out = nullptr;
  const int rc = validate_fit_params(prm);
  if (rc != ITERGP_OK) return rc;
  return fit_many(prm, 1, out, report, static_cast<cudaStream_t>(stream), false);
}

int itergp_fit_batch(const itergp_fit_params* params, int32_t count, itergp_model** models,
                     itergp_fit_report* reports, itergp_stream stream) {
  clear_stale_error();
  if (!params || !models || count < 1 || count > 65535) return ITERGP_EINVAL;
  for (int i = 0; i < count; ++i) models[i] = nullptr;
  const itergp_fit_params& a = params[0];
  for (int i = 0; i < count; ++i) {
    const int rc = validate_fit_params(&params[i]);
    if (rc != ITERGP_OK) return rc;
    const itergp_fit_params& b = params[i];
    if (b.kernel.kind != a.kernel.kind || b.precision != a.precision || b.policy != a.policy ||
        b.max_newton != a.max_newton || b.max_iters != a.max_iters || b.rank != a.rank ||
        b.recycle != a.recycle || b.literal_kv != 0 || b.tol_newton != a.tol_newton ||
        b.tol_abs != a.tol_abs || b.tol_rel != a.tol_rel || b.graph != a.graph ||
        b.likelihood != a.likelihood)
      return ITERGP_EINVAL;
  }
  bool per_class = false;
  for (int i = 0; i < count; ++i) per_class = per_class || params[i].class_kernels != nullptr;
  if (!per_class) return fit_many(params, count, models, reports, static_cast<cudaStream_t>(stream), true);
  // grouped per-class products do not share a launch across problems: one fit each, with
  // the batched call's per-problem error semantics
  for (int i = 0; i < count; ++i) {
    itergp_fit_report rep{};
    const int rc = fit_many(&params[i], 1, &models[i], &rep, static_cast<cudaStream_t>(stream), false);
    if (rc == ITERGP_ECUDA || rc == ITERGP_ENOMEM || rc == ITERGP_ETIMEOUT) {
      for (int k = 0; k < i; ++k) {
        itergp_model_free(models[k]);
        models[k] = nullptr;
      }
      return rc;
    }
    if (rc != ITERGP_OK) {
      models[i] = nullptr;
      rep.status = rc;
    }
    if (reports) reports[i] = rep;
  }
  return ITERGP_OK;
}

int itergp_predict(const itergp_model* mdl, const float* Xs, int64_t m, float* mean, float* var,
                   float* probs, itergp_stream stream) {
  clear_stale_error();
  if (!mdl || m < 0 || (m > 0 && (!Xs || !mean))) return ITERGP_EINVAL;
  if (m == 0) return ITERGP_OK;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  if (ctx->device != mdl->device) return ITERGP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int C = mdl->c;
  const int B = (var || probs) ? mdl->B : 0;
  const int64_t P = static_cast<int64_t>(C) * (1 + B);
  const size_t rb = rows_workspace_bytes(mdl->precision, m, static_cast<int>(mdl->d));
  const size_t sb = align_up(sizeof(float) * mdl->n * P, 256);
  const size_t yb = align_up(sizeof(float) * m * P, 256);
  Scratch ws;
  ITERGP_CUDA_TRY(ws.alloc(ctx, rb + sb + yb, s));
  RowOperand op;
  int rc = prepare_rows(mdl->precision, Xs, m, static_cast<int>(mdl->d), mdl->d, ws.as<void>(), &op, s);
  if (rc != ITERGP_OK) return rc;
  float* Sv = ws.as<float>(rb);
  float* Y = ws.as<float>(rb + sb);
  {
    const int64_t total = mdl->n * P;
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(ceil_div(total, 256), 8LL * ctx->num_sms));
    gather_vq_kernel<<<blocks, 256, 0, s>>>(mdl->v, mdl->Q, mdl->n, C, B, Sv), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
  }
  // [v | Q] columns of class c are c, c + C, ... (CN ordering): with one kernel per class
  // the product runs as C grouped products
  ClassScales cs{};
  if (!mdl->class_kernels.empty()) {
    std::vector<KParams> kps;
    for (const itergp_kernel& kc : mdl->class_kernels) kps.push_back(make_kparams(kc));
    for (int c = 0; c < C; ++c) cs.s[c] = mdl->class_kernels[c].outputscale;
    cs.n = C;
    rc = kmv_classes(ctx, kps.data(), C, op, mdl->xop, Sv, P, P, Y, P, s, nullptr);
  } else {
    rc = kmv_execute(ctx, make_kparams(mdl->kernel), op, mdl->xop, Sv, P, P, Y, P, s, nullptr);
  }
  if (rc != ITERGP_OK) return rc;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(ceil_div(m, 256), 8LL * ctx->num_sms));
  predict_epilogue_kernel<<<blocks, 256, 0, s>>>(Y, m, C, B, P, mdl->kernel.outputscale, cs, mean, var, probs,
                                                 mdl->likelihood), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  if (mdl->used) ITERGP_CUDA_TRY(cudaEventRecord(mdl->used, s));   // the model's last use
  return ITERGP_OK;
}

int itergp_selftest_wait(uint64_t limit_ns, itergp_stream stream) {
  clear_stale_error();
  if (limit_ns < 100000u || limit_ns > 5000000000ull) return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  return wait_selftest_launch(ctx, limit_ns, static_cast<cudaStream_t>(stream));
}

int itergp_autotune(const itergp_kernel* kernel, int32_t precision, int64_t n, int64_t d, int64_t p,
                    int32_t items, itergp_tune_result* result, itergp_stream stream) {
  clear_stale_error();
  if (!kernel_ok(kernel) || !result || !precision_is_tensor(precision) || n < 128 || n > (int64_t(1) << 26) ||
      d < 1 || d > 4096 || p < 1 || p > (items ? 128 : 4096))
    return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  if (!ctx->tcgen05) return ITERGP_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bx = align_up(sizeof(float) * n * d, 256), bs = align_up(sizeof(float) * n * p, 256);
  const size_t br = rows_workspace_bytes(precision, n, static_cast<int>(d));
  Scratch ws;
  ITERGP_CUDA_TRY(ws.alloc(ctx, bx + 2 * bs + br, s));
  float* X = ws.as<float>();
  float* S = ws.as<float>(bx);
  float* Y = ws.as<float>(bx + bs);
  const unsigned blocks = static_cast<unsigned>(8 * ctx->num_sms);
  fill_hash_kernel<<<blocks, 256, 0, s>>>(X, n * d, 0x1234u, 0.f, 1.f), ::itergp::note_launch();
  fill_hash_kernel<<<blocks, 256, 0, s>>>(S, n * p, 0x9876u, -1.f, 1.f), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  RowOperand op;
  int rc = prepare_rows(precision, X, n, static_cast<int>(d), d, ws.as<char>(bx + 2 * bs), &op, s);
  if (rc != ITERGP_OK) return rc;
  int count = 0, best = -1, epi[ITERGP_TUNE_MAX], ns[ITERGP_TUNE_MAX], pr[ITERGP_TUNE_MAX];
  double ms[ITERGP_TUNE_MAX];
  rc = kmv_tc_tune(ctx, make_kparams(*kernel), op, S, p, Y, items ? 1 : 0, ITERGP_TUNE_MAX, &count, epi,
                   ns, pr, ms, &best, s);
  if (rc != ITERGP_OK) return rc;
  result->count = count;
  result->best = best;
  for (int i = 0; i < count; ++i) {
    result->variants[i].epilogue_warps = epi[i];
    result->variants[i].stages = ns[i];
    result->variants[i].cta_pair = pr[i];
    result->variants[i].ms = ms[i];
  }
  return ITERGP_OK;
}

int itergp_model_get_view(const itergp_model* mdl, itergp_model_view* view) {
  if (!mdl || !view) return ITERGP_EINVAL;
  view->n = mdl->n;
  view->d = mdl->d;
  view->c = mdl->c;
  view->buffer_cols = mdl->B;
  view->kernel = mdl->kernel;
  view->X = mdl->X;
  view->v = mdl->v;
  view->f = mdl->f;
  view->Q = mdl->Q;
  return ITERGP_OK;
}

void itergp_model_free(itergp_model* mdl) {
  if (!mdl) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != mdl->device) cudaSetDevice(mdl->device);
  // wait for the model's last fit or predict (an event recorded there), then free on the
  // library's own non-blocking stream: no device-wide synchronisation, no legacy stream
  // (either would break a stream capture that another thread has open)
  if (mdl->used) {
    cudaEventSynchronize(mdl->used);
    cudaEventDestroy(mdl->used);
  }
  DeviceContext* ctx = current_context();
  cudaStream_t rs = ctx ? ctx->release : nullptr;
  if (mdl->mem) {
    cudaFreeAsync(mdl->mem, rs);
    cudaStreamSynchronize(rs);
  }
  if (prev >= 0 && prev != mdl->device) cudaSetDevice(prev);
  delete mdl;
}

}  // extern "C"
