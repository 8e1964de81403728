// Serving: fits and predictive queries over many resident models with continuous batching.
//
// One server owns a slab of device memory for resident models and two host threads, each
// with its own stream:
//  - the fit thread admits the fits waiting when it frees up (arrival order, while the
//    slab and the work budget allow; idle models are evicted least recently used first),
//    runs them as one batched fit (every phase of Alg. 1-3 one launch over the batch) and
//    installs each model in the slab: prepared rows of X and the weights [v | Q];
//  - the predict thread admits the predicts waiting when it frees up, across models, and
//    answers them with one batched product per part, mean = K(X*, X) v and the variance
//    term K(X*, X) Q (Eqs. 9-10 with C_j = Q Q^T), then one epilogue with the probit
//    approximation (App. C.3).
// Predicts run while fits are on the GPU; both share the slab, which only the fit thread
// writes (rows of a model are written before it becomes visible to predicts and freed
// only when no predict uses it).
//
// Slab layout (rows in 128-row blocks, one block range per model):
//  tensor precisions: 16-bit hi (and lo) rows [slab_rows][d_pad], FP32 norms [slab_rows],
//                     split rows: tile scales [slab_rows / 128],
//                     weights transposed [144][slab_rows]: FP16 hi and lo with per-model
//                     column scales (BF16X3, TF32), one BF16 plane otherwise;
//  FP32:              FP32 rows [slab_rows][d_max], norms, weights [slab_rows][144].
// Weight row w of a model: w < 16: v[:, w] (zero for w >= C); w >= 16: column
// (w - 16) = b C + c of Q, i.e. Q_b[:, c] (zero beyond C B).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_fp16.h>

#include "internal.h"

namespace itergp {
namespace {

constexpr int kMeanRows = 16;    // weight rows holding v (C <= 16)
constexpr int kVarRows = 128;    // weight rows holding Q (C B <= 128)
constexpr int kWeightRows = kMeanRows + kVarRows;

// ------------------------------------------------------------------ install kernels
// FP32 rows of a model into the slab (pitch d_max), zero beyond d and beyond n.
__global__ void slab_rows32_kernel(const float* __restrict__ X, int64_t n, int d, int64_t rows_pad,
                                   int d_max, float* __restrict__ out) {
  const int64_t total = rows_pad * d_max;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / d_max;
    const int col = static_cast<int>(e % d_max);
    out[e] = (r < n && col < d) ? X[r * d + col] : 0.f;
  }
}

__device__ __forceinline__ float weight_value(const float* __restrict__ v, const float* __restrict__ Q,
                                              int64_t n, int C, int B, int64_t r, int w) {
  if (r >= n) return 0.f;
  if (w < kMeanRows) return w < C ? v[r * C + w] : 0.f;
  const int col = w - kMeanRows;
  if (col >= C * B) return 0.f;
  const int b = col / C, c = col % C;
  return Q[static_cast<int64_t>(b) * n * C + r * C + c];
}

// Largest |weight| of each of a model's weight rows (columns of [v | Q]), as float bits,
// into wmax [kWeightRows] (zeroed by the caller): a shared maximum per row and block, then
// one atomicMax per row and block.
__global__ void slab_wmax_kernel(const float* __restrict__ v, const float* __restrict__ Q, int64_t n, int C,
                                 int B, uint32_t* __restrict__ wmax) {
  __shared__ uint32_t m[kWeightRows];
  for (int w = threadIdx.x; w < kWeightRows; w += blockDim.x) m[w] = 0u;
  __syncthreads();
  const int64_t total = n * kWeightRows;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int w = static_cast<int>(e % kWeightRows);
    atomicMax(&m[w], __float_as_uint(fabsf(weight_value(v, Q, n, C, B, e / kWeightRows, w))));
  }
  __syncthreads();
  for (int w = threadIdx.x; w < kWeightRows; w += blockDim.x)
    if (m[w] != 0u) atomicMax(&wmax[w], m[w]);
}

// Weights of a model, transposed [kWeightRows][slab_rows].  SPLIT (BF16X3, TF32): FP16 hi
// and lo of 2^e_w times weight row w, e_w from its maximum (wmax) so that it lies in
// [128, 256), scales 2^-e_w into wscale [kWeightRows]; otherwise one BF16 plane.
template <bool SPLIT>
__global__ void slab_weights_tc_kernel(const float* __restrict__ v, const float* __restrict__ Q,
                                       int64_t n, int C, int B, int64_t rows_pad, int64_t row0,
                                       int64_t slab_rows, __nv_bfloat16* __restrict__ hi,
                                       __nv_bfloat16* __restrict__ lo, const uint32_t* __restrict__ wmax,
                                       float* __restrict__ wscale) {
  const int64_t total = rows_pad * kWeightRows;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int w = static_cast<int>(e / rows_pad);
    const int64_t r = e % rows_pad;
    const float x = weight_value(v, Q, n, C, B, r, w);
    if constexpr (SPLIT) {
      const int ex = scale_exp_of_max(wmax[w]);
      const float xs = x * pow2i(ex);
      const __half h = __float2half_rn(xs);
      reinterpret_cast<__half*>(hi)[w * slab_rows + row0 + r] = h;
      reinterpret_cast<__half*>(lo)[w * slab_rows + row0 + r] = __float2half_rn(xs - __half2float(h));
      if (r == 0) wscale[w] = pow2i(-ex);
    } else {
      hi[w * slab_rows + row0 + r] = __float2bfloat16_rn(x);
    }
  }
}

// Weights of a model, FP32 [slab_rows][kWeightRows].
__global__ void slab_weights32_kernel(const float* __restrict__ v, const float* __restrict__ Q,
                                      int64_t n, int C, int B, int64_t rows_pad,
                                      float* __restrict__ out) {
  const int64_t total = rows_pad * kWeightRows;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[e] = weight_value(v, Q, n, C, B, e / kWeightRows, static_cast<int>(e % kWeightRows));
}

// ------------------------------------------------------------------ predict epilogue
struct PredDesc {
  const float* y;    // [m][144]: columns 0..C-1 K(X*, X) v, columns 16 + b C + c K(X*, X) Q_b
  float* out;        // [3][m][C]: mean, variance, probabilities
  int64_t m;
  int32_t c, b;
  float s;
  int32_t pad;
};

// Eqs. 9-10 with C_j = Q Q^T: var_c = s - sum_b ((K(X*, X) Q_b)_c)^2; probit probabilities
// softmax(mean / sqrt(1 + pi var / 8)) (App. C.3).
__global__ void serve_epilogue_kernel(const PredDesc* __restrict__ descs) {
  const PredDesc q = descs[blockIdx.y];
  const int C = q.c;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < q.m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float* mean = q.out + i * C;
    float* var = q.out + q.m * C + i * C;
    float* probs = q.out + 2 * q.m * C + i * C;
    float mx = -INFINITY;
    for (int c = 0; c < C; ++c) {
      const float mu = q.y[i * kWeightRows + c];
      float acc = 0.f;
      for (int b = 0; b < q.b; ++b) {
        const float t = q.y[i * kWeightRows + kMeanRows + b * C + c];
        acc = fmaf(t, t, acc);
      }
      const float vc = q.s - acc;
      mean[c] = mu;
      var[c] = vc;
      const float a = mu / sqrtf(1.f + 0.39269908169872414f * vc);
      probs[c] = a;
      mx = fmaxf(mx, a);
    }
    float se = 0.f;
    for (int c = 0; c < C; ++c) {
      const float e = expf(probs[c] - mx);
      probs[c] = e;
      se += e;
    }
    for (int c = 0; c < C; ++c) probs[c] /= se;
  }
}

// ------------------------------------------------------------------ host side
// First-fit allocator of row ranges of the slab (multiples of 128 rows).
class RowBlocks {
 public:
  void init(int64_t total) {
    free_.clear();
    if (total > 0) free_[0] = total;
    used_ = 0;
  }
  int64_t alloc(int64_t rows) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < rows) continue;
      const int64_t start = it->first, len = it->second;
      free_.erase(it);
      if (len > rows) free_[start + rows] = len - rows;
      used_ += rows;
      return start;
    }
    return -1;
  }
  void release(int64_t start, int64_t rows) {
    used_ -= rows;
    auto it = free_.emplace(start, rows).first;
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
  int64_t used() const { return used_; }

 private:
  std::map<int64_t, int64_t> free_;
  int64_t used_ = 0;
};

// Pinned host staging that grows geometrically.
struct Pinned {
  char* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t bytes) {
    if (bytes <= cap) return true;
    size_t want = std::max(bytes, cap * 2);
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&p), want, cudaHostAllocDefault) != cudaSuccess) return false;
    cap = want;
    return true;
  }
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

struct Resident {
  int64_t n = 0;
  int d = 0, c = 0, B = 0;
  KParams kp{};
  float outputscale = 1.f;
  int64_t row0 = -1, rows_pad = 0;
  uint64_t last_use = 0;
  bool release_requested = false;
};

struct FitReq {
  int64_t id = 0;
  double t_submit = 0;
  std::vector<float> X;
  std::vector<int32_t> y;
  int64_t n = 0;
  int d = 0, c = 0;
  float ell = 1.f, s = 1.f;
  int64_t row0 = -1, rows_pad = 0;
  size_t work = 0;
};

struct PredReq {
  int64_t id = 0, model = 0;
  double t_submit = 0;
  std::vector<float> Xs;
  int64_t m = 0;
  int d = 0;
  float *mean = nullptr, *var = nullptr, *probs = nullptr;
};

int64_t round128(int64_t n) { return (n + 127) / 128 * 128; }

}  // namespace
}  // namespace itergp

using namespace itergp;

struct itergp_server {
  itergp_server_config cfg{};
  int device = 0;
  DeviceContext* ctx = nullptr;
  cudaStream_t fit_stream = nullptr, pred_stream = nullptr;
  std::chrono::steady_clock::time_point t0;
  // slab
  void* slab = nullptr;
  int64_t slab_rows = 0;
  int d_pad = 0;
  int bcap = 0;
  RowOperand rows_op;                 // problem side of the predict products (rows = slab)
  __nv_bfloat16 *w_hi = nullptr, *w_lo = nullptr;
  uint32_t* w_max = nullptr;          // split weights: scratch of an install [kWeightRows]
  float* w_scale = nullptr;           // split weights: per 128-row block [slab_rows / 128][kWeightRows]
  float* w32 = nullptr;
  RowBlocks blocks;
  // state (guarded by mu)
  std::mutex mu;
  std::condition_variable cv_fit, cv_pred, cv_events;
  std::deque<FitReq*> fit_q;
  std::deque<PredReq*> pred_q;
  std::map<int64_t, Resident> resident;
  std::map<int64_t, int> in_fit;      // queued or running fits (id -> 1)
  std::map<int64_t, int> gone;        // id -> status (failed fit, evicted, released)
  std::map<int64_t, int> pending;     // id -> predicts queued or running
  std::map<int64_t, int> dims;        // id -> input dimension of every model submitted
  std::deque<itergp_server_event> events;
  itergp_server_stats stats{};
  uint64_t tick = 0;
  int64_t next_id = 1;
  bool stop = false;
  std::thread fit_thr, pred_thr;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  bool tensor() const { return precision_is_tensor(cfg.precision); }

  // workspace bytes of one fit in flight (model + fit workspace + staging), an upper bound
  size_t fit_work_bytes(int64_t n, int d, int c) const {
    const int64_t nc = n * c;
    const size_t model = sizeof(float) * (n * d + 2 * nc + nc * bcap) +
                         rows_workspace_bytes(cfg.precision, n, d) + 4096;
    const size_t work = sizeof(float) * (3 * nc * bcap + 12 * nc) +
                        static_cast<size_t>(bcap) * bcap * (4 + 8 + 8) + sizeof(double) * 64 * bcap * bcap;
    const size_t arena = sizeof(float) * round128(n) * cfg.d_max +
                         rows_workspace_bytes(cfg.precision, n, cfg.d_max) +
                         sizeof(__nv_bfloat16) * 2 * 16 * round128(n) + sizeof(float) * round128(n) * 16;
    return model + work + arena + sizeof(float) * n * d + sizeof(int32_t) * n + (1 << 20);
  }

  void push_event(int64_t id, int64_t model, int kind, int status, double t_submit, double t_start,
                  int batch) {
    itergp_server_event e{};
    e.id = id;
    e.model = model;
    e.kind = kind;
    e.status = status;
    e.submit_s = t_submit;
    e.start_s = t_start;
    e.done_s = now();
    e.batch = batch;
    events.push_back(e);
  }

  // Evicts the least recently used resident model without queued predicts; false if none.
  bool evict_one() {
    auto victim = resident.end();
    for (auto it = resident.begin(); it != resident.end(); ++it) {
      auto p = pending.find(it->first);
      if (p != pending.end() && p->second > 0) continue;
      if (victim == resident.end() || it->second.last_use < victim->second.last_use) victim = it;
    }
    if (victim == resident.end()) return false;
    blocks.release(victim->second.row0, victim->second.rows_pad);
    gone[victim->first] = ITERGP_EGONE;
    resident.erase(victim);
    ++stats.evicted;
    return true;
  }

  // ---------------------------------------------------------------- fit thread
  void fit_loop();
  void run_fits(std::vector<FitReq*>& batch);
  int install(itergp_model* m, const FitReq& r);
  // ---------------------------------------------------------------- predict thread
  void pred_loop();
  void run_predicts(std::vector<PredReq*>& batch, const std::vector<Resident>& models,
                    std::vector<int>* status, double* t_start);
  Pinned fit_pin, pred_pin, pred_out_pin;
};

void itergp_server::fit_loop() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<FitReq*> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_fit.wait(lk, [&] { return stop || !fit_q.empty(); });
      if (fit_q.empty()) break;   // stop requested and nothing left
      size_t work = 0;
      while (!fit_q.empty() && static_cast<int>(batch.size()) < cfg.max_fit_batch) {
        FitReq* r = fit_q.front();
        if (r->work > static_cast<size_t>(cfg.work_bytes) || r->rows_pad > slab_rows) {
          fit_q.pop_front();
          in_fit.erase(r->id);
          gone[r->id] = ITERGP_ENOMEM;
          push_event(r->id, r->id, ITERGP_REQ_FIT, ITERGP_ENOMEM, r->t_submit, now(), 0);
          delete r;
          continue;
        }
        if (!batch.empty() && work + r->work > static_cast<size_t>(cfg.work_bytes)) break;
        int64_t row0 = blocks.alloc(r->rows_pad);
        while (row0 < 0 && evict_one()) row0 = blocks.alloc(r->rows_pad);
        if (row0 < 0) break;   // rows free up when predicts on resident models finish
        r->row0 = row0;
        work += r->work;
        batch.push_back(r);
        fit_q.pop_front();
      }
      stats.queued_fits = static_cast<int64_t>(fit_q.size());
      if (batch.empty()) {
        cv_events.notify_all();
        cv_fit.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    run_fits(batch);
  }
}

int itergp_server::install(itergp_model* m, const FitReq& r) {
  const int64_t n = m->n;
  const int64_t rows_pad = r.rows_pad;
  cudaStream_t s = fit_stream;
  const unsigned blocks_rows = static_cast<unsigned>(std::min<int64_t>(ceil_div(rows_pad * kWeightRows, 256), 4096));
  if (tensor()) {
    __nv_bfloat16* lo = precision_splits_rows(cfg.precision)
                            ? const_cast<__nv_bfloat16*>(rows_op.lo) + r.row0 * d_pad : nullptr;
    // TF32 rows are FP32 values: the block starts r.row0 rows of 4-byte elements in
    __nv_bfloat16* hi = precision_tf32_rows(cfg.precision)
                            ? reinterpret_cast<__nv_bfloat16*>(
                                  const_cast<float*>(reinterpret_cast<const float*>(rows_op.hi)) + r.row0 * d_pad)
                            : const_cast<__nv_bfloat16*>(rows_op.hi) + r.row0 * d_pad;
    float* ts = rows_op.tscale ? const_cast<float*>(rows_op.tscale) + r.row0 / kRowTile : nullptr;
    int rc = prepare_rows_into(cfg.precision, m->X, n, static_cast<int>(m->d), m->d, rows_pad, d_pad,
                               hi, lo, const_cast<float*>(rows_op.norms) + r.row0, ts, s);
    if (rc != ITERGP_OK) return rc;
    if (precision_splits_weights(cfg.precision)) {
      ITERGP_CUDA_TRY(cudaMemsetAsync(w_max, 0, sizeof(uint32_t) * kWeightRows, s));
      const unsigned blocks_max = static_cast<unsigned>(std::min<int64_t>(ceil_div(n * kWeightRows, 256), 1024));
      slab_wmax_kernel<<<blocks_max, 256, 0, s>>>(m->v, m->Q, n, m->c, m->B, w_max), ::itergp::note_launch();
      slab_weights_tc_kernel<true><<<blocks_rows, 256, 0, s>>>(m->v, m->Q, n, m->c, m->B, rows_pad, r.row0,
                                                              slab_rows, w_hi, w_lo, w_max,
                                                              w_scale + (r.row0 / 128) * kWeightRows),
          ::itergp::note_launch();
    } else {
      slab_weights_tc_kernel<false><<<blocks_rows, 256, 0, s>>>(m->v, m->Q, n, m->c, m->B, rows_pad, r.row0,
                                                               slab_rows, w_hi, w_lo, nullptr, nullptr),
          ::itergp::note_launch();
    }
    ITERGP_CUDA_TRY(cudaGetLastError());
  } else {
    float* x32 = const_cast<float*>(rows_op.X) + r.row0 * cfg.d_max;
    const unsigned b2 = static_cast<unsigned>(std::min<int64_t>(ceil_div(rows_pad * cfg.d_max, 256), 4096));
    slab_rows32_kernel<<<b2, 256, 0, s>>>(m->X, n, static_cast<int>(m->d), rows_pad, cfg.d_max, x32), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
    int rc = prepare_rows_into(ITERGP_FP32, x32, rows_pad, cfg.d_max, cfg.d_max, rows_pad, cfg.d_max,
                               nullptr, nullptr, const_cast<float*>(rows_op.norms) + r.row0, nullptr, s);
    if (rc != ITERGP_OK) return rc;
    slab_weights32_kernel<<<blocks_rows, 256, 0, s>>>(m->v, m->Q, n, m->c, m->B, rows_pad,
                                                      w32 + r.row0 * kWeightRows), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
  }
  return ITERGP_OK;
}

void itergp_server::run_fits(std::vector<FitReq*>& batch) {
  const int count = static_cast<int>(batch.size());
  const double t_start = now();
  std::vector<int> status(count, ITERGP_OK);
  std::vector<itergp_model*> models(count, nullptr);
  std::vector<itergp_fit_report> reps(count);
  int rc = ITERGP_OK;
  // stage X and y of the batch in pinned memory, one copy to the device
  size_t bytes = 0;
  std::vector<size_t> off_x(count), off_y(count);
  for (int i = 0; i < count; ++i) {
    off_x[i] = bytes;
    bytes += align_up(sizeof(float) * batch[i]->X.size(), 256);
    off_y[i] = bytes;
    bytes += align_up(sizeof(int32_t) * batch[i]->y.size(), 256);
  }
  Scratch dev;
  if (!fit_pin.reserve(bytes)) rc = ITERGP_ENOMEM;
  if (rc == ITERGP_OK && dev.alloc(ctx, bytes, fit_stream) != cudaSuccess) rc = ITERGP_ENOMEM;
  if (rc == ITERGP_OK) {
    for (int i = 0; i < count; ++i) {
      std::memcpy(fit_pin.p + off_x[i], batch[i]->X.data(), sizeof(float) * batch[i]->X.size());
      std::memcpy(fit_pin.p + off_y[i], batch[i]->y.data(), sizeof(int32_t) * batch[i]->y.size());
    }
    if (cudaMemcpyAsync(dev.as<char>(), fit_pin.p, bytes, cudaMemcpyHostToDevice, fit_stream) != cudaSuccess)
      rc = ITERGP_ECUDA;
  }
  if (rc == ITERGP_OK) {
    std::vector<itergp_fit_params> prm(count);
    for (int i = 0; i < count; ++i) {
      itergp_fit_params& p = prm[i];
      std::memset(&p, 0, sizeof(p));
      p.n = batch[i]->n;
      p.d = batch[i]->d;
      p.c = batch[i]->c;
      p.X = dev.as<float>(off_x[i]);
      p.y = reinterpret_cast<const int32_t*>(dev.as<char>(off_y[i]));
      p.kernel = itergp_kernel{cfg.kind, batch[i]->ell, batch[i]->s};
      p.precision = cfg.precision;
      p.policy = ITERGP_POLICY_CG;
      p.max_newton = cfg.max_newton;
      p.max_iters = cfg.max_iters;
      p.rank = cfg.rank;
      p.recycle = 1;
      p.literal_kv = 0;
      p.tol_newton = 0.0;
      p.tol_abs = cfg.tol_abs;
      p.tol_rel = cfg.tol_rel;
      p.graph = cfg.graph;
    }
    rc = fit_many(prm.data(), count, models.data(), reps.data(), fit_stream, true);
  }
  for (int i = 0; i < count; ++i) {
    if (rc != ITERGP_OK) {
      status[i] = rc;
    } else if (!models[i]) {
      status[i] = reps[i].status != ITERGP_OK ? reps[i].status : ITERGP_ENUMERIC;
    } else {
      status[i] = install(models[i], *batch[i]);
    }
  }
  cudaStreamSynchronize(fit_stream);    // installed rows are in the slab
  for (int i = 0; i < count; ++i) model_release(models[i], fit_stream);
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < count; ++i) {
    FitReq* r = batch[i];
    in_fit.erase(r->id);
    if (status[i] == ITERGP_OK) {
      Resident& res = resident[r->id];
      res.n = r->n;
      res.d = r->d;
      res.c = r->c;
      res.B = models[i]->B;
      res.kp = make_kparams(itergp_kernel{cfg.kind, r->ell, r->s});
      res.outputscale = r->s;
      res.row0 = r->row0;
      res.rows_pad = r->rows_pad;
      res.last_use = ++tick;
      ++stats.fits_done;
    } else {
      blocks.release(r->row0, r->rows_pad);
      gone[r->id] = status[i];
    }
    push_event(r->id, r->id, ITERGP_REQ_FIT, status[i], r->t_submit, t_start, count);
    delete r;
  }
  ++stats.fit_batches;
  cv_pred.notify_all();
  cv_events.notify_all();
}

void itergp_server::pred_loop() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<PredReq*> batch;
    std::vector<Resident> models;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        // answer predicts whose model is gone; take those whose model is resident
        int64_t rows = 0;
        for (auto it = pred_q.begin(); it != pred_q.end();) {
          PredReq* q = *it;
          auto g = gone.find(q->model);
          if (g != gone.end()) {
            push_event(q->id, q->model, ITERGP_REQ_PREDICT, ITERGP_EGONE, q->t_submit, now(), 0);
            if (--pending[q->model] == 0) pending.erase(q->model);
            delete q;
            it = pred_q.erase(it);
            continue;
          }
          auto r = resident.find(q->model);
          if (r == resident.end() || static_cast<int>(batch.size()) >= cfg.max_predict_batch ||
              (!batch.empty() && rows + round128(q->m) > cfg.max_predict_rows)) {
            ++it;
            continue;
          }
          r->second.last_use = ++tick;
          rows += round128(q->m);
          batch.push_back(q);
          models.push_back(r->second);
          it = pred_q.erase(it);
        }
        stats.queued_predicts = static_cast<int64_t>(pred_q.size());
        if (!batch.empty()) break;
        cv_events.notify_all();
        if (stop && pred_q.empty()) break;
        cv_pred.wait(lk);
      }
      if (batch.empty()) break;   // stopped
    }
    std::vector<int> status;
    double t_start = 0;
    run_predicts(batch, models, &status, &t_start);
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < batch.size(); ++i) {
      PredReq* q = batch[i];
      push_event(q->id, q->model, ITERGP_REQ_PREDICT, status[i], q->t_submit, t_start,
                 static_cast<int>(batch.size()));
      if (--pending[q->model] == 0) {
        pending.erase(q->model);
        auto r = resident.find(q->model);
        if (r != resident.end() && r->second.release_requested) {
          blocks.release(r->second.row0, r->second.rows_pad);
          gone[q->model] = ITERGP_EGONE;
          resident.erase(r);
        }
      }
      ++stats.predicts_done;
      delete q;
    }
    ++stats.predict_batches;
    cv_fit.notify_all();
    cv_events.notify_all();
  }
}

void itergp_server::run_predicts(std::vector<PredReq*>& batch, const std::vector<Resident>& models,
                                 std::vector<int>* status_out, double* t_start) {
  const int count = static_cast<int>(batch.size());
  std::vector<int>& status = *status_out;
  status.assign(count, ITERGP_OK);
  *t_start = now();
  cudaStream_t s = pred_stream;
  const int dm = cfg.d_max;
  // ---- host tables
  std::vector<int64_t> q0(count), o0(count), oo(count);
  int64_t q_rows = 0, m_total = 0, out_total = 0;
  int max_c = 1, max_cb = 0;
  for (int i = 0; i < count; ++i) {
    q0[i] = q_rows;
    q_rows += round128(batch[i]->m);
    o0[i] = m_total;
    m_total += batch[i]->m;
    oo[i] = out_total;
    out_total += 3 * batch[i]->m * models[i].c;
    max_c = std::max(max_c, models[i].c);
    max_cb = std::max(max_cb, models[i].c * models[i].B);
  }
  std::vector<WorkItem> items_mean, items_var;
  for (int i = 0; i < count; ++i) {
    const Resident& r = models[i];
    const int tiles = static_cast<int>(ceil_div(batch[i]->m, 128));
    for (int t = 0; t < tiles; ++t) {
      WorkItem it{i, static_cast<int32_t>(q0[i] + 128 * t), 128 * t, static_cast<int32_t>(r.row0),
                  static_cast<int32_t>(r.rows_pad / 128), static_cast<int32_t>(r.n), 0, 0};
      items_mean.push_back(it);
      if (r.c * r.B > 0) items_var.push_back(it);
    }
  }
  const bool tc = tensor();
  std::vector<WorkItem> ord_mean, ord_var;
  std::vector<int32_t> beg_mean, beg_var;
  int g_mean = 0, g_var = 0;
  if (tc) {
    g_mean = static_cast<int>(std::min<int64_t>(ctx->num_sms, static_cast<int64_t>(items_mean.size())));
    plan_items(items_mean, g_mean, &ord_mean, &beg_mean);
    // the variance columns ride in the same launch as the mean (weight rows [0, 16 + C B))
  } else {
    ord_mean = items_mean;
    ord_var = items_var;
  }
  // ---- device memory: queries, prepared rows, products, outputs, tables
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += align_up(std::max<size_t>(b, 1), 256); return o; };
  const size_t o_q = take(sizeof(float) * q_rows * dm);
  const size_t o_rows = take(rows_workspace_bytes(cfg.precision, q_rows, dm));
  const size_t o_y = take(sizeof(float) * m_total * kWeightRows);
  const size_t o_out = take(sizeof(float) * out_total);
  const size_t o_tab = off;   // tables: items, begins, probs, descs (staged with the queries)
  size_t toff = 0;
  auto ttake = [&](size_t b) { const size_t o = toff; toff += align_up(std::max<size_t>(b, 1), 256); return o; };
  const size_t t_im = ttake(sizeof(WorkItem) * ord_mean.size());
  const size_t t_iv = ttake(sizeof(WorkItem) * ord_var.size());
  const size_t t_bm = ttake(sizeof(int32_t) * beg_mean.size());
  const size_t t_bv = ttake(sizeof(int32_t) * beg_var.size());
  const size_t t_pm = ttake(sizeof(TcProb) * count);
  const size_t t_pv = ttake(sizeof(TcProb) * count);
  const size_t t_d = ttake(sizeof(PredDesc) * count);
  off += toff;
  Scratch dev;
  const size_t stage_bytes = sizeof(float) * q_rows * dm + toff;
  if (!pred_pin.reserve(stage_bytes) || !pred_out_pin.reserve(sizeof(float) * std::max<int64_t>(out_total, 1)) ||
      dev.alloc(ctx, off, s) != cudaSuccess) {
    status.assign(count, ITERGP_ENOMEM);
    return;
  }
  char* base = dev.as<char>();
  float* qX = reinterpret_cast<float*>(base + o_q);
  float* ybuf = reinterpret_cast<float*>(base + o_y);
  float* out = reinterpret_cast<float*>(base + o_out);
  char* tab = base + o_tab;
  // ---- stage queries (rows padded with zeros to 128 and to d_max) and tables
  float* hq = reinterpret_cast<float*>(pred_pin.p);
  std::memset(hq, 0, sizeof(float) * q_rows * dm);
  for (int i = 0; i < count; ++i) {
    const PredReq& q = *batch[i];
    if (q.d == dm) {
      std::memcpy(hq + q0[i] * dm, q.Xs.data(), sizeof(float) * q.m * dm);
    } else {
      for (int64_t r = 0; r < q.m; ++r)
        std::memcpy(hq + (q0[i] + r) * dm, q.Xs.data() + r * q.d, sizeof(float) * q.d);
    }
  }
  char* ht = pred_pin.p + sizeof(float) * q_rows * dm;
  std::vector<TcProb> pm(count), pv(count);
  std::vector<PredDesc> ds(count);
  for (int i = 0; i < count; ++i) {
    const Resident& r = models[i];
    float* yi = ybuf + o0[i] * kWeightRows;
    if (tc) {   // one pass over weight rows [0, 16 + C B): mean and variance columns together
      const float* wsc = w_scale ? w_scale + (r.row0 / 128) * kWeightRows : nullptr;
      pm[i] = TcProb{yi, kWeightRows, batch[i]->m, kMeanRows + r.c * r.B, 0, r.kp, nullptr, wsc};
    } else {    // FP32: a mean pass (columns 0..C-1) and a variance pass (columns 16..)
      pm[i] = TcProb{yi, kWeightRows, batch[i]->m, r.c, 0, r.kp, nullptr, nullptr};
      pv[i] = TcProb{yi + kMeanRows, kWeightRows, batch[i]->m, r.c * r.B, 0, r.kp, nullptr, nullptr};
    }
    ds[i] = PredDesc{yi, out + oo[i], batch[i]->m, r.c, r.B, r.outputscale, 0};
  }
  std::memcpy(ht + t_im, ord_mean.data(), sizeof(WorkItem) * ord_mean.size());
  std::memcpy(ht + t_iv, ord_var.data(), sizeof(WorkItem) * ord_var.size());
  std::memcpy(ht + t_bm, beg_mean.data(), sizeof(int32_t) * beg_mean.size());
  std::memcpy(ht + t_bv, beg_var.data(), sizeof(int32_t) * beg_var.size());
  std::memcpy(ht + t_pm, pm.data(), sizeof(TcProb) * count);
  std::memcpy(ht + t_pv, pv.data(), sizeof(TcProb) * count);
  std::memcpy(ht + t_d, ds.data(), sizeof(PredDesc) * count);
  int rc = ITERGP_OK;
  if (cudaMemcpyAsync(qX, hq, sizeof(float) * q_rows * dm, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(tab, ht, toff, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = ITERGP_ECUDA;
  RowOperand qop;
  if (rc == ITERGP_OK) rc = prepare_rows(cfg.precision, qX, q_rows, dm, dm, base + o_rows, &qop, s);
  KmvItemTables tm, tv;
  tm.items = reinterpret_cast<const WorkItem*>(tab + t_im);
  tm.item_begin = reinterpret_cast<const int32_t*>(tab + t_bm);
  tm.probs = reinterpret_cast<const TcProb*>(tab + t_pm);
  tm.G = tc ? g_mean : 0;
  tm.n_items = static_cast<int>(ord_mean.size());
  tv.items = reinterpret_cast<const WorkItem*>(tab + t_iv);
  tv.item_begin = reinterpret_cast<const int32_t*>(tab + t_bv);
  tv.probs = reinterpret_cast<const TcProb*>(tab + t_pv);
  tv.G = tc ? g_var : 0;
  tv.n_items = static_cast<int>(ord_var.size());
  if (rc == ITERGP_OK) {
    if (tc) {
      rc = kmv_tc_items(ctx, cfg.kind, qop, rows_op, tm, w_hi, w_lo, kWeightRows, 0,
                        kMeanRows + static_cast<int>((max_cb + 15) / 16 * 16), s);
    } else {
      rc = kmv_simt_items(ctx, cfg.kind, qop, rows_op, tm, w32, kWeightRows, max_c, s);
      if (rc == ITERGP_OK && tv.n_items > 0)
        rc = kmv_simt_items(ctx, cfg.kind, qop, rows_op, tv, w32 + kMeanRows, kWeightRows, max_cb, s);
    }
  }
  if (rc == ITERGP_OK) {
    int64_t max_m = 1;
    for (int i = 0; i < count; ++i) max_m = std::max(max_m, batch[i]->m);
    dim3 grid(static_cast<unsigned>(std::min<int64_t>(ceil_div(max_m, 256), 64)), static_cast<unsigned>(count));
    serve_epilogue_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const PredDesc*>(tab + t_d)), ::itergp::note_launch();
    if (cudaGetLastError() != cudaSuccess) rc = ITERGP_ECUDA;
  }
  if (rc == ITERGP_OK &&
      cudaMemcpyAsync(pred_out_pin.p, out, sizeof(float) * out_total, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = ITERGP_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == ITERGP_OK) rc = ITERGP_ECUDA;
  if (rc != ITERGP_OK) {
    status.assign(count, rc);
    return;
  }
  const float* ho = reinterpret_cast<const float*>(pred_out_pin.p);
  for (int i = 0; i < count; ++i) {
    const PredReq& q = *batch[i];
    const int64_t mc = q.m * models[i].c;
    std::memcpy(q.mean, ho + oo[i], sizeof(float) * mc);
    if (q.var) std::memcpy(q.var, ho + oo[i] + mc, sizeof(float) * mc);
    if (q.probs) std::memcpy(q.probs, ho + oo[i] + 2 * mc, sizeof(float) * mc);
  }
}

extern "C" {

int itergp_server_create(const itergp_server_config* cfg, itergp_server** out) {
  if (!cfg || !out) return ITERGP_EINVAL;
  *out = nullptr;
  if (cfg->model_bytes <= 0 || cfg->work_bytes <= 0 || cfg->d_max < 1 || cfg->d_max > 1024 ||
      cfg->c_max < 2 || cfg->c_max > kMeanRows || cfg->max_fit_batch < 1 || cfg->max_predict_batch < 1 ||
      cfg->max_predict_rows < 4096 || cfg->max_newton < 1 || cfg->max_iters < 1 ||
      !(cfg->kind == ITERGP_RBF || cfg->kind == ITERGP_MATERN32) || cfg->precision < ITERGP_FP32 ||
      cfg->precision > ITERGP_TF32 || !(cfg->tol_abs >= 0) || !(cfg->tol_rel >= 0))
    return ITERGP_EINVAL;
  itergp_fit_params probe{};
  probe.n = int64_t(1) << 40;
  probe.c = cfg->c_max;
  probe.max_newton = cfg->max_newton;
  probe.max_iters = cfg->max_iters;
  probe.rank = cfg->rank;
  probe.recycle = 1;
  const int64_t bcap = buffer_capacity(probe);
  if (static_cast<int64_t>(cfg->c_max) * bcap > kVarRows) return ITERGP_EINVAL;
  DeviceContext* ctx = current_context();
  if (!ctx) return ITERGP_ECUDA;
  if (precision_is_tensor(cfg->precision) && !ctx->tcgen05) return ITERGP_EUNSUPPORTED;
  auto* srv = new itergp_server();
  srv->cfg = *cfg;
  srv->ctx = ctx;
  srv->device = ctx->device;
  srv->bcap = static_cast<int>(bcap);
  srv->t0 = std::chrono::steady_clock::now();
  const bool tc = precision_is_tensor(cfg->precision);
  srv->d_pad = tc ? (cfg->d_max + 63) / 64 * 64 : cfg->d_max;
  const int planes = tc ? precision_row_planes(cfg->precision) : 0;   // 2-byte planes per row
  const int wplanes = tc ? (precision_splits_weights(cfg->precision) ? 2 : 1) : 0;
  // bytes per slab row: rows, norm, weights
  const size_t per_row = tc ? (static_cast<size_t>(planes) * srv->d_pad * 2 + 4 + static_cast<size_t>(wplanes) * kWeightRows * 2)
                            : (sizeof(float) * cfg->d_max + 4 + sizeof(float) * kWeightRows);
  srv->slab_rows = (static_cast<int64_t>(cfg->model_bytes) - 8 * 256) / static_cast<int64_t>(per_row) / 128 * 128;
  if (srv->slab_rows < 128) {
    delete srv;
    return ITERGP_EINVAL;
  }
  const int64_t R = srv->slab_rows;
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += align_up(b, 256); return o; };
  const size_t o_norm = take(sizeof(float) * R);
  // split rows: one scale per 128-row block (R is a multiple of 128)
  const size_t o_tscale = precision_splits_rows(cfg->precision) ? take(sizeof(float) * (R / 128)) : 0;
  size_t o_hi = 0, o_lo = 0, o_whi = 0, o_wlo = 0, o_x = 0, o_w = 0, o_wmax = 0, o_wscale = 0;
  if (tc) {
    // TF32: one FP32 plane in the bytes of two BF16 planes
    const bool tf32 = precision_tf32_rows(cfg->precision);
    o_hi = take(static_cast<size_t>(R) * srv->d_pad * 2 * (tf32 ? 2 : 1));
    if (planes == 2 && !tf32) o_lo = take(static_cast<size_t>(R) * srv->d_pad * 2);
    o_whi = take(static_cast<size_t>(R) * kWeightRows * 2);
    if (wplanes == 2) o_wlo = take(static_cast<size_t>(R) * kWeightRows * 2);
    if (wplanes == 2) {   // a model's weight scales live at its first 128-row block's entry
      o_wmax = take(sizeof(uint32_t) * kWeightRows);
      o_wscale = take(sizeof(float) * (R / 128) * kWeightRows);
    }
  } else {
    o_x = take(sizeof(float) * R * cfg->d_max);
    o_w = take(sizeof(float) * R * kWeightRows);
  }
  // every allocation and copy of the server is stream-ordered on its own non-blocking
  // streams (a synchronising call would break stream captures that other threads have open)
  if (cudaStreamCreateWithFlags(&srv->fit_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&srv->pred_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (srv->fit_stream) cudaStreamDestroy(srv->fit_stream);
    delete srv;
    return ITERGP_ECUDA;
  }
  auto fail = [&](int code) {
    if (srv->slab) {
      cudaFreeAsync(srv->slab, srv->fit_stream);
      cudaStreamSynchronize(srv->fit_stream);
    }
    cudaStreamDestroy(srv->fit_stream);
    cudaStreamDestroy(srv->pred_stream);
    delete srv;
    return code;
  };
  if (cudaMallocFromPoolAsync(&srv->slab, off, ctx->pool, srv->fit_stream) != cudaSuccess) {
    srv->slab = nullptr;
    return fail(ITERGP_ENOMEM);
  }
  char* b = static_cast<char*>(srv->slab);
  // zero once: rows never written by a model (free blocks) are never read, but weights
  // beyond a model's columns must read as zeros
  if (cudaMemsetAsync(srv->slab, 0, off, srv->fit_stream) != cudaSuccess ||
      cudaStreamSynchronize(srv->fit_stream) != cudaSuccess)
    return fail(ITERGP_ECUDA);
  // predict staging at its largest size now: no pinned reallocation while running
  {
    const int64_t rows = cfg->max_predict_rows + 128LL * cfg->max_predict_batch;
    const size_t tabs = static_cast<size_t>(rows / 128 + cfg->max_predict_batch) * sizeof(WorkItem) * 2 +
                        static_cast<size_t>(cfg->max_predict_batch) * (2 * sizeof(TcProb) + 64) +
                        static_cast<size_t>(ctx->num_sms + 1) * 8 + 64 * 1024;
    if (!srv->pred_pin.reserve(sizeof(float) * rows * cfg->d_max + tabs) ||
        !srv->pred_out_pin.reserve(sizeof(float) * 3 * cfg->max_predict_rows * cfg->c_max))
      return fail(ITERGP_ENOMEM);
  }
  RowOperand& op = srv->rows_op;
  op.rows = R;
  op.rows_pad = R;
  op.d = cfg->d_max;
  op.d_pad = srv->d_pad;
  op.precision = cfg->precision;
  op.norms = reinterpret_cast<float*>(b + o_norm);
  op.tscale = precision_splits_rows(cfg->precision) ? reinterpret_cast<float*>(b + o_tscale) : nullptr;
  if (tc) {
    op.X = nullptr;
    op.ldX = cfg->d_max;
    op.hi = reinterpret_cast<__nv_bfloat16*>(b + o_hi);
    op.lo = precision_splits_rows(cfg->precision) ? reinterpret_cast<__nv_bfloat16*>(b + o_lo) : nullptr;
    srv->w_hi = reinterpret_cast<__nv_bfloat16*>(b + o_whi);
    srv->w_lo = wplanes == 2 ? reinterpret_cast<__nv_bfloat16*>(b + o_wlo) : nullptr;
    srv->w_max = wplanes == 2 ? reinterpret_cast<uint32_t*>(b + o_wmax) : nullptr;
    srv->w_scale = wplanes == 2 ? reinterpret_cast<float*>(b + o_wscale) : nullptr;
  } else {
    op.X = reinterpret_cast<float*>(b + o_x);
    op.ldX = cfg->d_max;
    srv->w32 = reinterpret_cast<float*>(b + o_w);
  }
  srv->blocks.init(R);
  srv->stats.slab_rows = R;
  srv->fit_thr = std::thread([srv] { srv->fit_loop(); });
  srv->pred_thr = std::thread([srv] { srv->pred_loop(); });
  *out = srv;
  return ITERGP_OK;
}

int itergp_server_destroy(itergp_server* srv) {
  if (!srv) return ITERGP_EINVAL;
  {
    // queued requests are dropped; batches already on the GPU finish
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (FitReq* r : srv->fit_q) delete r;
    srv->fit_q.clear();
    for (PredReq* q : srv->pred_q) delete q;
    srv->pred_q.clear();
  }
  srv->cv_fit.notify_all();
  srv->cv_pred.notify_all();
  if (srv->fit_thr.joinable()) srv->fit_thr.join();
  if (srv->pred_thr.joinable()) srv->pred_thr.join();
  cudaStreamSynchronize(srv->pred_stream);
  cudaFreeAsync(srv->slab, srv->fit_stream);   // stream-ordered, after the last fit
  cudaStreamSynchronize(srv->fit_stream);
  cudaStreamDestroy(srv->fit_stream);
  cudaStreamDestroy(srv->pred_stream);
  delete srv;
  return ITERGP_OK;
}

int itergp_server_submit_fit(itergp_server* srv, const float* X, const int32_t* y, int64_t n,
                             int64_t d, int32_t c, float lengthscale, float outputscale,
                             int64_t* model_id) {
  if (!srv || !X || !y || !model_id || n < 1 || d < 1 || d > srv->cfg.d_max || c < 2 ||
      c > srv->cfg.c_max || !(lengthscale > 0.f) || !(outputscale > 0.f) || n > (int64_t(1) << 31) - 1024)
    return ITERGP_EINVAL;
  auto* r = new FitReq();
  r->X.assign(X, X + n * d);
  r->y.assign(y, y + n);
  r->n = n;
  r->d = static_cast<int>(d);
  r->c = c;
  r->ell = lengthscale;
  r->s = outputscale;
  r->rows_pad = round128(n);
  r->work = srv->fit_work_bytes(n, static_cast<int>(d), c);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) {
      delete r;
      return ITERGP_EINVAL;
    }
    r->id = srv->next_id++;
    r->t_submit = srv->now();
    srv->in_fit[r->id] = 1;
    srv->dims[r->id] = r->d;
    srv->fit_q.push_back(r);
    srv->stats.queued_fits = static_cast<int64_t>(srv->fit_q.size());
    *model_id = r->id;
  }
  srv->cv_fit.notify_one();
  return ITERGP_OK;
}

int itergp_server_submit_predict(itergp_server* srv, int64_t model_id, const float* Xs, int64_t m,
                                 float* mean, float* var, float* probs, int64_t* request_id) {
  if (!srv || !Xs || !mean || !request_id || m < 1 || m > srv->cfg.max_predict_rows) return ITERGP_EINVAL;
  auto* q = new PredReq();
  q->model = model_id;
  q->m = m;
  q->mean = mean;
  q->var = var;
  q->probs = probs;
  {
    // the model must be queued, fitting or resident (and not released)
    std::lock_guard<std::mutex> lk(srv->mu);
    const auto r = srv->resident.find(model_id);
    const bool live = (r != srv->resident.end() && !r->second.release_requested) ||
                      srv->in_fit.count(model_id) != 0;
    if (!live || srv->stop) {
      delete q;
      return srv->gone.count(model_id) ? ITERGP_EGONE : ITERGP_EINVAL;
    }
    q->d = srv->dims[model_id];
    ++srv->pending[model_id];   // keeps the model from eviction until this request is done
    q->t_submit = srv->now();
  }
  q->Xs.assign(Xs, Xs + m * q->d);   // copied outside the lock
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    q->id = srv->next_id++;
    *request_id = q->id;
    srv->pred_q.push_back(q);
    srv->stats.queued_predicts = static_cast<int64_t>(srv->pred_q.size());
  }
  srv->cv_pred.notify_one();
  return ITERGP_OK;
}

int itergp_server_poll(itergp_server* srv, itergp_server_event* events, int32_t capacity,
                       int32_t* count, int64_t timeout_us) {
  if (!srv || !count || capacity < 0 || (capacity > 0 && !events)) return ITERGP_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto ready = [&] { return !srv->events.empty(); };
  if (timeout_us < 0)
    srv->cv_events.wait(lk, ready);
  else if (timeout_us > 0)
    srv->cv_events.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
  int32_t n = 0;
  while (n < capacity && !srv->events.empty()) {
    events[n++] = srv->events.front();
    srv->events.pop_front();
  }
  *count = n;
  return ITERGP_OK;
}

int itergp_server_release(itergp_server* srv, int64_t model_id) {
  if (!srv) return ITERGP_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto r = srv->resident.find(model_id);
  if (r == srv->resident.end()) return srv->gone.count(model_id) ? ITERGP_EGONE : ITERGP_EINVAL;
  auto p = srv->pending.find(model_id);
  if (p != srv->pending.end() && p->second > 0) {
    r->second.release_requested = true;   // freed when its last predict completes
    return ITERGP_OK;
  }
  srv->blocks.release(r->second.row0, r->second.rows_pad);
  srv->gone[model_id] = ITERGP_EGONE;
  srv->resident.erase(r);
  srv->cv_fit.notify_all();
  return ITERGP_OK;
}

int itergp_server_get_stats(itergp_server* srv, itergp_server_stats* st) {
  if (!srv || !st) return ITERGP_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  *st = srv->stats;
  st->resident_models = static_cast<int64_t>(srv->resident.size());
  st->resident_rows = srv->blocks.used();
  st->queued_fits = static_cast<int64_t>(srv->fit_q.size());
  st->queued_predicts = static_cast<int64_t>(srv->pred_q.size());
  return ITERGP_OK;
}

}  // extern "C"
