// Internal interfaces between the translation units of libitergp (not exported).
#pragma once
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace itergp {

// One side of the kernel product k(A, B): the FP32 rows plus, for the tensor-core
// paths, their 16-bit copies and row norms, zero-padded to tile multiples.
//
// Split-row precisions (BF16X3, BF16_COMP) store each 128-row tile T scaled by a power of
// two 2^e_T that brings the tile's largest |x| into [128, 256), as FP16 hi = fp16(2^e x)
// and lo = fp16(2^e x - hi): 22 significant bits, and the exponent range of FP16 no
// longer limits the data.  tscale[T] = 2^-e_T; a product of tiles I and J reads
// a.b = tscale[I] tscale[J] (a_hi.b_hi + a_hi.b_lo + a_lo.b_hi) exactly as scaled.
struct RowOperand {
  const float* X = nullptr;          // rows x d, row pitch ldX (FP32, caller-owned)
  int64_t rows = 0;
  int d = 0;
  int64_t ldX = 0;
  int64_t rows_pad = 0;              // multiple of 128
  int d_pad = 0;                     // multiple of 64 (tensor paths) / d (FP32 path)
  int precision = ITERGP_FP32;
  const float* norms = nullptr;      // [rows_pad] squared row norms (see prepare_rows)
  const __nv_bfloat16* hi = nullptr; // [rows_pad][d_pad] (TF32: FP32 values; split rows: FP16 bits)
  const __nv_bfloat16* lo = nullptr; // [rows_pad][d_pad] (split precisions only, FP16 bits)
  const float* tscale = nullptr;     // [rows_pad / 128] tile scales (split precisions only)
};

constexpr int kRowTile = 128;
constexpr int kColTile = 64;

inline bool precision_is_tensor(int p) {
  return p == ITERGP_BF16X3 || p == ITERGP_BF16 || p == ITERGP_BF16_COMP || p == ITERGP_TF32;
}
inline bool precision_splits_rows(int p) { return p == ITERGP_BF16X3 || p == ITERGP_BF16_COMP; }
inline bool precision_splits_weights(int p) { return p == ITERGP_BF16X3 || p == ITERGP_TF32; }
// TF32 rows: one FP32 plane (rows_pad x d_pad, values rounded to TF32) in the bytes of two
// BF16 planes; RowOperand::hi then points at FP32 data.
inline bool precision_tf32_rows(int p) { return p == ITERGP_TF32; }
inline int precision_row_planes(int p) { return precision_splits_rows(p) || precision_tf32_rows(p) ? 2 : 1; }

// Bytes of device memory prepare_rows needs for `rows` x `d` at `precision`.
size_t rows_workspace_bytes(int precision, int64_t rows, int d);

// Fill `op` (norms and, for tensor precisions, BF16 copies) using `mem` (device memory of
// rows_workspace_bytes).  Enqueued on `stream`.
int prepare_rows(int precision, const float* X, int64_t rows, int d, int64_t ldX, void* mem,
                 RowOperand* op, cudaStream_t stream);

// Y[i, 0:p] = sum_j k(A_i, B_j) S[j, 0:p]  (row pitches ldS, ldY).  A and B must be
// prepared with the same precision.  If `active` is non-null and *active == 0 on the
// device, every launch returns immediately (used by the device-side solver loop).
int kmv_execute(DeviceContext* ctx, const KParams& kp, const RowOperand& A, const RowOperand& B,
                const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY,
                cudaStream_t stream, const int* active);
// The product with one kernel per class: column j of S and Y belongs to class j mod C and
// uses kps[j mod C].  Runs C grouped products, each over its class's columns gathered into
// a contiguous block (scratch from the pool) and scattered back into Y.
int kmv_classes(DeviceContext* ctx, const KParams* kps, int C, const RowOperand& A, const RowOperand& B,
                const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY, cudaStream_t stream,
                const int* active);

// Plain FP32 path (kmv_simt.cu).
int kmv_simt(DeviceContext* ctx, const KParams& kp, const RowOperand& A, const RowOperand& B,
             const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY, cudaStream_t stream,
             const int* active);

// Tensor-core path (kmv_tc.cu).
int kmv_tc(DeviceContext* ctx, const KParams& kp, const RowOperand& A, const RowOperand& B,
           const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY, cudaStream_t stream,
           const int* active);

// Static work partition of the tensor-core kernel: G CTAs share U = R * J units
// (row tile, column chunk) in contiguous ranges [start(g), start(g+1)).
__host__ __device__ inline int64_t part_start(int64_t g, int64_t U, int64_t G) { return g * U / G; }
__host__ __device__ inline int64_t part_owner(int64_t u, int64_t U, int64_t G) {
  return ((u + 1) * G - 1) / U;
}


// ---------------------------------------------------------------- batched products
// One row tile of one problem of a batched product, processed over all column chunks.
struct WorkItem {
  int32_t prob;      // index into the problem table
  int32_t a_row;     // arena row of the tile's first row (multiple of 128)
  int32_t tile_row;  // first output row of the tile within its problem
  int32_t b_row0;    // arena row (= transposed-S column) of the problem's first row
  int32_t chunks;    // 128-row column chunks of the problem
  int32_t n_rows;    // rows of the problem
  int32_t pad0, pad1;
};

// Per-problem output and kernel of a batched product launch.
struct TcProb {
  float* Y;          // output rows (already offset to the P tile's first column)
  int64_t ldY;
  int64_t m;         // valid rows
  int32_t p_valid;   // valid output columns
  int32_t pad;
  KParams kp;
  const int* active; // the problem's solver flag (nullptr: always active)
  const float* wscale;   // split weights: 2^-e per weight row of the problem's staged S
};

// Device-side tables of a batched product.
struct KmvItemTables {
  const WorkItem* items = nullptr;      // [n_items], grouped per CTA
  const int32_t* item_begin = nullptr;  // [G + 1] (tensor-core path)
  const TcProb* probs = nullptr;        // [nprob]
  int G = 0;
  int n_items = 0;
};

// Tensor-core product in item mode: item rows a_row of A (query side) against the rows
// b_row0 .. of B (problem side, both prepared with the same precision and d_pad).
// s_hi/s_lo: transposed split weights [s_rows][B.rows_pad]; this call reads weight rows
// [s_row0, s_row0 + p_pad) (p_pad a multiple of 16, <= 256; launched in P tiles of at
// most 128 that fit the shared memory).  All problems share `kind`.
int kmv_tc_items(DeviceContext* ctx, int kind, const RowOperand& A, const RowOperand& B,
                 const KmvItemTables& tab, const __nv_bfloat16* s_hi, const __nv_bfloat16* s_lo,
                 int64_t s_rows, int s_row0, int p_pad, cudaStream_t stream);

// FP32 SIMT product in item mode: one CTA per item; FP32 rows of A and B (pitch ldX, same
// d), S = FP32 weights [B rows][ldS] with up to p_max (<= 128) columns.  All problems
// share `kind`.
int kmv_simt_items(DeviceContext* ctx, int kind, const RowOperand& A, const RowOperand& B,
                   const KmvItemTables& tab, const float* S, int64_t ldS, int p_max,
                   cudaStream_t stream);


// ---------------------------------------------------------------- fits (solver.cu)
// One problem of a (batched) fit: its parameters, prepared rows and the model arrays the
// fit writes (v, f, Q), plus where its outcome goes.
struct FitProblem {
  const itergp_fit_params* prm;
  KParams kp;
  std::vector<KParams> class_kp;   // one per class, or empty for the shared kernel
  const RowOperand* xop;   // prepared rows of the problem (model memory)
  float *v, *f, *Q;
  int bcap;
  itergp_fit_report* rep;
  int* final_B;
  int* status;             // the problem's own outcome (ITERGP_OK, ITERGP_EINVAL, ITERGP_ENUMERIC)
};

// Runs Alg. 1-3 for all problems with one schedule (params of probs[0]) on `stream`,
// optionally captured into one CUDA graph; waits for the stream.  Returns errors of the
// call (CUDA, memory, a wait limit); device errors of single problems go to their status.
int fit_run_batch(DeviceContext* ctx, const std::vector<FitProblem>& probs, cudaStream_t stream,
                  bool use_graph);

// ---------------------------------------------------------------- models (api.cu)
// Host-side argument checks shared by the entry points: a known kernel kind with finite,
// positive lengthscale and outputscale; a known precision.
inline bool kernel_ok(const itergp_kernel* k) {
  return k && (k->kind == ITERGP_RBF || k->kind == ITERGP_MATERN32) && std::isfinite(k->lengthscale) &&
         k->lengthscale > 0.f && std::isfinite(k->outputscale) && k->outputscale > 0.f;
}
inline bool precision_ok(int p) { return p >= ITERGP_FP32 && p <= ITERGP_TF32; }

int validate_fit_params(const itergp_fit_params* prm);
void clear_stale_error();
// Buffer columns a fit keeps at most: min(max_newton * max_iters, R + max_iters, N C).
int64_t buffer_capacity(const itergp_fit_params& p);
// Fits params[0..count) with one schedule (allocating the models from the library pool on
// `s`) and waits.  batch = false: a device error of the problem is the return value;
// batch = true: failed problems get out[i] = NULL and their report's status.
int fit_many(const itergp_fit_params* params, int count, itergp_model** out,
             itergp_fit_report* reports, cudaStream_t s, bool batch);
// Stream-ordered release of a model no other stream still reads.
void model_release(itergp_model* m, cudaStream_t s);

// LPT (longest processing time first) assignment of whole-row items to G CTAs; items of
// one problem stay together within a CTA.  begin: [G + 1] offsets into `ordered`.
void plan_items(const std::vector<WorkItem>& items, int G, std::vector<WorkItem>* ordered,
                std::vector<int32_t>* begin);

// Times every launch variant of the tensor-core product (epilogue warps x stages x form:
// one CTA with a streamed or resident-A ring, or CTA pairs) on X
// (A = B = X, weights S: rows x p, output Y) in the single (items = 0) or item-mode
// schedule, records the fastest for (precision, kind, d_pad, P tile, schedule) and
// returns the timings (up to cap variants).
int kmv_tc_tune(DeviceContext* ctx, const KParams& kp, const RowOperand& X, const float* S,
                int64_t p, float* Y, int items, int cap, int* count, int* epi_out, int* ns_out,
                int* pair_out, double* ms_out, int* best, cudaStream_t stream);

// Self-test of the bounded waits: one CTA waits on an mbarrier nothing arrives on and
// records ITERGP_ETIMEOUT in ctx->status after limit_ns.
int wait_selftest_launch(DeviceContext* ctx, uint64_t limit_ns, cudaStream_t stream);

// Prepared rows written into caller-provided planes with pitch d_pad (>= d, multiple of
// 64 for tensor precisions): the 16-bit hi (and lo for split precisions) [rows_pad][d_pad],
// FP32 squared norms [rows_pad] and, for split precisions, the tile scales
// [rows_pad / 128] (rows_pad a multiple of 128 there); rows beyond `rows` are zero.
int prepare_rows_into(int precision, const float* X, int64_t rows, int d, int64_t ldX,
                      int64_t rows_pad, int d_pad, __nv_bfloat16* hi, __nv_bfloat16* lo,
                      float* norms, float* tscale, cudaStream_t stream);

}  // namespace itergp

// A fitted model: one pool allocation with X, its prepared rows, v, f and Q.
struct itergp_model {
  int device = -1;
  int64_t n = 0, d = 0;
  int c = 0, bcap = 0, B = 0;
  itergp_kernel kernel{};
  std::vector<itergp_kernel> class_kernels;   // one per class, or empty for the shared kernel
  int precision = 0;
  int likelihood = ITERGP_LIK_SOFTMAX;
  void* mem = nullptr;
  cudaEvent_t used = nullptr;   // recorded after the model's last fit / predict
  float* X = nullptr;
  float* v = nullptr;
  float* f = nullptr;
  float* Q = nullptr;     // [bcap][n c]: buffer column b at Q + b n c
  itergp::RowOperand xop;
  int64_t bytes = 0;
};
