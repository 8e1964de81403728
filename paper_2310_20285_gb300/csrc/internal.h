// Internal interfaces between the translation units of libitergp (not exported).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace itergp {

// One side of the kernel product k(A, B): the FP32 rows plus, for the tensor-core
// paths, their BF16 hi/lo split copies and row norms, zero-padded to tile multiples.
struct RowOperand {
  const float* X = nullptr;          // rows x d, row pitch ldX (FP32, caller-owned)
  int64_t rows = 0;
  int d = 0;
  int64_t ldX = 0;
  int64_t rows_pad = 0;              // multiple of 128
  int d_pad = 0;                     // multiple of 64 (tensor paths) / d (FP32 path)
  int precision = ITERGP_FP32;
  const float* norms = nullptr;      // [rows_pad] squared row norms (see prepare_rows)
  const __nv_bfloat16* hi = nullptr; // [rows_pad][d_pad]
  const __nv_bfloat16* lo = nullptr; // [rows_pad][d_pad] (split precisions only)
};

constexpr int kRowTile = 128;
constexpr int kColTile = 64;

inline bool precision_is_tensor(int p) { return p == ITERGP_BF16X3 || p == ITERGP_BF16 || p == ITERGP_BF16_COMP; }
inline bool precision_splits_rows(int p) { return p == ITERGP_BF16X3 || p == ITERGP_BF16_COMP; }
inline bool precision_splits_weights(int p) { return p == ITERGP_BF16X3; }

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
};

// Device-side tables of a batched product.
struct KmvItemTables {
  const WorkItem* items = nullptr;      // [n_items], grouped per CTA
  const int32_t* item_begin = nullptr;  // [G + 1] (tensor-core path)
  const TcProb* probs = nullptr;        // [nprob]
  int G = 0;
  int n_items = 0;
};

// Tensor-core product in item mode over an arena of rows (A = B = arena); s_hi/s_lo:
// transposed split weights [p16][arena.rows_pad].  All problems share `kind`.
int kmv_tc_items(DeviceContext* ctx, int kind, const RowOperand& arena, const KmvItemTables& tab,
                 int p16, const __nv_bfloat16* s_hi, const __nv_bfloat16* s_lo, cudaStream_t stream);

// FP32 SIMT product in item mode: one CTA per item; FP32 arena rows (ld = arena.d_pad),
// S = FP32 arena [rows_pad][p_max].  All problems share `kind`.
int kmv_simt_items(DeviceContext* ctx, int kind, const RowOperand& arena, const KmvItemTables& tab,
                   const float* S, int p_max, cudaStream_t stream);

}  // namespace itergp
