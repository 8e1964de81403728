// Operand preparation and dispatch of the kernel product Y = k(A, B) S.
#include <algorithm>

#include <cuda_fp16.h>

#include "internal.h"

namespace itergp {
namespace {

// Split rows (BF16X3, BF16_COMP), one CTA of 8 warps per 128-row tile.  Pass 1 finds the
// tile's largest |x| = m 2^k (m in [0.5, 1)) and takes e = 8 - k, so that 2^e |x| < 256
// with the largest in [128, 256); pass 2 writes hi = fp16(2^e x) and
// lo = fp16(2^e x - hi), zero-padded to d_pad (2^e x and the difference are exact in FP32,
// so hi + lo holds 2^e x to 22 bits), and the squared norm of the unscaled FP32 row.
// tscale = 2^-e.  FP16 keeps its relative precision over the whole scaled range: elements
// below 4 (of up to 256) only lose lo bits below 2^-24, i.e. an absolute 2^-33 of the
// tile's largest value.
// The norm is summed per lane in FP32 with the exact error of each square (FMA) and of
// each addition (TwoSum) carried in a second FP32 word, then across lanes in FP64: FP64
// accuracy for the few dozen terms of a lane at FP32 speed (this GPU's FP64 unit is about
// 1/64 of its FP32 rate).  VEC: rows 16-byte aligned with d a multiple of 4, loaded as
// float4 and stored as pairs of half2.
__device__ __forceinline__ void sq_accumulate(float x, float& s, float& c) {
  const float p = x * x;
  const float pe = fmaf(x, x, -p);        // x^2 = p + pe exactly
  const float t = s + p;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (p - bp);   // s + p = t + err exactly (TwoSum)
  s = t;
  c += err + pe;
}

template <bool VEC>
__global__ void prep_rows_split_kernel(const float* __restrict__ X, int64_t ldX, int64_t rows, int d, int d_pad,
                                       __half* __restrict__ hi, __half* __restrict__ lo, float* __restrict__ norms,
                                       float* __restrict__ tscale) {
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 128;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __shared__ float wmax[8];
  __shared__ int e_s;
  float mx = 0.f;
  for (int rr = warp; rr < 128 && r0 + rr < rows; rr += 8) {
    if constexpr (VEC) {
      const float4* xr = reinterpret_cast<const float4*>(X + (r0 + rr) * ldX);
#pragma unroll 2
      for (int c4 = lane; c4 < d / 4; c4 += 32) {
        const float4 v = xr[c4];
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
    } else {
#pragma unroll 4
      for (int col = lane; col < d; col += 32) mx = fmaxf(mx, fabsf(X[(r0 + rr) * ldX + col]));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) wmax[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < 8; ++w) m = fmaxf(m, wmax[w]);
    const int e = scale_exp_of_max(__float_as_uint(m));   // non-finite data: no scaling
    e_s = e;
    tscale[blockIdx.x] = pow2i(-e);
  }
  __syncthreads();
  const float sc = pow2i(e_s);
  for (int rr = warp; rr < 128; rr += 8) {
    const int64_t row = r0 + rr;
    float s = 0.f, c = 0.f;
    if constexpr (VEC) {
      const float4* xr = reinterpret_cast<const float4*>(X + row * ldX);
      __half2* h2 = reinterpret_cast<__half2*>(hi + row * d_pad);
      __half2* l2 = reinterpret_cast<__half2*>(lo + row * d_pad);
#pragma unroll 2
      for (int c4 = lane; c4 < d_pad / 4; c4 += 32) {
        const float4 v = (row < rows && c4 < d / 4) ? xr[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
        sq_accumulate(v.x, s, c);
        sq_accumulate(v.y, s, c);
        sq_accumulate(v.z, s, c);
        sq_accumulate(v.w, s, c);
        const float a0 = v.x * sc, a1 = v.y * sc, a2 = v.z * sc, a3 = v.w * sc;
        const __half2 hA = __floats2half2_rn(a0, a1), hB = __floats2half2_rn(a2, a3);
        const float2 fA = __half22float2(hA), fB = __half22float2(hB);
        h2[2 * c4] = hA;
        h2[2 * c4 + 1] = hB;
        l2[2 * c4] = __floats2half2_rn(a0 - fA.x, a1 - fA.y);
        l2[2 * c4 + 1] = __floats2half2_rn(a2 - fB.x, a3 - fB.y);
      }
    } else {
#pragma unroll 4
      for (int col = lane; col < d_pad; col += 32) {
        const float x = (row < rows && col < d) ? X[row * ldX + col] : 0.f;
        const float xs = x * sc;
        const __half h = __float2half_rn(xs);
        hi[row * d_pad + col] = h;
        lo[row * d_pad + col] = __float2half_rn(xs - __half2float(h));
        sq_accumulate(x, s, c);
      }
    }
    double acc = static_cast<double>(s) + static_cast<double>(c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) norms[row] = static_cast<float>(acc);
  }
}

// The split-row preparation of rows_pad / 128 tiles, with 16-byte row loads where the
// rows allow them.
void launch_prep_split(const float* X, int64_t ldX, int64_t rows, int d, int64_t rows_pad, int d_pad,
                       void* hi, void* lo, float* norms, float* tscale, cudaStream_t stream) {
  const bool vec = (d % 4) == 0 && (ldX % 4) == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0;
  const unsigned grid = static_cast<unsigned>(rows_pad / kRowTile);
  __half* h = reinterpret_cast<__half*>(hi);
  __half* l = reinterpret_cast<__half*>(lo);
  if (vec)
    prep_rows_split_kernel<true><<<grid, 256, 0, stream>>>(X, ldX, rows, d, d_pad, h, l, norms, tscale),
        ::itergp::note_launch();
  else
    prep_rows_split_kernel<false><<<grid, 256, 0, stream>>>(X, ldX, rows, d, d_pad, h, l, norms, tscale),
        ::itergp::note_launch();
}

// BF16 rows (one warp per row): BF16 copies zero-padded to d_pad and the squared norm of
// the BF16-rounded row, which keeps r^2 = |a|^2 + |b|^2 - 2 a.b the exact distance between
// the rounded points (the dot product is formed from those same values).
__global__ void prep_rows_kernel(const float* __restrict__ X, int64_t ldX, int64_t rows, int d,
                                 int64_t rows_pad, int d_pad, __nv_bfloat16* __restrict__ hi,
                                 float* __restrict__ norms) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= rows_pad) return;
  float s = 0.f, c = 0.f;   // compensated FP32 (see sq_accumulate)
  for (int col = lane; col < d_pad; col += 32) {
    const float x = (row < rows && col < d) ? X[row * ldX + col] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float hf = __bfloat162float(h);
    hi[row * d_pad + col] = h;
    sq_accumulate(hf, s, c);
  }
  double acc = static_cast<double>(s) + static_cast<double>(c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) norms[row] = static_cast<float>(acc);
}

// TF32 rows: each value rounded to 10 mantissa bits (round to nearest, ties to even, on
// the bit pattern; infinities and NaNs pass unchanged) and stored as FP32, zero padding;
// squared norms of the rounded rows, so that |a|^2 + |b|^2 - 2 a.b describes one pair of
// points.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) != 0x7F800000u) {
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
  }
  return __uint_as_float(u);
}

__global__ void prep_rows_tf32_kernel(const float* __restrict__ X, int64_t ldX, int64_t rows, int d,
                                      int64_t rows_pad, int d_pad, float* __restrict__ out,
                                      float* __restrict__ norms) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= rows_pad) return;
  float s = 0.f, c = 0.f;   // compensated FP32 (see sq_accumulate)
  for (int col = lane; col < d_pad; col += 32) {
    const float x = round_tf32((row < rows && col < d) ? X[row * ldX + col] : 0.f);
    out[row * d_pad + col] = x;
    sq_accumulate(x, s, c);
  }
  double acc = static_cast<double>(s) + static_cast<double>(c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) norms[row] = static_cast<float>(acc);
}

// FP32 path: squared row norms only.
__global__ void row_norms_kernel(const float* __restrict__ X, int64_t ldX, int64_t rows, int d,
                                 float* __restrict__ norms) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= rows) return;
  float s = 0.f, c = 0.f;   // compensated FP32 (see sq_accumulate)
  for (int col = lane; col < d; col += 32) sq_accumulate(X[row * ldX + col], s, c);
  double acc = static_cast<double>(s) + static_cast<double>(c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) norms[row] = static_cast<float>(acc);
}

__global__ void zero_rows_kernel(float* __restrict__ Y, int64_t m, int64_t p, int64_t ldY,
                                 const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  const int64_t total = m * p;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    Y[(e / p) * ldY + e % p] = 0.f;
}

}  // namespace

int prepare_rows_into(int precision, const float* X, int64_t rows, int d, int64_t ldX,
                      int64_t rows_pad, int d_pad, __nv_bfloat16* hi, __nv_bfloat16* lo,
                      float* norms, float* tscale, cudaStream_t stream) {
  if (rows_pad <= 0) return ITERGP_OK;
  if (rows_pad < rows || d_pad < d || !norms) return ITERGP_EINVAL;
  if (!precision_is_tensor(precision)) {
    if (rows > 0) {
      row_norms_kernel<<<static_cast<unsigned>(ceil_div(rows, 8)), 256, 0, stream>>>(X, ldX, rows, d, norms), ::itergp::note_launch();
      ITERGP_CUDA_TRY(cudaGetLastError());
    }
    return ITERGP_OK;
  }
  if (!hi || d_pad % 64 != 0 || (precision_splits_rows(precision) && (!lo || !tscale || rows_pad % kRowTile != 0)))
    return ITERGP_EINVAL;
  const unsigned blocks = static_cast<unsigned>(ceil_div(rows_pad, 8));
  if (precision_tf32_rows(precision))
    prep_rows_tf32_kernel<<<blocks, 256, 0, stream>>>(X, ldX, rows, d, rows_pad, d_pad, reinterpret_cast<float*>(hi), norms), ::itergp::note_launch();
  else if (precision_splits_rows(precision))
    launch_prep_split(X, ldX, rows, d, rows_pad, d_pad, hi, lo, norms, tscale, stream);
  else
    prep_rows_kernel<<<blocks, 256, 0, stream>>>(X, ldX, rows, d, rows_pad, d_pad, hi, norms), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  return ITERGP_OK;
}

size_t rows_workspace_bytes(int precision, int64_t rows, int d) {
  const int64_t rows_pad = (rows + kRowTile - 1) / kRowTile * kRowTile;
  size_t bytes = align_up(sizeof(float) * std::max<int64_t>(rows_pad, 1), 256);
  if (precision_splits_rows(precision)) bytes += align_up(sizeof(float) * std::max<int64_t>(rows_pad / kRowTile, 1), 256);
  if (precision_is_tensor(precision)) {
    const int64_t d_pad = (d + 63) / 64 * 64;
    const size_t plane = align_up(static_cast<size_t>(rows_pad) * d_pad * 2, 256);
    bytes += plane * precision_row_planes(precision);
  }
  return bytes;
}

int prepare_rows(int precision, const float* X, int64_t rows, int d, int64_t ldX, void* mem,
                 RowOperand* op, cudaStream_t stream) {
  op->X = X;
  op->rows = rows;
  op->d = d;
  op->ldX = ldX;
  op->precision = precision;
  op->rows_pad = (rows + kRowTile - 1) / kRowTile * kRowTile;
  char* base = static_cast<char*>(mem);
  float* norms = reinterpret_cast<float*>(base);
  op->norms = norms;
  const size_t norm_bytes = align_up(sizeof(float) * std::max<int64_t>(op->rows_pad, 1), 256);
  if (!precision_is_tensor(precision)) {
    op->d_pad = d;
    op->hi = op->lo = nullptr;
    op->tscale = nullptr;
    if (rows > 0) {
      row_norms_kernel<<<static_cast<unsigned>(ceil_div(rows, 8)), 256, 0, stream>>>(X, ldX, rows, d, norms), ::itergp::note_launch();
      ITERGP_CUDA_TRY(cudaGetLastError());
    }
    return ITERGP_OK;
  }
  op->d_pad = (d + 63) / 64 * 64;
  const size_t plane = align_up(static_cast<size_t>(op->rows_pad) * op->d_pad * 2, 256);
  // split rows: the tile scales follow the norms
  const bool split = precision_splits_rows(precision);
  float* tscale = split ? reinterpret_cast<float*>(base + norm_bytes) : nullptr;
  const size_t planes0 =
      norm_bytes + (split ? align_up(sizeof(float) * std::max<int64_t>(op->rows_pad / kRowTile, 1), 256) : 0);
  __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(base + planes0);
  __nv_bfloat16* lo = split ? reinterpret_cast<__nv_bfloat16*>(base + planes0 + plane) : nullptr;
  op->hi = hi;
  op->lo = lo;
  op->tscale = tscale;
  if (op->rows_pad == 0) return ITERGP_OK;
  const unsigned blocks = static_cast<unsigned>(ceil_div(op->rows_pad, 8));
  if (precision_tf32_rows(precision))   // one FP32 plane in the bytes of two BF16 planes
    prep_rows_tf32_kernel<<<blocks, 256, 0, stream>>>(X, ldX, rows, d, op->rows_pad, op->d_pad,
                                                      reinterpret_cast<float*>(hi), norms), ::itergp::note_launch();
  else if (lo)
    launch_prep_split(X, ldX, rows, d, op->rows_pad, op->d_pad, hi, lo, norms, tscale, stream);
  else
    prep_rows_kernel<<<blocks, 256, 0, stream>>>(X, ldX, rows, d, op->rows_pad, op->d_pad, hi, norms), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  return ITERGP_OK;
}

namespace {
// out[r, q] = S[r, c0 + C q]  (r < rows, q < pc): one class's columns of a CN-ordered block
__global__ void gather_class_cols_kernel(const float* __restrict__ S, int64_t ldS, int64_t rows, int c0, int C,
                                         int64_t pc, float* __restrict__ out, const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  const int64_t total = rows * pc;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / pc, q = e % pc;
    out[e] = S[r * ldS + c0 + C * q];
  }
}

// Y[r, c0 + C q] = in[r, q]
__global__ void scatter_class_cols_kernel(const float* __restrict__ in, int64_t rows, int c0, int C, int64_t pc,
                                          float* __restrict__ Y, int64_t ldY, const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  const int64_t total = rows * pc;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / pc, q = e % pc;
    Y[r * ldY + c0 + C * q] = in[e];
  }
}
}  // namespace

int kmv_classes(DeviceContext* ctx, const KParams* kps, int C, const RowOperand& A, const RowOperand& B,
                const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY, cudaStream_t stream,
                const int* active) {
  if (A.rows == 0 || p == 0) return ITERGP_OK;
  if (C < 1 || C > 64) return ITERGP_EINVAL;
  const int64_t pc_max = (p + C - 1) / C;
  const size_t sb = align_up(sizeof(float) * std::max<int64_t>(B.rows, 1) * pc_max, 256);
  const size_t yb = align_up(sizeof(float) * A.rows * pc_max, 256);
  Scratch buf;
  ITERGP_CUDA_TRY(buf.alloc(ctx, sb + yb, stream));
  float* Sc = buf.as<float>();
  float* Yc = buf.as<float>(sb);
  for (int c = 0; c < C && c < p; ++c) {
    const int64_t pc = (p - c + C - 1) / C;   // columns c, c + C, ... below p
    if (B.rows > 0) {
      const unsigned g = static_cast<unsigned>(std::min<int64_t>(ceil_div(B.rows * pc, 256), 8LL * ctx->num_sms));
      gather_class_cols_kernel<<<g, 256, 0, stream>>>(S, ldS, B.rows, c, C, pc, Sc, active), ::itergp::note_launch();
      ITERGP_CUDA_TRY(cudaGetLastError());
    }
    int rc = kmv_execute(ctx, kps[c], A, B, Sc, pc, pc, Yc, pc, stream, active);
    if (rc != ITERGP_OK) return rc;
    const unsigned g = static_cast<unsigned>(std::min<int64_t>(ceil_div(A.rows * pc, 256), 8LL * ctx->num_sms));
    scatter_class_cols_kernel<<<g, 256, 0, stream>>>(Yc, A.rows, c, C, pc, Y, ldY, active), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
  }
  return ITERGP_OK;
}

int kmv_execute(DeviceContext* ctx, const KParams& kp, const RowOperand& A, const RowOperand& B,
                const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY,
                cudaStream_t stream, const int* active) {
  if (A.rows == 0 || p == 0) return ITERGP_OK;
  if (B.rows == 0) {
    const int64_t total = A.rows * p;
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(ceil_div(total, 256), 4096));
    zero_rows_kernel<<<blocks, 256, 0, stream>>>(Y, A.rows, p, ldY, active), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
    return ITERGP_OK;
  }
  if (precision_is_tensor(A.precision)) {
    if (!ctx->tcgen05) return ITERGP_EUNSUPPORTED;
    return kmv_tc(ctx, kp, A, B, S, ldS, p, Y, ldY, stream, active);
  }
  return kmv_simt(ctx, kp, A, B, S, ldS, p, Y, ldY, stream, active);
}

}  // namespace itergp
