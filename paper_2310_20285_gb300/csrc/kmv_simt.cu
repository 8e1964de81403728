// Plain FP32 kernel product Y = k(A, B) S on the CUDA cores (FFMA), K never stored.
//
// CTA tile: 128 rows of A x 64 rows of B per step.  The squared distances come from the
// expansion |a|^2 + |b|^2 - 2 a.b (App. B.3.1 leaves the product to the implementation;
// the expansion turns the D-contraction into a register-blocked dot product), the
// kernel tile is formed in registers, staged in shared memory and contracted with the
// matching 64 rows of S into a per-CTA accumulator that stays in registers across the
// whole row range.  Column ranges are split over grid.y when there are too few row tiles
// to fill the GPU; split partial sums are reduced in a fixed order afterwards, so the
// result is deterministic.
#include <algorithm>

#include "internal.h"

namespace itergp {
namespace {

constexpr int BM = 128, BN = 64, BK = 16;
constexpr int APAD = BM + 4, BPAD = BN + 4, KPAD = BM + 4;

template <int PJ>
struct SimtSmem {
  float As[2][BK][APAD];
  float Bs[2][BK][BPAD];
  float Ks[BN][KPAD];
  float Ss[BN][16 * PJ + 4];
};

template <int KIND, int PJ>
__global__ void __launch_bounds__(256, PJ >= 8 ? 1 : 2)
kmv_simt_kernel(const float* __restrict__ A, int64_t ldA, const float* __restrict__ na, int64_t m,
                const float* __restrict__ B, int64_t ldB, const float* __restrict__ nb, int64_t n,
                int d, const float* __restrict__ S, int64_t ldS, int64_t p, float* __restrict__ out,
                int64_t ldo, int64_t split_stride, int chunks_per_split, KParams kp,
                const int* __restrict__ active, const WorkItem* __restrict__ items,
                const TcProb* __restrict__ probs) {
  if (active != nullptr && *active == 0) return;
  constexpr int PT = 16 * PJ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SimtSmem<PJ>& sm = *reinterpret_cast<SimtSmem<PJ>*>(smem_raw);

  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  int64_t m0 = static_cast<int64_t>(blockIdx.x) * BM;
  if (items != nullptr) {
    // item mode: one whole row tile of one problem of a batch (A = B = the row arena)
    const WorkItem it = items[blockIdx.x];
    const TcProb pr = probs[it.prob];
    if (pr.active != nullptr && *pr.active == 0) return;
    A += static_cast<int64_t>(it.a_row) * ldA;
    na += it.a_row;
    m = pr.m - it.tile_row < BM ? pr.m - it.tile_row : BM;
    m0 = 0;
    B += static_cast<int64_t>(it.b_row0) * ldB;
    nb += it.b_row0;
    n = it.n_rows;
    S += static_cast<int64_t>(it.b_row0) * ldS;
    p = pr.p_valid;
    out = pr.Y + static_cast<int64_t>(it.tile_row) * pr.ldY;
    ldo = pr.ldY;
    kp = pr.kp;
    chunks_per_split = static_cast<int>((n + BN - 1) / BN);
  }
  const int64_t p0 = static_cast<int64_t>(blockIdx.z) * PT;
  const int64_t n_chunks = (n + BN - 1) / BN;
  const int64_t c_begin = static_cast<int64_t>(blockIdx.y) * chunks_per_split;
  const int64_t c_end = c_begin + chunks_per_split < n_chunks ? c_begin + chunks_per_split : n_chunks;

  float o[8][PJ];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < PJ; ++j) o[i][j] = 0.f;

  float na_r[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + ty * 8 + i;
    na_r[i] = r < m ? na[r] : 0.f;
  }
  const int nkt = (d + BK - 1) / BK;

  for (int64_t c = c_begin; c < c_end; ++c) {
    const int64_t n0 = c * BN;
    // ---- GEMM1: acc = A_tile . B_tile^T over d, double-buffered through shared memory
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    float ra[8], rb[4];
    auto load_tiles = [&](int kt) {
      const int k0 = kt * BK;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = tid + 256 * t, row = e / BK, kk = e % BK;
        const int64_t gr = m0 + row;
        ra[t] = (gr < m && k0 + kk < d) ? A[gr * ldA + k0 + kk] : 0.f;
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = tid + 256 * t, row = e / BK, kk = e % BK;
        const int64_t gr = n0 + row;
        rb[t] = (gr < n && k0 + kk < d) ? B[gr * ldB + k0 + kk] : 0.f;
      }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = tid + 256 * t;
        sm.As[buf][e % BK][e / BK] = ra[t];
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = tid + 256 * t;
        sm.Bs[buf][e % BK][e / BK] = rb[t];
      }
    };
    __syncthreads();  // previous chunk finished with Ks/Ss/As/Bs
    load_tiles(0);
    store_tiles(0);
    __syncthreads();
    for (int kt = 0; kt < nkt; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nkt) load_tiles(kt + 1);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&sm.As[buf][k][ty * 8]);
        const float4 a1 = *reinterpret_cast<const float4*>(&sm.As[buf][k][ty * 8 + 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&sm.Bs[buf][k][tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (kt + 1 < nkt) store_tiles(buf ^ 1);
      __syncthreads();
    }

    // ---- kernel tile: k(r^2) with r^2 = max(0, |a|^2 + |b|^2 - 2 a.b) -> Ks[col][row]
    float nb_c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t cc = n0 + tx * 4 + j;
      nb_c[j] = cc < n ? nb[cc] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float kv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float r2 = fmaxf(fmaf(-2.f, acc[i][j], na_r[i] + nb_c[j]), 0.f);
        kv[i] = kernel_eval_accurate<KIND>(r2, kp);
      }
      float4* dst = reinterpret_cast<float4*>(&sm.Ks[tx * 4 + j][ty * 8]);
      dst[0] = make_float4(kv[0], kv[1], kv[2], kv[3]);
      dst[1] = make_float4(kv[4], kv[5], kv[6], kv[7]);
    }
    // ---- S rows of this chunk (zero beyond n and beyond p)
    for (int e = tid; e < BN * PT; e += 256) {
      const int row = e / PT, col = e % PT;
      const int64_t gr = n0 + row, gc = p0 + col;
      sm.Ss[row][col] = (gr < n && gc < p) ? S[gr * ldS + gc] : 0.f;
    }
    __syncthreads();
    // ---- GEMM2: o += Ks^T (128 x 64) . Ss (64 x PT)
#pragma unroll 4
    for (int cc = 0; cc < BN; ++cc) {
      const float4 k0 = *reinterpret_cast<const float4*>(&sm.Ks[cc][ty * 8]);
      const float4 k1 = *reinterpret_cast<const float4*>(&sm.Ks[cc][ty * 8 + 4]);
      const float kv[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
      float sv[PJ];
      if constexpr (PJ >= 4) {
#pragma unroll
        for (int j = 0; j < PJ; j += 4) {
          const float4 q = *reinterpret_cast<const float4*>(&sm.Ss[cc][tx * PJ + j]);
          sv[j] = q.x; sv[j + 1] = q.y; sv[j + 2] = q.z; sv[j + 3] = q.w;
        }
      } else if constexpr (PJ == 2) {
        const float2 q = *reinterpret_cast<const float2*>(&sm.Ss[cc][tx * 2]);
        sv[0] = q.x; sv[1] = q.y;
      } else {
        sv[0] = sm.Ss[cc][tx];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < PJ; ++j) o[i][j] = fmaf(kv[i], sv[j], o[i][j]);
    }
  }

  float* dst = out + static_cast<int64_t>(blockIdx.y) * split_stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + ty * 8 + i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < PJ; ++j) {
      const int64_t cidx = p0 + tx * PJ + j;
      if (cidx < p) dst[r * ldo + cidx] = o[i][j];
    }
  }
}

// Y[i, :] = sum_s part[s][i, :] in split order (deterministic).
__global__ void reduce_splits_kernel(const float* __restrict__ part, int splits, int64_t m,
                                     int64_t p, float* __restrict__ Y, int64_t ldY,
                                     const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  const int64_t total = m * p;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < splits; ++s) acc += part[s * total + e];
    Y[(e / p) * ldY + e % p] = acc;
  }
}

template <int KIND, int PJ>
cudaError_t launch_simt(dim3 grid, cudaStream_t st, const RowOperand& A, const RowOperand& B,
                        const float* S, int64_t ldS, int64_t p, float* out, int64_t ldo,
                        int64_t split_stride, int cps, const KParams& kp, const int* active,
                        const WorkItem* items = nullptr, const TcProb* probs = nullptr) {
  const size_t smem = sizeof(SimtSmem<PJ>);
  auto fn = kmv_simt_kernel<KIND, PJ>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  timing_begin(st);
  fn<<<grid, 256, smem, st>>>(A.X, A.ldX, A.norms, A.rows, B.X, B.ldX, B.norms, B.rows, A.d, S, ldS,
                              p, out, ldo, split_stride, cps, kp, active, items, probs), ::itergp::note_launch();
  timing_end(st);
  return cudaGetLastError();
}

template <int KIND>
cudaError_t dispatch_pj(int pj, dim3 grid, cudaStream_t st, const RowOperand& A,
                        const RowOperand& B, const float* S, int64_t ldS, int64_t p, float* out,
                        int64_t ldo, int64_t split_stride, int cps, const KParams& kp,
                        const int* active) {
  switch (pj) {
    case 1: return launch_simt<KIND, 1>(grid, st, A, B, S, ldS, p, out, ldo, split_stride, cps, kp, active);
    case 2: return launch_simt<KIND, 2>(grid, st, A, B, S, ldS, p, out, ldo, split_stride, cps, kp, active);
    case 4: return launch_simt<KIND, 4>(grid, st, A, B, S, ldS, p, out, ldo, split_stride, cps, kp, active);
    default: return launch_simt<KIND, 8>(grid, st, A, B, S, ldS, p, out, ldo, split_stride, cps, kp, active);
  }
}

template <int KIND>
cudaError_t dispatch_items(int pj, dim3 grid, cudaStream_t st, const RowOperand& A,
                           const RowOperand& B, const float* S, int64_t ldS, int p_max,
                           const KParams& kp, const KmvItemTables& tab) {
  switch (pj) {
    case 1: return launch_simt<KIND, 1>(grid, st, A, B, S, ldS, p_max, nullptr, 0, 0, 0, kp, nullptr, tab.items, tab.probs);
    case 2: return launch_simt<KIND, 2>(grid, st, A, B, S, ldS, p_max, nullptr, 0, 0, 0, kp, nullptr, tab.items, tab.probs);
    case 4: return launch_simt<KIND, 4>(grid, st, A, B, S, ldS, p_max, nullptr, 0, 0, 0, kp, nullptr, tab.items, tab.probs);
    default: return launch_simt<KIND, 8>(grid, st, A, B, S, ldS, p_max, nullptr, 0, 0, 0, kp, nullptr, tab.items, tab.probs);
  }
}

}  // namespace

int kmv_simt_items(DeviceContext* ctx, int kind, const RowOperand& A, const RowOperand& B,
                   const KmvItemTables& tab, const float* S, int64_t ldS, int p_max,
                   cudaStream_t stream) {
  (void)ctx;
  if (tab.n_items <= 0) return ITERGP_OK;
  if (p_max < 1 || p_max > 128 || ldS < p_max || A.d != B.d || A.precision != ITERGP_FP32)
    return ITERGP_EINVAL;
  const int pj = p_max <= 16 ? 1 : p_max <= 32 ? 2 : p_max <= 64 ? 4 : 8;
  dim3 grid(static_cast<unsigned>(tab.n_items), 1, 1);
  const KParams kp = make_kparams(itergp_kernel{kind, 1.f, 1.f});   // per-item values from the table
  cudaError_t e = kind == ITERGP_RBF ? dispatch_items<ITERGP_RBF>(pj, grid, stream, A, B, S, ldS, p_max, kp, tab)
                                     : dispatch_items<ITERGP_MATERN32>(pj, grid, stream, A, B, S, ldS, p_max, kp, tab);
  ITERGP_CUDA_TRY(e);
  return ITERGP_OK;
}

int kmv_simt(DeviceContext* ctx, const KParams& kp, const RowOperand& A, const RowOperand& B,
             const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY, cudaStream_t stream,
             const int* active) {
  const int pj = p <= 16 ? 1 : p <= 32 ? 2 : p <= 64 ? 4 : 8;
  const int64_t p_tiles = ceil_div(p, 16 * pj);
  const int64_t row_tiles = ceil_div(A.rows, BM);
  const int64_t chunks = ceil_div(B.rows, BN);
  // enough CTAs for ~2 waves at 2 CTAs per SM; split the column range if needed
  const int64_t target = 4LL * ctx->num_sms;
  int64_t splits = 1;
  if (row_tiles * p_tiles < target) splits = ceil_div(target, row_tiles * p_tiles);
  if (splits > chunks) splits = chunks;
  const int64_t cps = ceil_div(chunks, splits);
  splits = ceil_div(chunks, cps);
  dim3 grid(static_cast<unsigned>(row_tiles), static_cast<unsigned>(splits),
            static_cast<unsigned>(p_tiles));
  Scratch part;
  float* out = Y;
  int64_t ldo = ldY, split_stride = 0;
  if (splits > 1) {
    ITERGP_CUDA_TRY(part.alloc(ctx, sizeof(float) * splits * A.rows * p, stream));
    out = part.as<float>();
    ldo = p;
    split_stride = A.rows * p;
  }
  cudaError_t e = kp.kind == ITERGP_RBF
                      ? dispatch_pj<ITERGP_RBF>(pj, grid, stream, A, B, S, ldS, p, out, ldo, split_stride, (int)cps, kp, active)
                      : dispatch_pj<ITERGP_MATERN32>(pj, grid, stream, A, B, S, ldS, p, out, ldo, split_stride, (int)cps, kp, active);
  ITERGP_CUDA_TRY(e);
  if (splits > 1) {
    const int64_t total = A.rows * p;
    const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(total, 256), 8LL * ctx->num_sms));
    reduce_splits_kernel<<<blocks, 256, 0, stream>>>(part.as<float>(), (int)splits, A.rows, p, Y, ldY, active), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
  }
  return ITERGP_OK;
}

}  // namespace itergp
