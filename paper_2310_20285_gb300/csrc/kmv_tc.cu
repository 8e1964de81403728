// Tensor-core kernel product Y = k(A, B) S for sm_103a (tcgen05 + TMEM + TMA): host side,
// the one-CTA instantiations, the tail fix-up, the weight staging and the tuner.
//
// The product of App. B.3.1 is evaluated flash-style and K is never stored:
//   for each (row tile of A, column chunk of B):
//     G   = A_tile . B_chunk^T        tcgen05.mma, 16-bit operands, FP32 accumulator in TMEM
//     P   = k(|a|^2 + |b|^2 - 2 G)    epilogue warps: TMEM -> registers -> 16-bit -> TMEM
//     O  += P . S_chunk               tcgen05.mma with P read from TMEM (A operand)
// Operands are staged by TMA with 128-byte swizzle.  The split precisions use FP16 hi/lo
// parts with power-of-two scales (rows per 128-row tile, weights per column, kernel
// values by 2^ke): a.b ~ ah.bh + ah.bl + al.bh and P S ~ Ph Sh + Ph Sl + Pl Sh.
//
// Forms (kmv_tc_impl.cuh): one CTA per 128-row tile (128-row chunks; instantiated here),
// and CTA pairs sharing 256-row tiles through cta_group::2 MMAs with 128- or 192-row
// chunks (kmv_tc2.cu).  Warp roles: warp 0 issues the A/B TMA loads, warp 1 the MMAs
// (one thread), warp 2 owns TMEM, warp 3 loads the weight tiles, warps 4-7 (or 4-11) run
// the kernel evaluation and the output stores.
//
// The tensor core accumulates in FP32 with truncation, which biases long sums; O is
// therefore accumulated over sub-runs of a few chunks and each sub-run is added into a
// running sum (TMEM, or registers in the wide form) by the epilogue with ordinary FP32
// adds.
//
// Work partition (G persistent CTAs or pairs, R row tiles, J column chunks): the first
// floor(R / G) * G row tiles are processed whole, one wave at a time, and every CTA sweeps
// the column chunks in the same order 0 .. J-1, so at any moment all CTAs read the same
// tile of B and the L2 serves it to all of them (B is larger than the L2 at the large
// sizes).  The remaining R mod G row tiles form Ut = (R mod G) * J units split into equal
// contiguous ranges over the G CTAs; partial runs there (at most the first and last of a
// CTA) go to scratch and a fix-up kernel adds them in CTA order, so results are
// deterministic.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cstring>

#include "kmv_tc_impl.cuh"
#include "tma_host.h"

namespace itergp {
namespace {

using namespace tcimpl;

// Adds the partial runs of tail row tiles (of tm rows) shared by several CTAs (or pairs),
// in their order.
__global__ void tc_fixup_kernel(const float* __restrict__ partial, int64_t R, int64_t G, int J, int tm,
                                int64_t m, int p_pad, int p_valid, float* __restrict__ Y,
                                int64_t ldY, const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  const int64_t rt0 = (R / G) * G, ut = (R - rt0) * J;
  const int64_t r = rt0 + blockIdx.x;
  if (r >= R) return;
  const int64_t u0 = (r - rt0) * J, u1 = u0 + J - 1;
  const int64_t g_lo = part_owner(u0, ut, G), g_hi = part_owner(u1, ut, G);
  if (g_lo == g_hi) return;   // one CTA covered the whole row tile and stored it
  // grid: (tail row tiles, blocks per tile); every element of the tile is one thread's sum
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < tm * p_valid; e += gridDim.y * blockDim.x) {
    const int row = e / p_valid, col = e % p_valid;
    const int64_t grow = r * tm + row;
    if (grow >= m) continue;
    float acc = 0.f;
    for (int64_t gg = g_lo; gg <= g_hi; ++gg) {
      const int64_t s0 = part_start(gg, ut, G);
      if (s0 == part_start(gg + 1, ut, G)) continue;   // CTA without tail units
      const int64_t slot = 2 * gg + (s0 < u0 ? 1 : 0);
      acc += partial[(slot * tm + row) * p_pad + col];
    }
    Y[grow * ldY + col] = acc;
  }
}


// Largest |S[:, c]| of each column c < p, as float bits (non-negative floats order like
// their bit patterns): one block per 256-row band and 32-column group, one atomicMax per
// column and block into cmax (zeroed by the caller).
__global__ void colmax_kernel(const float* __restrict__ S, int64_t ldS, int64_t n, int64_t p,
                              uint32_t* __restrict__ cmax, const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  __shared__ float part[8][33];
  const int64_t c = static_cast<int64_t>(blockIdx.y) * 32 + threadIdx.x;
  const int64_t j0 = static_cast<int64_t>(blockIdx.x) * 256;
  float m = 0.f;
  if (c < p)
    for (int64_t j = j0 + threadIdx.y; j < j0 + 256 && j < n; j += 8) m = fmaxf(m, fabsf(S[j * ldS + c]));
  part[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && c < p) {
    for (int i = 1; i < 8; ++i) m = fmaxf(m, part[i][threadIdx.x]);
    atomicMax(&cmax[c], __float_as_uint(m));
  }
}

// S (n x p, row pitch ldS) -> transposed weights [p16][n_pad], zero padded.  SPLIT (the
// BF16X3 and TF32 forms): FP16 hi and lo of 2^e_c S[:, c], with e_c from the column's
// largest |value| (cmax, see colmax_kernel) so that it lies in [128, 256); wscale[c] =
// 2^-e_c (22 significant bits at any magnitude).  Otherwise one BF16 plane.
template <bool SPLIT>
__global__ void prep_s_kernel(const float* __restrict__ S, int64_t ldS, int64_t n, int64_t p,
                              int64_t n_pad, int64_t p16, __nv_bfloat16* __restrict__ hi,
                              __nv_bfloat16* __restrict__ lo, const uint32_t* __restrict__ cmax,
                              float* __restrict__ wscale, const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  __shared__ float tile[32][33];
  const int64_t j0 = static_cast<int64_t>(blockIdx.x) * 32, c0 = static_cast<int64_t>(blockIdx.y) * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t j = j0 + i, cc = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (j < n && cc < p) ? S[j * ldS + cc] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t cc = c0 + i, j = j0 + threadIdx.x;
    if (cc < p16 && j < n_pad) {
      const float x = tile[threadIdx.x][i];
      if constexpr (SPLIT) {
        const int e = cc < p ? scale_exp_of_max(cmax[cc]) : 0;
        const float xs = x * pow2i(e);
        const __half h = __float2half_rn(xs);
        reinterpret_cast<__half*>(hi)[cc * n_pad + j] = h;
        reinterpret_cast<__half*>(lo)[cc * n_pad + j] = __float2half_rn(xs - __half2float(h));
        if (blockIdx.x == 0 && threadIdx.x == 0) wscale[cc] = pow2i(-e);
      } else {
        hi[cc * n_pad + j] = __float2bfloat16_rn(x);
      }
    }
  }
}

// Column maxima, then the transposed (split) weights; cmax / wscale: [p16] device scratch.
cudaError_t stage_weights(const float* S, int64_t ldS, int64_t n, int64_t p, int64_t n_pad, int64_t p16,
                          __nv_bfloat16* hi, __nv_bfloat16* lo, uint32_t* cmax, float* wscale, bool split,
                          const int* active, cudaStream_t stream) {
  dim3 grid(static_cast<unsigned>(n_pad / 32), static_cast<unsigned>(ceil_div(p16, 32)));
  if (split) {
    cudaError_t e = cudaMemsetAsync(cmax, 0, sizeof(uint32_t) * p16, stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
      colmax_kernel<<<dim3(static_cast<unsigned>(ceil_div(n, 256)), static_cast<unsigned>(ceil_div(p, 32))),
                      dim3(32, 8), 0, stream>>>(S, ldS, n, p, cmax, active), ::itergp::note_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    prep_s_kernel<true><<<grid, dim3(32, 8), 0, stream>>>(S, ldS, n, p, n_pad, p16, hi, lo, cmax, wscale, active), ::itergp::note_launch();
  } else {
    prep_s_kernel<false><<<grid, dim3(32, 8), 0, stream>>>(S, ldS, n, p, n_pad, p16, hi, lo, nullptr, nullptr, active), ::itergp::note_launch();
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- launch variants
// A variant: epilogue warps (4 or 8) and pipeline stages (0: the deepest that fits).
// The table holds what the autotuner measured per (precision, kind, d_pad, P tile,
// schedule); a thread may force a variant while it times candidates.
struct TcVariant {
  int epi = 4;
  int nstage = 0;
  int ares = -1;   // resident A (one K slice only): 1 on, 0 off, -1 on where possible
  int pair = -1;   // CTA-pair form (single-problem streamed ring): 1 on with 128-row chunks, 2 on
                   // with wide (192-row) chunks, 0 off, -1 on where possible (wide for P <= 80)
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, TcVariant> g_tune;
thread_local const TcVariant* t_forced = nullptr;

TcVariant tc_variant(int prec, int kind, int d_pad, int p_pad, int items) {
  if (t_forced) return *t_forced;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(prec, kind, d_pad, std::min(p_pad, 128), items));
  return it == g_tune.end() ? TcVariant{} : it->second;
}

// Deepest instantiated stage count (<= want, 0 = no limit) that fits with P tile p_tile;
// 0 if none.  Streamed rings: 2, 3, 4 stages of A+B; resident A: 3 or 5 B-only stages.
// The one-CTA form keeps one weight-tile slot per G buffer; the pair form's stages come
// first and its weight ring takes what is left (at least one slot, at most one per G buffer).
size_t smem_cap_bytes(const DeviceContext* ctx) { return std::min<size_t>(ctx->smem_optin, 232448) - 2048; }

int stages_that_fit(const DeviceContext* ctx, int nt1, int nt2, int p_tile, int epi, int want,
                    bool ares = false, bool pair = false, int cw = BN) {
  const size_t smem_cap = smem_cap_bytes(ctx);
  const size_t a_bytes = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BM * BK * 2 : 0;
  const size_t stage = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BN * BK * 2 : stage_bytes(nt1, pair, cw);
  const size_t fixed = (pair ? 1 : g_bufs(p_tile)) * s_buf_bytes(nt2, p_tile, pair, cw) + smem_extra(epi, cw) + a_bytes;
  const int fit = static_cast<int>((smem_cap > fixed ? smem_cap - fixed : 0) / stage);
  if (cw != BN)   // wide chunks: P tiles <= 80 (TMEM), three streamed stages only
    return (pair && !ares && p_tile <= 80 && fit >= 3 && (want <= 0 || want == 3)) ? 3 : 0;
  int ns = ares ? (fit >= 5 ? 5 : fit >= 3 ? 3 : 0) : (fit >= 4 ? 4 : fit >= 3 ? 3 : fit >= 2 ? 2 : 0);
  if (want >= 2 && ns > want) ns = ares ? (want >= 5 ? 5 : want >= 3 ? 3 : 0) : want;
  return ns;
}

int tc_nt1(int prec) { return precision_tf32_rows(prec) ? 2 : precision_splits_rows(prec) ? 3 : 1; }

// MMA K steps (32 bytes of a row each) of the last D slice that hold data: rows are zero
// padded from d to d_pad, and the steps past d are skipped.
int last_slice_ksteps(int d, int d_pad, int nt1) {
  const int slice = slice_elems(nt1), step = nt1 == 2 ? 8 : 16;
  const int rem = d - (d_pad / slice - 1) * slice;   // values in the last slice, 1 .. slice
  return rem <= 0 ? slice / step : static_cast<int>(ceil_div(rem, step));
}

// Tensor maps of the row operands (maps[1] and [3] repeat the hi planes when rows are not
// split).  Boxes: 128 rows of A; 128 rows of B, or 64 in the pair form (each CTA of a pair
// stages half of every chunk).
bool encode_rows(CUtensorMap* maps, const RowOperand& A, const RowOperand& B, int nt1, bool pair = false,
                 int cw = BN) {
  const uint32_t bb = static_cast<uint32_t>(b_rows_cta(pair, cw));
  if (nt1 == 2)
    return encode_f32_sw128(&maps[0], A.hi, A.rows_pad, A.d_pad, A.d_pad, BM) &&
           encode_f32_sw128(&maps[1], A.hi, A.rows_pad, A.d_pad, A.d_pad, BM) &&
           encode_f32_sw128(&maps[2], B.hi, B.rows_pad, B.d_pad, B.d_pad, bb) &&
           encode_f32_sw128(&maps[3], B.hi, B.rows_pad, B.d_pad, B.d_pad, bb);
  // split rows are FP16 hi/lo planes, plain 16-bit rows BF16
  const CUtensorMapDataType ty = nt1 == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return encode_bf16_sw128(&maps[0], A.hi, A.rows_pad, A.d_pad, A.d_pad, BM, ty) &&
         encode_bf16_sw128(&maps[1], nt1 == 3 ? A.lo : A.hi, A.rows_pad, A.d_pad, A.d_pad, BM, ty) &&
         encode_bf16_sw128(&maps[2], B.hi, B.rows_pad, B.d_pad, B.d_pad, bb, ty) &&
         encode_bf16_sw128(&maps[3], nt1 == 3 ? B.lo : B.hi, B.rows_pad, B.d_pad, B.d_pad, bb, ty);
}

// Weight-tile slots with nstage stages (see stages_that_fit).
int weight_slots(const DeviceContext* ctx, int nt1, int nt2, int p_tile, int epi, int nstage, bool pair,
                 int cw = BN) {
  if (!pair) return g_bufs(p_tile);
  const size_t used = nstage * static_cast<size_t>(stage_bytes(nt1, true, cw)) + smem_extra(epi, cw);
  const size_t cap = smem_cap_bytes(ctx);
  const size_t fit = cap > used ? (cap - used) / s_buf_bytes(nt2, p_tile, true, cw) : 0;
  const int bufs = cw == BN ? g_bufs(p_tile) : 2;   // wide chunks: two G buffers
  return static_cast<int>(std::max<size_t>(1, std::min<size_t>(fit, bufs)));
}

size_t tc_smem_bytes(int nt1, int nt2, int p_pad, int epi, int nstage, bool ares, int slots, bool pair = false,
                     int cw = BN) {
  const size_t a_bytes = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BM * BK * 2 : 0;
  const size_t stage = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BN * BK * 2 : stage_bytes(nt1, pair, cw);
  return nstage * stage + a_bytes + slots * s_buf_bytes(nt2, p_pad, pair, cw) + smem_extra(epi, cw);
}

// Pairs of the pair form that can be resident at once with this configuration (cached per
// configuration: the answer depends on the GPU's GPC layout, not on the problem).
int pair_clusters(int kind, int prec, int nstage, int epi, size_t smem, int cw = BN) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, size_t, int>, int> cache;
  const auto key = std::make_tuple(kind, prec, nstage, epi, smem, cw);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const int n = pair_max_clusters(kind, prec, nstage, epi, smem, cw);
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = n;
  return n;
}

}  // namespace

int kmv_tc_items(DeviceContext* ctx, int kind, const RowOperand& A, const RowOperand& B,
                 const KmvItemTables& tab, const __nv_bfloat16* s_hi, const __nv_bfloat16* s_lo,
                 int64_t s_rows, int s_row0, int p16, cudaStream_t stream) {
  const int prec = B.precision;
  const int nt1 = tc_nt1(prec);
  const int nt2 = precision_splits_weights(prec) ? 3 : 1;
  if (p16 > 256 || p16 < 16 || p16 % 16 != 0 || tab.G <= 0 || A.precision != prec ||
      A.d_pad != B.d_pad || s_row0 < 0 || s_row0 + p16 > s_rows)
    return ITERGP_EINVAL;
  // P tile: the widest multiple of 16 (<= p16) that leaves room for >= 2 stages
  const TcVariant var = tc_variant(prec, kind, B.d_pad, p16, 1);
  const bool can_ares = B.d_pad == BK && var.ares != 0 && nt1 != 2;   // one K slice: A can stay resident
  int p_tile = std::min(p16, 128), nstage = 0;
  bool ares = false;
  for (; p_tile >= 16; p_tile -= 16) {
    if (can_ares && (nstage = stages_that_fit(ctx, nt1, nt2, p_tile, var.epi, var.nstage, true)) >= 3) {
      ares = true;
      break;
    }
    nstage = stages_that_fit(ctx, nt1, nt2, p_tile, var.epi, var.nstage);
    if (nstage >= 2) break;
  }
  if (nstage < 2) return ITERGP_EUNSUPPORTED;
  CUtensorMap maps[6];
  bool ok = encode_rows(maps, A, B, nt1);
  if (!ok) return ITERGP_ECUDA;
  for (int p0 = 0; p0 < p16; p0 += p_tile) {
    const int pp = std::min(p_tile, p16 - p0);   // multiple of 16
    const CUtensorMapDataType wty = nt2 == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    ok = encode_bf16_sw128(&maps[4], s_hi, s_rows, B.rows_pad, B.rows_pad, pp, wty) &&
         encode_bf16_sw128(&maps[5], nt2 == 3 ? s_lo : s_hi, s_rows, B.rows_pad, B.rows_pad, pp, wty);
    if (!ok) return ITERGP_ECUDA;
    TcArgs a{};
    a.na = A.norms;
    a.nb = B.norms;
    a.ua = A.tscale;
    a.ub = B.tscale;
    a.wait_ns = thread_wait_limit();
    a.a_rows_pad = A.rows_pad;
    a.b_rows_pad = B.rows_pad;
    a.nk = B.d_pad / slice_elems(nt1);
    a.klast = last_slice_ksteps(std::max(A.d, B.d), B.d_pad, nt1);
    a.p_pad = pp;
    a.p_valid = pp;
    a.s_row0 = s_row0 + p0;
    a.p_col0 = p0;
    a.status = ctx->status;
    a.active = nullptr;
    a.items = tab.items;
    a.item_begin = tab.item_begin;
    a.probs = tab.probs;
    a.kp = make_kparams(itergp_kernel{kind, 1.f, 1.f});   // per-item values come from the table
    a.w_slots = g_bufs(pp);
    a.diag = &A == &B || (A.hi == B.hi && A.norms == B.norms && A.rows == B.rows);
    const size_t smem = tc_smem_bytes(nt1, nt2, pp, var.epi, nstage, ares, a.w_slots);
    cudaError_t e = kind == ITERGP_RBF
                        ? launch_prec<ITERGP_RBF, false>(prec, nstage, ares, var.epi, tab.G, smem, stream, maps, a)
                        : launch_prec<ITERGP_MATERN32, false>(prec, nstage, ares, var.epi, tab.G, smem, stream, maps, a);
    ITERGP_CUDA_TRY(e);
  }
  return ITERGP_OK;
}

int kmv_tc(DeviceContext* ctx, const KParams& kp, const RowOperand& A, const RowOperand& B,
           const float* S, int64_t ldS, int64_t p, float* Y, int64_t ldY, cudaStream_t stream,
           const int* active) {
  const int prec = A.precision;
  const int nt1 = tc_nt1(prec);
  const int nt2 = precision_splits_weights(prec) ? 3 : 1;

  // P tile: the largest multiple of 16 (<= 128) that leaves room for >= 2 stages; then the
  // deepest instantiated stage count (2, 3, 4) that fits.  (Deeper rings help only while a
  // stage's arrival is on the critical path; the issue of the MMAs by one thread bounds
  // the loop otherwise.)
  const int64_t p16 = (p + 15) / 16 * 16;
  const TcVariant var = tc_variant(prec, kp.kind, A.d_pad, static_cast<int>(std::min<int64_t>(p16, 128)), 0);
  const bool can_ares = A.d_pad == BK && var.ares != 0 && nt1 != 2;   // one K slice: A can stay resident
  int p_tile = static_cast<int>(std::min<int64_t>(p16, 128));
  int nstage = 0;
  bool ares = false;
  for (; p_tile >= 16; p_tile -= 16) {
    if (can_ares && (nstage = stages_that_fit(ctx, nt1, nt2, p_tile, var.epi, var.nstage, true)) >= 3) {
      ares = true;
      break;
    }
    nstage = stages_that_fit(ctx, nt1, nt2, p_tile, var.epi, var.nstage);
    if (nstage >= 2) break;
  }
  if (nstage < 2) return ITERGP_EUNSUPPORTED;

  // The CTA-pair form (streamed ring) replaces the one-CTA form unless the variant says
  // otherwise: by default wherever A is not kept resident and there is a full 256-row tile.
  // Wide chunks (192 rows of B) where the whole P fits one tile of <= 80 columns.
  bool pair = false;
  int cw = BN;
  int64_t pair_cap = 0;
  if ((var.pair == 2 || (var.pair == -1 && !ares)) && A.rows >= 2 * BM && p16 <= 80) {
    const int pt = static_cast<int>(p16);
    const int ns = stages_that_fit(ctx, nt1, nt2, pt, var.epi, var.nstage, false, true, kWideCW);
    if (ns == 3) {
      const int ws = weight_slots(ctx, nt1, nt2, pt, var.epi, ns, true, kWideCW);
      pair_cap = pair_clusters(kp.kind, prec, ns, var.epi,
                               tc_smem_bytes(nt1, nt2, pt, var.epi, ns, false, ws, true, kWideCW), kWideCW);
      if (pair_cap >= 1) {
        pair = true;
        cw = kWideCW;
        ares = false;
        p_tile = pt;
        nstage = ns;
      }
    }
  }
  if (!pair && (var.pair == 1 || (var.pair == -1 && !ares)) && A.rows >= 2 * BM) {
    int pt = static_cast<int>(std::min<int64_t>(p16, 128)), ns = 0;
    for (; pt >= 16; pt -= 16)
      if ((ns = stages_that_fit(ctx, nt1, nt2, pt, var.epi, var.nstage, false, true)) >= 2) break;
    if (ns >= 2) {
      const int ws = weight_slots(ctx, nt1, nt2, pt, var.epi, ns, true);
      pair_cap = pair_clusters(kp.kind, prec, ns, var.epi, tc_smem_bytes(nt1, nt2, pt, var.epi, ns, false, ws, true));
      if (pair_cap >= 1) {
        pair = true;
        ares = false;
        p_tile = pt;
        nstage = ns;
      }
    }
  }

  // transposed (split) S, with the split form's column maxima and scales after the planes
  const int64_t n_pad = B.rows_pad;
  Scratch sbuf;
  const size_t s_elems = static_cast<size_t>(p16) * n_pad;
  const size_t s_planes = align_up(s_elems * 2 * (nt2 == 3 ? 2 : 1), 256);
  ITERGP_CUDA_TRY(sbuf.alloc(ctx, s_planes + sizeof(uint32_t) * p16 * 2, stream));
  __nv_bfloat16* s_hi = sbuf.as<__nv_bfloat16>();
  __nv_bfloat16* s_lo = nt2 == 3 ? s_hi + s_elems : nullptr;
  uint32_t* s_cmax = sbuf.as<uint32_t>(s_planes);
  float* s_scale = reinterpret_cast<float*>(s_cmax + p16);
  ITERGP_CUDA_TRY(stage_weights(S, ldS, B.rows, p, n_pad, p16, s_hi, s_lo, s_cmax, s_scale, nt2 == 3, active, stream));

  CUtensorMap maps[6];
  bool ok = encode_rows(maps, A, B, nt1, pair, cw);
  if (!ok) return ITERGP_ECUDA;

  const int tm = tile_rows(pair);
  const int64_t row_tiles = ceil_div(A.rows, tm);
  const int64_t chunks = ceil_div(B.rows, static_cast<int64_t>(cw));
  const int64_t units = row_tiles * chunks;
  // persistent grid: one CTA per SM, or as many pairs as can be resident together
  const int64_t G = std::min<int64_t>(pair ? pair_cap : ctx->num_sms, units);
  const int64_t tail_rows = row_tiles - (row_tiles / G) * G;
  Scratch part;
  ITERGP_CUDA_TRY(part.alloc(ctx, sizeof(float) * 2 * G * tm * p_tile, stream));

  for (int64_t p0 = 0; p0 < p; p0 += p_tile) {
    const int pw = static_cast<int>(std::min<int64_t>(p_tile, p - p0));
    const int pp = (pw + 15) / 16 * 16;
    const uint32_t s_box_rows = static_cast<uint32_t>(pair ? pp / 2 : pp);   // pair: each CTA's half
    const CUtensorMapDataType wty = nt2 == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    ok = encode_bf16_sw128(&maps[4], s_hi, p16, n_pad, n_pad, s_box_rows, wty) &&
         encode_bf16_sw128(&maps[5], nt2 == 3 ? s_lo : s_hi, p16, n_pad, n_pad, s_box_rows, wty);
    if (!ok) return ITERGP_ECUDA;
    TcArgs a{};   // items/item_begin/probs stay null: single-problem schedule
    a.na = A.norms;
    a.nb = B.norms;
    a.ua = A.tscale;
    a.ub = B.tscale;
    a.wait_ns = thread_wait_limit();
    a.m = A.rows;
    a.a_rows_pad = A.rows_pad;
    a.b_rows_pad = B.rows_pad;
    a.row_tiles = row_tiles;
    a.chunks = static_cast<int>(chunks);
    a.nk = A.d_pad / slice_elems(nt1);
    a.klast = last_slice_ksteps(std::max(A.d, B.d), A.d_pad, nt1);
    a.p_pad = pp;
    a.p_valid = pw;
    a.s_row0 = static_cast<int>(p0);
    a.Y = Y + p0;
    a.ldY = ldY;
    a.partial = part.as<float>();
    a.wscale = s_scale;
    a.kp = kp;
    a.status = ctx->status;
    a.active = active;
    a.items = nullptr;
    a.item_begin = nullptr;
    a.probs = nullptr;
    a.w_slots = weight_slots(ctx, nt1, nt2, pp, var.epi, nstage, pair, cw);
    a.diag = A.hi == B.hi && A.norms == B.norms && A.rows == B.rows;
    const size_t smem_t = tc_smem_bytes(nt1, nt2, pp, var.epi, nstage, ares, a.w_slots, pair, cw);
    cudaError_t e;
    if (pair)
      e = launch_pair_form(kp.kind, prec, nstage, var.epi, (int)G, smem_t, stream, maps, a, cw);
    else
      e = kp.kind == ITERGP_RBF
              ? launch_prec<ITERGP_RBF, false>(prec, nstage, ares, var.epi, (int)G, smem_t, stream, maps, a)
              : launch_prec<ITERGP_MATERN32, false>(prec, nstage, ares, var.epi, (int)G, smem_t, stream, maps, a);
    ITERGP_CUDA_TRY(e);
    if (tail_rows > 0) {
      const unsigned per_tile = static_cast<unsigned>(std::min<int64_t>(ceil_div(static_cast<int64_t>(tm) * pw, 256), 64));
      tc_fixup_kernel<<<dim3(static_cast<unsigned>(tail_rows), per_tile), 256, 0, stream>>>(
          part.as<float>(), row_tiles, G, (int)chunks, tm, A.rows, pp, pw, Y + p0, ldY, active), ::itergp::note_launch();
      ITERGP_CUDA_TRY(cudaGetLastError());
    }
  }
  return ITERGP_OK;
}

}  // namespace itergp

// ---------------------------------------------------------------- autotuning
namespace itergp {

int kmv_tc_tune(DeviceContext* ctx, const KParams& kp, const RowOperand& X, const float* S,
                int64_t p, float* Y, int items, int cap, int* count, int* epi_out, int* ns_out,
                int* pair_out, double* ms_out, int* best, cudaStream_t stream) {
  const int prec = X.precision;
  const int nt1 = tc_nt1(prec);
  const int nt2 = precision_splits_weights(prec) ? 3 : 1;
  const int p16 = static_cast<int>(std::min<int64_t>((p + 15) / 16 * 16, 128));
  // item mode: one problem covering all rows, weights staged as the batched fit stages them
  Scratch tabs, sbuf;
  KmvItemTables tab;
  __nv_bfloat16 *s_hi = nullptr, *s_lo = nullptr;
  if (items) {
    if (p > 128) return ITERGP_EINVAL;
    const int chunks = static_cast<int>(ceil_div(X.rows, BM));
    std::vector<WorkItem> its;
    for (int r = 0; r < chunks; ++r)
      its.push_back(WorkItem{0, 128 * r, 128 * r, 0, chunks, static_cast<int32_t>(X.rows), 0, 0});
    const int G = static_cast<int>(std::min<int64_t>(ctx->num_sms, chunks));
    std::vector<WorkItem> ord;
    std::vector<int32_t> beg;
    plan_items(its, G, &ord, &beg);
    // weights first (the table entry points at their scales)
    const size_t s_elems = static_cast<size_t>(p16) * X.rows_pad;
    const size_t s_planes = align_up(s_elems * 2 * 2, 256);
    ITERGP_CUDA_TRY(sbuf.alloc(ctx, s_planes + sizeof(uint32_t) * p16 * 2, stream));
    s_hi = sbuf.as<__nv_bfloat16>();
    s_lo = s_hi + s_elems;
    uint32_t* cmax = sbuf.as<uint32_t>(s_planes);
    float* wsc = reinterpret_cast<float*>(cmax + p16);
    ITERGP_CUDA_TRY(stage_weights(S, p, X.rows, p, X.rows_pad, p16, s_hi, s_lo, cmax, wsc, nt2 == 3, nullptr, stream));
    TcProb pr{Y, p, X.rows, static_cast<int32_t>(p), 0, kp, nullptr, wsc};
    const size_t b_items = align_up(sizeof(WorkItem) * ord.size(), 256);
    const size_t b_beg = align_up(sizeof(int32_t) * beg.size(), 256);
    ITERGP_CUDA_TRY(tabs.alloc(ctx, b_items + b_beg + sizeof(TcProb), stream));
    ITERGP_CUDA_TRY(cudaMemcpyAsync(tabs.as<char>(), ord.data(), sizeof(WorkItem) * ord.size(), cudaMemcpyHostToDevice, stream));
    ITERGP_CUDA_TRY(cudaMemcpyAsync(tabs.as<char>(b_items), beg.data(), sizeof(int32_t) * beg.size(), cudaMemcpyHostToDevice, stream));
    ITERGP_CUDA_TRY(cudaMemcpyAsync(tabs.as<char>(b_items + b_beg), &pr, sizeof(TcProb), cudaMemcpyHostToDevice, stream));
    tab.items = tabs.as<WorkItem>();
    tab.item_begin = reinterpret_cast<const int32_t*>(tabs.as<char>(b_items));
    tab.probs = reinterpret_cast<const TcProb*>(tabs.as<char>(b_items + b_beg));
    tab.G = G;
    tab.n_items = static_cast<int>(ord.size());
  }
  cudaEvent_t e0, e1;
  ITERGP_CUDA_TRY(cudaEventCreate(&e0));
  ITERGP_CUDA_TRY(cudaEventCreate(&e1));
  int n = 0, rc = ITERGP_OK;
  *best = -1;
  // forms: 0 one CTA, streamed ring; 1 one CTA, resident A; 2 CTA pairs (single schedule);
  // 3 CTA pairs with wide chunks (P <= 80)
  for (int form : {0, 1, 2, 3}) for (int epi : {4, 8}) {
    const int ares = form == 1 ? 1 : 0;
    const bool pair = form >= 2;
    const int cw = form == 3 ? kWideCW : BN;
    if (ares && (X.d_pad != BK || nt1 == 2)) continue;
    if (pair && (items || X.rows < 2 * BM)) continue;
    if (form == 3 && p16 > 80) continue;
    // the P tile the launchers use with this variant: the widest that fits its ring
    int p_tile = p16;
    const int min_ns = ares ? 3 : 2;
    while (p_tile > 16 && stages_that_fit(ctx, nt1, nt2, p_tile, epi, 0, ares != 0, pair, cw) < min_ns) p_tile -= 16;
    for (int ns : {2, 3, 4, 5}) {
      if (n >= cap) break;
      if (stages_that_fit(ctx, nt1, nt2, p_tile, epi, ns, ares != 0, pair, cw) != ns) continue;
      if (pair && pair_clusters(kp.kind, prec, ns, epi,
                                tc_smem_bytes(nt1, nt2, p_tile, epi, ns, false,
                                              weight_slots(ctx, nt1, nt2, p_tile, epi, ns, true, cw), true, cw),
                                cw) < 1)
        continue;
      const TcVariant v{epi, ns, ares, form == 3 ? 2 : pair ? 1 : 0};
      t_forced = &v;
      auto run = [&] {
        return items ? kmv_tc_items(ctx, kp.kind, X, X, tab, s_hi, s_lo, p16, 0, p16, stream)
                     : kmv_tc(ctx, kp, X, X, S, p, p, Y, p, stream, nullptr);
      };
      rc = run();   // warm-up
      int reps = 0;
      float ms = 0.f;
      if (rc == ITERGP_OK && cudaEventRecord(e0, stream) == cudaSuccess) {
        for (reps = 0; reps < 5 && rc == ITERGP_OK; ++reps) rc = run();
        if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          rc = ITERGP_ECUDA;
      }
      t_forced = nullptr;
      if (rc != ITERGP_OK) break;
      epi_out[n] = epi;
      ns_out[n] = ares ? -ns : ns;   // negative: resident-A ring
      pair_out[n] = form == 3 ? 2 : pair ? 1 : 0;
      ms_out[n] = ms / reps;
      if (*best < 0 || ms_out[n] < ms_out[*best]) *best = n;
      ++n;
    }
    if (rc != ITERGP_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *count = n;
  if (rc != ITERGP_OK) return rc;
  if (*best >= 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int bns = ns_out[*best];
    g_tune[std::make_tuple(prec, kp.kind, X.d_pad, p16, items ? 1 : 0)] =
        TcVariant{epi_out[*best], bns < 0 ? -bns : bns, bns < 0 ? 1 : 0, pair_out[*best]};
  }
  return ITERGP_OK;
}

}  // namespace itergp

extern "C" int itergp_tune_save(const char* path) {
  if (!path) return ITERGP_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (!f) return ITERGP_EINVAL;
  std::lock_guard<std::mutex> lk(itergp::g_tune_mu);
  std::fprintf(f, "# precision kind d_pad p_tile items epilogue_warps stages resident_a cta_pair\n");
  for (const auto& kv : itergp::g_tune)
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second.epi,
                 kv.second.nstage, kv.second.ares, kv.second.pair);
  std::fclose(f);
  return ITERGP_OK;
}

extern "C" int itergp_tune_load(const char* path) {
  if (!path) return ITERGP_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return ITERGP_EINVAL;
  char line[256];
  int rc = ITERGP_OK;
  std::lock_guard<std::mutex> lk(itergp::g_tune_mu);
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int a[9];
    a[7] = -1;   // resident A and the pair form: automatic when the column is absent
    a[8] = -1;
    const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4],
                                &a[5], &a[6], &a[7], &a[8]);
    if (got < 7 || (a[5] != 4 && a[5] != 8) || a[6] < 0 || a[6] > 5 || a[7] < -1 || a[7] > 1 || a[8] < -1 ||
        a[8] > 2) {
      rc = ITERGP_EINVAL;
      continue;
    }
    itergp::g_tune[std::make_tuple(a[0], a[1], a[2], a[3], a[4])] = itergp::TcVariant{a[5], a[6], a[7], a[8]};
  }
  std::fclose(f);
  return rc;
}

extern "C" int itergp_tune_clear(void) {
  std::lock_guard<std::mutex> lk(itergp::g_tune_mu);
  itergp::g_tune.clear();
  return ITERGP_OK;
}

// ---------------------------------------------------------------- wait self-test
namespace itergp {
namespace {

// One thread waits, with the product kernel's bounded wait, on an mbarrier that nothing
// ever arrives on (phase 0 of a fresh barrier never completes); when the limit runs out
// the kernel records ITERGP_ETIMEOUT and returns, leaving the context usable.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_s;
  if (threadIdx.x == 0) {
    abort_s = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* ab = &abort_s;
    if (!mbar_wait(&bar, 0u, ab, limit_ns)) atomicExch(status, ITERGP_ETIMEOUT);
  }
  __syncthreads();
}

}  // namespace

int wait_selftest_launch(DeviceContext* ctx, uint64_t limit_ns, cudaStream_t stream) {
  wait_selftest_kernel<<<1, 32, 0, stream>>>(limit_ns, ctx->status), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  return ITERGP_OK;
}

}  // namespace itergp

