// Shared device code of the tensor-core kernel product Y = k(A, B) S (sm_103a): the
// constants, the work partition, the issue helpers and the kernel template, in two forms:
//   one CTA per tile (PAIR = false): 128 rows of A per CTA, MMAs of M = 128;
//   CTA pairs (PAIR = true): clusters of two CTAs on two SMs share one 256-row tile; the
//     even CTA issues cta_group::2 MMAs of M = 256 for both, each CTA stages its own 128
//     rows of A and half of each B chunk and of each weight tile, and the accumulators of
//     each CTA's rows stay in its own TMEM.  Half the MMA instructions per unit of work
//     and three quarters of the shared-memory bytes per chunk.
// kmv_tc.cu instantiates the one-CTA form and kmv_tc2.cu the pair form (separate
// translation units compile in parallel).
#pragma once
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace itergp {
namespace tcimpl {

constexpr int BM = 128;   // rows of A per CTA (MMA M of the one-CTA form; half the pair's M = 256)
constexpr int BN = 128;   // rows of B per chunk (MMA N of the distance GEMM, K of the product)
constexpr int BK = 64;    // D slice per stage (one 128-byte swizzle row of BF16)
// The wide pair form takes chunks of 192 rows of B (MMA N = 192): each SM's share of the
// MMA then reads 10 KB of shared memory per 1.5 128 x 128 x 16 blocks instead of 8 KB per
// block, and its ring refills 56 KB per 18 blocks instead of 48 KB per 12, which lets the
// tensor pipe run at its issue rate while TMA refills the ring (at N = 128 the shared-memory
// traffic of the operands and the refills holds it near three quarters of it).
constexpr int kWideCW = 192;
// Rows of A per tile and rows of each B chunk staged per CTA, in either form.
__host__ __device__ constexpr int tile_rows(bool pair) { return pair ? 2 * BM : BM; }
__host__ __device__ constexpr int b_rows_cta(bool pair, int cw = BN) { return pair ? cw / 2 : cw; }
// Row operand forms (NT1): 1 BF16 rows, 3 split BF16 rows (hi, lo), 2 TF32 rows (FP32
// storage, 32 values per 128-byte swizzle row, kind::tf32 MMAs of K = 8).  A stage holds
// one 128-byte row per tile row in every form, so the ring layout is the same.
__host__ __device__ constexpr int slice_elems(int nt1) { return nt1 == 2 ? BK / 2 : BK; }
// Threads: warps 0-3 (TMA loads of A and B, MMA issue, TMEM owner, TMA loads of the
// weights) plus EPI epilogue warps (4 or 8; with 8, two warps share each TMEM lane
// quadrant and split the columns).
__host__ __device__ constexpr int tc_threads(int epi) { return (4 + epi) * 32; }
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kOCol = 256;
constexpr uint32_t kO2Col = 384;   // FP32 running sum of flushed O (IEEE round-to-nearest adds)
// G buffers (and weight-tile slots): 3 for P tiles <= 48, else 2.  With three, GEMM2 of a
// chunk is issued two chunks behind its GEMM1, so the epilogue of chunk t overlaps GEMM1
// of t + 1 and t + 2 (at small D the epilogue is longer than one GEMM1).  TMEM then holds
// G 3 x 128 columns, O at 384 and O2 at 384 + P (384 + 2P when GEMM2 runs packed, see
// issue_gemm2).
__host__ __device__ constexpr int g_bufs(int p_pad) { return p_pad <= 48 ? 3 : 2; }
constexpr int kFlushChunks = 4;    // O is flushed into O2 at least every 4 chunks (512 rows)
// Chunks per flush group for a chunk width: 4 x 128 or 3 x 192 rows of B.
__host__ __device__ constexpr int flush_chunks(int cw) { return cw == BN ? kFlushChunks : 3; }
// Waits for work of the kernel's own roles are bounded by TcArgs::wait_ns; the drains after
// an abort (copies and MMAs already in flight) by a fixed 4 s.
constexpr uint64_t kDrainLimitNs = 4000000000ull;

struct TcArgs {
  const float* na;        // [A.rows_pad] row norms of A
  const float* nb;        // [B.rows_pad] row norms of B
  const float* ua;        // split rows: tile scales of A [A.rows_pad / 128] (else unused)
  const float* ub;        // split rows: tile scales of B [B.rows_pad / 128] (else unused)
  int64_t m;              // valid rows of A
  int64_t b_rows_pad;     // rows of B's norms and tile scales (a wide chunk may pass the end)
  int64_t a_rows_pad;     // rows of A's prepared planes and norms (rows beyond read as zero)
  int64_t row_tiles;      // R (tiles of tile_rows(pair) rows)
  int chunks;             // J
  int nk;                 // D slices (d_pad / 64)
  int klast;              // MMA K steps of the last slice that hold data (1 .. 4; the rest of
                          // the padded slice is zeros, whose products are skipped)
  int p_pad;              // MMA N of the product (multiple of 16, <= 128)
  int p_valid;            // valid output columns of this P tile
  int s_row0;             // first row of this P tile in the transposed S
  int p_col0;             // item mode: first output column of this P tile
  float* Y;               // output, already offset to the tile's first column
  int64_t ldY;
  float* partial;         // [2 G][tile_rows][p_pad] (G: CTAs, or pairs in the pair form)
  int w_slots;            // weight-tile slots of the shared-memory layout (1 .. 3)
  int diag;               // A and B are the same rows: k(x_i, x_i) = s is set exactly
  const float* wscale;    // split weights: per transposed-S row (output column) 2^-e of its
                          // FP16 scaling (single-problem mode; item mode: TcProb::wscale)
  uint64_t wait_ns;       // bound of each wait for another role's work (ns)
  KParams kp;
  int* status;
  const int* active;
  // item mode (batched problems): per-CTA lists of whole row tiles
  const WorkItem* items;            // nullptr: single-problem schedule
  const int32_t* item_begin;        // [G + 1]
  const TcProb* probs;
};

__host__ __device__ constexpr uint32_t stage_bytes(int nt1, bool pair = false, int cw = BN) {
  return (nt1 == 3 ? 2u : 1u) * (BM * BK * 2u) + (nt1 == 3 ? 2u : 1u) * (b_rows_cta(pair, cw) * BK * 2u);
}
// One 64-row-wide box of the chunk's transposed weights: P rows (the pair form stages
// P / 2 of them per CTA, its half of the product's N) x 128 bytes.
__host__ __device__ constexpr uint32_t s_box_bytes(int p_pad, bool pair = false) {
  return static_cast<uint32_t>(pair ? p_pad / 2 : p_pad) * 128u;
}
// A weight tile: the chunk's cw / 64 boxes per plane.
__host__ __device__ constexpr uint32_t s_buf_bytes(int nt2, int p_pad, bool pair = false, int cw = BN) {
  return static_cast<uint32_t>(cw / 64) * s_box_bytes(p_pad, pair) * (nt2 == 3 ? 2u : 1u);
}
// alignment slack + per-epilogue-warp staging of one chunk's column norms
__host__ __device__ constexpr uint32_t smem_extra(int epi, int cw = BN) {
  return 1024u + static_cast<uint32_t>(epi) * static_cast<uint32_t>(cw) * 4u;
}

// Per-CTA sequence of (row tile, chunk) steps of the partition described above.
struct Schedule {
  int64_t G, g, J, fw, rt0, ut, tb, T;
  __host__ __device__ void init(int64_t R, int64_t J_, int64_t G_, int64_t g_) {
    G = G_;
    g = g_;
    J = J_;
    fw = R / G;                      // whole-row waves
    rt0 = fw * G;                    // first tail row tile
    ut = (R - rt0) * J;              // tail units
    tb = part_start(g, ut, G);
    const int64_t te = part_start(g + 1, ut, G);
    T = fw * J + (te - tb);
  }
  __host__ __device__ int64_t row(int64_t t) const {
    return t < fw * J ? (t / J) * G + g : rt0 + (tb + (t - fw * J)) / J;
  }
  __host__ __device__ int col(int64_t t) const {
    return static_cast<int>(t < fw * J ? t % J : (tb + (t - fw * J)) % J);
  }
  __host__ __device__ bool first(int64_t t) const { return t == 0 || row(t - 1) != row(t); }
  __host__ __device__ bool last(int64_t t) const { return t == T - 1 || row(t + 1) != row(t); }
};

struct StepInfo {
  int32_t a_row;   // A-arena row of this CTA's first row of the current tile
  int32_t b_row;   // B-arena row (transposed-S column) of the current chunk
  int32_t c;       // chunk index within the row tile (flush boundaries)
  int32_t item;    // item index (item mode) or -1
  bool first, last;// first / last chunk of the CTA's run on this row tile
};

// Walks a CTA's steps in order; every role owns one and advances it in lockstep with the
// step counter t.  Single mode follows Schedule; item mode walks the CTA's items, skipping
// problems whose solver has stopped.
struct Walker {
  Schedule sch;
  int64_t t = 0;
  const WorkItem* items = nullptr;
  const TcProb* probs = nullptr;
  int32_t k = 0, k_end = 0, c = 0;
  // The position advances with compares and adds only (every role steps it once per
  // chunk; divisions there cost the single issuing threads about a thousand cycles).
  int64_t row = 0, lock = 0;                      // single problem: row tile, fw * J
  int32_t it_a_row = 0, it_b_row0 = 0, it_chunks = 0;   // item mode: the current item
  int32_t rows_per_tile = BM, row_off = 0;        // single problem: tile height, this CTA's rows in it
  int32_t cw = BN;                                // rows of B per chunk

  __device__ bool item_active(int32_t kk) const {
    const int* a = probs[items[kk].prob].active;
    return a == nullptr || *a != 0;
  }
  __device__ void load_item() {   // skip stopped problems, cache the item's fields
    while (k < k_end && !item_active(k)) ++k;
    c = 0;
    if (k < k_end) {
      const WorkItem it = items[k];
      it_a_row = it.a_row;
      it_b_row0 = it.b_row0;
      it_chunks = it.chunks;
    }
  }
  __device__ void seek() {        // single problem: position of step t (with divisions)
    row = sch.row(t);
    c = sch.col(t);
  }
  // G CTAs (or pairs) and this one's index g; pair form: tiles of 256 rows, of which the
  // CTA of rank h owns rows [128 h, 128 h + 128)
  __device__ void init(const TcArgs& a, int64_t G, int64_t g, int32_t tile_h = BM, int32_t off = 0,
                       int32_t chunk_w = BN) {
    items = a.items;
    probs = a.probs;
    rows_per_tile = tile_h;
    row_off = off;
    cw = chunk_w;
    t = 0;
    if (items == nullptr) {
      sch.init(a.row_tiles, a.chunks, G, g);
      lock = sch.fw * sch.J;
      seek();
    } else {
      k = a.item_begin[g];
      k_end = a.item_begin[g + 1];
      load_item();
    }
  }
  __device__ int64_t total() const {   // number of steps
    if (items == nullptr) return sch.T;
    int64_t n = 0;
    for (int32_t kk = k; kk < k_end; ++kk)
      if (item_active(kk)) n += items[kk].chunks;
    return n;
  }
  __device__ StepInfo cur() const {
    StepInfo s;
    if (items == nullptr) {
      s.a_row = static_cast<int32_t>(row * rows_per_tile) + row_off;
      s.b_row = c * cw;
      s.c = c;
      // a row run starts at chunk 0, at step 0 and where the tail begins; it ends at the
      // row's last chunk and at the CTA's last step
      s.first = t == 0 || c == 0 || t == lock;
      s.last = t == sch.T - 1 || c == sch.J - 1;
      s.item = -1;
    } else {
      s.a_row = it_a_row;
      s.b_row = it_b_row0 + c * cw;
      s.c = c;
      s.first = (c == 0);
      s.last = (c == it_chunks - 1);
      s.item = k;
    }
    return s;
  }
  __device__ void next() {
    ++t;
    if (items == nullptr) {
      if (t == lock) {
        seek();                       // first tail step
      } else if (++c == sch.J) {
        c = 0;
        row += t < lock ? sch.G : 1;  // next wave's row tile, or the next tail row
      }
    } else if (++c >= it_chunks) {
      ++k;
      load_item();
    }
  }
};

// The pair form's launcher (kmv_tc2.cu): grid_pairs clusters of two CTAs; chunks of cw
// (128, or kWideCW) rows of B.
cudaError_t launch_pair_form(int kind, int prec, int nstage, int epi, int grid_pairs, size_t smem, cudaStream_t st,
                             const CUtensorMap* maps, const TcArgs& a, int cw = BN);
// Clusters of two CTAs of the pair form with this configuration that can be resident at
// once (the SM pairs available within the GPCs); 0 if it cannot launch.
int pair_max_clusters(int kind, int prec, int nstage, int epi, size_t smem, int cw = BN);

namespace {

// Out-of-line slow path of a bounded mbarrier wait (the fast path is one try_wait).
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                            uint64_t limit_ns) {
  return mbar_wait(bar, parity, abort_flag, limit_ns);
}
// The same for barriers the other CTA of a pair arrives on (acquire at cluster scope).
__device__ __noinline__ bool mbar_wait_cluster_slow(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                    uint64_t limit_ns) {
  return mbar_wait_cluster(bar, parity, abort_flag, limit_ns);
}

// The MMA and commit instructions of either form: cta_group::1 on this CTA's tile, or
// cta_group::2 on the pair's (issued by the even CTA; commits arrive on the barrier at the
// same offset in both CTAs).
template <bool PAIR>
__device__ __forceinline__ void mma_ss_x(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (PAIR) mma_ss_pair(d, a, b, id, acc); else mma_ss(d, a, b, id, acc);
}
template <bool PAIR>
__device__ __forceinline__ void mma_ss_tf32_x(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (PAIR) mma_ss_tf32_pair(d, a, b, id, acc); else mma_ss_tf32(d, a, b, id, acc);
}
template <bool PAIR>
__device__ __forceinline__ void mma_ts_x(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (PAIR) mma_ts_pair(d, a, b, id, acc); else mma_ts(d, a, b, id, acc);
}
template <bool PAIR>
__device__ __forceinline__ void commit_x(uint64_t* bar) {
  if constexpr (PAIR) mma_commit_pair_both(bar); else mma_commit(bar);
}

// GEMM1 of one chunk: G = A . B^T over the nk D slices of the stage ring (12 MMAs per
// slice for split rows: the correction terms hi.lo and lo.hi, then hi.hi, K = 16 each),
// releasing each stage to the producer with a commit.  The tensor core adds each MMA into
// the FP32 accumulator with truncation, an error relative to the accumulator's value: the
// small correction terms go first, so that in a one-slice product (D <= 64) only the four
// hi.hi steps add at the full magnitude of G.  `pos` packs the ring position
// (stage | phase << 8); returns the position after the chunk, or -1 if a wait gave up.  A
// small out-of-line function: the issuing thread must keep up with one MMA every few
// dozen cycles.
// In the pair form a stage holds this CTA's 128 rows of A and 64 rows of B; the same
// descriptors address the other CTA's stage, and the MMA's M = 256.
template <int NT1, int NSTAGE, bool ARES, bool PAIR, int CW>
__device__ __noinline__ int issue_gemm1(uint32_t gt, int nk, int klast, uint64_t dStage0, uint64_t dAres,
                                        uint64_t* full_bar, uint64_t* empty_bar, volatile int* ab, uint32_t idesc1,
                                        int pos, uint64_t lim) {
  constexpr uint32_t A_PART = BM * BK * 2, B_PART = b_rows_cta(PAIR, CW) * BK * 2;
  constexpr uint32_t SB = ARES ? (NT1 == 3 ? 2u : 1u) * B_PART : stage_bytes(NT1, PAIR, CW);
  int stage = pos & 0xFF;
  uint32_t phase = static_cast<uint32_t>(pos >> 8);
  for (int ks = 0; ks < nk; ++ks) {
    // operands arrive by TMA with completion on the mbarrier (async proxy on both sides):
    // no tcgen05 fence is needed here
    if (!mbar_try_wait(&full_bar[stage], phase) && !mbar_wait_slow(&full_bar[stage], phase, ab, lim)) return -1;
    const uint64_t dSt = dStage0 + static_cast<uint64_t>(stage) * (SB >> 4);
    const uint64_t dAh = ARES ? dAres : dSt;
    const uint64_t dBh = ARES ? dSt : dSt + ((NT1 == 3 ? 2 : 1) * A_PART >> 4);
    const uint64_t dAl = dAh + (A_PART >> 4);
    const uint64_t dBl = dBh + (B_PART >> 4);
    // one MMA order for every ring and form, so that launch variants agree
    if (ks + 1 == nk && klast < BK / 16) {
      // the last slice with zero padding: its K steps past the data are skipped (adding
      // zero products leaves the FP32 sums as they are)
      for (int kk = 0; kk < klast; ++kk) {
        if constexpr (NT1 == 3) {
          mma_ss_x<PAIR>(gt, dAh + 2 * kk, dBl + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
          mma_ss_x<PAIR>(gt, dAl + 2 * kk, dBh + 2 * kk, idesc1, 1u);
        } else if constexpr (NT1 == 2) {
          mma_ss_tf32_x<PAIR>(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
        } else {
          mma_ss_x<PAIR>(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
        }
      }
      if constexpr (NT1 == 3)
        for (int kk = 0; kk < klast; ++kk) mma_ss_x<PAIR>(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, 1u);
    } else if constexpr (NT1 == 3) {
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        mma_ss_x<PAIR>(gt, dAh + 2 * kk, dBl + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
        mma_ss_x<PAIR>(gt, dAl + 2 * kk, dBh + 2 * kk, idesc1, 1u);
      }
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) mma_ss_x<PAIR>(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, 1u);
    } else {
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {   // K steps of 32 bytes: 16 16-bit or 8 TF32 values
        if constexpr (NT1 == 2)
          mma_ss_tf32_x<PAIR>(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
        else
          mma_ss_x<PAIR>(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
      }
    }
    commit_x<PAIR>(&empty_bar[stage]);
    if (++stage == NSTAGE) {
      stage = 0;
      phase ^= 1u;
    }
  }
  return stage | static_cast<int>(phase << 8);
}

// GEMM2 of one chunk: O (+)= P . S with P (the chunk's kernel values, 16-bit hi/lo pairs
// packed in the G buffer's TMEM columns) as the A operand and the chunk's transposed
// weights from shared memory as B; CW / 16 K steps of 16 rows, 3 MMAs each for split
// weights (hi.hi, hi.lo, lo.hi).  Packed (pk2: one CTA, split weights, P tiles <= 32): the weight tile holds each
// 64-row box's hi and lo planes back to back, so one MMA of N = 2P multiplies P's hi plane
// by both (O columns [0, P) take hi.hi, [P, 2P) hi.lo) and a second of N = P adds lo.hi
// into [P, 2P): 2 MMAs per K step instead of 3.  The hi.hi sum then takes one accumulation
// per K step (not three) and the correction terms are summed apart at their own magnitude;
// the flush adds the two column halves.
// Waits for the epilogue's P (pfull, parity par of its G buffer) and the weight tile (sfull,
// parity spar of its slot); releases the weight tile (sempty) and, at the end of a flush
// group, hands O to the epilogue (ofull).
// In the pair form P comes from both CTAs' TMEM and each CTA holds half of the weight
// tile's P columns (the MMA's N).
template <int NT2, bool PAIR, int CW>
__device__ __noinline__ bool issue_gemm2(uint32_t tb, uint32_t a_col0, uint32_t o_col, uint32_t par, uint32_t spar,
                                         bool first, bool last, uint64_t* pfull_b, uint64_t* sfull_b, uint64_t* sempty_b,
                                         uint64_t* ofull_b, volatile int* ab, uint64_t dS0, uint64_t sbox16,
                                         uint32_t idesc2, uint32_t idesc2w, bool pk2, uint32_t p_pad, uint64_t lim) {
  if constexpr (PAIR) {   // both CTAs' epilogue warps arrive on pfull
    if (!mbar_try_wait_cluster(pfull_b, par) && !mbar_wait_cluster_slow(pfull_b, par, ab, lim)) return false;
  } else {
    if (!mbar_try_wait(pfull_b, par) && !mbar_wait_slow(pfull_b, par, ab, lim)) return false;
  }
  if (!mbar_try_wait(sfull_b, spar) && !mbar_wait_slow(sfull_b, spar, ab, lim)) return false;
  tc_fence_after();   // P was written by the epilogue's tcgen05.st
  if (NT2 == 3 && !PAIR && pk2) {
#pragma unroll
    for (int ks2 = 0; ks2 < CW / 16; ++ks2) {
      const int grp = ks2 >> 1, h = ks2 & 1;
      const uint32_t a_hi = tb + a_col0 + static_cast<uint32_t>(32 * grp + 8 * h);
      const uint64_t dSh = dS0 + static_cast<uint64_t>(ks2 >> 2) * 2 * sbox16 + static_cast<uint64_t>((ks2 & 3) * 2);
      mma_ts_x<PAIR>(tb + o_col, a_hi, dSh, idesc2w, (first && ks2 == 0) ? 0u : 1u);
      mma_ts_x<PAIR>(tb + o_col + p_pad, a_hi + 16, dSh, idesc2, 1u);
    }
    commit_x<PAIR>(sempty_b);
    if (last) commit_x<PAIR>(ofull_b);
    return true;
  }
#pragma unroll
  for (int ks2 = 0; ks2 < CW / 16; ++ks2) {
    const int grp = ks2 >> 1, h = ks2 & 1;
    const uint32_t a_hi = tb + a_col0 + static_cast<uint32_t>(32 * grp + 8 * h);
    const uint64_t dSh = dS0 + static_cast<uint64_t>(ks2 >> 2) * sbox16 + static_cast<uint64_t>((ks2 & 3) * 2);
    mma_ts_x<PAIR>(tb + o_col, a_hi, dSh, idesc2, (first && ks2 == 0) ? 0u : 1u);
    if (NT2 == 3) {   // the lo plane's boxes follow the hi plane's CW / 64
      mma_ts_x<PAIR>(tb + o_col, a_hi, dSh + (CW / 64) * sbox16, idesc2, 1u);
      mma_ts_x<PAIR>(tb + o_col, a_hi + 16, dSh, idesc2, 1u);
    }
  }
  commit_x<PAIR>(sempty_b);
  if (last) commit_x<PAIR>(ofull_b);
  return true;
}

// ARES (D <= 64, one K slice): the A tile of a row segment stays resident in shared
// memory for all of its chunks and only B streams through the ring.
// PAIR: launched as clusters of two CTAs (single-problem schedule, streamed ring only);
// G below counts pairs, g is the pair and h the CTA's rank in it.  Every early return is
// taken by both CTAs of a pair (the conditions read the same values), so both always
// meet at the cluster barriers.
template <int KIND, int NT1, int NT2, int NSTAGE, int EPI, bool ARES, bool PAIR, int CW = BN>
__global__ void __launch_bounds__(tc_threads(EPI), 1)
kmv_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
              const __grid_constant__ CUtensorMap mSh, const __grid_constant__ CUtensorMap mSl,
              const TcArgs args) {
  static_assert(!(PAIR && ARES), "the pair form streams A");
  static_assert(CW == BN || (CW == kWideCW && PAIR), "wide chunks are a pair-form layout");
  // Wide chunks: two G buffers of 192 columns and O at 384 (P tiles <= 80); O2, the flushed
  // running sum, lives in the epilogue threads' registers instead of TMEM.
  constexpr bool O2REG = CW != BN;
  constexpr int FC = flush_chunks(CW);
  if (args.active != nullptr && *args.active == 0) return;
  if (PAIR && args.items != nullptr) return;   // the pair form has no item mode
  const uint32_t h = PAIR ? cluster_rank() : 0u;
  const bool leader = h == 0;   // the pair's MMA issuer and owner of its shared barriers
  const int64_t G = PAIR ? gridDim.x / 2 : gridDim.x, g = PAIR ? blockIdx.x / 2 : blockIdx.x;
  Walker walk0;
  walk0.init(args, G, g, tile_rows(PAIR), static_cast<int32_t>(BM * h), CW);
  const int64_t T = walk0.total();
  if (T <= 0) return;
  const Schedule& sch = walk0.sch;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  constexpr uint32_t A_PART = BM * BK * 2, B_PART = b_rows_cta(PAIR, CW) * BK * 2;
  constexpr uint32_t A_BYTES = (NT1 == 3 ? 2u : 1u) * A_PART;   // resident A (ARES)
  constexpr uint32_t SB = ARES ? (NT1 == 3 ? 2u : 1u) * B_PART : stage_bytes(NT1, PAIR, CW);
  const int ng = O2REG ? 2 : g_bufs(args.p_pad);         // G buffers
  const int nsl = args.w_slots;                          // weight-tile slots (1 .. 3)
  // packed GEMM2 (see issue_gemm2): O takes 2P columns, so O2 moves to 384 + 2P (<= 448)
  const bool pk2 = NT2 == 3 && !PAIR && CW == BN && args.p_pad <= 32;
  const uint32_t ocol = O2REG ? 2u * CW : ng == 3 ? 384u : kOCol;
  const uint32_t o2col = ng == 3 ? 384u + static_cast<uint32_t>((pk2 ? 2 : 1) * args.p_pad) : kO2Col;   // TMEM O2 forms
  const uint32_t SBOX = s_box_bytes(args.p_pad, PAIR);
  const uint32_t SBUF = s_buf_bytes(NT2, args.p_pad, PAIR, CW);
  uint8_t* a_region = smem + NSTAGE * SB;                        // ARES only
  uint8_t* s_region = a_region + (ARES ? A_BYTES : 0u);
  float* nb_all = reinterpret_cast<float*>(s_region + nsl * SBUF);   // [EPI warps][CW]

  __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE];
  __shared__ __align__(8) uint64_t gfull[3], pfull[3], sfull[3], sempty[3], ofull, oempty, drain;
  __shared__ __align__(8) uint64_t afull, aempty;               // resident A (ARES)
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    // pfull and oempty count one arrival per epilogue warp (after the warp's lanes meet), of
    // each CTA in the pair form (on the even CTA's barriers)
    for (int i = 0; i < 3; ++i) {
      mbar_init(&gfull[i], 1);
      mbar_init(&pfull[i], PAIR ? 2 * EPI : EPI);
      mbar_init(&sfull[i], 1);
      mbar_init(&sempty[i], 1);
    }
    mbar_init(&ofull, 1);
    mbar_init(&oempty, PAIR ? 2 * EPI : EPI);
    mbar_init(&drain, 1);
    mbar_init(&afull, 1);
    mbar_init(&aempty, 1);
    fence_mbar_init();
  }
  if (warp == 2) {   // pair form: one warp of each CTA allocates the same columns in both
    if constexpr (PAIR) {
      tmem_alloc_pair(&tmem_base_s, kTmemCols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(&tmem_base_s, kTmemCols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync_all();   // both CTAs' barriers are initialised before any remote use
  tc_fence_after();
  const uint32_t tb = tmem_base_s;
  volatile int* ab = &abort_s;
  // shared::cluster address of a barrier of the even CTA (pair form), where both CTAs'
  // loads, and both CTAs' epilogue hand-offs, are counted
  auto lead = [](uint64_t* bar) -> uint32_t { return cluster_addr(smem_u32(bar), 0u); };

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&mAh);
      tma_prefetch_desc(&mBh);
      tma_prefetch_desc(&mSh);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t armed = 0, armed_par = 0;      // bit i: stage i armed / parity of last arm
      bool a_armed = false;
      uint32_t a_par = 0;
      int64_t seg = -1;
      Walker wk = walk0;
      for (int64_t t = 0; t < T && !*ab; ++t, wk.next()) {
        const StepInfo st = wk.cur();
        const int32_t a_y = st.a_row;
        // this CTA's rows of the B chunk (the pair form stages half of them per CTA)
        const int32_t b_y = st.b_row + (PAIR ? b_rows_cta(true, CW) * static_cast<int32_t>(h) : 0);
        if (ARES) {
          if (st.first) {
            // a new row segment: reload A once the previous segment's MMAs are done with it
            ++seg;
            if (seg >= 1 && !mbar_wait(&aempty, static_cast<uint32_t>((seg - 1) & 1), ab, args.wait_ns)) break;
            mbar_arrive_expect_tx(&afull, A_BYTES);
            a_armed = true;
            a_par = static_cast<uint32_t>(seg & 1);
            tma_load_2d(a_region, &mAh, &afull, 0, a_y);
            if (NT1 == 3) tma_load_2d(a_region + A_PART, &mAl, &afull, 0, a_y);
          }
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, ab, args.wait_ns)) break;
          mbar_arrive_expect_tx(&full_bar[stage], SB);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          uint8_t* bbase = smem + stage * SB;
          tma_load_2d(bbase, &mBh, &full_bar[stage], 0, b_y);
          if (NT1 == 3) tma_load_2d(bbase + B_PART, &mBl, &full_bar[stage], 0, b_y);
          if (++stage == NSTAGE) {
            stage = 0;
            phase ^= 1u;
          }
        }
        for (int ks = 0; !ARES && ks < args.nk; ++ks) {
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, ab, args.wait_ns)) break;
          uint8_t* base = smem + stage * SB;
          uint8_t* bbase = base + (NT1 == 3 ? 2 : 1) * A_PART;
          if constexpr (PAIR) {
            // both CTAs' loads complete on the even CTA's barrier, which expects them all
            if (leader) {
              mbar_arrive_expect_tx(&full_bar[stage], 2 * SB);
              armed |= 1u << stage;
              armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            }
            const uint32_t fb = lead(&full_bar[stage]);
            tma_load_2d_pair(base, &mAh, fb, ks * slice_elems(NT1), a_y);
            tma_load_2d_pair(bbase, &mBh, fb, ks * slice_elems(NT1), b_y);
            if (NT1 == 3) {
              tma_load_2d_pair(base + A_PART, &mAl, fb, ks * BK, a_y);
              tma_load_2d_pair(bbase + B_PART, &mBl, fb, ks * BK, b_y);
            }
          } else {
            mbar_arrive_expect_tx(&full_bar[stage], SB);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            tma_load_2d(base, &mAh, &full_bar[stage], ks * slice_elems(NT1), a_y);
            tma_load_2d(bbase, &mBh, &full_bar[stage], ks * slice_elems(NT1), b_y);
            if (NT1 == 3) {
              tma_load_2d(base + A_PART, &mAl, &full_bar[stage], ks * BK, a_y);
              tma_load_2d(bbase + B_PART, &mBl, &full_bar[stage], ks * BK, b_y);
            }
          }
          if (++stage == NSTAGE) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (*ab) {
        // let every load this thread issued land before the CTA can exit (pair form: the
        // even CTA's barriers count both CTAs' loads; the odd CTA waits at the end)
        for (int i = 0; i < NSTAGE; ++i)
          if (armed & (1u << i)) mbar_wait_drain(&full_bar[i], (armed_par >> i) & 1u, kDrainLimitNs);
        if (a_armed) mbar_wait_drain(&afull, a_par, kDrainLimitNs);
      }
    }
  } else if (warp == 3) {
    // ------------------------------------------------------------------ weight-tile producer
    // The chunk's transposed weights go through their own ring of nsl slots (slot t % nsl,
    // parity (t / nsl) & 1), loaded by this warp so that the A/B ring never waits for a
    // slot: a weight tile is read only by GEMM2, a chunk after its GEMM1, so even one
    // slot has a whole GEMM1 to refill.
    if (lane == 0) {
      uint32_t s_armed = 0, s_par = 0;
      int s_slot = 0;
      uint32_t s_phase = 0;
      Walker wk = walk0;
      for (int64_t t = 0; t < T && !*ab; ++t, wk.next()) {
        const int32_t j0 = wk.cur().b_row;
        const int sb = s_slot;
        if (!mbar_wait(&sempty[sb], s_phase ^ 1u, ab, args.wait_ns)) break;
        if (!PAIR || leader) {
          mbar_arrive_expect_tx(&sfull[sb], PAIR ? 2 * SBUF : SBUF);
          s_armed |= 1u << sb;
          s_par = (s_par & ~(1u << sb)) | (s_phase << sb);
        }
        if (++s_slot == nsl) {
          s_slot = 0;
          s_phase ^= 1u;
        }
        uint8_t* sbase = s_region + sb * SBUF;
        if constexpr (PAIR) {   // this CTA's half of the tile's P rows (the MMA's N)
          const uint32_t fb = lead(&sfull[sb]);
          const int32_t srow = args.s_row0 + static_cast<int32_t>(h) * (args.p_pad / 2);
#pragma unroll
          for (int bx = 0; bx < CW / 64; ++bx) {
            tma_load_2d_pair(sbase + bx * SBOX, &mSh, fb, j0 + 64 * bx, srow);
            if (NT2 == 3) tma_load_2d_pair(sbase + (CW / 64 + bx) * SBOX, &mSl, fb, j0 + 64 * bx, srow);
          }
        } else {
          // plain order hi0 hi1 lo0 lo1; packed GEMM2 hi0 lo0 hi1 lo1
          const uint32_t hs = pk2 ? 2u : 1u, lo0 = pk2 ? 1u : 2u;
          tma_load_2d(sbase, &mSh, &sfull[sb], j0, args.s_row0);
          tma_load_2d(sbase + hs * SBOX, &mSh, &sfull[sb], j0 + 64, args.s_row0);
          if (NT2 == 3) {
            tma_load_2d(sbase + lo0 * SBOX, &mSl, &sfull[sb], j0, args.s_row0);
            tma_load_2d(sbase + (lo0 + hs) * SBOX, &mSl, &sfull[sb], j0 + 64, args.s_row0);
          }
        }
      }
      if (*ab)   // let every weight load this thread armed land before the CTA can exit
        for (int i = 0; i < 3; ++i)
          if (s_armed & (1u << i)) mbar_wait_drain(&sfull[i], (s_par >> i) & 1u, kDrainLimitNs);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0 && leader) {   // pair form: the even CTA issues for both
      constexpr uint32_t TM = tile_rows(PAIR);
      // split rows are FP16 hi/lo, BF16 rows BF16, TF32 rows TF32
      const uint32_t idesc1 = NT1 == 2 ? idesc_tf32_f32(TM, CW) : NT1 == 3 ? idesc_f16_f32(TM, CW) : idesc_bf16_f32(TM, CW);
      // split weights are FP16 hi/lo (kernel values too), single weights BF16
      const uint32_t idesc2 = NT2 == 3 ? idesc_f16_f32(TM, static_cast<uint32_t>(args.p_pad))
                                       : idesc_bf16_f32(TM, static_cast<uint32_t>(args.p_pad));
      const uint32_t idesc2w = idesc_f16_f32(TM, static_cast<uint32_t>(2 * args.p_pad));   // pk2 only
      // shared-memory descriptors of stage 0, the resident A and the weight buffers; the
      // start-address field (bits 0-13, 16-byte units) takes offsets by plain addition
      // because every operand lies below 256 KB of the shared window
      const uint64_t dStage0 = sdesc_kmajor_sw128(smem_u32(smem));
      const uint64_t dAres = sdesc_kmajor_sw128(smem_u32(a_region));
      const uint64_t dS_base = sdesc_kmajor_sw128(smem_u32(s_region));
      const uint64_t sbox16 = SBOX >> 4;
      int stage = 0;
      uint32_t phase = 0;
      int64_t sub = -1;
      bool ok = true;
      // The issuing thread has to keep up with one MMA every few dozen cycles, so the hot
      // loop holds only the fast path of each wait; slow waits and the weighted-sum GEMM2
      // are out-of-line calls (inlined, they measurably slowed the issue of GEMM1).
      Walker wk2 = walk0;   // lags the GEMM1 loop by ng - 1 steps
      int g2 = 0;           // GEMM2's G buffer (t % ng) and its parity ((t / ng) & 1)
      uint32_t g2par = 0;
      int w2 = 0;           // GEMM2's weight slot (t % nsl) and its parity ((t / nsl) & 1)
      uint32_t w2par = 0;
      auto gemm2 = [&](int64_t t) -> bool {
        const StepInfo st = wk2.cur();
        wk2.next();
        const int c = st.c;
        const bool first = st.first || (c % FC == 0);
        const bool last = st.last || ((c + 1) % FC == 0);
        if (first) {
          ++sub;
          const uint32_t opar = static_cast<uint32_t>((sub - 1) & 1);
          if (sub >= 1 && !(PAIR ? mbar_wait_cluster_slow(&oempty, opar, ab, args.wait_ns)
                                 : mbar_wait_slow(&oempty, opar, ab, args.wait_ns)))
            return false;
        }
        (void)t;
        const int gb = g2, wb = w2;
        const uint32_t par = g2par, wpar = w2par;
        if (++g2 == ng) {
          g2 = 0;
          g2par ^= 1u;
        }
        if (++w2 == nsl) {
          w2 = 0;
          w2par ^= 1u;
        }
        return issue_gemm2<NT2, PAIR, CW>(tb, static_cast<uint32_t>(gb) * CW, ocol, par, wpar, first, last, &pfull[gb],
                                      &sfull[wb], &sempty[wb], &ofull, ab,
                                      dS_base + static_cast<uint64_t>(wb) * (SBUF >> 4), sbox16, idesc2,
                                      idesc2w, pk2, static_cast<uint32_t>(args.p_pad), args.wait_ns);
      };
      Walker wk1 = walk0;    // GEMM1 steps (segment boundaries for the resident A)
      int64_t aseg = -1;
      const int nk = args.nk;
      const int lag = ng - 1;
      int g1 = 0;           // GEMM1's buffer (t % ng)
      for (int64_t t = 0; t < T && ok; ++t, wk1.next()) {
        const int gb = g1;
        if (++g1 == ng) g1 = 0;
        const uint32_t gt = tb + static_cast<uint32_t>(gb) * CW;
        bool seg_last = false;
        if (ARES) {
          const StepInfo st1 = wk1.cur();
          seg_last = st1.last;
          if (st1.first) {
            ++aseg;
            if (!mbar_wait_slow(&afull, static_cast<uint32_t>(aseg & 1), ab, args.wait_ns)) {
              ok = false;
              break;
            }
          }
        }
        const int pos = issue_gemm1<NT1, NSTAGE, ARES, PAIR, CW>(gt, nk, args.klast, dStage0, dAres, full_bar, empty_bar, ab, idesc1,
                                                             stage | static_cast<int>(phase << 8), args.wait_ns);
        if (pos < 0) {
          ok = false;
          break;
        }
        stage = pos & 0xFF;
        phase = static_cast<uint32_t>(pos >> 8);
        if (!ok) break;
        if (ARES && seg_last) mma_commit(&aempty);   // the segment's A is no longer read
        commit_x<PAIR>(&gfull[gb]);
        if (t >= lag && !gemm2(t - lag)) ok = false;
      }
      for (int64_t t = T > lag ? T - lag : 0; ok && t < T; ++t)
        if (!gemm2(t)) ok = false;
      // all issued MMAs must retire before TMEM is released
      if constexpr (PAIR) mma_commit_pair_local(&drain); else mma_commit(&drain);
      mbar_wait_drain(&drain, 0, kDrainLimitNs);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ epilogue
    constexpr int NH = EPI / 4;     // epilogue warps per TMEM lane quadrant
    const int e = warp - 4;
    const int q = e & 3;            // lane quadrant (= warp % 4, the warp's TMEM lanes)
    const int hc = e >> 2;          // this warp's share of the columns
    const int row = 32 * q + lane;
    const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
    int64_t seg = -1, sub = -1;
    int seg_c0 = 0, sub_in_seg = 0;
    float na_r = 0.f;
    int64_t grow = 0;
    KParams kp = args.kp;
    float rowc = 0.f;   // RBF: c_exp |a|^2 + log2 s of this thread's row
    float ua_t = 1.f;   // split rows: scale of this row's tile (G reads 2^(e_I + e_J) a.b)
    float ke = 0.f, kls = kp.log2s, kmul = 1.f;   // split weights: kernel-value scale 2^ke
    const float* item_ws = nullptr;               // item mode: the problem's weight scales
    const int J = args.chunks;
    float* out_row = nullptr;       // item mode: this row's output
    bool out_valid = false;
    int out_lim = 0;
    Walker wk = walk0;
    int gbuf = 0;                   // G buffer of the current chunk (t % ng) and its parity
    uint32_t gpar = 0;
    // column norms of the next step are loaded while the current chunk is processed
    Walker wkn = walk0;
    // (a wide chunk may pass the end of B's rows: norms there read as 0, the weights and
    // rows there are TMA zero fill, so those columns add nothing)
    auto nb_at = [&](int64_t r) -> float { return r < args.b_rows_pad ? args.nb[r] : 0.f; };
    float nb_next[CW / 32];
    {
      const StepInfo s0 = wkn.cur();
#pragma unroll
      for (int k = 0; k < CW / 32; ++k) nb_next[k] = nb_at(static_cast<int64_t>(s0.b_row) + lane + 32 * k);
    }
    constexpr int O2G = O2REG ? (NH == 1 ? 5 : 3) : 1;   // 16-column groups of O per thread (P <= 80)
    // the next 32-column group of G is loaded while the current one is computed, except in
    // the wide form with 8 epilogue warps, whose 168 registers per thread leave no room for
    // the second buffer beside the running sum (two warps per SMSP hide the load instead)
    constexpr bool PREF = !(O2REG && NH == 2);
    float o2r[O2G][16];                                  // wide chunks: O2 of this thread's row
    for (int64_t t = 0; t < T; ++t, wk.next()) {
      const StepInfo st = wk.cur();
      const int c = st.c;
      const bool first = st.first;
      const bool last = st.last;
      const bool sub_last = last || ((c + 1) % FC == 0);
      if (first) {
        ++seg;
        seg_c0 = c;
        sub_in_seg = 0;
        grow = static_cast<int64_t>(st.a_row) + row;
        na_r = grow < args.a_rows_pad ? args.na[grow] : 0.f;   // pair tiles may pass the last row
        if constexpr (NT1 == 3) ua_t = grow < args.a_rows_pad ? args.ua[grow / BM] : 1.f;
        if (st.item >= 0) {
          const WorkItem& it = args.items[st.item];
          const TcProb& pr = args.probs[it.prob];
          kp = pr.kp;
          const int64_t prow = static_cast<int64_t>(it.tile_row) + row;
          out_valid = prow < pr.m;
          out_row = pr.Y + prow * pr.ldY + args.p_col0;
          out_lim = pr.p_valid - args.p_col0;   // <= 0: nothing of this tile to write
          item_ws = pr.wscale;
        }
        // split weights: kernel values are formed as 2^ke k with ke = 14 - floor(log2 s),
        // which puts them in [0, 2^15) for FP16 (an exact power of two, undone at the
        // output).  The headroom keeps the lo half normal down to k = 2^-17 s and the
        // absolute rounding near 2^-39 s, so rows whose kernel values are all small (test
        // points far from the data) keep their relative accuracy.
        if constexpr (NT2 == 3) {
          ke = fminf(fmaxf(14.f - floorf(kp.log2s), -100.f), 100.f);
          kls = kp.log2s + ke;
          kmul = pow2i(static_cast<int>(ke));
        }
        rowc = fmaf(kp.c_exp, na_r, kls);
      }
      float* nb_s = nb_all + e * CW;
      __syncwarp();
      // RBF stages c_exp |b|^2 (the column term of the exponent), Matern |b|^2
#pragma unroll
      for (int k = 0; k < CW / 32; ++k) nb_s[lane + 32 * k] = KIND == ITERGP_RBF ? kp.c_exp * nb_next[k] : nb_next[k];
      __syncwarp();
      wkn.next();
      if (t + 1 < T) {
        const StepInfo sn = wkn.cur();
#pragma unroll
        for (int k = 0; k < CW / 32; ++k) nb_next[k] = nb_at(static_cast<int64_t>(sn.b_row) + lane + 32 * k);
      }
      const int gb = gbuf;
      if (!mbar_wait_warp(&gfull[gb], gpar, ab, args.wait_ns)) break;
      if (++gbuf == ng) {
        gbuf = 0;
        gpar ^= 1u;
      }
      tc_fence_after();
      const uint32_t gcol = tb + lane_base + gb * CW;
      // this row's own column, when the chunk holds it (dcol in [0, CW)); the test is
      // warp-uniform so that chunks without a diagonal skip the patch below
      const int64_t dcol64 = grow - st.b_row;
      const bool dhit = args.diag != 0 && dcol64 >= 0 && dcol64 < CW;
      const bool dchunk = __any_sync(0xffffffffu, dhit);
      const int dcol = dhit ? static_cast<int>(dcol64) : -1024;
      // the TMEM load of the next 32-column group is in flight while this one is computed
      const int grp0 = hc * (CW / 32 / NH), grp1 = (hc + 1) * (CW / 32 / NH);
      uint32_t v[32];
      tmem_ld32(gcol + 32 * grp0, v);
      tmem_ld_wait();
#pragma unroll 1
      for (int grp = grp0; grp < grp1; ++grp) {
        uint32_t vn[32];
        const bool more = grp + 1 < grp1;   // warp-uniform
        if (PREF && more) tmem_ld32(gcol + 32 * (grp + 1), vn);
        uint32_t ph[16], pl[16];
        if (dchunk) {
          // the row's own column: a huge a.b clamps r^2 to 0 below, so the kernel value is
          // s itself rather than the rounding left by |a|^2 + |a|^2 - 2 a.a
          const int dj = dcol - 32 * grp;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j == dj) v[j] = __float_as_uint(1e30f);
        }
        // -2 a.b = gsc G: the tile scales of the row and of this group's columns undo the
        // split rows' powers of two exactly (a wide chunk spans two 128-row tiles of B)
        float gsc = -2.f;
        if constexpr (NT1 == 3) {
          const int64_t br = static_cast<int64_t>(st.b_row) + 32 * grp;
          gsc = -2.f * ua_t * (br < args.b_rows_pad ? args.ub[br / BM] : 1.f);
        }
        if (KIND == ITERGP_RBF) {
          // k = s 2^(c_exp r^2) = 2^t, t = c_exp (|a|^2 + |b|^2 - 2 a.b) + log2 s, formed two
          // lanes at a time; r^2 >= 0 is t <= log2 s (c_exp < 0)
          const uint64_t m2c = f2_pack(gsc * kp.c_exp, gsc * kp.c_exp);
          const uint64_t rc2 = f2_pack(rowc, rowc);
          const float* cnb = nb_s + 32 * grp;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float2 cb = *reinterpret_cast<const float2*>(cnb + 2 * i);
            const uint64_t t2 = f2_fma(f2_pack(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1])), m2c,
                                       f2_add(f2_pack(cb.x, cb.y), rc2));
            const float k0 = ex2_approx(fminf(f2_lo(t2), kls));
            const float k1 = ex2_approx(fminf(f2_hi(t2), kls));
            if constexpr (NT2 == 3) {   // FP16 hi and lo (22 significant bits)
              ph[i] = pack_f16x2(k0, k1);
              const uint64_t hh = f2_pack(f16_lo_to_f32(ph[i]), f16_hi_to_f32(ph[i]));
              const uint64_t lo2 = f2_sub(f2_pack(k0, k1), hh);
              pl[i] = pack_f16x2(f2_lo(lo2), f2_hi(lo2));
            } else {
              ph[i] = pack_bf16x2(k0, k1);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float r0 = fmaxf(fmaf(gsc, __uint_as_float(v[2 * i]), na_r + nb_s[32 * grp + 2 * i]), 0.f);
            const float r1 = fmaxf(fmaf(gsc, __uint_as_float(v[2 * i + 1]), na_r + nb_s[32 * grp + 2 * i + 1]), 0.f);
            const float k0 = kernel_eval_fast<KIND>(r0, kp) * kmul;
            const float k1 = kernel_eval_fast<KIND>(r1, kp) * kmul;
            if constexpr (NT2 == 3) {
              ph[i] = pack_f16x2(k0, k1);
              pl[i] = pack_f16x2(k0 - f16_lo_to_f32(ph[i]), k1 - f16_hi_to_f32(ph[i]));
            } else {
              ph[i] = pack_bf16x2(k0, k1);
            }
          }
        }
        tmem_st16(gcol + 32 * grp, ph);
        if (NT2 == 3) tmem_st16(gcol + 32 * grp + 16, pl);
        if (more) {
          if constexpr (PREF) {
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = vn[i];
          } else {
            tmem_ld32(gcol + 32 * (grp + 1), v);
            tmem_ld_wait();
          }
        }
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();   // one arrival per warp (the pair form's on the even CTA's barrier)
      if (lane == 0) {
        if constexpr (PAIR) mbar_arrive_remote(lead(&pfull[gb])); else mbar_arrive(&pfull[gb]);
      }
      if (sub_last) {
        ++sub;
        if (!mbar_wait_warp(&ofull, static_cast<uint32_t>(sub & 1), ab, args.wait_ns)) break;
        tc_fence_after();
        const bool full_row = st.item >= 0 || ((seg_c0 == 0) && (c == J - 1));
        float* dst = nullptr;
        bool valid = true;
        if (last) {
          if (st.item >= 0) {
            dst = out_row;
            valid = out_valid;
          } else if (full_row) {
            dst = args.Y + grow * args.ldY;
            valid = grow < args.m;
          } else {
            // partial runs only occur in the tail phase; segment index there -> slot
            const int64_t slot = 2 * g + (seg - sch.fw == 0 ? 0 : 1);
            dst = args.partial + (slot * tile_rows(PAIR) + BM * static_cast<int64_t>(h) + row) * args.p_pad;
          }
        }
        const int lim = st.item >= 0 ? out_lim : (full_row ? args.p_valid : args.p_pad);
        if constexpr (O2REG) {
          // O2 in registers: add the flushed O (IEEE round-to-nearest), write at the run's end
          const int np16 = args.p_pad / 16;
#pragma unroll
          for (int gi = 0; gi < O2G; ++gi) {
            const int c16 = hc + gi * NH;
            if (c16 < np16) {   // warp-uniform
              uint32_t o[16];
              tmem_ld16(tb + lane_base + ocol + 16 * c16, o);
              tmem_ld_wait();
#pragma unroll
              for (int i = 0; i < 16; ++i)
                o2r[gi][i] = sub_in_seg > 0 ? o2r[gi][i] + __uint_as_float(o[i]) : __uint_as_float(o[i]);
              if (last && valid) {
                if constexpr (NT2 == 3) {   // undo the weights' and the kernel values' scales
                  const float* ws = (st.item >= 0 ? item_ws : args.wscale) + args.s_row0 + 16 * c16;
                  const float kinv = pow2i(-static_cast<int>(ke));
#pragma unroll
                  for (int i = 0; i < 16; ++i)
                    if (16 * c16 + i < lim) dst[16 * c16 + i] = (o2r[gi][i] * ws[i]) * kinv;
                } else {
#pragma unroll
                  for (int i = 0; i < 16; ++i)
                    if (16 * c16 + i < lim) dst[16 * c16 + i] = o2r[gi][i];
                }
              }
            }
          }
        }
        for (int c16 = hc; !O2REG && c16 < args.p_pad / 16; c16 += NH) {
          uint32_t o[16];
          tmem_ld16(tb + lane_base + ocol + 16 * c16, o);
          if (pk2) {   // the correction half (hi.lo + lo.hi) of the packed GEMM2's columns
            uint32_t ox[16];
            tmem_ld16(tb + lane_base + ocol + static_cast<uint32_t>(args.p_pad) + 16 * c16, ox);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = __float_as_uint(__uint_as_float(o[i]) + __uint_as_float(ox[i]));
          }
          if (sub_in_seg > 0) {
            uint32_t o2[16];
            tmem_ld16(tb + lane_base + o2col + 16 * c16, o2);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = __float_as_uint(__uint_as_float(o[i]) + __uint_as_float(o2[i]));
          } else {
            tmem_ld_wait();
          }
          if (last) {
            if (valid) {
              if constexpr (NT2 == 3) {   // undo the weights' and the kernel values' scales
                const float* ws = (st.item >= 0 ? item_ws : args.wscale) + args.s_row0 + 16 * c16;
                const float kinv = pow2i(-static_cast<int>(ke));
#pragma unroll
                for (int i = 0; i < 16; ++i)
                  if (16 * c16 + i < lim) dst[16 * c16 + i] = (__uint_as_float(o[i]) * ws[i]) * kinv;
              } else {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                  if (16 * c16 + i < lim) dst[16 * c16 + i] = __uint_as_float(o[i]);
              }
            }
          } else {
            tmem_st16(tb + lane_base + o2col + 16 * c16, o);
          }
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR) mbar_arrive_remote(lead(&oempty)); else mbar_arrive(&oempty);
        }
        ++sub_in_seg;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) {
    // After an abort the odd CTA cannot see its own loads land (they count on the even
    // CTA's barriers): give copies in flight 1 ms before it may exit.  Then neither CTA
    // leaves while the other may still address its shared memory or TMEM.
    if (abort_s) {
      const uint64_t t0 = globaltimer_ns();
      while (globaltimer_ns() - t0 < 1000000ull) {
      }
    }
    cluster_sync_all();
  }
  if (warp == 2) {
    tc_fence_after();
    if constexpr (PAIR) tmem_dealloc_pair(tb, kTmemCols); else tmem_dealloc(tb, kTmemCols);
  }
  if (threadIdx.x == 0 && abort_s) atomicExch(args.status, ITERGP_ETIMEOUT);
}

// One launch of an instantiation, or (max_clusters non-null, pair form) the number of
// its clusters that can be resident at once.  The pair form launches 2 * grid CTAs in
// clusters of two.
template <int KIND, int NT1, int NT2, int NSTAGE, int EPI, bool ARES, bool PAIR, int CW = BN>
cudaError_t launch_tc(int grid, size_t smem, cudaStream_t st, const CUtensorMap* maps, const TcArgs& a,
                      int* max_clusters) {
  auto fn = kmv_tc_kernel<KIND, NT1, NT2, NSTAGE, EPI, ARES, PAIR, CW>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (PAIR) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(2 * grid));
    cfg.blockDim = dim3(tc_threads(EPI));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (max_clusters) return cudaOccupancyMaxActiveClusters(max_clusters, fn, &cfg);
    timing_begin(st);
    e = cudaLaunchKernelEx(&cfg, fn, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], a);
    ::itergp::note_launch();
    timing_end(st);
    return e != cudaSuccess ? e : cudaGetLastError();
  } else {
    if (max_clusters) return cudaErrorInvalidValue;
    timing_begin(st);
    fn<<<grid, tc_threads(EPI), smem, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], a), ::itergp::note_launch();
    timing_end(st);
    return cudaGetLastError();
  }
}

// Instantiated rings: streamed A+B 2, 3, 4 stages; resident A (B-only stages) 3, 5 (one-CTA
// form only); wide chunks (pair form): 3 streamed stages.
template <int KIND, int NT1, int NT2, int EPI, bool PAIR, int CW = BN>
cudaError_t launch_stages(int nstage, bool ares, int grid, size_t smem, cudaStream_t st,
                          const CUtensorMap* maps, const TcArgs& a, int* mc) {
  if constexpr (CW != BN) {
    if (ares || nstage != 3) return cudaErrorInvalidValue;
    return launch_tc<KIND, NT1, NT2, 3, EPI, false, true, CW>(grid, smem, st, maps, a, mc);
  } else {
    if (ares) {
      if constexpr (NT1 == 2 || PAIR)   // TF32 rows take two slices per 64 columns; pairs stream A
        return cudaErrorInvalidValue;
      else
        return nstage == 5 ? launch_tc<KIND, NT1, NT2, 5, EPI, true, false>(grid, smem, st, maps, a, mc)
                           : launch_tc<KIND, NT1, NT2, 3, EPI, true, false>(grid, smem, st, maps, a, mc);
    }
    switch (nstage) {
      case 2: return launch_tc<KIND, NT1, NT2, 2, EPI, false, PAIR>(grid, smem, st, maps, a, mc);
      case 3: return launch_tc<KIND, NT1, NT2, 3, EPI, false, PAIR>(grid, smem, st, maps, a, mc);
      default: return launch_tc<KIND, NT1, NT2, 4, EPI, false, PAIR>(grid, smem, st, maps, a, mc);
    }
  }
}

template <int KIND, int EPI, bool PAIR, int CW = BN>
cudaError_t launch_prec_epi(int prec, int nstage, bool ares, int grid, size_t smem, cudaStream_t st,
                            const CUtensorMap* maps, const TcArgs& a, int* mc) {
  switch (prec) {
    case ITERGP_BF16X3: return launch_stages<KIND, 3, 3, EPI, PAIR, CW>(nstage, ares, grid, smem, st, maps, a, mc);
    case ITERGP_BF16_COMP: return launch_stages<KIND, 3, 1, EPI, PAIR, CW>(nstage, ares, grid, smem, st, maps, a, mc);
    case ITERGP_TF32: return launch_stages<KIND, 2, 3, EPI, PAIR, CW>(nstage, ares, grid, smem, st, maps, a, mc);
    default: return launch_stages<KIND, 1, 1, EPI, PAIR, CW>(nstage, ares, grid, smem, st, maps, a, mc);
  }
}

template <int KIND, bool PAIR, int CW = BN>
cudaError_t launch_prec(int prec, int nstage, bool ares, int epi, int grid, size_t smem,
                        cudaStream_t st, const CUtensorMap* maps, const TcArgs& a, int* mc = nullptr) {
  return epi == 8 ? launch_prec_epi<KIND, 8, PAIR, CW>(prec, nstage, ares, grid, smem, st, maps, a, mc)
                  : launch_prec_epi<KIND, 4, PAIR, CW>(prec, nstage, ares, grid, smem, st, maps, a, mc);
}

}  // namespace
}  // namespace tcimpl
}  // namespace itergp
