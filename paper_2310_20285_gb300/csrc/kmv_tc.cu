// Tensor-core kernel product Y = k(A, B) S for sm_103a (tcgen05 + TMEM + TMA).
//
// The product of App. B.3.1 is evaluated flash-style and K is never stored:
//   for each CTA-owned (row tile of A, column chunk of B):
//     G   = A_tile . B_chunk^T        tcgen05.mma, BF16 operands, FP32 accumulator in TMEM
//     P   = k(|a|^2 + |b|^2 - 2 G)    epilogue warps: TMEM -> registers -> BF16 -> TMEM
//     O  += P . S_chunk               tcgen05.mma with P read from TMEM (A operand)
// Operands are staged by TMA with 128-byte swizzle.  Split precisions use BF16 hi/lo
// parts: a.b ~ ah.bh + ah.bl + al.bh and P S ~ Ph Sh + Ph Sl + Pl Sh.
//
// Warp roles (256 threads): warp 0 issues TMA loads, warp 1 issues the MMAs (one thread),
// warp 2 owns the TMEM allocation, warps 4-7 (one per TMEM lane quadrant) run the kernel
// evaluation and the output stores.  TMEM columns: G0 [0,128), G1 [128,256) (double
// buffer, P aliases the G it came from), O [256, 256 + p_tile).
//
// The tensor core accumulates in FP32 with truncation, which biases long sums; O is
// therefore accumulated over sub-runs of at most kFlushChunks chunks and each sub-run
// is added into the running sum O2 [384, 384 + p_tile) by the epilogue with ordinary
// FP32 adds.
//
// Work partition (G persistent CTAs, R row tiles, J column chunks): the first
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

#include "internal.h"
#include "tc_ptx.cuh"
#include "tma_host.h"

namespace itergp {
namespace {

constexpr int BM = 128;   // rows of A per tile (MMA M)
constexpr int BN = 128;   // rows of B per chunk (MMA N of the distance GEMM, K of the product)
constexpr int BK = 64;    // D slice per stage (one 128-byte swizzle row of BF16)
// Row operand forms (NT1): 1 BF16 rows, 3 split BF16 rows (hi, lo), 2 TF32 rows (FP32
// storage, 32 values per 128-byte swizzle row, kind::tf32 MMAs of K = 8).  A stage holds
// one 128-byte row per tile row in every form, so the ring layout is the same.
__host__ __device__ constexpr int slice_elems(int nt1) { return nt1 == 2 ? BK / 2 : BK; }
// Threads: warps 0-3 (TMA, MMA, TMEM owner, idle) plus EPI epilogue warps (4 or 8; with 8,
// two warps share each TMEM lane quadrant and split the columns).
__host__ __device__ constexpr int tc_threads(int epi) { return (4 + epi) * 32; }
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kOCol = 256;
constexpr uint32_t kO2Col = 384;   // FP32 running sum of flushed O (IEEE round-to-nearest adds)
// G buffers (and weight-tile slots): 3 for P tiles <= 48, else 2.  With three, GEMM2 of a
// chunk is issued two chunks behind its GEMM1, so the epilogue of chunk t overlaps GEMM1
// of t + 1 and t + 2 (at small D the epilogue is longer than one GEMM1).  TMEM then holds
// G 3 x 128 columns, O at 384 and O2 at 384 + P.
__host__ __device__ constexpr int g_bufs(int p_pad) { return p_pad <= 48 ? 3 : 2; }
constexpr int kFlushChunks = 4;    // O is flushed into O2 at least every 4 chunks (512 rows)
constexpr uint64_t kWaitLimitNs = 4000000000ull;   // 4 s per wait

struct TcArgs {
  const float* na;        // [A.rows_pad] row norms of A
  const float* nb;        // [B.rows_pad] row norms of B
  int64_t m;              // valid rows of A
  int64_t row_tiles;      // R
  int chunks;             // J
  int nk;                 // D slices (d_pad / 64)
  int p_pad;              // MMA N of the product (multiple of 16, <= 128)
  int p_valid;            // valid output columns of this P tile
  int s_row0;             // first row of this P tile in the transposed S
  int p_col0;             // item mode: first output column of this P tile
  float* Y;               // output, already offset to the tile's first column
  int64_t ldY;
  float* partial;         // [2 G][BM][p_pad]
  KParams kp;
  int* status;
  const int* active;
  // item mode (batched problems): per-CTA lists of whole row tiles
  const WorkItem* items;            // nullptr: single-problem schedule
  const int32_t* item_begin;        // [G + 1]
  const TcProb* probs;
};

__host__ __device__ constexpr uint32_t stage_bytes(int nt1) {
  return (nt1 == 3 ? 2u : 1u) * (BM * BK * 2u) + (nt1 == 3 ? 2u : 1u) * (BN * BK * 2u);
}
// Split arrival: with a two-stage ring of split rows the stage's arrival is on the critical
// path, so its hi halves are tracked by their own barrier and the hi.hi MMAs start as soon
// as they land (measured faster there; with deeper rings the extra wait costs more than it
// saves).
__host__ __device__ constexpr bool split_arrival(int nt1, int nstage, bool ares) {
  return nt1 == 3 && nstage == 2 && !ares;
}
__host__ __device__ constexpr uint32_t s_box_bytes(int p_pad) { return static_cast<uint32_t>(p_pad) * 128u; }
__host__ __device__ constexpr uint32_t s_buf_bytes(int nt2, int p_pad) {
  return 2u * s_box_bytes(p_pad) * (nt2 == 3 ? 2u : 1u);
}
// alignment slack + per-epilogue-warp staging of 128 column norms
__host__ __device__ constexpr uint32_t smem_extra(int epi) { return 1024u + static_cast<uint32_t>(epi) * 512u; }

// Out-of-line slow path of a bounded mbarrier wait (the fast path is one try_wait).
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                            uint64_t limit_ns) {
  return mbar_wait(bar, parity, abort_flag, limit_ns);
}

// GEMM1 of one chunk: G = A . B^T over the nk D slices of the stage ring (12 MMAs per
// slice for split rows: hi.hi + hi.lo + lo.hi, K = 16 each), releasing each stage to the
// producer with a commit.  `pos` packs the ring position (stage | phase << 8); returns the
// position after the chunk, or -1 if a wait gave up.  A small out-of-line function: the
// issuing thread must keep up with one MMA every few dozen cycles.
template <int NT1, int NSTAGE, bool ARES>
__device__ __noinline__ int issue_gemm1(uint32_t gt, int nk, uint64_t dStage0, uint64_t dAres, uint64_t* full_bar,
                                        uint64_t* full_lo, uint64_t* empty_bar, volatile int* ab, uint32_t idesc1,
                                        int pos) {
  constexpr uint32_t A_PART = BM * BK * 2, B_PART = BN * BK * 2;
  constexpr uint32_t SB = ARES ? (NT1 == 3 ? 2u : 1u) * B_PART : stage_bytes(NT1);
  constexpr bool SPLIT = split_arrival(NT1, NSTAGE, ARES);
  int stage = pos & 0xFF;
  uint32_t phase = static_cast<uint32_t>(pos >> 8);
  for (int ks = 0; ks < nk; ++ks) {
    // operands arrive by TMA with completion on the mbarrier (async proxy on both sides):
    // no tcgen05 fence is needed here
    if (!mbar_wait(&full_bar[stage], phase, ab, kWaitLimitNs)) return -1;
    const uint64_t dSt = dStage0 + static_cast<uint64_t>(stage) * (SB >> 4);
    const uint64_t dAh = ARES ? dAres : dSt;
    const uint64_t dBh = ARES ? dSt : dSt + ((NT1 == 3 ? 2 : 1) * A_PART >> 4);
    const uint64_t dAl = dAh + (A_PART >> 4);
    const uint64_t dBl = dBh + (B_PART >> 4);
    // one MMA order for every ring, so that all launch variants give bitwise the same
    // product: the slice's hi.hi terms, then its correction terms hi.lo and lo.hi
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {   // K steps of 32 bytes: 16 BF16 or 8 TF32 values
      if constexpr (NT1 == 2)
        mma_ss_tf32(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
      else
        mma_ss(gt, dAh + 2 * kk, dBh + 2 * kk, idesc1, (ks | kk) != 0 ? 1u : 0u);
    }
    if (NT1 == 3) {
      if (SPLIT && !mbar_wait(&full_lo[stage], phase, ab, kWaitLimitNs)) return -1;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        mma_ss(gt, dAh + 2 * kk, dBl + 2 * kk, idesc1, 1u);
        mma_ss(gt, dAl + 2 * kk, dBh + 2 * kk, idesc1, 1u);
      }
    }
    mma_commit(&empty_bar[stage]);
    if (++stage == NSTAGE) {
      stage = 0;
      phase ^= 1u;
    }
  }
  return stage | static_cast<int>(phase << 8);
}

// GEMM2 of one chunk: O (+)= P . S with P (the chunk's kernel values, BF16 hi/lo pairs
// packed in the G buffer's TMEM columns) as the A operand and the chunk's transposed
// weights from shared memory as B; 8 K steps of 16 rows, 3 MMAs each for split weights.
// Waits for the epilogue's P (pfull) and the weight tile (sfull); releases the weight tile
// (sempty) and, at the end of a flush group, hands O to the epilogue (ofull).
template <int NT2>
__device__ __noinline__ bool issue_gemm2(uint32_t tb, uint32_t a_col0, uint32_t o_col, uint32_t par, bool first, bool last,
                                         uint64_t* pfull_b, uint64_t* sfull_b, uint64_t* sempty_b, uint64_t* ofull_b,
                                         volatile int* ab, uint64_t dS0, uint64_t sbox16, uint32_t idesc2) {
  if (!mbar_try_wait(pfull_b, par) && !mbar_wait(pfull_b, par, ab, kWaitLimitNs)) return false;
  if (!mbar_try_wait(sfull_b, par) && !mbar_wait(sfull_b, par, ab, kWaitLimitNs)) return false;
  tc_fence_after();   // P was written by the epilogue's tcgen05.st
#pragma unroll
  for (int ks2 = 0; ks2 < BN / 16; ++ks2) {
    const int grp = ks2 >> 1, h = ks2 & 1;
    const uint32_t a_hi = tb + a_col0 + static_cast<uint32_t>(32 * grp + 8 * h);
    const uint64_t dSh = dS0 + static_cast<uint64_t>(ks2 >> 2) * sbox16 + static_cast<uint64_t>((ks2 & 3) * 2);
    mma_ts(tb + o_col, a_hi, dSh, idesc2, (first && ks2 == 0) ? 0u : 1u);
    if (NT2 == 3) {
      mma_ts(tb + o_col, a_hi, dSh + 2 * sbox16, idesc2, 1u);
      mma_ts(tb + o_col, a_hi + 16, dSh, idesc2, 1u);
    }
  }
  mma_commit(sempty_b);
  if (last) mma_commit(ofull_b);
  return true;
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
  int32_t a_row;   // A-arena row of the current tile
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
  __device__ void init(const TcArgs& a, int64_t G, int64_t g) {
    items = a.items;
    probs = a.probs;
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
      s.a_row = static_cast<int32_t>(row * BM);
      s.b_row = c * BN;
      s.c = c;
      // a row run starts at chunk 0, at step 0 and where the tail begins; it ends at the
      // row's last chunk and at the CTA's last step
      s.first = t == 0 || c == 0 || t == lock;
      s.last = t == sch.T - 1 || c == sch.J - 1;
      s.item = -1;
    } else {
      s.a_row = it_a_row;
      s.b_row = it_b_row0 + c * BN;
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

// ARES (D <= 64, one K slice): the A tile of a row segment stays resident in shared
// memory for all of its chunks and only B streams through the ring.
template <int KIND, int NT1, int NT2, int NSTAGE, int EPI, bool ARES>
__global__ void __launch_bounds__(tc_threads(EPI), 1)
kmv_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
              const __grid_constant__ CUtensorMap mSh, const __grid_constant__ CUtensorMap mSl,
              const TcArgs args) {
  if (args.active != nullptr && *args.active == 0) return;
  const int64_t G = gridDim.x, g = blockIdx.x;
  Walker walk0;
  walk0.init(args, G, g);
  const int64_t T = walk0.total();
  if (T <= 0) return;
  const Schedule& sch = walk0.sch;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  constexpr uint32_t A_PART = BM * BK * 2, B_PART = BN * BK * 2;
  constexpr uint32_t A_BYTES = (NT1 == 3 ? 2u : 1u) * A_PART;   // resident A (ARES)
  constexpr uint32_t SB = ARES ? (NT1 == 3 ? 2u : 1u) * B_PART : stage_bytes(NT1);
  constexpr bool SPLIT = split_arrival(NT1, NSTAGE, ARES);
  const int ng = g_bufs(args.p_pad);                     // G buffers = weight-tile slots
  const uint32_t ocol = ng == 3 ? 384u : kOCol;
  const uint32_t o2col = ng == 3 ? 384u + static_cast<uint32_t>(args.p_pad) : kO2Col;
  const uint32_t SBOX = s_box_bytes(args.p_pad);
  const uint32_t SBUF = s_buf_bytes(NT2, args.p_pad);
  uint8_t* a_region = smem + NSTAGE * SB;                        // ARES only
  uint8_t* s_region = a_region + (ARES ? A_BYTES : 0u);
  float* nb_all = reinterpret_cast<float*>(s_region + ng * SBUF);   // [EPI warps][128]

  // full_bar: a whole stage, or with split arrival its hi halves (A_hi and B_hi, enough for
  // the hi.hi MMAs) while full_lo tracks the lo halves
  __shared__ __align__(8) uint64_t full_bar[NSTAGE], full_lo[NSTAGE], empty_bar[NSTAGE];
  __shared__ __align__(8) uint64_t gfull[3], pfull[3], sfull[3], sempty[3], ofull, oempty, drain;
  __shared__ __align__(8) uint64_t afull, aempty;               // resident A (ARES)
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&full_lo[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    for (int i = 0; i < 3; ++i) {
      mbar_init(&gfull[i], 1);
      mbar_init(&pfull[i], 32 * EPI);
      mbar_init(&sfull[i], 1);
      mbar_init(&sempty[i], 1);
    }
    mbar_init(&ofull, 1);
    mbar_init(&oempty, 32 * EPI);
    mbar_init(&drain, 1);
    mbar_init(&afull, 1);
    mbar_init(&aempty, 1);
    fence_mbar_init();
  }
  if (warp == 2) {
    tmem_alloc(&tmem_base_s, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tmem_base_s;
  volatile int* ab = &abort_s;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&mAh);
      tma_prefetch_desc(&mBh);
      tma_prefetch_desc(&mSh);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t armed = 0, armed_par = 0;      // bit i: stage i armed / parity of last arm
      uint32_t s_armed = 0, s_par = 0;
      int s_slot = 0;
      uint32_t s_phase = 0;                   // weight-tile ring: slot t % ng, parity (t / ng) & 1
      bool a_armed = false;
      uint32_t a_par = 0;
      int64_t seg = -1;
      Walker wk = walk0;
      for (int64_t t = 0; t < T && !*ab; ++t, wk.next()) {
        const StepInfo st = wk.cur();
        const int32_t a_y = st.a_row;
        const int32_t b_y = st.b_row;
        if (ARES) {
          if (st.first) {
            // a new row segment: reload A once the previous segment's MMAs are done with it
            ++seg;
            if (seg >= 1 && !mbar_wait(&aempty, static_cast<uint32_t>((seg - 1) & 1), ab, kWaitLimitNs)) break;
            mbar_arrive_expect_tx(&afull, A_BYTES);
            a_armed = true;
            a_par = static_cast<uint32_t>(seg & 1);
            tma_load_2d(a_region, &mAh, &afull, 0, a_y);
            if (NT1 == 3) tma_load_2d(a_region + A_PART, &mAl, &afull, 0, a_y);
          }
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, ab, kWaitLimitNs)) break;
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
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, ab, kWaitLimitNs)) break;
          uint64_t* lo_bar = SPLIT ? &full_lo[stage] : &full_bar[stage];
          mbar_arrive_expect_tx(&full_bar[stage], SPLIT ? A_PART + B_PART : SB);
          if (SPLIT) mbar_arrive_expect_tx(lo_bar, A_PART + B_PART);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          uint8_t* base = smem + stage * SB;
          uint8_t* bbase = base + (NT1 == 3 ? 2 : 1) * A_PART;
          tma_load_2d(base, &mAh, &full_bar[stage], ks * slice_elems(NT1), a_y);
          tma_load_2d(bbase, &mBh, &full_bar[stage], ks * slice_elems(NT1), b_y);
          if (NT1 == 3) {
            tma_load_2d(base + A_PART, &mAl, lo_bar, ks * BK, a_y);
            tma_load_2d(bbase + B_PART, &mBl, lo_bar, ks * BK, b_y);
          }
          if (++stage == NSTAGE) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (*ab) break;
        const int sb = s_slot;
        if (!mbar_wait(&sempty[sb], s_phase ^ 1u, ab, kWaitLimitNs)) break;
        mbar_arrive_expect_tx(&sfull[sb], SBUF);
        s_armed |= 1u << sb;
        s_par = (s_par & ~(1u << sb)) | (s_phase << sb);
        if (++s_slot == ng) {
          s_slot = 0;
          s_phase ^= 1u;
        }
        uint8_t* sbase = s_region + sb * SBUF;
        tma_load_2d(sbase, &mSh, &sfull[sb], b_y, args.s_row0);
        tma_load_2d(sbase + SBOX, &mSh, &sfull[sb], b_y + 64, args.s_row0);
        if (NT2 == 3) {
          tma_load_2d(sbase + 2 * SBOX, &mSl, &sfull[sb], b_y, args.s_row0);
          tma_load_2d(sbase + 3 * SBOX, &mSl, &sfull[sb], b_y + 64, args.s_row0);
        }
      }
      if (*ab) {
        // let every load this thread issued land before the CTA can exit
        for (int i = 0; i < NSTAGE; ++i)
          if (armed & (1u << i)) {
            mbar_wait_drain(&full_bar[i], (armed_par >> i) & 1u, kWaitLimitNs);
            if (SPLIT) mbar_wait_drain(&full_lo[i], (armed_par >> i) & 1u, kWaitLimitNs);
          }
        for (int i = 0; i < 3; ++i)
          if (s_armed & (1u << i)) mbar_wait_drain(&sfull[i], (s_par >> i) & 1u, kWaitLimitNs);
        if (a_armed) mbar_wait_drain(&afull, a_par, kWaitLimitNs);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc1 = NT1 == 2 ? idesc_tf32_f32(BM, BN) : idesc_bf16_f32(BM, BN);
      const uint32_t idesc2 = idesc_bf16_f32(BM, static_cast<uint32_t>(args.p_pad));
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
      int g2 = 0;           // GEMM2's buffer / slot (t % ng) and its parity ((t / ng) & 1)
      uint32_t g2par = 0;
      auto gemm2 = [&](int64_t t) -> bool {
        const StepInfo st = wk2.cur();
        wk2.next();
        const int c = st.c;
        const bool first = st.first || (c % kFlushChunks == 0);
        const bool last = st.last || ((c + 1) % kFlushChunks == 0);
        if (first) {
          ++sub;
          if (sub >= 1 && !mbar_wait_slow(&oempty, static_cast<uint32_t>((sub - 1) & 1), ab, kWaitLimitNs))
            return false;
        }
        (void)t;
        const int gb = g2;
        const uint32_t par = g2par;
        if (++g2 == ng) {
          g2 = 0;
          g2par ^= 1u;
        }
        return issue_gemm2<NT2>(tb, static_cast<uint32_t>(gb) * BN, ocol, par, first, last, &pfull[gb], &sfull[gb],
                                &sempty[gb], &ofull, ab, dS_base + static_cast<uint64_t>(gb) * (SBUF >> 4), sbox16,
                                idesc2);
      };
      Walker wk1 = walk0;    // GEMM1 steps (segment boundaries for the resident A)
      int64_t aseg = -1;
      const int nk = args.nk;
      const int lag = ng - 1;
      int g1 = 0;           // GEMM1's buffer (t % ng)
      for (int64_t t = 0; t < T && ok; ++t, wk1.next()) {
        const int gb = g1;
        if (++g1 == ng) g1 = 0;
        const uint32_t gt = tb + static_cast<uint32_t>(gb) * BN;
        bool seg_last = false;
        if (ARES) {
          const StepInfo st1 = wk1.cur();
          seg_last = st1.last;
          if (st1.first) {
            ++aseg;
            if (!mbar_wait_slow(&afull, static_cast<uint32_t>(aseg & 1), ab, kWaitLimitNs)) {
              ok = false;
              break;
            }
          }
        }
        const int pos = issue_gemm1<NT1, NSTAGE, ARES>(gt, nk, dStage0, dAres, full_bar, full_lo, empty_bar, ab, idesc1,
                                                       stage | static_cast<int>(phase << 8));
        if (pos < 0) {
          ok = false;
          break;
        }
        stage = pos & 0xFF;
        phase = static_cast<uint32_t>(pos >> 8);
        if (!ok) break;
        if (ARES && seg_last) mma_commit(&aempty);   // the segment's A is no longer read
        mma_commit(&gfull[gb]);
        if (t >= lag && !gemm2(t - lag)) ok = false;
      }
      for (int64_t t = T > lag ? T - lag : 0; ok && t < T; ++t)
        if (!gemm2(t)) ok = false;
      // all issued MMAs must retire before TMEM is released
      mma_commit(&drain);
      mbar_wait_drain(&drain, 0, kWaitLimitNs);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ epilogue
    constexpr int NH = EPI / 4;     // epilogue warps per TMEM lane quadrant
    const int e = warp - 4;
    const int q = e & 3;            // lane quadrant (= warp % 4, the warp's TMEM lanes)
    const int h = e >> 2;           // this warp's share of the columns
    const int row = 32 * q + lane;
    const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
    int64_t seg = -1, sub = -1;
    int seg_c0 = 0, sub_in_seg = 0;
    float na_r = 0.f;
    int64_t grow = 0;
    KParams kp = args.kp;
    float rowc = 0.f;   // RBF: c_exp |a|^2 + log2 s of this thread's row
    const int J = args.chunks;
    float* out_row = nullptr;       // item mode: this row's output
    bool out_valid = false;
    int out_lim = 0;
    Walker wk = walk0;
    int gbuf = 0;                   // G buffer of the current chunk (t % ng) and its parity
    uint32_t gpar = 0;
    // column norms of the next step are loaded while the current chunk is processed
    Walker wkn = walk0;
    float nb_next[BN / 32];
    {
      const StepInfo s0 = wkn.cur();
#pragma unroll
      for (int k = 0; k < BN / 32; ++k) nb_next[k] = args.nb[static_cast<int64_t>(s0.b_row) + lane + 32 * k];
    }
    for (int64_t t = 0; t < T; ++t, wk.next()) {
      const StepInfo st = wk.cur();
      const int c = st.c;
      const bool first = st.first;
      const bool last = st.last;
      const bool sub_last = last || ((c + 1) % kFlushChunks == 0);
      if (first) {
        ++seg;
        seg_c0 = c;
        sub_in_seg = 0;
        grow = static_cast<int64_t>(st.a_row) + row;
        na_r = args.na[grow];
        if (st.item >= 0) {
          const WorkItem& it = args.items[st.item];
          const TcProb& pr = args.probs[it.prob];
          kp = pr.kp;
          const int64_t prow = static_cast<int64_t>(it.tile_row) + row;
          out_valid = prow < pr.m;
          out_row = pr.Y + prow * pr.ldY + args.p_col0;
          out_lim = pr.p_valid - args.p_col0;   // <= 0: nothing of this tile to write
        }
        rowc = fmaf(kp.c_exp, na_r, kp.log2s);
      }
      float* nb_s = nb_all + e * BN;
      __syncwarp();
      // RBF stages c_exp |b|^2 (the column term of the exponent), Matern |b|^2
#pragma unroll
      for (int k = 0; k < BN / 32; ++k) nb_s[lane + 32 * k] = KIND == ITERGP_RBF ? kp.c_exp * nb_next[k] : nb_next[k];
      __syncwarp();
      wkn.next();
      if (t + 1 < T) {
        const StepInfo sn = wkn.cur();
#pragma unroll
        for (int k = 0; k < BN / 32; ++k) nb_next[k] = args.nb[static_cast<int64_t>(sn.b_row) + lane + 32 * k];
      }
      const int gb = gbuf;
      if (!mbar_wait_warp(&gfull[gb], gpar, ab, kWaitLimitNs)) break;
      if (++gbuf == ng) {
        gbuf = 0;
        gpar ^= 1u;
      }
      tc_fence_after();
      const uint32_t gcol = tb + lane_base + gb * BN;
      // the TMEM load of the next 32-column group is in flight while this one is computed
      const int grp0 = h * (BN / 32 / NH), grp1 = (h + 1) * (BN / 32 / NH);
      uint32_t v[32];
      tmem_ld32(gcol + 32 * grp0, v);
      tmem_ld_wait();
#pragma unroll 1
      for (int grp = grp0; grp < grp1; ++grp) {
        uint32_t vn[32];
        const bool more = grp + 1 < grp1;   // warp-uniform
        if (more) tmem_ld32(gcol + 32 * (grp + 1), vn);
        uint32_t ph[16], pl[16];
        if (KIND == ITERGP_RBF) {
          // k = s 2^(c_exp r^2) = 2^t, t = c_exp (|a|^2 + |b|^2 - 2 a.b) + log2 s, formed two
          // lanes at a time; r^2 >= 0 is t <= log2 s (c_exp < 0)
          const uint64_t m2c = f2_pack(-2.f * kp.c_exp, -2.f * kp.c_exp);
          const uint64_t rc2 = f2_pack(rowc, rowc);
          const float* cnb = nb_s + 32 * grp;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float2 cb = *reinterpret_cast<const float2*>(cnb + 2 * i);
            const uint64_t t2 = f2_fma(f2_pack(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1])), m2c,
                                       f2_add(f2_pack(cb.x, cb.y), rc2));
            const float k0 = ex2_approx(fminf(f2_lo(t2), kp.log2s));
            const float k1 = ex2_approx(fminf(f2_hi(t2), kp.log2s));
            ph[i] = pack_bf16x2(k0, k1);
            if (NT2 == 3) {
              const uint64_t hh = f2_pack(__uint_as_float(ph[i] << 16), __uint_as_float(ph[i] & 0xFFFF0000u));
              const uint64_t lo2 = f2_sub(f2_pack(k0, k1), hh);
              pl[i] = pack_bf16x2(f2_lo(lo2), f2_hi(lo2));
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float r0 = fmaxf(fmaf(-2.f, __uint_as_float(v[2 * i]), na_r + nb_s[32 * grp + 2 * i]), 0.f);
            const float r1 = fmaxf(fmaf(-2.f, __uint_as_float(v[2 * i + 1]), na_r + nb_s[32 * grp + 2 * i + 1]), 0.f);
            const float k0 = kernel_eval_fast<KIND>(r0, kp);
            const float k1 = kernel_eval_fast<KIND>(r1, kp);
            ph[i] = pack_bf16x2(k0, k1);
            if (NT2 == 3) {
              const float h0 = __uint_as_float(ph[i] << 16);
              const float h1 = __uint_as_float(ph[i] & 0xFFFF0000u);
              pl[i] = pack_bf16x2(k0 - h0, k1 - h1);
            }
          }
        }
        tmem_st16(gcol + 32 * grp, ph);
        if (NT2 == 3) tmem_st16(gcol + 32 * grp + 16, pl);
        if (more) {
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = vn[i];
        }
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&pfull[gb]);
      if (sub_last) {
        ++sub;
        if (!mbar_wait_warp(&ofull, static_cast<uint32_t>(sub & 1), ab, kWaitLimitNs)) break;
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
            dst = args.partial + (slot * BM + row) * args.p_pad;
          }
        }
        const int lim = st.item >= 0 ? out_lim : (full_row ? args.p_valid : args.p_pad);
        for (int c16 = h; c16 < args.p_pad / 16; c16 += NH) {
          uint32_t o[16];
          tmem_ld16(tb + lane_base + ocol + 16 * c16, o);
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
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (16 * c16 + i < lim) dst[16 * c16 + i] = __uint_as_float(o[i]);
            }
          } else {
            tmem_st16(tb + lane_base + o2col + 16 * c16, o);
          }
        }
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(&oempty);
        ++sub_in_seg;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tb, kTmemCols);
  }
  if (threadIdx.x == 0 && abort_s) atomicExch(args.status, ITERGP_ETIMEOUT);
}

// Adds the partial runs of tail row tiles shared by several CTAs, in CTA order.
__global__ void tc_fixup_kernel(const float* __restrict__ partial, int64_t R, int64_t G, int J,
                                int64_t m, int p_pad, int p_valid, float* __restrict__ Y,
                                int64_t ldY, const int* __restrict__ active) {
  if (active != nullptr && *active == 0) return;
  const int64_t rt0 = (R / G) * G, ut = (R - rt0) * J;
  const int64_t r = rt0 + blockIdx.x;
  if (r >= R) return;
  const int64_t u0 = (r - rt0) * J, u1 = u0 + J - 1;
  const int64_t g_lo = part_owner(u0, ut, G), g_hi = part_owner(u1, ut, G);
  if (g_lo == g_hi) return;   // one CTA covered the whole row tile and stored it
  for (int e = threadIdx.x; e < BM * p_valid; e += blockDim.x) {
    const int row = e / p_valid, col = e % p_valid;
    const int64_t grow = r * BM + row;
    if (grow >= m) continue;
    float acc = 0.f;
    for (int64_t gg = g_lo; gg <= g_hi; ++gg) {
      const int64_t s0 = part_start(gg, ut, G);
      if (s0 == part_start(gg + 1, ut, G)) continue;   // CTA without tail units
      const int64_t slot = 2 * gg + (s0 < u0 ? 1 : 0);
      acc += partial[(slot * BM + row) * p_pad + col];
    }
    Y[grow * ldY + col] = acc;
  }
}

// S (n x p, row pitch ldS) -> transposed BF16 hi [p16][n_pad] (+ lo), zero padded.
template <bool SPLIT>
__global__ void prep_s_kernel(const float* __restrict__ S, int64_t ldS, int64_t n, int64_t p,
                              int64_t n_pad, int64_t p16, __nv_bfloat16* __restrict__ hi,
                              __nv_bfloat16* __restrict__ lo, const int* __restrict__ active) {
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
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      hi[cc * n_pad + j] = h;
      if (SPLIT) lo[cc * n_pad + j] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
}

template <int KIND, int NT1, int NT2, int NSTAGE, int EPI, bool ARES>
cudaError_t launch_tc(int grid, size_t smem, cudaStream_t st, const CUtensorMap* maps,
                      const TcArgs& a) {
  auto fn = kmv_tc_kernel<KIND, NT1, NT2, NSTAGE, EPI, ARES>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  timing_begin(st);
  fn<<<grid, tc_threads(EPI), smem, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], a), ::itergp::note_launch();
  timing_end(st);
  return cudaGetLastError();
}

// Instantiated rings: streamed A+B 2, 3, 4 stages; resident A (B-only stages) 3, 5.
template <int KIND, int NT1, int NT2, int EPI>
cudaError_t launch_stages(int nstage, bool ares, int grid, size_t smem, cudaStream_t st,
                          const CUtensorMap* maps, const TcArgs& a) {
  if (ares) {
    if constexpr (NT1 == 2)   // TF32 rows take two slices per 64 columns: no resident A
      return cudaErrorInvalidValue;
    else
      return nstage == 5 ? launch_tc<KIND, NT1, NT2, 5, EPI, true>(grid, smem, st, maps, a)
                         : launch_tc<KIND, NT1, NT2, 3, EPI, true>(grid, smem, st, maps, a);
  }
  switch (nstage) {
    case 2: return launch_tc<KIND, NT1, NT2, 2, EPI, false>(grid, smem, st, maps, a);
    case 3: return launch_tc<KIND, NT1, NT2, 3, EPI, false>(grid, smem, st, maps, a);
    default: return launch_tc<KIND, NT1, NT2, 4, EPI, false>(grid, smem, st, maps, a);
  }
}

template <int KIND, int EPI>
cudaError_t launch_prec_epi(int prec, int nstage, bool ares, int grid, size_t smem, cudaStream_t st,
                            const CUtensorMap* maps, const TcArgs& a) {
  switch (prec) {
    case ITERGP_BF16X3: return launch_stages<KIND, 3, 3, EPI>(nstage, ares, grid, smem, st, maps, a);
    case ITERGP_BF16_COMP: return launch_stages<KIND, 3, 1, EPI>(nstage, ares, grid, smem, st, maps, a);
    case ITERGP_TF32: return launch_stages<KIND, 2, 3, EPI>(nstage, ares, grid, smem, st, maps, a);
    default: return launch_stages<KIND, 1, 1, EPI>(nstage, ares, grid, smem, st, maps, a);
  }
}

template <int KIND>
cudaError_t launch_prec(int prec, int nstage, bool ares, int epi, int grid, size_t smem,
                        cudaStream_t st, const CUtensorMap* maps, const TcArgs& a) {
  return epi == 8 ? launch_prec_epi<KIND, 8>(prec, nstage, ares, grid, smem, st, maps, a)
                  : launch_prec_epi<KIND, 4>(prec, nstage, ares, grid, smem, st, maps, a);
}

// ---------------------------------------------------------------- launch variants
// A variant: epilogue warps (4 or 8) and pipeline stages (0: the deepest that fits).
// The table holds what the autotuner measured per (precision, kind, d_pad, P tile,
// schedule); a thread may force a variant while it times candidates.
struct TcVariant {
  int epi = 4;
  int nstage = 0;
  int ares = -1;   // resident A (one K slice only): 1 on, 0 off, -1 on where possible
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
int stages_that_fit(const DeviceContext* ctx, int nt1, int nt2, int p_tile, int epi, int want,
                    bool ares = false) {
  const size_t smem_cap = std::min<size_t>(ctx->smem_optin, 232448) - 2048;
  const size_t a_bytes = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BM * BK * 2 : 0;
  const size_t stage = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BN * BK * 2 : stage_bytes(nt1);
  const size_t fixed = g_bufs(p_tile) * s_buf_bytes(nt2, p_tile) + smem_extra(epi) + a_bytes;
  const int fit = static_cast<int>((smem_cap > fixed ? smem_cap - fixed : 0) / stage);
  int ns = ares ? (fit >= 5 ? 5 : fit >= 3 ? 3 : 0) : (fit >= 4 ? 4 : fit >= 3 ? 3 : fit >= 2 ? 2 : 0);
  if (want >= 2 && ns > want) ns = ares ? (want >= 5 ? 5 : want >= 3 ? 3 : 0) : want;
  return ns;
}

int tc_nt1(int prec) { return precision_tf32_rows(prec) ? 2 : precision_splits_rows(prec) ? 3 : 1; }

// Tensor maps of the row operands (maps[1] and [3] repeat the hi planes when rows are not split).
bool encode_rows(CUtensorMap* maps, const RowOperand& A, const RowOperand& B, int nt1) {
  if (nt1 == 2)
    return encode_f32_sw128(&maps[0], A.hi, A.rows_pad, A.d_pad, A.d_pad, BM) &&
           encode_f32_sw128(&maps[1], A.hi, A.rows_pad, A.d_pad, A.d_pad, BM) &&
           encode_f32_sw128(&maps[2], B.hi, B.rows_pad, B.d_pad, B.d_pad, BN) &&
           encode_f32_sw128(&maps[3], B.hi, B.rows_pad, B.d_pad, B.d_pad, BN);
  return encode_bf16_sw128(&maps[0], A.hi, A.rows_pad, A.d_pad, A.d_pad, BM) &&
         encode_bf16_sw128(&maps[1], nt1 == 3 ? A.lo : A.hi, A.rows_pad, A.d_pad, A.d_pad, BM) &&
         encode_bf16_sw128(&maps[2], B.hi, B.rows_pad, B.d_pad, B.d_pad, BN) &&
         encode_bf16_sw128(&maps[3], nt1 == 3 ? B.lo : B.hi, B.rows_pad, B.d_pad, B.d_pad, BN);
}

size_t tc_smem_bytes(int nt1, int nt2, int p_pad, int epi, int nstage, bool ares) {
  const size_t a_bytes = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BM * BK * 2 : 0;
  const size_t stage = ares ? static_cast<size_t>(nt1 == 3 ? 2 : 1) * BN * BK * 2 : stage_bytes(nt1);
  return nstage * stage + a_bytes + g_bufs(p_pad) * s_buf_bytes(nt2, p_pad) + smem_extra(epi);
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
    ok = encode_bf16_sw128(&maps[4], s_hi, s_rows, B.rows_pad, B.rows_pad, pp) &&
         encode_bf16_sw128(&maps[5], nt2 == 3 ? s_lo : s_hi, s_rows, B.rows_pad, B.rows_pad, pp);
    if (!ok) return ITERGP_ECUDA;
    TcArgs a{};
    a.na = A.norms;
    a.nb = B.norms;
    a.nk = B.d_pad / slice_elems(nt1);
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
    const size_t smem = tc_smem_bytes(nt1, nt2, pp, var.epi, nstage, ares);
    cudaError_t e = kind == ITERGP_RBF
                        ? launch_prec<ITERGP_RBF>(prec, nstage, ares, var.epi, tab.G, smem, stream, maps, a)
                        : launch_prec<ITERGP_MATERN32>(prec, nstage, ares, var.epi, tab.G, smem, stream, maps, a);
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

  // transposed, split S
  const int64_t n_pad = B.rows_pad;
  Scratch sbuf;
  const size_t s_elems = static_cast<size_t>(p16) * n_pad;
  ITERGP_CUDA_TRY(sbuf.alloc(ctx, s_elems * 2 * (nt2 == 3 ? 2 : 1), stream));
  __nv_bfloat16* s_hi = sbuf.as<__nv_bfloat16>();
  __nv_bfloat16* s_lo = nt2 == 3 ? s_hi + s_elems : nullptr;
  {
    dim3 grid(static_cast<unsigned>(n_pad / 32), static_cast<unsigned>(ceil_div(p16, 32)));
    if (nt2 == 3)
      prep_s_kernel<true><<<grid, dim3(32, 8), 0, stream>>>(S, ldS, B.rows, p, n_pad, p16, s_hi, s_lo, active), ::itergp::note_launch();
    else
      prep_s_kernel<false><<<grid, dim3(32, 8), 0, stream>>>(S, ldS, B.rows, p, n_pad, p16, s_hi, s_lo, active), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
  }

  CUtensorMap maps[6];
  bool ok = encode_rows(maps, A, B, nt1);
  if (!ok) return ITERGP_ECUDA;

  const int64_t row_tiles = ceil_div(A.rows, BM);
  const int64_t chunks = ceil_div(B.rows, BN);
  const int64_t units = row_tiles * chunks;
  const int64_t G = std::min<int64_t>(ctx->num_sms, units);
  const int64_t tail_rows = row_tiles - (row_tiles / G) * G;
  Scratch part;
  ITERGP_CUDA_TRY(part.alloc(ctx, sizeof(float) * 2 * G * BM * p_tile, stream));

  for (int64_t p0 = 0; p0 < p; p0 += p_tile) {
    const int pw = static_cast<int>(std::min<int64_t>(p_tile, p - p0));
    const int pp = (pw + 15) / 16 * 16;
    ok = encode_bf16_sw128(&maps[4], s_hi, p16, n_pad, n_pad, pp) &&
         encode_bf16_sw128(&maps[5], nt2 == 3 ? s_lo : s_hi, p16, n_pad, n_pad, pp);
    if (!ok) return ITERGP_ECUDA;
    TcArgs a{};   // items/item_begin/probs stay null: single-problem schedule
    a.na = A.norms;
    a.nb = B.norms;
    a.m = A.rows;
    a.row_tiles = row_tiles;
    a.chunks = static_cast<int>(chunks);
    a.nk = A.d_pad / slice_elems(nt1);
    a.p_pad = pp;
    a.p_valid = pw;
    a.s_row0 = static_cast<int>(p0);
    a.Y = Y + p0;
    a.ldY = ldY;
    a.partial = part.as<float>();
    a.kp = kp;
    a.status = ctx->status;
    a.active = active;
    a.items = nullptr;
    a.item_begin = nullptr;
    a.probs = nullptr;
    const size_t smem_t = tc_smem_bytes(nt1, nt2, pp, var.epi, nstage, ares);
    cudaError_t e = kp.kind == ITERGP_RBF
                        ? launch_prec<ITERGP_RBF>(prec, nstage, ares, var.epi, (int)G, smem_t, stream, maps, a)
                        : launch_prec<ITERGP_MATERN32>(prec, nstage, ares, var.epi, (int)G, smem_t, stream, maps, a);
    ITERGP_CUDA_TRY(e);
    if (tail_rows > 0) {
      tc_fixup_kernel<<<static_cast<unsigned>(tail_rows), 256, 0, stream>>>(
          part.as<float>(), row_tiles, G, (int)chunks, A.rows, pp, pw, Y + p0, ldY, active), ::itergp::note_launch();
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
                double* ms_out, int* best, cudaStream_t stream) {
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
    TcProb pr{Y, p, X.rows, static_cast<int32_t>(p), 0, kp, nullptr};
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
    const size_t s_elems = static_cast<size_t>(p16) * X.rows_pad;
    ITERGP_CUDA_TRY(sbuf.alloc(ctx, s_elems * 2 * 2, stream));
    s_hi = sbuf.as<__nv_bfloat16>();
    s_lo = s_hi + s_elems;
    dim3 grid(static_cast<unsigned>(X.rows_pad / 32), static_cast<unsigned>(ceil_div(p16, 32)));
    prep_s_kernel<true><<<grid, dim3(32, 8), 0, stream>>>(S, p, X.rows, p, X.rows_pad, p16, s_hi, s_lo, nullptr), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
  }
  cudaEvent_t e0, e1;
  ITERGP_CUDA_TRY(cudaEventCreate(&e0));
  ITERGP_CUDA_TRY(cudaEventCreate(&e1));
  int n = 0, rc = ITERGP_OK;
  *best = -1;
  for (int ares : {0, 1}) for (int epi : {4, 8}) {
    if (ares && (X.d_pad != BK || nt1 == 2)) continue;
    // the P tile the launchers use with this variant: the widest that fits its ring
    int p_tile = p16;
    const int min_ns = ares ? 3 : 2;
    while (p_tile > 16 && stages_that_fit(ctx, nt1, nt2, p_tile, epi, 0, ares != 0) < min_ns) p_tile -= 16;
    for (int ns : {2, 3, 4, 5}) {
      if (n >= cap) break;
      if (stages_that_fit(ctx, nt1, nt2, p_tile, epi, ns, ares != 0) != ns) continue;
      const TcVariant v{epi, ns, ares};
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
        TcVariant{epi_out[*best], bns < 0 ? -bns : bns, bns < 0 ? 1 : 0};
  }
  return ITERGP_OK;
}

}  // namespace itergp

extern "C" int itergp_tune_save(const char* path) {
  if (!path) return ITERGP_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (!f) return ITERGP_EINVAL;
  std::lock_guard<std::mutex> lk(itergp::g_tune_mu);
  std::fprintf(f, "# precision kind d_pad p_tile items epilogue_warps stages resident_a\n");
  for (const auto& kv : itergp::g_tune)
    std::fprintf(f, "%d %d %d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second.epi,
                 kv.second.nstage, kv.second.ares);
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
    int a[8];
    a[7] = -1;   // resident A: automatic when the column is absent
    const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4],
                                &a[5], &a[6], &a[7]);
    if (got < 7 || (a[5] != 4 && a[5] != 8) || a[6] < 0 || a[6] > 5 || a[7] < -1 || a[7] > 1) {
      rc = ITERGP_EINVAL;
      continue;
    }
    itergp::g_tune[std::make_tuple(a[0], a[1], a[2], a[3], a[4])] = itergp::TcVariant{a[5], a[6], a[7]};
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
