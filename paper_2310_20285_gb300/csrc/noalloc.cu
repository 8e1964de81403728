// itergp_kmatvec_noalloc: the kernel product for callers that may not allocate device
// memory.  The same kernels as itergp_kmatvec run on the same arguments; their scratch
// comes from one file-scope static device array instead of the library's pool.
#include <algorithm>
#include <mutex>

#include "internal.h"

namespace itergp {
namespace {

// Scratch for every call of the entry point, held by each GPU that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ITERGP_NOALLOC_SCRATCH_BYTES];
// Fallback status word when the caller passes no device_status.
static __device__ int g_noalloc_status;

struct NoAllocDevice {
  bool ready = false;
  DeviceContext ctx;          // properties only: no pool, no allocated status word
  char* scratch = nullptr;    // device address of g_noalloc_scratch
  int* status = nullptr;      // device address of g_noalloc_status
};

std::mutex g_mu;
NoAllocDevice g_dev[64];

// Device set-up, once per device with that device current: properties and the device
// addresses of the static arrays (host code only sees a host-side stand-in symbol).
int setup_current_device(NoAllocDevice** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ITERGP_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocDevice& d = g_dev[dev];
  if (!d.ready) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return ITERGP_ECUDA;
    void* scratch = nullptr;
    void* status = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess) return ITERGP_ECUDA;
    if (cudaGetSymbolAddress(&status, g_noalloc_status) != cudaSuccess) return ITERGP_ECUDA;
    d.ctx.device = dev;
    d.ctx.num_sms = prop.multiProcessorCount;
    d.ctx.cc_major = prop.major;
    d.ctx.cc_minor = prop.minor;
    d.ctx.smem_optin = prop.sharedMemPerBlockOptin;
    d.ctx.tcgen05 = (prop.major == 10);
    d.ctx.pool = nullptr;
    d.scratch = static_cast<char*>(scratch);
    d.status = static_cast<int*>(status);
    d.ready = true;
  }
  *out = &d;
  return ITERGP_OK;
}

// Upper bound of the scratch one call takes (rows of A and B, transposed S, partials),
// following the sizes the kernel-product launchers request.
size_t scratch_bound(const DeviceContext& ctx, int prec, int64_t m, int64_t n, int d, int64_t p,
                     bool same) {
  size_t bytes = 8 * 256;   // alignment slack for up to eight carved blocks
  bytes += align_up(rows_workspace_bytes(prec, m, d), 256);
  if (!same) bytes += align_up(rows_workspace_bytes(prec, n, d), 256);
  if (n == 0) return bytes;
  if (precision_is_tensor(prec)) {
    const int64_t p16 = (p + 15) / 16 * 16;
    const int64_t n_pad = (n + kRowTile - 1) / kRowTile * kRowTile;
    bytes += align_up(static_cast<size_t>(p16) * n_pad * 2 * (precision_splits_weights(prec) ? 2 : 1), 256) +
             sizeof(uint32_t) * p16 * 2;   // column maxima and scales of split weights
    const int64_t units = ceil_div(m, kRowTile) * ceil_div(n, kRowTile);
    const int64_t G = std::min<int64_t>(ctx.num_sms, units);
    bytes += align_up(sizeof(float) * 2 * G * kRowTile * std::min<int64_t>(p16, 128), 256);
  } else {
    const int pj = p <= 16 ? 1 : p <= 32 ? 2 : p <= 64 ? 4 : 8;
    const int64_t p_tiles = ceil_div(p, 16 * pj);
    const int64_t row_tiles = ceil_div(m, kRowTile);
    const int64_t chunks = ceil_div(n, kColTile);
    const int64_t target = 4LL * ctx.num_sms;
    int64_t splits = 1;
    if (row_tiles * p_tiles < target) splits = ceil_div(target, row_tiles * p_tiles);
    splits = std::min(splits, chunks);
    if (splits > 1) bytes += align_up(sizeof(float) * splits * m * p, 256);
  }
  return bytes;
}

struct ArenaGuard {
  explicit ArenaGuard(ScratchArena* a) { set_thread_arena(a); }
  ~ArenaGuard() { set_thread_arena(nullptr); }
};

}  // namespace
}  // namespace itergp

using namespace itergp;

extern "C" int itergp_kmatvec_noalloc(const itergp_kernel* kernel, int32_t precision,
                                      const float* A, int64_t m, const float* B, int64_t n,
                                      int64_t d, const float* S, int64_t p, float* Y,
                                      int* device_status, itergp_stream stream) {
  clear_stale_error();
  if (!kernel_ok(kernel) || !precision_ok(precision)) return ITERGP_EINVAL;
  if (m < 0 || n < 0 || p < 0 || d < 1 || d > 4096 || p > 65536) return ITERGP_EINVAL;
  // device set-up first, so that a call with m = 0 or p = 0 performs only the set-up
  NoAllocDevice* nd = nullptr;
  int rc = setup_current_device(&nd);
  if (rc != ITERGP_OK) return rc;
  if (m == 0 || p == 0) return ITERGP_OK;
  if (!Y || (n > 0 && (!A || !B || !S))) return ITERGP_EINVAL;
  if (precision_is_tensor(precision) && !nd->ctx.tcgen05) return ITERGP_EUNSUPPORTED;
  const bool same = (A == B) && (m == n);
  if (scratch_bound(nd->ctx, precision, m, n, static_cast<int>(d), p, same) > ITERGP_NOALLOC_SCRATCH_BYTES)
    return ITERGP_ESCRATCH;

  DeviceContext ctx = nd->ctx;
  ctx.status = device_status ? device_status : nd->status;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScratchArena arena;
  arena.base = nd->scratch;
  arena.size = ITERGP_NOALLOC_SCRATCH_BYTES;
  ArenaGuard guard(&arena);
  const size_t ba = rows_workspace_bytes(precision, m, static_cast<int>(d));
  const size_t bb = same ? 0 : rows_workspace_bytes(precision, n, static_cast<int>(d));
  Scratch ws;   // carved from the static array while the arena is installed
  if (ws.alloc(&ctx, ba + bb, s) != cudaSuccess) return ITERGP_ESCRATCH;
  RowOperand opA, opB;
  rc = prepare_rows(precision, A, m, static_cast<int>(d), d, ws.as<void>(), &opA, s);
  if (rc != ITERGP_OK) return rc;
  if (same) {
    opB = opA;
  } else {
    rc = prepare_rows(precision, B, n, static_cast<int>(d), d, ws.as<char>(ba), &opB, s);
    if (rc != ITERGP_OK) return rc;
  }
  rc = kmv_execute(&ctx, make_kparams(*kernel), opA, opB, S, p, p, Y, p, s, nullptr);
  return rc == ITERGP_ENOMEM ? ITERGP_ESCRATCH : rc;
}
