// Device-side IterNCGP: Newton outer loop (Alg. 1), IterGP inner loop (Alg. 2) and the
// virtual solver run with compression (Alg. 3), for the softmax likelihood with the
// pseudo-inverse W^+ of Lemma A.6.
//
// The host enqueues a fixed schedule (max_newton x (prologue + Alg. 3 + max_iters x
// iteration)) without waiting; every kernel reads device-side flags and returns at once
// when its loop has stopped (inner tolerance, eta <= 0, outer tolerance), so the whole
// fit runs without a host round trip.  Scalars (alpha, eta, norms, objective) are
// reduced in FP64 with a fixed block order, so results are deterministic.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace itergp {

constexpr int kMaxC = 64;
constexpr int kMaxBcap = 512;   // buffer columns a fit keeps at most (checked by the API)
constexpr int kRedThreads = 256;

struct FitState {
  int newton_active;   // outer loop still running
  int active;          // inner loop still running
  int B;               // committed buffer columns
  int B0;              // columns after the virtual solver run
  int pending;         // a new column waits to be committed
  int j;               // completed iterations in this Newton step
  int newton;          // current Newton step
  int newton_steps;
  int total_iters;
  int stop_reason;
  int status;
  int zdone;           // blocks of zproj_kernel finished in this iteration (the last resets it)
  double alpha, eta, coef, inv_sqrt_eta;
  double bnorm, thresh, rnorm;
  int iters[ITERGP_MAX_REPORT_STEPS];
  int stops[ITERGP_MAX_REPORT_STEPS];
  int kept[ITERGP_MAX_REPORT_STEPS];
  double objective[ITERGP_MAX_REPORT_STEPS];
  double rel_change[ITERGP_MAX_REPORT_STEPS];
};

// Per-problem device descriptor of a (batched) fit: sizes, state and every array.  Kernels
// receive the table and select their problem with blockIdx.y (per-problem kernels with
// blockIdx.x).
struct ProbDev {
  FitState* st;
  int64_t n, nc;
  int c, bcap;
  const int32_t* y;
  int lik;                           // itergp_likelihood
  float noise;                       // Gaussian noise variance
  const float* yr;                   // Gaussian real targets (n x c)
  float *f, *v, *Q;                  // model arrays
  float *S, *T, *KQ;                 // buffers [bcap][nc]
  float *u, *b, *r, *z, *gp, *ip, *s_cur, *t_cur;
  float *w, *sq, *W;
  double *Am, *Vm, *pg, *pv, *ps;
  int* bold;
};

namespace {

__device__ __forceinline__ double block_reduce_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += sh[i];
  }
  return t;  // valid in thread 0
}

// Softmax: out_n = P diag(inv_pi_n) P x_n, P = I - 11^T/C (Lemma A.6).  Likelihoods with a
// diagonal W (one latent per point: Bernoulli, Poisson; Gaussian): out = ip * x with ip
// the diagonal of W^-1 -- the same formula with the class means m1, m2 set to zero.
__device__ __forceinline__ void winv_point(const float* __restrict__ x, const float* __restrict__ ip,
                                           int C, float* __restrict__ out, bool diag = false) {
  float m1 = 0.f, m2 = 0.f;
  if (!diag) {
    for (int c = 0; c < C; ++c) m1 += x[c];
    m1 /= C;
    for (int c = 0; c < C; ++c) m2 += (x[c] - m1) * ip[c];
    m2 /= C;
  }
  for (int c = 0; c < C; ++c) out[c] = (x[c] - m1) * ip[c] - m2;
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// -------------------------------------------------------------------- Newton prologue
// For every point: pi = softmax(f_n), 1/pi = exp(lse - f), grad = e_y - pi,
// b = y_hat - m = f + W^+ grad (m = 0).  Partial sums: |b|^2, log p(y|f), v.(f - m),
// |g - g_prev|^2, |g|^2 with g = f - m; g_prev <- g.
__global__ void newton_prologue_kernel(const ProbDev* __restrict__ probs, int project) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  int* status = &P.st->status;   // errors stop this problem only
  const int64_t n = P.n;
  const int C = P.c;
  const float* __restrict__ f = P.f;
  const int32_t* __restrict__ y = P.y;
  const float* __restrict__ v = P.v;
  float* __restrict__ g_prev = P.gp;
  float* __restrict__ inv_pi = P.ip;
  float* __restrict__ b = P.b;
  double* __restrict__ part = P.ps;
  if (!st->newton_active) return;
  __shared__ double sh[32];
  double s_b2 = 0, s_ll = 0, s_vf = 0, s_dg = 0, s_g2 = 0;
  const bool diag = P.lik != ITERGP_LIK_SOFTMAX;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* fi = f + i * C;
    float* ipi = inv_pi + i * C;
    float grad[kMaxC];
    float m1 = 0.f, m2 = 0.f;
    if (P.lik == ITERGP_LIK_SOFTMAX) {
      float mx = fi[0];
      for (int c = 1; c < C; ++c) mx = fmaxf(mx, fi[c]);
      float se = 0.f;
      for (int c = 0; c < C; ++c) se += expf(fi[c] - mx);
      const float lse = mx + logf(se);
      int yi = y[i];
      if (yi < 0 || yi >= C) {
        set_status(status, ITERGP_EINVAL);
        yi = 0;
      }
      float gsum = 0.f;
      for (int c = 0; c < C; ++c) {
        const float e = expf(lse - fi[c]);
        if (!isfinite(e)) set_status(status, ITERGP_ENUMERIC);
        ipi[c] = e;
        grad[c] = (c == yi ? 1.f : 0.f) - expf(fi[c] - lse);
        gsum += grad[c];
      }
      // W^+ grad with P applied on both sides
      m1 = gsum / C;
      for (int c = 0; c < C; ++c) m2 += (grad[c] - m1) * ipi[c];
      m2 /= C;
      s_ll += static_cast<double>(fi[yi]) - lse;
    } else if (P.lik == ITERGP_LIK_BERNOULLI) {
      // pi = 1 / (1 + e^-f), grad = y - pi, W^-1 = 2 + e^f + e^-f (App. C)
      const int yi = y[i];
      if (yi != 0 && yi != 1) set_status(status, ITERGP_EINVAL);
      const float fv = fi[0];
      const float ef = expf(fv), emf = expf(-fv);
      const float w = 2.f + ef + emf;
      if (!isfinite(w)) set_status(status, ITERGP_ENUMERIC);
      ipi[0] = w;
      grad[0] = static_cast<float>(yi == 1) - 1.f / (1.f + emf);
      s_ll += static_cast<double>(yi == 1 ? fv : 0.f) - (fmaxf(fv, 0.f) + log1pf(expf(-fabsf(fv))));
    } else if (P.lik == ITERGP_LIK_POISSON) {
      // rate e^f, grad = y - e^f, W^-1 = e^-f (App. A)
      const int yi = y[i];
      if (yi < 0) set_status(status, ITERGP_EINVAL);
      const float fv = fi[0];
      const float ef = expf(fv), emf = expf(-fv);
      if (!isfinite(ef) || !isfinite(emf)) set_status(status, ITERGP_ENUMERIC);
      ipi[0] = emf;
      grad[0] = static_cast<float>(yi) - ef;
      s_ll += static_cast<double>(yi) * fv - ef;
    } else {
      // Gaussian: grad = (y - f) / sigma^2, W^-1 = sigma^2 I (Thm. A.2)
      for (int c = 0; c < C; ++c) {
        const float rr = P.yr[i * C + c] - fi[c];
        ipi[c] = P.noise;
        grad[c] = rr / P.noise;
        s_ll += -0.5 * static_cast<double>(rr) * rr / P.noise;
      }
    }
    float* bi = b + i * C;
    float* gp = g_prev + i * C;
    const float* vi = v + i * C;
    // With residual (CG) actions b lies in the class-contrast subspace range(I kron P) in
    // exact arithmetic (f = K v with v there, W^+ maps into it); removing the per-point
    // mean keeps rounding out of the class-sum directions, where K_hat reduces to the
    // near-singular k(X, X).  Unit-vector actions leave that subspace: no projection.
    float bmean = 0.f;
    if (project && !diag) {
      for (int c = 0; c < C; ++c) bmean += fi[c] + ((grad[c] - m1) * ipi[c] - m2);
      bmean /= C;
    }
    for (int c = 0; c < C; ++c) {
      const float bc = fi[c] + ((grad[c] - m1) * ipi[c] - m2) - bmean;
      bi[c] = bc;
      s_b2 += static_cast<double>(bc) * bc;
      s_vf += static_cast<double>(vi[c]) * fi[c];
      const double dg = static_cast<double>(fi[c]) - gp[c];
      s_dg += dg * dg;
      s_g2 += static_cast<double>(fi[c]) * fi[c];
      gp[c] = fi[c];
    }
  }
  double r;
  r = block_reduce_sum(s_b2, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 0] = r;
  r = block_reduce_sum(s_ll, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 1] = r;
  r = block_reduce_sum(s_vf, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 2] = r;
  r = block_reduce_sum(s_dg, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 3] = r;
  r = block_reduce_sum(s_g2, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 4] = r;
}

__global__ void newton_finalize_kernel(const ProbDev* __restrict__ probs, int nblk, int step,
                                       double tol_newton, double tol_abs, double tol_rel,
                                       int recycle, double floor_rel) {
  const ProbDev& P = probs[blockIdx.x];
  FitState* st = P.st;
  const double* __restrict__ part = P.ps;
  if (threadIdx.x != 0 || !st->newton_active) return;
  if (st->status != ITERGP_OK) {
    // a label out of range or a non-finite 1/pi in the prologue: this problem stops here
    // with f of the last completed step; the others continue
    st->newton_active = 0;
    st->active = 0;
    return;
  }
  double s[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblk; ++b)
    for (int k = 0; k < 5; ++k) s[k] += part[b * 5 + k];
  st->newton = step;
  if (step < ITERGP_MAX_REPORT_STEPS) st->objective[step] = s[1] - 0.5 * s[2];
  if (step >= 1) {
    const double rc = s[4] > 0 ? sqrt(s[3]) / sqrt(s[4]) : 0.0;
    if (step < ITERGP_MAX_REPORT_STEPS) st->rel_change[step] = rc;
    if (tol_newton > 0 && rc <= tol_newton) {
      st->newton_active = 0;
      st->active = 0;
      return;
    }
  }
  st->bnorm = sqrt(s[0]);
  // App. B.2: |r| < max(tol_abs, tol_rel |b|); with BF16 products (2^-9 relative) the
  // solve also stops at their rounding level floor_rel |b|, below which the residual
  // actions are rounding noise
  st->thresh = fmax(fmax(tol_abs, tol_rel * st->bnorm), floor_rel * st->bnorm);
  st->j = 0;
  st->pending = 0;
  st->active = 1;
  if (!recycle) st->B = 0;
  st->B0 = st->B;
}

// -------------------------------------------------------------------- Alg. 3 pieces
// Z = T + W^+ S for the B committed columns (written into the Q buffer as scratch).
__global__ void vsr_z_kernel(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const int64_t n = P.n, nc = P.nc;
  const int C = P.c;
  const float* __restrict__ S = P.S;
  const float* __restrict__ T = P.T;
  const float* __restrict__ inv_pi = P.ip;
  float* __restrict__ Z = P.Q;
  if (!st->newton_active) return;
  const int B = st->B;
  const int64_t total = static_cast<int64_t>(B) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t col = e / n, i = e % n;
    const float* s = S + col * nc + i * C;
    float w[kMaxC];
    winv_point(s, inv_pi + i * C, C, w, P.lik != ITERGP_LIK_SOFTMAX);
    const float* t = T + col * nc + i * C;
    float* z = Z + col * nc + i * C;
    for (int c = 0; c < C; ++c) z[c] = t[c] + w[c];
  }
}

// Gram partials G[split][a][b] = sum_{e in split} X[a][e] Y[b][e], a, b < B (32 x 32
// tiles, FP32 products summed in FP64).
constexpr int kGT = 32;
__global__ void gram_partial_kernel(const ProbDev* __restrict__ probs, int tiles) {
  const ProbDev& P = probs[blockIdx.z];
  const FitState* st = P.st;
  const float* __restrict__ X = P.S;
  const float* __restrict__ Y = P.Q;
  const int64_t nc = P.nc;
  const int bcap = P.bcap;
  double* __restrict__ part = P.pg;
  if (!st->newton_active) return;
  const int B = st->B;
  const int a0 = (blockIdx.x / tiles) * kGT, b0 = (blockIdx.x % tiles) * kGT;
  if (a0 >= B || b0 >= B) return;
  const int64_t per_split = (nc + gridDim.y - 1) / gridDim.y;
  const int64_t e0 = static_cast<int64_t>(blockIdx.y) * per_split;
  const int64_t e1 = std::min<int64_t>(e0 + per_split, nc);
  __shared__ float xs[64][kGT + 1], ys[64][kGT + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;   // 2 x 2 outputs each
  double acc[2][2] = {{0, 0}, {0, 0}};
  for (int64_t base = e0; base < e1; base += 64) {
    for (int k = tid; k < 64 * kGT; k += blockDim.x) {
      const int col = k / 64, ee = k % 64;
      const int64_t e = base + ee;
      xs[ee][col] = (a0 + col < B && e < e1) ? X[(a0 + col) * nc + e] : 0.f;
      ys[ee][col] = (b0 + col < B && e < e1) ? Y[(b0 + col) * nc + e] : 0.f;
    }
    __syncthreads();
    float loc[2][2] = {{0, 0}, {0, 0}};
#pragma unroll 8
    for (int ee = 0; ee < 64; ++ee) {
      const float x0 = xs[ee][2 * ty], x1 = xs[ee][2 * ty + 1];
      const float y0 = ys[ee][2 * tx], y1 = ys[ee][2 * tx + 1];
      loc[0][0] = fmaf(x0, y0, loc[0][0]);
      loc[0][1] = fmaf(x0, y1, loc[0][1]);
      loc[1][0] = fmaf(x1, y0, loc[1][0]);
      loc[1][1] = fmaf(x1, y1, loc[1][1]);
    }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) acc[i][j] += loc[i][j];
    __syncthreads();
  }
  double* out = part + static_cast<int64_t>(blockIdx.y) * bcap * bcap;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + 2 * ty + i, bb = b0 + 2 * tx + j;
      if (a < B && bb < B) out[a * bcap + bb] = acc[i][j];
    }
}

// ---------------------------------------------------------------- FP64 Jacobi (1 CTA)
// Cyclic Jacobi with round-robin (tournament) pairing: in each round the m/2 disjoint pairs
// (m = n rounded up to even; index n is a dummy) are rotated simultaneously.  A rotation
// J_k acts on the index pair (lo_k, hi_k); the pairs partition the indices, so A' = J^T A J
// splits into independent 2 x 2 blocks A[{lo_a, hi_a}, {lo_b, hi_b}] <- J_a^T X J_b.  Each
// thread updates whole blocks of the upper block triangle and mirrors them (A stays exactly
// symmetric), half the FP64 work of separate column and row passes; the rotated pairs'
// diagonal entries take the usual t-form (a_pp - t a_pq, a_qq + t a_pq) and their
// off-diagonal entry is set to 0.  A rotation whose off-diagonal entry is below 1e-18 of
// the geometric mean of its diagonal is replaced by setting that entry to 0.  V accumulates
// the rotations (A_in = V diag V^T).  The SM's FP64 rate bounds the routine (one SM has
// about 1.7 FP64 FMA per cycle here).
// Rotation (c, s) = (1, t) / sqrt(1 + t^2) that zeroes a_pq, t the smaller root of
// a_pq t^2 + (a_qq - a_pp) t - a_pq = 0.  The operands are scaled by a power of two into
// [-1, 1]; t is found in FP32 and polished by one FP64 Newton step on the quadratic, and
// 1 / sqrt(1 + t^2) by two FP64 Newton steps from an FP32 seed: a few FP64 operations in
// place of the FP64 divisions and square roots (each a long sequence on this GPU's small
// FP64 unit), with t and c accurate to FP64 rounding.
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double* c_out, double* s_out) {
  const double mx = fmax(fmax(fabs(app), fabs(aqq)), fabs(apq));
  const int ex = static_cast<int>((__double_as_longlong(mx) >> 52) & 0x7FF) - 1023;   // mx = m 2^ex, m in [1, 2)
  const double sc = __longlong_as_double(static_cast<long long>(1023 - ex - 1) << 52);   // 2^-(ex + 1)
  const double a = apq * sc, d = (aqq - app) * sc;   // |a| < 1, |d| < 2
  const float a32 = static_cast<float>(a), d32 = static_cast<float>(d);
  float t32;
  if (a32 == 0.f) {
    t32 = 0.f;
  } else {
    const float th = d32 / (2.f * a32);
    t32 = fabsf(th) > 1e18f ? 0.5f / th : copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
  }
  double t = t32;
  const double q = fma(a * t, t, fma(d, t, -a));        // a t^2 + d t - a
  const double qp = fma(2.0 * a, t, d);                 // its derivative (|qp| >= 2|a| at the root)
  t -= q * static_cast<double>(1.f / static_cast<float>(qp));
  const double y = fma(t, t, 1.0);                      // in [1, 2]
  double r = static_cast<double>(rsqrtf(static_cast<float>(y)));
  r = r * fma(-0.5 * y, r * r, 1.5);
  r = r * fma(-0.5 * y, r * r, 1.5);
  *c_out = r;
  *s_out = t * r;
}

__device__ __forceinline__ void rr_pair(int k, int r, int m, int* lo, int* hi) {
  const int i0 = k, i1 = m - 1 - k;
  const int p = (i0 == 0) ? 0 : ((i0 - 1 + r) % (m - 1)) + 1;
  const int q = ((i1 - 1 + r) % (m - 1)) + 1;
  *lo = p < q ? p : q;
  *hi = p < q ? q : p;
}

// CL > 1: the eigenproblem is shared by the CL CTAs of a cluster (one SM each), so the
// rounds' FP64 updates run on several SMs' FP64 units.  The rank-0 CTA holds the rotation
// arrays (cs, sn, plo, phi: addresses in its shared memory), computes the norms, the
// stopping test and each round's rotations exactly as one CTA would, and applies the
// round's 2 x 2 block updates of A (about half the round's FP64 work) on its own memory;
// the V rotations (the other half) are split over the threads of the other CTAs, which
// reach V and the rotations through distributed shared memory (A and V may also be
// global).  Remote accesses cost far more than local ones, so A stays with rank 0.  Cluster barriers stand where one
// CTA has block barriers; every thread of every CTA passes the same sequence of them, and
// each element is still computed by one thread from the same operands, so the result is
// bitwise the one-CTA result.  The caller maps the pointers of a rank > 0 CTA to rank 0.
template <int CL>
__device__ void jacobi_eig(double* A, double* V, int n, int ld, double* cs, double* sn, int* plo, int* phi,
                           double* sh) {
  namespace cg = cooperative_groups;
  const int rank = CL > 1 ? static_cast<int>(cg::this_cluster().block_rank()) : 0;
  const bool lead = rank == 0;
  const int tid = threadIdx.x, nt = blockDim.x;
  // the V rotations' threads: those of ranks 1 .. CL - 1 (one CTA: all of its threads)
  const int vtid = CL > 1 ? (rank - 1) * nt + tid : tid, vnt = CL > 1 ? (CL - 1) * nt : nt;
  auto team_sync = [&]() {
    if constexpr (CL > 1) cg::this_cluster().sync(); else __syncthreads();
  };
  const int m = (n + 1) / 2 * 2;   // even number of players (index n is a dummy if n odd)
  const int h = m / 2;
  __shared__ double fro_s, off_s;
  __shared__ int stop_s;
  int* stop = &stop_s;
  if constexpr (CL > 1) stop = cg::this_cluster().map_shared_rank(&stop_s, 0);
  double tol2 = 0.0;
  if (lead) {
    for (int e = tid; e < n * n; e += nt) V[(e / n) * ld + e % n] = (e / n == e % n) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      const double a = A[(e / n) * ld + e % n];
      fro += a * a;
    }
    fro = block_reduce_sum(fro, sh);
    if (tid == 0) fro_s = fro;
    __syncthreads();
    tol2 = fro_s * 1e-30;
  }
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (lead) {
      double off = 0.0;
      for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        if (i < j) {
          const double a = A[i * ld + j];
          off += 2.0 * a * a;
        }
      }
      off = block_reduce_sum(off, sh);
      if (tid == 0) {
        off_s = off;
        stop_s = (off <= tol2 || off == 0.0) ? 1 : 0;
      }
    }
    team_sync();
    if (*stop) break;
    for (int r = 0; r < m - 1; ++r) {
      // the round's pairs and rotations; sn = 0 marks a pair left as it is
      for (int k = tid; lead && k < h; k += nt) {
        int lo, hi;
        rr_pair(k, r, m, &lo, &hi);
        plo[k] = lo;
        phi[k] = hi;
        double c = 1.0, s = 0.0;
        if (hi < n) {
          const double apq = A[lo * ld + hi];
          if (apq != 0.0) {
            const double app = A[lo * ld + lo], aqq = A[hi * ld + hi];
            if (apq * apq <= 1e-36 * fabs(app * aqq)) {
              A[lo * ld + hi] = 0.0;   // negligible: this pair's block is this thread's alone
              A[hi * ld + lo] = 0.0;
            } else {
              jacobi_rotation(app, aqq, apq, &c, &s);
            }
          }
        }
        cs[k] = c;
        sn[k] = s;
      }
      team_sync();
      // A <- J^T A J by 2 x 2 blocks (a <= b, enumerated densely: e = b (b + 1) / 2 + a),
      // mirrored; V <- V J (rows x pairs)
      for (int e = tid; lead && e < h * (h + 1) / 2; e += nt) {
        int b = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) - 1.f) * 0.5f);
        if ((b + 1) * (b + 2) / 2 <= e) ++b;
        if (b * (b + 1) / 2 > e) --b;
        const int a = e - b * (b + 1) / 2;
        const double s1 = sn[a], s2 = sn[b];
        if (s1 == 0.0 && s2 == 0.0) continue;
        const double c1 = cs[a], c2 = cs[b];
        const int p1 = plo[a], q1 = phi[a], p2 = plo[b], q2 = phi[b];
        const bool v1 = q1 < n, v2 = q2 < n;   // the dummy index has no row or column
        if (a == b) {   // the rotated pair itself: t-form of the new diagonal, zero off-diagonal
          const double apq = A[p1 * ld + q1];
          const double t = s1 / c1;
          A[p1 * ld + p1] -= t * apq;
          A[q1 * ld + q1] += t * apq;
          A[p1 * ld + q1] = 0.0;
          A[q1 * ld + p1] = 0.0;
          continue;
        }
        const double x00 = A[p1 * ld + p2];
        const double x01 = v2 ? A[p1 * ld + q2] : 0.0;
        const double x10 = v1 ? A[q1 * ld + p2] : 0.0;
        const double x11 = (v1 && v2) ? A[q1 * ld + q2] : 0.0;
        // X J_2: columns (p2, q2)
        const double y00 = c2 * x00 - s2 * x01, y01 = s2 * x00 + c2 * x01;
        const double y10 = c2 * x10 - s2 * x11, y11 = s2 * x10 + c2 * x11;
        // J_1^T (X J_2): rows (p1, q1)
        const double z00 = c1 * y00 - s1 * y10, z01 = c1 * y01 - s1 * y11;
        const double z10 = s1 * y00 + c1 * y10, z11 = s1 * y01 + c1 * y11;
        A[p1 * ld + p2] = z00;
        A[p2 * ld + p1] = z00;
        if (v2) {
          A[p1 * ld + q2] = z01;
          A[q2 * ld + p1] = z01;
        }
        if (v1) {
          A[q1 * ld + p2] = z10;
          A[p2 * ld + q1] = z10;
        }
        if (v1 && v2) {
          A[q1 * ld + q2] = z11;
          A[q2 * ld + q1] = z11;
        }
      }
      for (int e = vtid; (CL == 1 || !lead) && e < n * h; e += vnt) {
        const int row = e / h, k = e % h;
        const double s = sn[k];
        if (s == 0.0) continue;
        const int lo = plo[k], hi = phi[k];
        const double c = cs[k];
        const double x = V[row * ld + lo], y = V[row * ld + hi];
        V[row * ld + lo] = c * x - s * y;
        V[row * ld + hi] = s * x + c * y;
      }
      team_sync();
    }
  }
  // the other CTAs have read the stop flag and made their last accesses to rank 0's memory
  if constexpr (CL > 1) team_sync();
}

// Sort eigenpairs descending (ties by index): order[k] = index of the k-th largest.
__device__ void eig_order(const double* A, int n, int ld, int* order) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double li = A[i * ld + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[j * ld + j];
      if (lj > li || (lj == li && j < i)) ++rank;
    }
    order[rank] = i;
  }
  __syncthreads();
}

// Shared memory of the eigensolver kernels: rotations, pairs, order (b = largest buffer);
// with ab_smem, also A and V (FP64) of a b x b problem.
__host__ __device__ inline size_t eig_smem_base(int b) {
  return (sizeof(double) * (2 * (b / 2 + 1) + 32) + sizeof(int) * (3 * (b + 1)) + 15) / 16 * 16;
}
inline size_t eig_smem_bytes(int b, bool ab_smem = false) {
  return eig_smem_base(b) + (ab_smem ? static_cast<size_t>(b) * b * 2 * sizeof(double) : 0);
}
// Buffers up to this size keep A and V in shared memory (200 KB at 112).
constexpr int kEigSmemMax = 112;
// CTAs per eigenproblem when a few problems leave SMs idle (portable cluster size).
constexpr int kEigCluster = 8;

// Launch as clusters of cl CTAs, `groups` clusters.
template <typename... P, typename... Args>
cudaError_t launch_clustered(void (*fn)(P...), int groups, int cl, int threads, size_t smem, cudaStream_t st,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(groups * cl));
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = static_cast<unsigned>(cl);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}

// True when clusters of kEigCluster CTAs of fn (threads, smem) can be resident; sets fn's
// dynamic shared-memory limit to smem.
template <typename... P>
bool eig_cluster_fits(void (*fn)(P...), int threads, size_t smem) {
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kEigCluster);
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kEigCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

// The fit's eigen step: whether clusters fit with the largest layout (A and V of a
// kEigSmemMax buffer in shared memory), asked once per device.
bool vsr_eig_cluster_ok(const DeviceContext* ctx);

// Sum Gram partials, symmetrise, eigendecompose, drop lambda <= 1e-12 lambda_max, keep
// the R largest (Alg. 3), write rotation W[b][k] = U[b][k] lambda_k^-1/2 (FP32) and
// sqrt(lambda_k); set B = B0 = kept columns.  ab_smem: the launch gave room for A and V in
// shared memory.  (V stays FP64: a kept eigenvalue may be 1e-12 of the largest, and the
// rotation W = U lambda^-1/2 magnifies an eigenvector's error by up to lambda_max /
// lambda_k in the K-hat inner products of the compressed buffer.)
// CL > 1: launched as clusters of CL CTAs per problem (A and V in shared memory only); the
// rank-0 CTA does all but the eigendecomposition's rounds, which the cluster shares.
template <int CL>
__global__ void vsr_eig_kernel(const ProbDev* __restrict__ probs, int splits, int rank, int step, int ab_smem) {
  namespace cg = cooperative_groups;
  const ProbDev& P = probs[blockIdx.x / CL];
  const bool lead = CL == 1 || cg::this_cluster().block_rank() == 0;
  FitState* st = P.st;
  const double* __restrict__ part = P.pg;
  const int bcap = P.bcap;
  double* __restrict__ Amat = P.Am;
  double* __restrict__ Vmat = P.Vm;
  float* __restrict__ W = P.W;
  float* __restrict__ sq = P.sq;
  // every CTA of a cluster reads the same flags: rank 0 writes st->B only after the
  // eigendecomposition's first cluster barrier, which the others reach after these reads
  if (!st->newton_active) return;
  const int B = st->B;
  if (B == 0) {
    if (lead && threadIdx.x == 0 && step < ITERGP_MAX_REPORT_STEPS) st->kept[step] = 0;
    return;
  }
  extern __shared__ __align__(16) uint8_t esh[];
  double* cs = reinterpret_cast<double*>(esh);   // bcap/2 + 1
  double* sn = cs + bcap / 2 + 1;                // bcap/2 + 1
  double* red = sn + bcap / 2 + 1;               // 32
  int* plo = reinterpret_cast<int*>(red + 32);
  int* phi = plo + bcap + 1;
  int* order = phi + bcap + 1;
  double* A = Amat;
  double* V = Vmat;
  int ld = bcap;
  if (ab_smem) {   // B <= bcap <= kEigSmemMax: compact B x B copies in shared memory
    A = reinterpret_cast<double*>(esh + eig_smem_base(bcap));
    V = A + B * B;
    ld = B;
  }
  if constexpr (CL > 1) {
    if (!lead) {   // the cluster's other CTAs work on rank 0's arrays, then leave
      auto cl = cg::this_cluster();
      double* A0 = ab_smem ? cl.map_shared_rank(A, 0) : A;
      double* V0 = ab_smem ? cl.map_shared_rank(V, 0) : V;
      jacobi_eig<CL>(A0, V0, B, ld, cl.map_shared_rank(cs, 0), cl.map_shared_rank(sn, 0),
                     cl.map_shared_rank(plo, 0), cl.map_shared_rank(phi, 0), red);
      return;
    }
  }
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    const int a = e / B, b = e % B;
    double s1 = 0.0, s2 = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
      s1 += part[static_cast<int64_t>(sp) * bcap * bcap + a * bcap + b];
      s2 += part[static_cast<int64_t>(sp) * bcap * bcap + b * bcap + a];
    }
    A[a * ld + b] = 0.5 * (s1 + s2);
  }
  __syncthreads();
  jacobi_eig<CL>(A, V, B, ld, cs, sn, plo, phi, red);
  eig_order(A, B, ld, order);
  __shared__ int keep_s;
  if (threadIdx.x == 0) {
    const double lmax = A[order[0] * ld + order[0]];
    int keep = 0;
    while (keep < B && A[order[keep] * ld + order[keep]] > 1e-12 * fmax(lmax, 0.0)) ++keep;
    if (rank >= 0 && keep > rank) keep = rank;
    keep_s = keep;
    st->B = keep;
    st->B0 = keep;
    if (step < ITERGP_MAX_REPORT_STEPS) st->kept[step] = keep;
  }
  __syncthreads();
  const int keep = keep_s;
  for (int e = threadIdx.x; e < B * keep; e += blockDim.x) {
    const int b = e / keep, k = e % keep;
    const double lam = A[order[k] * ld + order[k]];
    W[b * bcap + k] = static_cast<float>(V[b * ld + order[k]] / sqrt(lam));
  }
  for (int k = threadIdx.x; k < keep; k += blockDim.x)
    sq[k] = static_cast<float>(sqrt(A[order[k] * ld + order[k]]));
}

bool vsr_eig_cluster_ok(const DeviceContext* ctx) {
  static std::mutex mu;
  static signed char known[64] = {};   // 0 not asked, 1 yes, -1 no
  const int dev = ctx->device;
  if (dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(mu);
  if (known[dev] == 0)
    known[dev] = eig_cluster_fits(vsr_eig_kernel<kEigCluster>, 512, eig_smem_bytes(kEigSmemMax, true)) ? 1 : -1;
  return known[dev] > 0;
}

// Q[:, k] = sum_b S[:, b] W[b][k];  KQ[:, k] = sum_b T[:, b] W[b][k]   (k < B_new, b < B_old)
// W is read with warp-uniform addresses (broadcast loads through L1).
__global__ void vsr_rotate_kernel(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const int* __restrict__ bold_ptr = P.bold;
  const int64_t nc = P.nc;
  const int bcap = P.bcap;
  const float* __restrict__ S = P.S;
  const float* __restrict__ T = P.T;
  const float* __restrict__ W = P.W;
  float* __restrict__ Q = P.Q;
  float* __restrict__ KQ = P.KQ;
  if (!st->newton_active) return;
  const int Bn = st->B, Bo = *bold_ptr;
  if (Bn == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nc;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int k0 = 0; k0 < Bn; k0 += 16) {
      float aq[16], ak[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) aq[k] = ak[k] = 0.f;
      for (int b = 0; b < Bo; ++b) {
        const float sv = S[b * nc + e], tv = T[b * nc + e];
        const float* wr = W + static_cast<int64_t>(b) * bcap + k0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          if (k0 + k < Bn) {
            const float w = __ldg(wr + k);
            aq[k] = fmaf(sv, w, aq[k]);
            ak[k] = fmaf(tv, w, ak[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k0 + k < Bn) {
          Q[(k0 + k) * nc + e] = aq[k];
          KQ[(k0 + k) * nc + e] = ak[k];
        }
    }
  }
}

// S[:, k] = Q[:, k] sqrt(lambda_k), T[:, k] = KQ[:, k] sqrt(lambda_k)  (= S U, T U)
__global__ void vsr_rescale_kernel(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const int64_t nc = P.nc;
  const float* __restrict__ sq = P.sq;
  const float* __restrict__ Q = P.Q;
  const float* __restrict__ KQ = P.KQ;
  float* __restrict__ S = P.S;
  float* __restrict__ T = P.T;
  if (!st->newton_active) return;
  const int Bn = st->B;
  const int64_t total = static_cast<int64_t>(Bn) * nc;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float w = sq[e / nc];
    S[e] = Q[e] * w;
    T[e] = KQ[e] * w;
  }
}

__global__ void copy_int_kernel(const ProbDev* __restrict__ probs) {
  if (threadIdx.x == 0) *probs[blockIdx.x].bold = probs[blockIdx.x].st->B;
}

// -------------------------------------------------------------------- projections
// Alg. 3's projection Q0^T b: part[blk][k] = sum_{e in blk} Q[k][e] b[e] for k < B (warp per
// column; the inner iteration's Q^T z is formed by zproj_kernel)
__global__ void proj_partial_kernel(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const float* __restrict__ Q = P.Q;
  const float* __restrict__ x = P.b;
  const int64_t nc = P.nc;
  const int bcap = P.bcap;
  double* __restrict__ part = P.pv;
  if (!st->newton_active) return;
  const int B = st->B;
  const int64_t per = (nc + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * per, e1 = std::min<int64_t>(e0 + per, nc);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int k = w; k < B; k += nw) {
    double acc = 0.0;
    const float* q = Q + static_cast<int64_t>(k) * nc;
    for (int64_t e = e0 + l; e < e1; e += 32) acc += static_cast<double>(q[e]) * x[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (l == 0) part[static_cast<int64_t>(blockIdx.x) * bcap + k] = acc;
  }
}

__global__ void proj_finalize_kernel(const ProbDev* __restrict__ probs, int nblk) {
  const ProbDev& P = probs[blockIdx.x];
  const FitState* st = P.st;
  const double* __restrict__ part = P.pv;
  const int bcap = P.bcap;
  float* __restrict__ w = P.w;
  if (!st->newton_active) return;
  const int B = st->B;
  for (int k = threadIdx.x; k < B; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[static_cast<int64_t>(b) * bcap + k];
    w[k] = static_cast<float>(s);
  }
}

// v = Q w, u = KQ w over the B0 recycled columns (v0 = C0 b, K v0)
__global__ void combine_kernel(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const float* __restrict__ Q = P.Q;
  const float* __restrict__ KQ = P.KQ;
  const float* __restrict__ w = P.w;
  const int64_t nc = P.nc;
  float* __restrict__ v = P.v;
  float* __restrict__ u = P.u;
  if (!st->newton_active) return;
  const int B = st->B;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nc;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float av = 0.f, au = 0.f;
    for (int k = 0; k < B; ++k) {
      av = fmaf(Q[k * nc + e], w[k], av);
      au = fmaf(KQ[k * nc + e], w[k], au);
    }
    v[e] = av;
    u[e] = au;
  }
}

// -------------------------------------------------------------------- inner iteration
// r = P(b - u - W^+ v)   (u = K v, P removes the per-point class mean); partial |r|^2.
// The residual is the small difference of large terms (u carries K's largest eigenvalues),
// so it is formed in FP64 arithmetic from the FP32 operands and rounded once; it is the
// quantity the inner convergence test reduces.
// The same pass writes the iteration's action (Alg. 2): s = r under the CG policy, or the
// unit vector e_{B0 + j}, into the staging vector and the next S column (B + pending;
// committed only if the solve goes on, see resid_finalize_kernel).
__global__ void resid_kernel(const ProbDev* __restrict__ probs, int project, int policy) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const int64_t n = P.n;
  const int C = P.c;
  const float* __restrict__ b = P.b;
  const float* __restrict__ u = P.u;
  const float* __restrict__ v = P.v;
  const float* __restrict__ inv_pi = P.ip;
  float* __restrict__ r = P.r;
  double* __restrict__ part = P.ps;
  if (!st->newton_active || !st->active) return;
  const int64_t nc = n * C;
  const int bnext = st->B + st->pending;
  float* __restrict__ s_cur = P.s_cur;
  float* __restrict__ scol = bnext < P.bcap ? P.S + static_cast<int64_t>(bnext) * nc : nullptr;
  const int64_t unit_idx = static_cast<int64_t>(st->B0) + st->j;
  const bool diag = P.lik != ITERGP_LIK_SOFTMAX;   // W^-1 diagonal: no class means
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* vi = v + i * C;
    const float* ipi = inv_pi + i * C;
    double m1 = 0.0, m2 = 0.0;
    if (!diag) {
      for (int c = 0; c < C; ++c) m1 += vi[c];
      m1 /= C;
      for (int c = 0; c < C; ++c) m2 += (vi[c] - m1) * static_cast<double>(ipi[c]);
      m2 /= C;
    }
    double rm = 0.0;
    if (project && !diag) {
      for (int c = 0; c < C; ++c)
        rm += static_cast<double>(b[i * C + c]) - u[i * C + c] - ((vi[c] - m1) * ipi[c] - m2);
      rm /= C;
    }
    for (int c = 0; c < C; ++c) {
      const double rv = static_cast<double>(b[i * C + c]) - u[i * C + c] - ((vi[c] - m1) * ipi[c] - m2) - rm;
      const float rf = static_cast<float>(rv);
      r[i * C + c] = rf;
      acc += rv * rv;
      const float sv = policy == ITERGP_POLICY_CG ? rf : (i * C + c == unit_idx ? 1.f : 0.f);
      s_cur[i * C + c] = sv;
      if (scol) scol[i * C + c] = sv;
    }
  }
  acc = block_reduce_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// commit the pending column; |r|; inner stopping test (App. B.2); alpha
__global__ void resid_finalize_kernel(const ProbDev* __restrict__ probs, int nblk, int policy) {
  const ProbDev& P = probs[blockIdx.x];
  FitState* st = P.st;
  const double* __restrict__ part = P.ps;
  const float* __restrict__ r = P.r;
  const int64_t nc = P.nc;
  if (threadIdx.x != 0 || !st->newton_active || !st->active) return;
  if (st->pending) {
    st->B += 1;
    st->pending = 0;
  }
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b];
  st->rnorm = sqrt(s);
  if (st->rnorm < st->thresh) {
    st->active = 0;
    st->stop_reason = ITERGP_STOP_TOL;
    return;
  }
  if (policy == ITERGP_POLICY_CG) {
    st->alpha = s;   // s_j^T r_{j-1} with s_j = r_{j-1}
  } else {
    const int64_t idx = static_cast<int64_t>(st->B0) + st->j;   // e_{B0 + j}, 0-based
    if (idx >= nc) {
      st->active = 0;
      st->stop_reason = ITERGP_STOP_MAXITER;
      return;
    }
    st->alpha = r[idx];
  }
}

// T[:, B] = t; z = t + W^+ s (Lemma A.6) over a block's segment of whole points, then the
// block's partial sums of Q_k^T z over the same segment (k < B), as proj_partial_kernel
// does for Alg. 3's projection.  The last block to finish adds the partial sums (FP64, in a
// fixed order) into w = Q^T z, rounded once.
__global__ void zproj_kernel(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  FitState* st = P.st;
  const int64_t n = P.n;
  const int C = P.c;
  const float* __restrict__ s_cur = P.s_cur;
  const float* __restrict__ t_cur = P.t_cur;
  const float* __restrict__ inv_pi = P.ip;
  const float* __restrict__ Q = P.Q;
  float* __restrict__ z = P.z;
  float* __restrict__ T = P.T;
  double* __restrict__ part = P.pv;
  if (!st->newton_active || !st->active) return;
  const int64_t nc = n * C;
  const int B = st->B;
  const int bcap = P.bcap;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;   // points per block
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * per, i1 = std::min<int64_t>(i0 + per, n);
  float* tcol = T + static_cast<int64_t>(B) * nc;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    float w[kMaxC];
    winv_point(s_cur + i * C, inv_pi + i * C, C, w, P.lik != ITERGP_LIK_SOFTMAX);
    for (int c = 0; c < C; ++c) {
      const float tv = t_cur[i * C + c];
      tcol[i * C + c] = tv;
      z[i * C + c] = tv + w[c];
    }
  }
  __syncthreads();   // the block reads back the z it wrote
  const int64_t e0 = std::min(i0, n) * C, e1 = i1 * C;
  const int wp = threadIdx.x / 32, l = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int k = wp; k < B; k += nw) {
    double acc = 0.0;
    const float* q = Q + static_cast<int64_t>(k) * nc;
    for (int64_t e = e0 + l; e < e1; e += 32) acc += static_cast<double>(q[e]) * z[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (l == 0) part[static_cast<int64_t>(blockIdx.x) * bcap + k] = acc;
  }
  __shared__ int last_s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_s = atomicAdd(&st->zdone, 1) == static_cast<int>(gridDim.x) - 1;
  __syncthreads();
  if (last_s) {   // one warp per column k: lanes take strided blocks, then a fixed shuffle tree
    __threadfence();
    for (int k = wp; k < B; k += nw) {
      double sum = 0.0;
      for (int b = l; b < static_cast<int>(gridDim.x); b += 32) sum += __ldcg(part + static_cast<int64_t>(b) * bcap + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (l == 0) P.w[k] = static_cast<float>(sum);
    }
    if (threadIdx.x == 0) st->zdone = 0;
  }
}

// d = s - Q w -> Q[:, B] (unnormalised); K d = t - KQ w -> KQ[:, B]; partial eta = z.d
// (w = Q^T z from zproj_kernel).
__global__ void direction_kernel(const ProbDev* __restrict__ probs, int track_kd) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const int64_t nc = P.nc;
  const float* __restrict__ s_cur = P.s_cur;
  const float* __restrict__ t_cur = P.t_cur;
  const float* __restrict__ z = P.z;
  float* __restrict__ Q = P.Q;
  float* __restrict__ KQ = P.KQ;
  double* __restrict__ part = P.ps;
  if (!st->newton_active || !st->active) return;
  __shared__ double sh[32];
  __shared__ float w[kMaxBcap];
  const int B = st->B;
  for (int k = threadIdx.x; k < B; k += blockDim.x) w[k] = P.w[k];
  __syncthreads();
  float* qcol = Q + static_cast<int64_t>(B) * nc;
  float* kcol = KQ + static_cast<int64_t>(B) * nc;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nc;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float d = s_cur[e], kd = t_cur[e];
    int k = 0;
    // eight columns' loads in flight at a time (the loop is bound by load latency)
    for (; k + 8 <= B; k += 8) {
      float qv[8], kv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        qv[i] = Q[(k + i) * nc + e];
        kv[i] = track_kd ? KQ[(k + i) * nc + e] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        d = fmaf(-qv[i], w[k + i], d);
        kd = fmaf(-kv[i], w[k + i], kd);
      }
    }
    for (; k < B; ++k) {
      d = fmaf(-Q[k * nc + e], w[k], d);
      if (track_kd) kd = fmaf(-KQ[k * nc + e], w[k], kd);
    }
    qcol[e] = d;
    if (track_kd) kcol[e] = kd;
    acc += static_cast<double>(z[e]) * d;
  }
  acc = block_reduce_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// eta = z^T d from direction_kernel's partial sums (every block adds them itself, in block
// order); block 0 records the step as eta's finalisation (stop if eta <= 0, App. B.2;
// otherwise the column is pending and the iteration counts); then
// Q[:, B] /= sqrt(eta); KQ[:, B] /= sqrt(eta); v += (alpha/eta) d; u += (alpha/eta) K d.
__global__ void update_kernel(const ProbDev* __restrict__ probs, int track_kd, int nblk) {
  const ProbDev& P = probs[blockIdx.y];
  FitState* st = P.st;
  const int64_t nc = P.nc;
  float* __restrict__ Q = P.Q;
  float* __restrict__ KQ = P.KQ;
  float* __restrict__ v = P.v;
  float* __restrict__ u = P.u;
  if (!st->newton_active || !st->active) return;
  __shared__ double eta_s;
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int b = 0; b < nblk; ++b) sum += P.ps[b];
    eta_s = sum;
  }
  __syncthreads();
  const double eta = eta_s;
  const int B = st->B;
  const double alpha = st->alpha;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->eta = eta;
    if (!(eta > 0.0)) {
      st->active = 0;
      st->stop_reason = ITERGP_STOP_ETA;
    } else {
      st->coef = alpha / eta;
      st->inv_sqrt_eta = 1.0 / sqrt(eta);
      st->pending = 1;
      st->j += 1;
      st->total_iters += 1;
    }
  }
  if (!(eta > 0.0)) return;
  const float coef = static_cast<float>(alpha / eta), ise = static_cast<float>(1.0 / sqrt(eta));
  float* qcol = Q + static_cast<int64_t>(B) * nc;
  float* kcol = KQ + static_cast<int64_t>(B) * nc;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nc;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float d = qcol[e];
    v[e] = fmaf(coef, d, v[e]);
    qcol[e] = d * ise;
    if (track_kd) {
      const float kd = kcol[e];
      u[e] = fmaf(coef, kd, u[e]);
      kcol[e] = kd * ise;
    }
  }
}

// end of a Newton step: commit the pending column, record the step
__global__ void step_end_kernel(const ProbDev* __restrict__ probs, int step) {
  FitState* st = probs[blockIdx.x].st;
  if (threadIdx.x != 0 || !st->newton_active) return;
  if (st->pending) {
    st->B += 1;
    st->pending = 0;
  }
  if (st->active) st->stop_reason = ITERGP_STOP_MAXITER;
  if (step < ITERGP_MAX_REPORT_STEPS) {
    st->iters[step] = st->j;
    st->stops[step] = st->stop_reason;
  }
  st->newton_steps = step + 1;
  st->active = 0;
}

// f_{i+1} = u + m  (u = K v, m = 0)
__global__ void copy_f_kernel(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const FitState* st = P.st;
  const int64_t nc = P.nc;
  const float* __restrict__ u = P.u;
  float* __restrict__ f = P.f;
  if (!st->newton_active) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nc;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    f[e] = u[e];
}

// standalone W^+ x and pseudo targets (verification entry points)
__global__ void winv_apply_kernel(const float* __restrict__ f, int64_t n, int C,
                                  const float* __restrict__ x, float* __restrict__ out, int* status) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* fi = f + i * C;
    float mx = fi[0];
    for (int c = 1; c < C; ++c) mx = fmaxf(mx, fi[c]);
    float se = 0.f;
    for (int c = 0; c < C; ++c) se += expf(fi[c] - mx);
    const float lse = mx + logf(se);
    float ip[kMaxC];
    for (int c = 0; c < C; ++c) {
      ip[c] = expf(lse - fi[c]);
      if (!isfinite(ip[c])) set_status(status, ITERGP_ENUMERIC);
    }
    winv_point(x + i * C, ip, C, out + i * C);
  }
}

__global__ void pseudo_targets_kernel(const float* __restrict__ f, const int32_t* __restrict__ y,
                                      int64_t n, int C, float* __restrict__ out, int* status) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* fi = f + i * C;
    float mx = fi[0];
    for (int c = 1; c < C; ++c) mx = fmaxf(mx, fi[c]);
    float se = 0.f;
    for (int c = 0; c < C; ++c) se += expf(fi[c] - mx);
    const float lse = mx + logf(se);
    int yi = y[i];
    if (yi < 0 || yi >= C) {
      set_status(status, ITERGP_EINVAL);
      yi = 0;
    }
    float ip[kMaxC], grad[kMaxC], w[kMaxC];
    for (int c = 0; c < C; ++c) {
      ip[c] = expf(lse - fi[c]);
      if (!isfinite(ip[c])) set_status(status, ITERGP_ENUMERIC);
      grad[c] = (c == yi ? 1.f : 0.f) - expf(fi[c] - lse);
    }
    winv_point(grad, ip, C, w);
    for (int c = 0; c < C; ++c) out[i * C + c] = fi[c] + w[c];
  }
}

// CL > 1: one cluster of CL CTAs (A and V global, the rotations in rank 0's shared memory).
template <int CL>
__global__ void sym_eig_kernel(const double* __restrict__ M, int b, double* __restrict__ lam,
                               double* __restrict__ U, double* __restrict__ A, double* __restrict__ V) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) uint8_t esh[];
  double* cs = reinterpret_cast<double*>(esh);
  double* sn = cs + b / 2 + 1;
  double* red = sn + b / 2 + 1;
  int* plo = reinterpret_cast<int*>(red + 32);
  int* phi = plo + b + 1;
  int* order = phi + b + 1;
  if constexpr (CL > 1) {
    if (cg::this_cluster().block_rank() != 0) {
      auto cl = cg::this_cluster();
      jacobi_eig<CL>(A, V, b, b, cl.map_shared_rank(cs, 0), cl.map_shared_rank(sn, 0),
                     cl.map_shared_rank(plo, 0), cl.map_shared_rank(phi, 0), red);
      return;
    }
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    A[i * b + j] = 0.5 * (M[i * b + j] + M[j * b + i]);
  }
  __syncthreads();
  jacobi_eig<CL>(A, V, b, b, cs, sn, plo, phi, red);
  eig_order(A, b, b, order);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, k = e % b;
    U[i * b + k] = V[i * b + order[k]];
  }
  for (int k = threadIdx.x; k < b; k += blockDim.x) lam[k] = A[order[k] * b + order[k]];
}

// ------------------------------------------------------------ batched product staging
// Row arena: FP32 rows of every problem, each block padded to a multiple of 128 rows and
// to d_max columns with zeros (zero columns leave distances unchanged).
struct ArenaCopy {
  const float* X;
  int64_t rows, row0;
  int d;
};
__global__ void arena_copy_kernel(const ArenaCopy* __restrict__ tab, float* __restrict__ arena,
                                  int d_max) {
  const ArenaCopy t = tab[blockIdx.y];
  const int64_t rows_pad = (t.rows + 127) / 128 * 128;
  const int64_t total = rows_pad * d_max;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / d_max;
    const int col = static_cast<int>(e % d_max);
    arena[(t.row0 + r) * d_max + col] = (r < t.rows && col < t.d) ? t.X[r * t.d + col] : 0.f;
  }
}

// Per-problem source of the weights S_p (n_p x C_p, row-major) of a batched product.
struct SSource {
  const float* S;
  int64_t rows, row0;
  int c;
  const int* active;
};
// Column maxima of every problem's weights (its N x C block), as float bits: per block a
// shared maximum per column, then one atomicMax per column into cmax [nprob][p16] (zeroed
// by the caller).
__global__ void s_colmax_kernel(const SSource* __restrict__ tab, int p16, uint32_t* __restrict__ cmax) {
  const SSource t = tab[blockIdx.y];
  if (t.active != nullptr && *t.active == 0) return;
  __shared__ uint32_t m[kMaxC];
  for (int c = threadIdx.x; c < kMaxC; c += blockDim.x) m[c] = 0u;
  __syncthreads();
  const int64_t total = t.rows * t.c;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicMax(&m[e % t.c], __float_as_uint(fabsf(t.S[e])));
  __syncthreads();
  for (int c = threadIdx.x; c < t.c && c < p16; c += blockDim.x)
    if (m[c] != 0u) atomicMax(&cmax[static_cast<int64_t>(blockIdx.y) * p16 + c], m[c]);
}

// Transposed weights [p16][arena rows] (tensor-core path).  SPLIT (BF16X3, TF32): FP16 hi
// and lo of 2^e_c S[:, c] with e_c from the column maximum (see prep_s_kernel), scale
// 2^-e_c into wsc [nprob][p16]; otherwise one BF16 plane.
template <bool SPLIT>
__global__ void s_stage_tc_kernel(const SSource* __restrict__ tab, int p16, int64_t arena_rows,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                  const uint32_t* __restrict__ cmax, float* __restrict__ wsc) {
  const SSource t = tab[blockIdx.y];
  if (t.active != nullptr && *t.active == 0) return;
  const int64_t rows_pad = (t.rows + 127) / 128 * 128;
  const int64_t total = rows_pad * p16;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int cc = static_cast<int>(e / rows_pad);
    const int64_t r = e % rows_pad;
    const float x = (r < t.rows && cc < t.c) ? t.S[r * t.c + cc] : 0.f;
    if constexpr (SPLIT) {
      const int ex = cc < t.c ? scale_exp_of_max(cmax[static_cast<int64_t>(blockIdx.y) * p16 + cc]) : 0;
      const float xs = x * pow2i(ex);
      const __half h = __float2half_rn(xs);
      reinterpret_cast<__half*>(hi)[cc * arena_rows + t.row0 + r] = h;
      reinterpret_cast<__half*>(lo)[cc * arena_rows + t.row0 + r] = __float2half_rn(xs - __half2float(h));
      if (r == 0) wsc[static_cast<int64_t>(blockIdx.y) * p16 + cc] = pow2i(-ex);
    } else {
      hi[cc * arena_rows + t.row0 + r] = __float2bfloat16_rn(x);
    }
  }
}
// FP32 weights [arena rows][p_max] (SIMT path).
__global__ void s_stage_simt_kernel(const SSource* __restrict__ tab, int p_max, float* __restrict__ out) {
  const SSource t = tab[blockIdx.y];
  if (t.active != nullptr && *t.active == 0) return;
  const int64_t rows_pad = (t.rows + 127) / 128 * 128;
  const int64_t total = rows_pad * p_max;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / p_max;
    const int cc = static_cast<int>(e % p_max);
    out[(t.row0 + r) * p_max + cc] = (r < t.rows && cc < t.c) ? t.S[r * t.c + cc] : 0.f;
  }
}

}  // namespace

// A batched kernel product over a fixed set of problems (built once per fit).
struct BatchProduct {
  int precision = 0, kind = 0, nprob = 0, p16 = 16, d_max = 0;
  int64_t arena_rows = 0;
  RowOperand arena;
  KmvItemTables tab;
  const SSource* src = nullptr;      // device [nprob]
  __nv_bfloat16 *s_hi = nullptr, *s_lo = nullptr;
  uint32_t* cmax = nullptr;          // split weights: column maxima [nprob][p16]
  float* wsc = nullptr;              // split weights: their scales 2^-e [nprob][p16]
  float* s32 = nullptr;
  int64_t max_rows_pad = 0;
};

// LPT (longest processing time first) assignment of whole-row items to G CTAs.
void plan_items(const std::vector<WorkItem>& items, int G, std::vector<WorkItem>* ordered,
                std::vector<int32_t>* begin) {
  std::vector<int> idx(items.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = static_cast<int>(i);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return items[a].chunks > items[b].chunks; });
  std::vector<int64_t> load(G, 0);
  std::vector<std::vector<int>> per(G);
  for (int i : idx) {
    int best = 0;
    for (int g = 1; g < G; ++g)
      if (load[g] < load[best]) best = g;
    load[best] += items[i].chunks;
    per[best].push_back(i);
  }
  ordered->clear();
  begin->assign(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    // within a CTA keep items of the same problem together (L2 reuse of its rows)
    std::stable_sort(per[g].begin(), per[g].end(), [&](int a, int b) { return items[a].prob < items[b].prob; });
    (*begin)[g] = static_cast<int32_t>(ordered->size());
    for (int i : per[g]) ordered->push_back(items[i]);
  }
  (*begin)[G] = static_cast<int32_t>(ordered->size());
}


// ======================================================================= host side

int fit_run_batch(DeviceContext* ctx, const std::vector<FitProblem>& probs, cudaStream_t stream,
                  bool use_graph) {
  const int np = static_cast<int>(probs.size());
  if (np == 0) return ITERGP_OK;
  const itergp_fit_params& prm = *probs[0].prm;    // schedule shared by the batch
  const int track_kd = prm.literal_kv ? 0 : 1;
  // the class-contrast projection belongs to the softmax likelihood (one latent per
  // point has no class-sum directions)
  // It is the identity in exact arithmetic only while K keeps the class contrasts in
  // place (one shared kernel, K = k kron I_C); one kernel per class mixes the per-point
  // class sums into K s, so there it would change the algorithm and is off.
  const int project = prm.policy == ITERGP_POLICY_CG && prm.likelihood == ITERGP_LIK_SOFTMAX &&
                              probs[0].class_kp.empty() ? 1 : 0;
  // the BF16 forms round kernel values (and weights) to 8 bits: residuals below 2^-8 |b|
  // are not resolved (FP32 and the BF16X3 split resolve far below the paper's 1e-5)
  const double floor_rel = (prm.precision == ITERGP_BF16 || prm.precision == ITERGP_BF16_COMP) ? 0x1p-8 : 0.0;
  int64_t max_n = 0, max_nc = 0;
  int max_bcap = 1, c_max = 2, d_max = 1;
  for (const FitProblem& fp : probs) {
    max_n = std::max<int64_t>(max_n, fp.prm->n);
    max_nc = std::max<int64_t>(max_nc, fp.prm->n * fp.prm->c);
    max_bcap = std::max(max_bcap, fp.bcap);
    c_max = std::max(c_max, static_cast<int>(fp.prm->c));
    d_max = std::max(d_max, static_cast<int>(fp.prm->d));
  }
  // Blocks of the per-iteration vector kernels, at most two per SM: a single problem spreads
  // even small vectors over many SMs (their FP64 partial sums run at the SM's low FP64
  // rate); a batch, whose grid repeats the largest problem's block count for every
  // problem, takes fewer, larger blocks.
  const int64_t per_pt = np > 1 ? 256 : 64, per_el = np > 1 ? 1024 : 64;
  const int nblk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(2LL * ctx->num_sms, ceil_div(max_n, per_pt))));
  const int nblk_e = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(2LL * ctx->num_sms, ceil_div(max_nc, per_el))));
  const int gram_splits = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(64, ceil_div(max_nc, 4096))));
  const int eb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(max_nc, 256), 8LL * ctx->num_sms)));
  const int maxblk = std::max(nblk, nblk_e);
  const int tiles = static_cast<int>(ceil_div(max_bcap, kGT));

  // ---- workspace: per-problem arrays
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(std::max<size_t>(bytes, 1), 256); return o; };
  struct Offs { size_t st, S, T, KQ, u, b, r, z, gp, ip, s, t, w, sq, W, A, V, pg, pv, ps, bold; };
  std::vector<Offs> offs(np);
  for (int i = 0; i < np; ++i) {
    const int64_t nc = probs[i].prm->n * probs[i].prm->c;
    const int bc = probs[i].bcap;
    Offs& o = offs[i];
    o.st = take(sizeof(FitState));
    o.S = take(sizeof(float) * nc * bc);
    o.T = take(sizeof(float) * nc * bc);
    o.KQ = take(sizeof(float) * nc * bc);
    o.u = take(sizeof(float) * nc); o.b = take(sizeof(float) * nc); o.r = take(sizeof(float) * nc);
    o.z = take(sizeof(float) * nc); o.gp = take(sizeof(float) * nc); o.ip = take(sizeof(float) * nc);
    o.s = take(sizeof(float) * nc); o.t = take(sizeof(float) * nc);
    o.w = take(sizeof(float) * bc); o.sq = take(sizeof(float) * bc);
    o.W = take(sizeof(float) * bc * bc);
    o.A = take(sizeof(double) * bc * bc); o.V = take(sizeof(double) * bc * bc);
    o.pg = take(sizeof(double) * gram_splits * bc * bc);
    o.pv = take(sizeof(double) * maxblk * bc);
    o.ps = take(sizeof(double) * 5 * maxblk);
    o.bold = take(sizeof(int));
  }
  const size_t o_probs = take(sizeof(ProbDev) * np);
  const size_t o_status = take(sizeof(int));

  // ---- batched product plan (np > 1)
  const bool batched = np > 1;
  BatchProduct bp;
  std::vector<WorkItem> items_host, ordered;
  std::vector<int32_t> begin_host;
  std::vector<TcProb> tcp_host;
  std::vector<SSource> src_host;
  std::vector<ArenaCopy> ac_host;
  size_t o_arena = 0, o_rows = 0, o_items = 0, o_begin = 0, o_tcp = 0, o_src = 0, o_ac = 0, o_shi = 0,
         o_slo = 0, o_s32 = 0, o_cmx = 0, o_wsc = 0;
  if (batched) {
    bp.precision = prm.precision;
    bp.kind = prm.kernel.kind;
    bp.nprob = np;
    bp.d_max = d_max;
    bp.p16 = (c_max + 15) / 16 * 16;
    int64_t row = 0;
    for (int i = 0; i < np; ++i) {
      const int64_t n = probs[i].prm->n;
      const int64_t rows_pad = ceil_div(n, 128) * 128;
      ac_host.push_back(ArenaCopy{probs[i].prm->X, n, row, static_cast<int>(probs[i].prm->d)});
      const int chunks = static_cast<int>(ceil_div(n, 128));
      for (int r = 0; r < chunks; ++r)
        items_host.push_back(WorkItem{i, static_cast<int32_t>(row + 128 * r), 128 * r,
                                      static_cast<int32_t>(row), chunks, static_cast<int32_t>(n), 0, 0});
      bp.max_rows_pad = std::max(bp.max_rows_pad, rows_pad);
      row += rows_pad;
    }
    bp.arena_rows = row;
    const int G = static_cast<int>(std::min<int64_t>(ctx->num_sms, static_cast<int64_t>(items_host.size())));
    plan_items(items_host, G, &ordered, &begin_host);
    bp.tab.G = G;
    bp.tab.n_items = static_cast<int>(ordered.size());
    o_arena = take(sizeof(float) * bp.arena_rows * d_max);
    o_rows = take(rows_workspace_bytes(prm.precision, bp.arena_rows, d_max));
    o_items = take(sizeof(WorkItem) * ordered.size());
    o_begin = take(sizeof(int32_t) * begin_host.size());
    o_tcp = take(sizeof(TcProb) * np);
    o_src = take(sizeof(SSource) * np);
    o_ac = take(sizeof(ArenaCopy) * np);
    if (precision_is_tensor(prm.precision)) {
      o_shi = take(sizeof(__nv_bfloat16) * bp.p16 * bp.arena_rows);
      o_slo = take(sizeof(__nv_bfloat16) * bp.p16 * bp.arena_rows);
      o_cmx = take(sizeof(uint32_t) * np * bp.p16);
      o_wsc = take(sizeof(float) * np * bp.p16);
    } else {
      o_s32 = take(sizeof(float) * bp.arena_rows * c_max);
    }
  }

  Scratch ws;
  ITERGP_CUDA_TRY(ws.alloc(ctx, off, stream));
  char* base = ws.as<char>();
  std::vector<ProbDev> pd(np);
  for (int i = 0; i < np; ++i) {
    const Offs& o = offs[i];
    ProbDev& d = pd[i];
    d.st = reinterpret_cast<FitState*>(base + o.st);
    d.n = probs[i].prm->n;
    d.c = probs[i].prm->c;
    d.nc = d.n * d.c;
    d.bcap = probs[i].bcap;
    d.y = probs[i].prm->y;
    d.lik = probs[i].prm->likelihood;
    d.noise = probs[i].prm->noise;
    d.yr = probs[i].prm->y_real;
    d.f = probs[i].f; d.v = probs[i].v; d.Q = probs[i].Q;
    d.S = reinterpret_cast<float*>(base + o.S); d.T = reinterpret_cast<float*>(base + o.T);
    d.KQ = reinterpret_cast<float*>(base + o.KQ);
    d.u = reinterpret_cast<float*>(base + o.u); d.b = reinterpret_cast<float*>(base + o.b);
    d.r = reinterpret_cast<float*>(base + o.r); d.z = reinterpret_cast<float*>(base + o.z);
    d.gp = reinterpret_cast<float*>(base + o.gp); d.ip = reinterpret_cast<float*>(base + o.ip);
    d.s_cur = reinterpret_cast<float*>(base + o.s); d.t_cur = reinterpret_cast<float*>(base + o.t);
    d.w = reinterpret_cast<float*>(base + o.w); d.sq = reinterpret_cast<float*>(base + o.sq);
    d.W = reinterpret_cast<float*>(base + o.W);
    d.Am = reinterpret_cast<double*>(base + o.A); d.Vm = reinterpret_cast<double*>(base + o.V);
    d.pg = reinterpret_cast<double*>(base + o.pg); d.pv = reinterpret_cast<double*>(base + o.pv);
    d.ps = reinterpret_cast<double*>(base + o.ps);
    d.bold = reinterpret_cast<int*>(base + o.bold);
  }
  ProbDev* pdev = reinterpret_cast<ProbDev*>(base + o_probs);
  // Kernel-level errors of this fit (a wait that ran out) go to a word of its own, so
  // fits and products on other streams never see them.
  DeviceContext fit_ctx = *ctx;
  fit_ctx.status = reinterpret_cast<int*>(base + o_status);
  ITERGP_CUDA_TRY(cudaMemsetAsync(fit_ctx.status, 0, sizeof(int), stream));
  ctx = &fit_ctx;
  ITERGP_CUDA_TRY(cudaMemcpyAsync(pdev, pd.data(), sizeof(ProbDev) * np, cudaMemcpyHostToDevice, stream));
  FitState init{};
  init.newton_active = 1;
  for (int i = 0; i < np; ++i) {
    ITERGP_CUDA_TRY(cudaMemcpyAsync(pd[i].st, &init, sizeof(FitState), cudaMemcpyHostToDevice, stream));
    if (probs[i].prm->f0)   // a given starting iterate (teacher forcing), else f_0 = m = 0
      ITERGP_CUDA_TRY(cudaMemcpyAsync(pd[i].f, probs[i].prm->f0, sizeof(float) * pd[i].nc,
                                      cudaMemcpyDeviceToDevice, stream));
    else
      ITERGP_CUDA_TRY(cudaMemsetAsync(pd[i].f, 0, sizeof(float) * pd[i].nc, stream));
    ITERGP_CUDA_TRY(cudaMemsetAsync(pd[i].v, 0, sizeof(float) * pd[i].nc, stream));
    ITERGP_CUDA_TRY(cudaMemsetAsync(pd[i].u, 0, sizeof(float) * pd[i].nc, stream));
    ITERGP_CUDA_TRY(cudaMemsetAsync(pd[i].gp, 0, sizeof(float) * pd[i].nc, stream));
  }

  // tables of the batched product, uploaded once
  if (batched) {
    for (int i = 0; i < np; ++i) {
      float* wsc_i = precision_is_tensor(prm.precision) ? reinterpret_cast<float*>(base + o_wsc) + i * bp.p16 : nullptr;
      tcp_host.push_back(TcProb{pd[i].t_cur, pd[i].c, pd[i].n, pd[i].c, 0, probs[i].kp, &pd[i].st->active, wsc_i});
      src_host.push_back(SSource{pd[i].s_cur, pd[i].n, ac_host[i].row0, pd[i].c, &pd[i].st->active});
    }
    bp.arena.X = nullptr;
    float* arena = reinterpret_cast<float*>(base + o_arena);
    ArenaCopy* ac = reinterpret_cast<ArenaCopy*>(base + o_ac);
    ITERGP_CUDA_TRY(cudaMemcpyAsync(ac, ac_host.data(), sizeof(ArenaCopy) * np, cudaMemcpyHostToDevice, stream));
    {
      dim3 grid(static_cast<unsigned>(std::min<int64_t>(ceil_div(bp.max_rows_pad * d_max, 256), 1024)), np);
      arena_copy_kernel<<<grid, 256, 0, stream>>>(ac, arena, d_max), ::itergp::note_launch();
      ITERGP_CUDA_TRY(cudaGetLastError());
    }
    int rc = prepare_rows(prm.precision, arena, bp.arena_rows, d_max, d_max, base + o_rows, &bp.arena, stream);
    if (rc != ITERGP_OK) return rc;
    WorkItem* items_dev = reinterpret_cast<WorkItem*>(base + o_items);
    int32_t* begin_dev = reinterpret_cast<int32_t*>(base + o_begin);
    TcProb* tcp_dev = reinterpret_cast<TcProb*>(base + o_tcp);
    SSource* src_dev = reinterpret_cast<SSource*>(base + o_src);
    ITERGP_CUDA_TRY(cudaMemcpyAsync(items_dev, ordered.data(), sizeof(WorkItem) * ordered.size(), cudaMemcpyHostToDevice, stream));
    ITERGP_CUDA_TRY(cudaMemcpyAsync(begin_dev, begin_host.data(), sizeof(int32_t) * begin_host.size(), cudaMemcpyHostToDevice, stream));
    ITERGP_CUDA_TRY(cudaMemcpyAsync(tcp_dev, tcp_host.data(), sizeof(TcProb) * np, cudaMemcpyHostToDevice, stream));
    ITERGP_CUDA_TRY(cudaMemcpyAsync(src_dev, src_host.data(), sizeof(SSource) * np, cudaMemcpyHostToDevice, stream));
    bp.tab.items = items_dev;
    bp.tab.item_begin = begin_dev;
    bp.tab.probs = tcp_dev;
    bp.src = src_dev;
    if (precision_is_tensor(prm.precision)) {
      bp.s_hi = reinterpret_cast<__nv_bfloat16*>(base + o_shi);
      bp.s_lo = reinterpret_cast<__nv_bfloat16*>(base + o_slo);
      bp.cmax = reinterpret_cast<uint32_t*>(base + o_cmx);
      bp.wsc = reinterpret_cast<float*>(base + o_wsc);
    } else {
      bp.s32 = reinterpret_cast<float*>(base + o_s32);
    }
    if (prm.literal_kv) return ITERGP_EINVAL;   // batched fits carry K v (validated by the API)
  }

  // the kernel products of an iteration: t_cur = K s_cur for every active problem
  // K w for one problem's N x C block (one kernel per class: C grouped products)
  auto kprod0 = [&](const float* w, float* out, const int* active) -> int {
    if (!probs[0].class_kp.empty())
      return kmv_classes(ctx, probs[0].class_kp.data(), pd[0].c, *probs[0].xop, *probs[0].xop, w, pd[0].c,
                         pd[0].c, out, pd[0].c, stream, active);
    return kmv_execute(ctx, probs[0].kp, *probs[0].xop, *probs[0].xop, w, pd[0].c, pd[0].c, out, pd[0].c,
                       stream, active);
  };
  auto products = [&]() -> int {
    if (!batched) return kprod0(pd[0].s_cur, pd[0].t_cur, &pd[0].st->active);
    dim3 grid(static_cast<unsigned>(std::min<int64_t>(ceil_div(bp.max_rows_pad * bp.p16, 256), 512)), np);
    if (precision_is_tensor(prm.precision)) {
      if (precision_splits_weights(prm.precision)) {
        ITERGP_CUDA_TRY(cudaMemsetAsync(bp.cmax, 0, sizeof(uint32_t) * np * bp.p16, stream));
        s_colmax_kernel<<<grid, 256, 0, stream>>>(bp.src, bp.p16, bp.cmax), ::itergp::note_launch();
        s_stage_tc_kernel<true><<<grid, 256, 0, stream>>>(bp.src, bp.p16, bp.arena_rows, bp.s_hi, bp.s_lo, bp.cmax,
                                                         bp.wsc), ::itergp::note_launch();
      } else {
        s_stage_tc_kernel<false><<<grid, 256, 0, stream>>>(bp.src, bp.p16, bp.arena_rows, bp.s_hi, bp.s_lo, nullptr,
                                                          nullptr), ::itergp::note_launch();
      }
      ITERGP_CUDA_TRY(cudaGetLastError());
      return kmv_tc_items(ctx, bp.kind, bp.arena, bp.arena, bp.tab, bp.s_hi, bp.s_lo, bp.p16, 0,
                          bp.p16, stream);
    }
    s_stage_simt_kernel<<<grid, 256, 0, stream>>>(bp.src, c_max, bp.s32), ::itergp::note_launch();
    ITERGP_CUDA_TRY(cudaGetLastError());
    return kmv_simt_items(ctx, bp.kind, bp.arena, bp.arena, bp.tab, bp.s32, c_max, c_max, stream);
  };

  const bool eig_ab_smem = max_bcap <= kEigSmemMax;
  const size_t eig_smem = eig_smem_bytes(max_bcap, eig_ab_smem);
  const int eig_threads = 512;
  ITERGP_CUDA_TRY(cudaFuncSetAttribute(vsr_eig_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(eig_smem)));
  // a few problems: each eigendecomposition on a cluster of SMs (bitwise the same result)
  const bool eig_cl = eig_ab_smem && eig_threads == 512 && static_cast<int64_t>(np) * kEigCluster <= ctx->num_sms &&
                      vsr_eig_cluster_ok(ctx);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // The schedule is captured on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured) and the graph is launched on the caller's stream,
  // after the set-up work enqueued above.
  cudaStream_t caller = stream;
  cudaStream_t cap = nullptr;
  if (use_graph) {
    ITERGP_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    const cudaError_t be = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (be != cudaSuccess) {
      cudaStreamDestroy(cap);
      ITERGP_CUDA_TRY(be);
    }
    stream = cap;
  }
  int rc = ITERGP_OK;
  for (int step = 0; step < prm.max_newton && rc == ITERGP_OK; ++step) {
    newton_prologue_kernel<<<dim3(nblk, np), kRedThreads, 0, stream>>>(pdev, project), ::itergp::note_launch();
    newton_finalize_kernel<<<np, 32, 0, stream>>>(pdev, nblk, step, prm.tol_newton, prm.tol_abs, prm.tol_rel,
                                                  prm.recycle, floor_rel), ::itergp::note_launch();
    // ---- Alg. 3: virtual solver run with compression
    if (prm.recycle && step > 0) {
      copy_int_kernel<<<np, 32, 0, stream>>>(pdev), ::itergp::note_launch();
      vsr_z_kernel<<<dim3(eb, np), 256, 0, stream>>>(pdev), ::itergp::note_launch();
      gram_partial_kernel<<<dim3(tiles * tiles, gram_splits, np), 256, 0, stream>>>(pdev, tiles), ::itergp::note_launch();
      if (eig_cl) {
        const cudaError_t le = launch_clustered(vsr_eig_kernel<kEigCluster>, np, kEigCluster, eig_threads, eig_smem,
                                                stream, static_cast<const ProbDev*>(pdev), gram_splits, prm.rank, step, 1);
        if (le != cudaSuccess) {
          ::itergp::record_cuda_error(le, "vsr_eig_kernel cluster launch", __FILE__, __LINE__);
          rc = ITERGP_ECUDA;
        }
      } else
        vsr_eig_kernel<1><<<np, eig_threads, eig_smem, stream>>>(pdev, gram_splits, prm.rank, step, eig_ab_smem ? 1 : 0);
      ::itergp::note_launch();
      if (rc != ITERGP_OK) break;
      vsr_rotate_kernel<<<dim3(eb, np), 256, 0, stream>>>(pdev), ::itergp::note_launch();
      vsr_rescale_kernel<<<dim3(eb, np), 256, 0, stream>>>(pdev), ::itergp::note_launch();
      // v0 = Q0 (Q0^T b), u0 = K v0 = KQ0 (Q0^T b)
      proj_partial_kernel<<<dim3(nblk_e, np), 256, 0, stream>>>(pdev), ::itergp::note_launch();
      proj_finalize_kernel<<<np, 256, 0, stream>>>(pdev, nblk_e), ::itergp::note_launch();
    }
    // v0 = C0 (y_hat - m) and K v0; with no recycled columns (B = 0) both are zero
    combine_kernel<<<dim3(eb, np), 256, 0, stream>>>(pdev), ::itergp::note_launch();
    // ---- Alg. 2 iterations
    for (int j = 0; j < prm.max_iters && rc == ITERGP_OK; ++j) {
      if (prm.literal_kv) {
        rc = kprod0(pd[0].v, pd[0].u, &pd[0].st->active);
        if (rc != ITERGP_OK) break;
      }
      // r and the action s; |r|, the stopping test and alpha; t = K s; z and Q^T z;
      // d, K d and eta; v, u and the new column (each reduction is finished by the next
      // kernel's blocks)
      resid_kernel<<<dim3(nblk, np), kRedThreads, 0, stream>>>(pdev, project, prm.policy), ::itergp::note_launch();
      resid_finalize_kernel<<<np, 32, 0, stream>>>(pdev, nblk, prm.policy), ::itergp::note_launch();
      rc = products();
      if (rc != ITERGP_OK) break;
      zproj_kernel<<<dim3(nblk_e, np), 256, 0, stream>>>(pdev), ::itergp::note_launch();
      direction_kernel<<<dim3(nblk_e, np), kRedThreads, 0, stream>>>(pdev, track_kd), ::itergp::note_launch();
      update_kernel<<<dim3(eb, np), 256, 0, stream>>>(pdev, track_kd, nblk_e), ::itergp::note_launch();
    }
    if (rc != ITERGP_OK) break;
    step_end_kernel<<<np, 32, 0, stream>>>(pdev, step), ::itergp::note_launch();
    if (prm.literal_kv) {
      // f_{i+1} = K v + m by a fresh product
      rc = kprod0(pd[0].v, pd[0].u, &pd[0].st->newton_active);
      if (rc != ITERGP_OK) break;
    }
    copy_f_kernel<<<dim3(eb, np), 256, 0, stream>>>(pdev), ::itergp::note_launch();
  }
  if (use_graph) {
    const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    stream = caller;
    if (rc != ITERGP_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (rc != ITERGP_OK) return rc;
      ITERGP_CUDA_TRY(ce);
    }
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    ITERGP_CUDA_TRY(ie);
    const cudaError_t le = cudaGraphLaunch(exec, stream);
    cudaGraphExecDestroy(exec);
    ITERGP_CUDA_TRY(le);
  }
  if (rc != ITERGP_OK) return rc;
  ITERGP_CUDA_TRY(cudaGetLastError());

  std::vector<FitState> hs(np);
  int fit_status = ITERGP_OK;
  for (int i = 0; i < np; ++i)
    ITERGP_CUDA_TRY(cudaMemcpyAsync(&hs[i], pd[i].st, sizeof(FitState), cudaMemcpyDeviceToHost, stream));
  ITERGP_CUDA_TRY(cudaMemcpyAsync(&fit_status, fit_ctx.status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  ITERGP_CUDA_TRY(cudaStreamSynchronize(stream));
  if (fit_status != ITERGP_OK) return fit_status;
  for (int i = 0; i < np; ++i) {
    itergp_fit_report* rep = probs[i].rep;
    if (rep) {
      rep->newton_steps = hs[i].newton_steps;
      rep->total_iters = hs[i].total_iters;
      rep->buffer_cols = hs[i].B;
      rep->stop_reason = hs[i].stop_reason;
      for (int k = 0; k < ITERGP_MAX_REPORT_STEPS; ++k) {
        rep->iters[k] = hs[i].iters[k];
        rep->stops[k] = hs[i].stops[k];
        rep->kept[k] = hs[i].kept[k];
        rep->objective[k] = hs[i].objective[k];
        rep->rel_change[k] = hs[i].rel_change[k];
      }
      rep->resid_norm = hs[i].rnorm;
      rep->status = hs[i].status;
    }
    *probs[i].status = hs[i].status;
    *probs[i].final_B = hs[i].B;
  }
  return ITERGP_OK;
}

int winv_apply_launch(DeviceContext* ctx, const float* f, int64_t n, int c, const float* x,
                      float* out, cudaStream_t s) {
  if (n == 0) return ITERGP_OK;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(ceil_div(n, 256), 8LL * ctx->num_sms));
  winv_apply_kernel<<<blocks, 256, 0, s>>>(f, n, c, x, out, ctx->status), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  return ITERGP_OK;
}

int pseudo_targets_launch(DeviceContext* ctx, const float* f, const int32_t* y, int64_t n, int c,
                          float* out, cudaStream_t s) {
  if (n == 0) return ITERGP_OK;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(ceil_div(n, 256), 8LL * ctx->num_sms));
  pseudo_targets_kernel<<<blocks, 256, 0, s>>>(f, y, n, c, out, ctx->status), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  return ITERGP_OK;
}

int sym_eig_launch(DeviceContext* ctx, const double* M, int b, double* lam, double* U,
                   cudaStream_t s) {
  Scratch ws;
  ITERGP_CUDA_TRY(ws.alloc(ctx, sizeof(double) * 2 * b * b, s));
  double* A = ws.as<double>();
  double* V = A + static_cast<size_t>(b) * b;
  const size_t smem = eig_smem_bytes(b);
  if (eig_cluster_fits(sym_eig_kernel<kEigCluster>, 512, smem))
    ITERGP_CUDA_TRY(launch_clustered(sym_eig_kernel<kEigCluster>, 1, kEigCluster, 512, smem, s, M, b, lam, U, A, V));
  else
    sym_eig_kernel<1><<<1, 512, smem, s>>>(M, b, lam, U, A, V);
  ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  return ITERGP_OK;
}

}  // namespace itergp
