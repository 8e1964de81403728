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
#include <vector>

#include "internal.h"

namespace itergp {

constexpr int kMaxC = 64;
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
  int pad_;
  double alpha, eta, coef, inv_sqrt_eta;
  double bnorm, thresh, rnorm;
  int iters[ITERGP_MAX_REPORT_STEPS];
  int stops[ITERGP_MAX_REPORT_STEPS];
  int kept[ITERGP_MAX_REPORT_STEPS];
  double objective[ITERGP_MAX_REPORT_STEPS];
  double rel_change[ITERGP_MAX_REPORT_STEPS];
};

struct FitConfig {
  int64_t n;
  int c;
  int64_t nc;
  int bcap;            // buffer capacity (columns)
  int policy;
  int rank;            // R (< 0: no limit)
  int max_iters;
  int literal_kv;
  int recycle;
  double tol_newton, tol_abs, tol_rel;
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

// out_n = P diag(inv_pi_n) P x_n, P = I - 11^T/C   (Lemma A.6)
__device__ __forceinline__ void winv_point(const float* __restrict__ x, const float* __restrict__ ip,
                                           int C, float* __restrict__ out) {
  float m1 = 0.f;
  for (int c = 0; c < C; ++c) m1 += x[c];
  m1 /= C;
  float m2 = 0.f;
  for (int c = 0; c < C; ++c) m2 += (x[c] - m1) * ip[c];
  m2 /= C;
  for (int c = 0; c < C; ++c) out[c] = (x[c] - m1) * ip[c] - m2;
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// -------------------------------------------------------------------- Newton prologue
// For every point: pi = softmax(f_n), 1/pi = exp(lse - f), grad = e_y - pi,
// b = y_hat - m = f + W^+ grad (m = 0).  Partial sums: |b|^2, log p(y|f), v.(f - m),
// |g - g_prev|^2, |g|^2 with g = f - m; g_prev <- g.
__global__ void newton_prologue_kernel(const FitState* __restrict__ st, int64_t n, int C,
                                       const float* __restrict__ f, const int32_t* __restrict__ y,
                                       const float* __restrict__ v, float* __restrict__ g_prev,
                                       float* __restrict__ inv_pi, float* __restrict__ b,
                                       double* __restrict__ part, int* status, int project) {
  if (!st->newton_active) return;
  __shared__ double sh[32];
  double s_b2 = 0, s_ll = 0, s_vf = 0, s_dg = 0, s_g2 = 0;
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
    float* ipi = inv_pi + i * C;
    float gsum = 0.f;
    float grad[kMaxC];
    for (int c = 0; c < C; ++c) {
      const float e = expf(lse - fi[c]);
      if (!isfinite(e)) set_status(status, ITERGP_ENUMERIC);
      ipi[c] = e;
      grad[c] = (c == yi ? 1.f : 0.f) - expf(fi[c] - lse);
      gsum += grad[c];
    }
    // W^+ grad with P applied on both sides
    const float m1 = gsum / C;
    float m2 = 0.f;
    for (int c = 0; c < C; ++c) m2 += (grad[c] - m1) * ipi[c];
    m2 /= C;
    float* bi = b + i * C;
    float* gp = g_prev + i * C;
    const float* vi = v + i * C;
    // With residual (CG) actions b lies in the class-contrast subspace range(I kron P) in
    // exact arithmetic (f = K v with v there, W^+ maps into it); removing the per-point
    // mean keeps rounding out of the class-sum directions, where K_hat reduces to the
    // near-singular k(X, X).  Unit-vector actions leave that subspace: no projection.
    float bmean = 0.f;
    if (project) {
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
    s_ll += static_cast<double>(fi[yi]) - lse;
  }
  double r;
  r = block_reduce_sum(s_b2, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 0] = r;
  r = block_reduce_sum(s_ll, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 1] = r;
  r = block_reduce_sum(s_vf, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 2] = r;
  r = block_reduce_sum(s_dg, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 3] = r;
  r = block_reduce_sum(s_g2, sh); if (threadIdx.x == 0) part[blockIdx.x * 5 + 4] = r;
}

__global__ void newton_finalize_kernel(FitState* st, const double* __restrict__ part, int nblk,
                                       int step, double tol_newton, double tol_abs,
                                       double tol_rel, int recycle) {
  if (threadIdx.x != 0 || !st->newton_active) return;
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
  st->thresh = fmax(tol_abs, tol_rel * st->bnorm);
  st->j = 0;
  st->pending = 0;
  st->active = 1;
  if (!recycle) st->B = 0;
  st->B0 = st->B;
}

// -------------------------------------------------------------------- Alg. 3 pieces
// Z = T + W^+ S for the B committed columns (written into the Q buffer as scratch).
__global__ void vsr_z_kernel(const FitState* __restrict__ st, int64_t n, int C, int64_t nc,
                             const float* __restrict__ S, const float* __restrict__ T,
                             const float* __restrict__ inv_pi, float* __restrict__ Z) {
  if (!st->newton_active) return;
  const int B = st->B;
  const int64_t total = static_cast<int64_t>(B) * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t col = e / n, i = e % n;
    const float* s = S + col * nc + i * C;
    float w[kMaxC];
    winv_point(s, inv_pi + i * C, C, w);
    const float* t = T + col * nc + i * C;
    float* z = Z + col * nc + i * C;
    for (int c = 0; c < C; ++c) z[c] = t[c] + w[c];
  }
}

// Gram partials G[split][a][b] = sum_{e in split} X[a][e] Y[b][e], a, b < B (32 x 32
// tiles, FP32 products summed in FP64).
constexpr int kGT = 32;
__global__ void gram_partial_kernel(const FitState* __restrict__ st, const float* __restrict__ X,
                                    const float* __restrict__ Y, int64_t nc, int bcap,
                                    int64_t per_split, double* __restrict__ part) {
  if (!st->newton_active) return;
  const int B = st->B;
  const int a0 = blockIdx.x * kGT, b0 = blockIdx.y * kGT;
  if (a0 >= B || b0 >= B) return;
  const int64_t e0 = static_cast<int64_t>(blockIdx.z) * per_split;
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
  double* out = part + static_cast<int64_t>(blockIdx.z) * bcap * bcap;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + 2 * ty + i, bb = b0 + 2 * tx + j;
      if (a < B && bb < B) out[a * bcap + bb] = acc[i][j];
    }
}

// ---------------------------------------------------------------- FP64 Jacobi (1 CTA)
// Cyclic Jacobi with round-robin (tournament) pairing: in each round the n/2 disjoint
// pairs are rotated simultaneously; column rotations then row rotations, each thread
// owning the two elements it updates.  A (n x n) is overwritten by a near-diagonal
// matrix, V accumulates the rotations (A_in = V diag V^T).
__device__ void jacobi_eig(double* A, double* V, int n, int ld, double* cs, double* sn, int* partner,
                           int* role, double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = (n + 1) / 2 * 2;   // even number of players (index n is a dummy if n odd)
  for (int e = tid; e < n * n; e += nt) V[(e / n) * ld + e % n] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();
  double fro = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    const double a = A[(e / n) * ld + e % n];
    fro += a * a;
  }
  fro = block_reduce_sum(fro, sh);
  __shared__ double fro_s, off_s;
  if (tid == 0) fro_s = fro;
  __syncthreads();
  const double tol2 = fro_s * 1e-30;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      if (i != j) {
        const double a = A[i * ld + j];
        off += a * a;
      }
    }
    off = block_reduce_sum(off, sh);
    if (tid == 0) off_s = off;
    __syncthreads();
    if (off_s <= tol2 || off_s == 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      // pairs of this round
      for (int k = tid; k < m / 2; k += nt) {
        const int i0 = k, i1 = m - 1 - k;
        const int p = (i0 == 0) ? 0 : ((i0 - 1 + r) % (m - 1)) + 1;
        const int q = ((i1 - 1 + r) % (m - 1)) + 1;
        const int lo = p < q ? p : q, hi = p < q ? q : p;
        double c = 1.0, s = 0.0;
        if (hi < n) {
          const double apq = A[lo * ld + hi];
          if (apq != 0.0) {
            const double app = A[lo * ld + lo], aqq = A[hi * ld + hi];
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        cs[k] = c;
        sn[k] = s;
        if (lo < n) { partner[lo] = hi; role[lo] = k; }
        if (hi < n) { partner[hi] = lo; role[hi] = -k - 1; }
      }
      __syncthreads();
      // columns: A[:, lo] = c A[:, lo] - s A[:, hi]; A[:, hi] = s A[:, lo] + c A[:, hi]
      for (int e = tid; e < n * (m / 2); e += nt) {
        const int row = e / (m / 2), k = e % (m / 2);
        const double c = cs[k], s = sn[k];
        if (s == 0.0) continue;
        const int i0 = k, i1 = m - 1 - k;
        const int p = (i0 == 0) ? 0 : ((i0 - 1 + r) % (m - 1)) + 1;
        const int q = ((i1 - 1 + r) % (m - 1)) + 1;
        const int lo = p < q ? p : q, hi = p < q ? q : p;
        if (hi >= n) continue;
        const double x = A[row * ld + lo], y = A[row * ld + hi];
        A[row * ld + lo] = c * x - s * y;
        A[row * ld + hi] = s * x + c * y;
        const double vx = V[row * ld + lo], vy = V[row * ld + hi];
        V[row * ld + lo] = c * vx - s * vy;
        V[row * ld + hi] = s * vx + c * vy;
      }
      __syncthreads();
      // rows: A[lo, :] = c A[lo, :] - s A[hi, :]; A[hi, :] = s A[lo, :] + c A[hi, :]
      for (int e = tid; e < n * (m / 2); e += nt) {
        const int col = e / (m / 2), k = e % (m / 2);
        const double c = cs[k], s = sn[k];
        if (s == 0.0) continue;
        const int i0 = k, i1 = m - 1 - k;
        const int p = (i0 == 0) ? 0 : ((i0 - 1 + r) % (m - 1)) + 1;
        const int q = ((i1 - 1 + r) % (m - 1)) + 1;
        const int lo = p < q ? p : q, hi = p < q ? q : p;
        if (hi >= n) continue;
        const double x = A[lo * ld + col], y = A[hi * ld + col];
        A[lo * ld + col] = c * x - s * y;
        A[hi * ld + col] = s * x + c * y;
      }
      __syncthreads();
      // the rotated pair's off-diagonal entries are zero in exact arithmetic
      for (int k = tid; k < m / 2; k += nt) {
        const int i0 = k, i1 = m - 1 - k;
        const int p = (i0 == 0) ? 0 : ((i0 - 1 + r) % (m - 1)) + 1;
        const int q = ((i1 - 1 + r) % (m - 1)) + 1;
        if (p < n && q < n && sn[k] != 0.0) {
          A[p * ld + q] = 0.0;
          A[q * ld + p] = 0.0;
        }
      }
      __syncthreads();
    }
  }
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

// Sum Gram partials, symmetrise, eigendecompose, drop lambda <= 1e-12 lambda_max, keep
// the R largest (Alg. 3), write rotation W[b][k] = U[b][k] lambda_k^-1/2 (FP32) and
// sqrt(lambda_k); set B = B0 = kept columns.
__global__ void vsr_eig_kernel(FitState* st, const double* __restrict__ part, int splits, int bcap,
                               int rank, double* __restrict__ Amat, double* __restrict__ Vmat,
                               float* __restrict__ W, float* __restrict__ sq, int step) {
  if (!st->newton_active) return;
  const int B = st->B;
  if (B == 0) {
    if (threadIdx.x == 0 && step < ITERGP_MAX_REPORT_STEPS) st->kept[step] = 0;
    return;
  }
  extern __shared__ double dsh[];
  double* cs = dsh;                 // bcap/2 + 1
  double* sn = cs + bcap / 2 + 1;   // bcap/2 + 1
  double* red = sn + bcap / 2 + 1;  // 32
  int* partner = reinterpret_cast<int*>(red + 32);
  int* role = partner + bcap + 1;
  int* order = role + bcap + 1;
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    const int a = e / B, b = e % B;
    double s1 = 0.0, s2 = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
      s1 += part[static_cast<int64_t>(sp) * bcap * bcap + a * bcap + b];
      s2 += part[static_cast<int64_t>(sp) * bcap * bcap + b * bcap + a];
    }
    Amat[a * bcap + b] = 0.5 * (s1 + s2);
  }
  __syncthreads();
  jacobi_eig(Amat, Vmat, B, bcap, cs, sn, partner, role, red);
  eig_order(Amat, B, bcap, order);
  __shared__ int keep_s;
  if (threadIdx.x == 0) {
    const double lmax = Amat[order[0] * bcap + order[0]];
    int keep = 0;
    while (keep < B && Amat[order[keep] * bcap + order[keep]] > 1e-12 * fmax(lmax, 0.0)) ++keep;
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
    const double lam = Amat[order[k] * bcap + order[k]];
    W[b * bcap + k] = static_cast<float>(Vmat[b * bcap + order[k]] / sqrt(lam));
  }
  for (int k = threadIdx.x; k < keep; k += blockDim.x)
    sq[k] = static_cast<float>(sqrt(Amat[order[k] * bcap + order[k]]));
}

// Q[:, k] = sum_b S[:, b] W[b][k];  KQ[:, k] = sum_b T[:, b] W[b][k]   (k < B_new, b < B_old)
// W is read with warp-uniform addresses (broadcast loads through L1).
__global__ void vsr_rotate_kernel(const FitState* __restrict__ st, const int* __restrict__ bold_ptr,
                                  int64_t nc, int bcap, const float* __restrict__ S,
                                  const float* __restrict__ T, const float* __restrict__ W,
                                  float* __restrict__ Q, float* __restrict__ KQ) {
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
__global__ void vsr_rescale_kernel(const FitState* __restrict__ st, int64_t nc,
                                   const float* __restrict__ sq, const float* __restrict__ Q,
                                   const float* __restrict__ KQ, float* __restrict__ S,
                                   float* __restrict__ T) {
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

__global__ void copy_int_kernel(const FitState* __restrict__ st, int* dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = st->B;
}

// -------------------------------------------------------------------- projections
// part[blk][k] = sum_{e in blk} Q[k][e] x[e]   for k < B   (warp per column)
__global__ void proj_partial_kernel(const FitState* __restrict__ st, int guard_inner,
                                    const float* __restrict__ Q, const float* __restrict__ x,
                                    int64_t nc, int bcap, double* __restrict__ part) {
  if (!st->newton_active || (guard_inner && !st->active)) return;
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

__global__ void proj_finalize_kernel(const FitState* __restrict__ st, int guard_inner,
                                     const double* __restrict__ part, int nblk, int bcap,
                                     float* __restrict__ w) {
  if (!st->newton_active || (guard_inner && !st->active)) return;
  const int B = st->B;
  for (int k = threadIdx.x; k < B; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[static_cast<int64_t>(b) * bcap + k];
    w[k] = static_cast<float>(s);
  }
}

// v = Q w, u = KQ w over the B0 recycled columns (v0 = C0 b, K v0)
__global__ void combine_kernel(const FitState* __restrict__ st, const float* __restrict__ Q,
                               const float* __restrict__ KQ, const float* __restrict__ w,
                               int64_t nc, float* __restrict__ v, float* __restrict__ u) {
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
__global__ void resid_kernel(const FitState* __restrict__ st, int64_t n, int C,
                             const float* __restrict__ b, const float* __restrict__ u,
                             const float* __restrict__ v, const float* __restrict__ inv_pi,
                             float* __restrict__ r, double* __restrict__ part, int project) {
  if (!st->newton_active || !st->active) return;
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* vi = v + i * C;
    const float* ipi = inv_pi + i * C;
    double m1 = 0.0;
    for (int c = 0; c < C; ++c) m1 += vi[c];
    m1 /= C;
    double m2 = 0.0;
    for (int c = 0; c < C; ++c) m2 += (vi[c] - m1) * static_cast<double>(ipi[c]);
    m2 /= C;
    double rm = 0.0;
    if (project) {
      for (int c = 0; c < C; ++c)
        rm += static_cast<double>(b[i * C + c]) - u[i * C + c] - ((vi[c] - m1) * ipi[c] - m2);
      rm /= C;
    }
    for (int c = 0; c < C; ++c) {
      const double rv = static_cast<double>(b[i * C + c]) - u[i * C + c] - ((vi[c] - m1) * ipi[c] - m2) - rm;
      r[i * C + c] = static_cast<float>(rv);
      acc += rv * rv;
    }
  }
  acc = block_reduce_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// commit the pending column; |r|; inner stopping test (App. B.2); alpha
__global__ void resid_finalize_kernel(FitState* st, const double* __restrict__ part, int nblk,
                                      const float* __restrict__ r, int64_t nc, int policy,
                                      int step) {
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

// s = r (CG) or e_{B0+j} (unit vectors) into the staging vector and S[:, B]
__global__ void action_kernel(const FitState* __restrict__ st, int64_t nc, int policy,
                              const float* __restrict__ r, float* __restrict__ s_cur,
                              float* __restrict__ S) {
  if (!st->newton_active || !st->active) return;
  float* col = S + static_cast<int64_t>(st->B) * nc;
  const int64_t idx = static_cast<int64_t>(st->B0) + st->j;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nc;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float sv = policy == ITERGP_POLICY_CG ? r[e] : (e == idx ? 1.f : 0.f);
    s_cur[e] = sv;
    col[e] = sv;
  }
}

// T[:, B] = t; z = t + W^+ s
__global__ void z_kernel(const FitState* __restrict__ st, int64_t n, int C,
                         const float* __restrict__ s_cur, const float* __restrict__ t_cur,
                         const float* __restrict__ inv_pi, float* __restrict__ z,
                         float* __restrict__ T) {
  if (!st->newton_active || !st->active) return;
  const int64_t nc = n * C;
  float* tcol = T + static_cast<int64_t>(st->B) * nc;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float w[kMaxC];
    winv_point(s_cur + i * C, inv_pi + i * C, C, w);
    for (int c = 0; c < C; ++c) {
      const float tv = t_cur[i * C + c];
      tcol[i * C + c] = tv;
      z[i * C + c] = tv + w[c];
    }
  }
}

// d = s - Q w -> Q[:, B] (unnormalised); K d = t - KQ w -> KQ[:, B]; partial eta = z.d
__global__ void direction_kernel(const FitState* __restrict__ st, int64_t nc,
                                 const float* __restrict__ s_cur, const float* __restrict__ t_cur,
                                 const float* __restrict__ z, const float* __restrict__ w,
                                 float* __restrict__ Q, float* __restrict__ KQ, int track_kd,
                                 double* __restrict__ part) {
  if (!st->newton_active || !st->active) return;
  __shared__ double sh[32];
  const int B = st->B;
  float* qcol = Q + static_cast<int64_t>(B) * nc;
  float* kcol = KQ + static_cast<int64_t>(B) * nc;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nc;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float d = s_cur[e], kd = t_cur[e];
    for (int k = 0; k < B; ++k) {
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

__global__ void eta_finalize_kernel(FitState* st, const double* __restrict__ part, int nblk) {
  if (threadIdx.x != 0 || !st->newton_active || !st->active) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b];
  st->eta = s;
  if (!(s > 0.0)) {
    st->active = 0;
    st->stop_reason = ITERGP_STOP_ETA;
    return;
  }
  st->coef = st->alpha / s;
  st->inv_sqrt_eta = 1.0 / sqrt(s);
  st->pending = 1;
  st->j += 1;
  st->total_iters += 1;
}

// Q[:, B] /= sqrt(eta); KQ[:, B] /= sqrt(eta); v += (alpha/eta) d; u += (alpha/eta) K d
__global__ void update_kernel(const FitState* __restrict__ st, int64_t nc, float* __restrict__ Q,
                              float* __restrict__ KQ, float* __restrict__ v, float* __restrict__ u,
                              int track_kd) {
  if (!st->newton_active || !st->active) return;
  const int B = st->B;
  const float coef = static_cast<float>(st->coef), ise = static_cast<float>(st->inv_sqrt_eta);
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
__global__ void step_end_kernel(FitState* st, int step) {
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
__global__ void copy_f_kernel(const FitState* __restrict__ st, int64_t nc, const float* __restrict__ u,
                              float* __restrict__ f) {
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

__global__ void sym_eig_kernel(const double* __restrict__ M, int b, double* __restrict__ lam,
                               double* __restrict__ U, double* __restrict__ A, double* __restrict__ V) {
  extern __shared__ double dsh[];
  double* cs = dsh;
  double* sn = cs + b / 2 + 1;
  double* red = sn + b / 2 + 1;
  int* partner = reinterpret_cast<int*>(red + 32);
  int* role = partner + b + 1;
  int* order = role + b + 1;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    A[i * b + j] = 0.5 * (M[i * b + j] + M[j * b + i]);
  }
  __syncthreads();
  jacobi_eig(A, V, b, b, cs, sn, partner, role, red);
  eig_order(A, b, b, order);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, k = e % b;
    U[i * b + k] = V[i * b + order[k]];
  }
  for (int k = threadIdx.x; k < b; k += blockDim.x) lam[k] = A[order[k] * b + order[k]];
}

inline size_t eig_smem_bytes(int b) {
  return sizeof(double) * (2 * (b / 2 + 1) + 32) + sizeof(int) * (3 * (b + 1));
}

}  // namespace

// ======================================================================= host side

int fit_run(DeviceContext* ctx, const itergp_fit_params& prm, const KParams& kp,
            const RowOperand& Xop, const int32_t* y, float* v, float* f, float* Q, int bcap,
            cudaStream_t stream, itergp_fit_report* rep, int* final_B) {
  const int64_t n = prm.n;
  const int C = prm.c;
  const int64_t nc = n * C;
  const int nblk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(2LL * ctx->num_sms, ceil_div(n, 256))));
  const int nblk_e = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(2LL * ctx->num_sms, ceil_div(nc, 1024))));
  const int gram_splits = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(64, ceil_div(nc, 4096))));
  const int64_t gram_per_split = ceil_div(nc, gram_splits);
  const int eb = static_cast<int>(std::min<int64_t>(ceil_div(nc, 256), 8LL * ctx->num_sms));
  const int nb_pts = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 8LL * ctx->num_sms));
  const int track_kd = prm.literal_kv ? 0 : 1;
  const int project = prm.policy == ITERGP_POLICY_CG ? 1 : 0;

  // ---- workspace
  const size_t vec = align_up(sizeof(float) * nc, 256);
  const size_t buf = align_up(sizeof(float) * nc * bcap, 256);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes, 256); return o; };
  const size_t o_state = take(sizeof(FitState));
  const size_t o_S = take(buf), o_T = take(buf), o_KQ = take(buf);
  const size_t o_u = take(vec), o_b = take(vec), o_r = take(vec), o_z = take(vec), o_gp = take(vec),
               o_ip = take(vec), o_s = take(vec), o_t = take(vec);
  const size_t o_w = take(sizeof(float) * bcap), o_sq = take(sizeof(float) * bcap);
  const size_t o_W = take(sizeof(float) * bcap * bcap);
  const size_t o_A = take(sizeof(double) * bcap * bcap), o_V = take(sizeof(double) * bcap * bcap);
  const size_t o_pg = take(sizeof(double) * gram_splits * bcap * bcap);
  const size_t o_pv = take(sizeof(double) * std::max(nblk_e, nblk) * bcap);
  const size_t o_ps = take(sizeof(double) * 5 * std::max(nblk_e, nblk));
  const size_t o_bold = take(sizeof(int));
  Scratch ws;
  ITERGP_CUDA_TRY(ws.alloc(ctx, off, stream));
  char* base = ws.as<char>();
  FitState* st = reinterpret_cast<FitState*>(base + o_state);
  float* S = reinterpret_cast<float*>(base + o_S);
  float* T = reinterpret_cast<float*>(base + o_T);
  float* KQ = reinterpret_cast<float*>(base + o_KQ);
  float* u = reinterpret_cast<float*>(base + o_u);
  float* b = reinterpret_cast<float*>(base + o_b);
  float* r = reinterpret_cast<float*>(base + o_r);
  float* z = reinterpret_cast<float*>(base + o_z);
  float* gp = reinterpret_cast<float*>(base + o_gp);
  float* ip = reinterpret_cast<float*>(base + o_ip);
  float* s_cur = reinterpret_cast<float*>(base + o_s);
  float* t_cur = reinterpret_cast<float*>(base + o_t);
  float* w = reinterpret_cast<float*>(base + o_w);
  float* sq = reinterpret_cast<float*>(base + o_sq);
  float* W = reinterpret_cast<float*>(base + o_W);
  double* Am = reinterpret_cast<double*>(base + o_A);
  double* Vm = reinterpret_cast<double*>(base + o_V);
  double* pg = reinterpret_cast<double*>(base + o_pg);
  double* pv = reinterpret_cast<double*>(base + o_pv);
  double* ps = reinterpret_cast<double*>(base + o_ps);
  int* bold = reinterpret_cast<int*>(base + o_bold);

  FitState init{};
  init.newton_active = 1;
  ITERGP_CUDA_TRY(cudaMemcpyAsync(st, &init, sizeof(FitState), cudaMemcpyHostToDevice, stream));
  ITERGP_CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(float) * nc, stream));
  ITERGP_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(float) * nc, stream));
  ITERGP_CUDA_TRY(cudaMemsetAsync(u, 0, sizeof(float) * nc, stream));
  ITERGP_CUDA_TRY(cudaMemsetAsync(gp, 0, sizeof(float) * nc, stream));

  const int* active = &st->active;
  const size_t eig_smem = eig_smem_bytes(bcap);
  const int eig_threads = 512;

  for (int step = 0; step < prm.max_newton; ++step) {
    newton_prologue_kernel<<<nblk, kRedThreads, 0, stream>>>(st, n, C, f, y, v, gp, ip, b, ps, ctx->status, project), ::itergp::note_launch();
    newton_finalize_kernel<<<1, 32, 0, stream>>>(st, ps, nblk, step, prm.tol_newton, prm.tol_abs, prm.tol_rel, prm.recycle), ::itergp::note_launch();
    // ---- Alg. 3: virtual solver run with compression
    if (prm.recycle && step > 0) {
      copy_int_kernel<<<1, 1, 0, stream>>>(st, bold), ::itergp::note_launch();
      vsr_z_kernel<<<eb, 256, 0, stream>>>(st, n, C, nc, S, T, ip, Q), ::itergp::note_launch();
      dim3 gg(ceil_div(bcap, kGT), ceil_div(bcap, kGT), gram_splits);
      gram_partial_kernel<<<gg, 256, 0, stream>>>(st, S, Q, nc, bcap, gram_per_split, pg), ::itergp::note_launch();
      vsr_eig_kernel<<<1, eig_threads, eig_smem, stream>>>(st, pg, gram_splits, bcap, prm.rank, Am, Vm, W, sq, step), ::itergp::note_launch();
      vsr_rotate_kernel<<<eb, 256, 0, stream>>>(st, bold, nc, bcap, S, T, W, Q, KQ), ::itergp::note_launch();
      vsr_rescale_kernel<<<eb, 256, 0, stream>>>(st, nc, sq, Q, KQ, S, T), ::itergp::note_launch();
      // v0 = Q0 (Q0^T b), u0 = K v0 = KQ0 (Q0^T b)
      proj_partial_kernel<<<nblk_e, 256, 0, stream>>>(st, 0, Q, b, nc, bcap, pv), ::itergp::note_launch();
      proj_finalize_kernel<<<1, 256, 0, stream>>>(st, 0, pv, nblk_e, bcap, w), ::itergp::note_launch();
    }
    // v0 = C0 (y_hat - m) and K v0; with no recycled columns (B = 0) both are zero
    combine_kernel<<<eb, 256, 0, stream>>>(st, Q, KQ, w, nc, v, u), ::itergp::note_launch();
    // ---- Alg. 2 iterations
    for (int j = 0; j < prm.max_iters; ++j) {
      if (prm.literal_kv) {
        int rc = kmv_execute(ctx, kp, Xop, Xop, v, C, C, u, C, stream, active);
        if (rc != ITERGP_OK) return rc;
      }
      resid_kernel<<<nblk, kRedThreads, 0, stream>>>(st, n, C, b, u, v, ip, r, ps, project), ::itergp::note_launch();
      resid_finalize_kernel<<<1, 32, 0, stream>>>(st, ps, nblk, r, nc, prm.policy, step), ::itergp::note_launch();
      action_kernel<<<eb, 256, 0, stream>>>(st, nc, prm.policy, r, s_cur, S), ::itergp::note_launch();
      int rc = kmv_execute(ctx, kp, Xop, Xop, s_cur, C, C, t_cur, C, stream, active);
      if (rc != ITERGP_OK) return rc;
      z_kernel<<<nb_pts, 256, 0, stream>>>(st, n, C, s_cur, t_cur, ip, z, T), ::itergp::note_launch();
      proj_partial_kernel<<<nblk_e, 256, 0, stream>>>(st, 1, Q, z, nc, bcap, pv), ::itergp::note_launch();
      proj_finalize_kernel<<<1, 256, 0, stream>>>(st, 1, pv, nblk_e, bcap, w), ::itergp::note_launch();
      direction_kernel<<<nblk_e, kRedThreads, 0, stream>>>(st, nc, s_cur, t_cur, z, w, Q, KQ, track_kd, ps), ::itergp::note_launch();
      eta_finalize_kernel<<<1, 32, 0, stream>>>(st, ps, nblk_e), ::itergp::note_launch();
      update_kernel<<<eb, 256, 0, stream>>>(st, nc, Q, KQ, v, u, track_kd), ::itergp::note_launch();
    }
    step_end_kernel<<<1, 32, 0, stream>>>(st, step), ::itergp::note_launch();
    if (prm.literal_kv) {
      // f_{i+1} = K v + m by a fresh product
      int rc = kmv_execute(ctx, kp, Xop, Xop, v, C, C, u, C, stream, &st->newton_active);
      if (rc != ITERGP_OK) return rc;
    }
    copy_f_kernel<<<eb, 256, 0, stream>>>(st, nc, u, f), ::itergp::note_launch();
  }
  ITERGP_CUDA_TRY(cudaGetLastError());

  FitState hs;
  ITERGP_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(FitState), cudaMemcpyDeviceToHost, stream));
  ITERGP_CUDA_TRY(cudaStreamSynchronize(stream));
  if (rep) {
    rep->newton_steps = hs.newton_steps;
    rep->total_iters = hs.total_iters;
    rep->buffer_cols = hs.B;
    rep->stop_reason = hs.stop_reason;
    for (int i = 0; i < ITERGP_MAX_REPORT_STEPS; ++i) {
      rep->iters[i] = hs.iters[i];
      rep->stops[i] = hs.stops[i];
      rep->kept[i] = hs.kept[i];
      rep->objective[i] = hs.objective[i];
      rep->rel_change[i] = hs.rel_change[i];
    }
    rep->resid_norm = hs.rnorm;
  }
  *final_B = hs.B;
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
  sym_eig_kernel<<<1, 512, smem, s>>>(M, b, lam, U, A, V), ::itergp::note_launch();
  ITERGP_CUDA_TRY(cudaGetLastError());
  return ITERGP_OK;
}

}  // namespace itergp
