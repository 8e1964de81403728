// CTA-pair form of the tensor-core kernel product (instantiations of kmv_tc_kernel with
// PAIR = true, see kmv_tc_impl.cuh): clusters of two CTAs on two SMs share each 256-row
// tile of A.  The even CTA's MMA thread issues cta_group::2 tcgen05.mma of M = 256 for
// both SMs, so the single issuing thread, which bounds the one-CTA form, issues half the
// instructions per unit of work; each CTA stages 128 rows of A and 64 rows of every B
// chunk (with 128-byte swizzle, as in the one-CTA form), and each CTA's accumulator rows
// stay in its own TMEM.  The arithmetic per output element (MMA order, flush cadence,
// epilogue) is the one-CTA form's.  The wide variant takes chunks of 192 rows of B (MMA
// N = 192, 96 rows staged per CTA) and keeps the flushed running sum in registers.
#include "kmv_tc_impl.cuh"

namespace itergp {
namespace tcimpl {

cudaError_t launch_pair_form(int kind, int prec, int nstage, int epi, int grid_pairs, size_t smem, cudaStream_t st,
                             const CUtensorMap* maps, const TcArgs& a, int cw) {
  if (cw == kWideCW)
    return kind == ITERGP_RBF
               ? launch_prec<ITERGP_RBF, true, kWideCW>(prec, nstage, false, epi, grid_pairs, smem, st, maps, a)
               : launch_prec<ITERGP_MATERN32, true, kWideCW>(prec, nstage, false, epi, grid_pairs, smem, st, maps, a);
  return kind == ITERGP_RBF
             ? launch_prec<ITERGP_RBF, true>(prec, nstage, false, epi, grid_pairs, smem, st, maps, a)
             : launch_prec<ITERGP_MATERN32, true>(prec, nstage, false, epi, grid_pairs, smem, st, maps, a);
}

int pair_max_clusters(int kind, int prec, int nstage, int epi, size_t smem, int cw) {
  const CUtensorMap maps[6] = {};
  const TcArgs a{};
  int n = 0;
  cudaError_t e;
  if (cw == kWideCW)
    e = kind == ITERGP_RBF
            ? launch_prec<ITERGP_RBF, true, kWideCW>(prec, nstage, false, epi, 1, smem, nullptr, maps, a, &n)
            : launch_prec<ITERGP_MATERN32, true, kWideCW>(prec, nstage, false, epi, 1, smem, nullptr, maps, a, &n);
  else
    e = kind == ITERGP_RBF ? launch_prec<ITERGP_RBF, true>(prec, nstage, false, epi, 1, smem, nullptr, maps, a, &n)
                           : launch_prec<ITERGP_MATERN32, true>(prec, nstage, false, epi, 1, smem, nullptr, maps, a, &n);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace tcimpl
}  // namespace itergp
