/* Throughput probes of the GB300's units (libitergp_probe.so): measurement tooling of the
 * bench, not part of the product library libitergp.so.  The paper has no counterpart; the
 * rates are the denominators of the product's roofline where no measured peak
 * exists (MUFU, FFMA, FP64, TF32 and the exact MMA shapes the product issues).
 *
 * itergp_probe_throughput: operations per second over the whole GPU on the current
 * device, timed with CUDA events on `stream` (it waits for the stream).
 *   what = 0: MUFU exp2 (ex2.approx); 1: FP32 FFMA (2 flops each); these bound the kernel
 *             product when D is small (one exp per kernel value).
 *   what = 2..6: tcgen05.mma flops (FP32 accumulate), one CTA per SM issuing back to back
 *             from one thread, in the shapes of the one-CTA product: 2 = SS M = 128,
 *             N = 128, BF16 (the distance GEMM); 3 = SS M = 128, N = 256; 4 = as 2 while
 *             four other warps stream tcgen05.ld (the epilogue's reads); 5 = TS (A from
 *             TMEM) M = 128, N = 80 (the weighted sum); 6 = as 2 with TF32 operands
 *             (kind::tf32, K = 8).
 *   what = 7: FP64 DFMA (2 flops each); 8: MUFU rsqrt (rsqrt.approx, Matern's distance).
 *   what = 9..11: the CTA-pair form (clusters of two CTAs; the even CTA issues
 *             cta_group::2 MMAs of M = 256 for both SMs, each SM holding 128 rows of A and
 *             half of B): 9 = SS N = 128, FP16 (the pair form's distance GEMM); 10 = SS
 *             N = 256; 11 = TS N = 80 (the pair form's weighted sum); 12 = SS N = 192,
 *             FP16 (the wide pair form's distance GEMM).
 *   what = 13, 14: the pair form's distance GEMM fed by a TMA ring (3 stages of K = 64, A and
 *             B hi/lo refilled from a 64 MB array through full/empty barriers, the
 *             product's three-term MMA order, no epilogue): 13 = N = 128, 14 = N = 192.
 *             Allocates (and frees) the 64 MB source array.
 * Returns ITERGP_EINVAL for another `what` or a null result, ITERGP_ETIMEOUT if a probe's
 * bounded wait (2 s) ran out, ITERGP_ENOMEM / ITERGP_ECUDA on a CUDA error. */
#ifndef ITERGP_PROBE_H
#define ITERGP_PROBE_H
#include <stdint.h>

#include "itergp.h"

#ifdef __cplusplus
extern "C" {
#endif

int itergp_probe_throughput(int32_t what, double* ops_per_s, itergp_stream stream);

#ifdef __cplusplus
}
#endif
#endif
