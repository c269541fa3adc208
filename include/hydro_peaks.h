/*
 * hydro_peaks.h — measured peak rate of the arithmetic pipes that bound the
 * patch-group kernels.
 *
 * The unsplit schemes (Sec. 2; the paper calls them arithmetic-intensive,
 * Sec. 3.2) are bound by plain FP32 / FP64 arithmetic, not by a dense
 * contraction and not by HBM, so their roofline denominator is the rate at
 * which the GPU retires fused multiply-adds.  This call launches a kernel of
 * independent FMA chains whose flop count is known exactly; the caller times
 * the launch (CUDA events on `stream`) and divides.
 */
#ifndef HYDRO_PEAKS_H
#define HYDRO_PEAKS_H

#include "hydro.h"

#ifdef __cplusplus
extern "C" {
#endif

#define HYDRO_PEAK_FP32 0   /* fma.rn.f32: 2 flops per instruction per thread        */
#define HYDRO_PEAK_FP32X2 1 /* fma.rn.f32x2 (packed pair): 4 flops per instruction   */
#define HYDRO_PEAK_FP64 2   /* fma.rn.f64: 2 flops per instruction per thread        */

/*
 * hydro_fma_peak — enqueue one FMA-loop launch of `ctas` CTAs x `threads`
 * threads, each thread running 8 independent chains for `iters` iterations.
 *   kind     HYDRO_PEAK_FP32 / HYDRO_PEAK_FP32X2 / HYDRO_PEAK_FP64.
 *   out      device buffer of ctas * threads elements (float for the FP32
 *            kinds, double for FP64), caller-owned; receives one sum per
 *            thread (meaningless values; written so the loop is kept).
 *   stream   cudaStream_t or NULL.
 *   flops_per_launch  (host, may be NULL) the exact flop count of the
 *            launch: 2 x 8 x iters x ctas x threads (x 2 for the packed kind).
 * Returns HYDRO_OK, HYDRO_EINVAL (kind, a size or out invalid; threads must
 * be a multiple of 32 in [32, 1024]) or HYDRO_ECUDA (launch failed; see
 * hydro_last_cuda_error).  Allocates nothing.
 */
int hydro_fma_peak(int kind, int ctas, int threads, int iters, void* out, void* stream, double* flops_per_launch);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_PEAKS_H */
