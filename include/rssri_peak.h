/*
 * rssri_peak.h - arithmetic-pipe peak measurement exported by librssri.so.
 *
 * The paper has no counterpart to this entry point: it measures the ceilings
 * that the library's fp64 and double-float kernels are reported against
 * (their roofline denominators), on the GPU the library runs on, so that no
 * peak has to be derived from an instruction recipe.
 */
#ifndef RSSRI_PEAK_H
#define RSSRI_PEAK_H

#include "rssri.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RSSRI_PEAK_DFMA = 0, /* fp64 fused multiply-add pipe (DFMA), 2 flop per FMA          */
  RSSRI_PEAK_DMMA = 1, /* fp64 mma.sync m8n8k4, 512 flop per warp instruction         */
  RSSRI_PEAK_FFMA = 2  /* fp32 fused multiply-add pipe (FFMA), 2 flop per FMA          */
};

/* Run compute-only kernels on every SM of `device` in several shapes (4 to 16
 * independent dependency chains per thread, 16 to 64 resident warps per SM,
 * shared or distinct operand registers), time each with CUDA events on the
 * legacy default stream (one warm-up and three timed launches of ~10 ms),
 * and return the best rate in TFLOP/s (*tflops) and that shape's mean launch
 * time in ms (*ms, may be NULL).  Allocates and frees one small device
 * buffer; makes `device` current; synchronises; takes about a second.
 * Errors: INVALID_ARG (unknown `which`, null tflops), OOM, CUDA. */
RSSRI_API int rssri_peak_measure(int which, int device, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* RSSRI_PEAK_H */
