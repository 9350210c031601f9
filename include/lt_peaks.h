/* Roofline denominators measured on the running GPU (no counterpart in the
 * paper).
 *
 * The projector kernels are bound on chip (shared-memory and L1 operand
 * traffic, FP32 issue), not by DRAM, so their roofline needs the peaks of
 * those levels.  Each call below launches one microbenchmark kernel on
 * `stream` and reports the algorithmic work it performs; the caller times
 * the launch with CUDA events on the same stream and divides.  The kernels
 * read only what they are given, change no device setting and run a bounded
 * amount of work.
 *
 *   lt_peak_smem_read   every CTA fills 32 KiB of shared memory once, then
 *                       reads it `reps` times with conflict-free 16-byte
 *                       loads; *bytes = bytes read from shared memory.
 *   lt_peak_l2_read     reads the device buffer buf[n16] of 16-byte words
 *                       `reps` times with L1-bypassing 16-byte loads (the
 *                       buffer should fit in L2, so that the repeats hit
 *                       it); *bytes = bytes read.  buf must be 16-byte
 *                       aligned.
 *   lt_peak_fp32_fma    independent FP32 FMA chains, `reps` rounds of 8 per
 *                       thread; *flops = 2 x FMAs.
 *
 * ctas: grid size (a multiple of the SM count is best); threads per CTA are
 * fixed (256).  sink: device float[ctas * 256] that receives one value per
 * thread so that the work cannot be removed.  Errors: LT_EINVAL for NULL
 * pointers or non-positive sizes, LT_ECUDA for a failed launch. */
#ifndef LT_PEAKS_H
#define LT_PEAKS_H

#include "lt.h"

#ifdef __cplusplus
extern "C" {
#endif

LT_API lt_status lt_peak_smem_read(float* sink, int32_t ctas, int32_t reps, void* stream, double* bytes);
LT_API lt_status lt_peak_l2_read(const void* buf, int64_t n16, float* sink, int32_t ctas, int32_t reps,
                                 void* stream, double* bytes);
LT_API lt_status lt_peak_fp32_fma(float* sink, int32_t ctas, int32_t reps, void* stream, double* flops);

#ifdef __cplusplus
}
#endif

#endif
