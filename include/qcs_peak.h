/*
 * qcs_peak.h -- measurement utility shipped beside libqcs (libqcs_peak.so):
 * the sustained 32-bit integer multiply-add (IMAD) and byte dot-product
 * (dp4a) throughput of the current GPU, used as the integer-ALU roofline of
 * the walk kernel, whose dominant work is multiply-adds.  The paper has no counterpart; it is not part
 * of the search.
 */
#ifndef QCS_PEAK_H
#define QCS_PEAK_H

#include <stdint.h>

#if defined(__GNUC__)
#define QCS_PEAK_API __attribute__((visibility("default")))
#else
#define QCS_PEAK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Runs `blocks_per_sm` x (number of SMs) CTAs of 256 threads, each thread
 * executing `iters` x 128 independent IMADs (8 chains), on the legacy default
 * stream, and reports the achieved IMAD/s (*imad_per_s) and the kernel time
 * (*ms, CUDA events).  Returns 0, or a negative cudaError_t on failure.  No
 * allocation outlives the call. */
QCS_PEAK_API int qcs_peak_imad(int blocks_per_sm, int iters, double *imad_per_s, double *ms);

/* Same for the 32-bit integer add / logic pipe (IADD3 chains). */
QCS_PEAK_API int qcs_peak_iadd(int blocks_per_sm, int iters, double *iadd_per_s, double *ms);

/* Same for the four-way byte dot product with accumulate (dp4a, unsigned
 * bytes times signed bytes), the instruction of the walk kernel's byte-plane
 * contraction; reports dp4a instructions per second. */
QCS_PEAK_API int qcs_peak_idp4a(int blocks_per_sm, int iters, double *dp4a_per_s, double *ms);

/* Legacy warp-level tensor-core MMA rates (mma.sync), reported as
 * multiply-adds per second: f16 x f16 with f32 accumulation (m16n8k16), the
 * form an exact small-integer contraction could take, and u8 x s8 with s32
 * accumulation (m16n8k32).  Same launch and return convention as above. */
QCS_PEAK_API int qcs_peak_hmma(int blocks_per_sm, int iters, double *mac_per_s, double *ms);
QCS_PEAK_API int qcs_peak_imma(int blocks_per_sm, int iters, double *mac_per_s, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* QCS_PEAK_H */
