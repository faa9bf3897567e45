/*
 * qb_diag -- diagnostics and measurement helpers of the qb library.  Neither
 * call computes anything of the paper's method (arXiv:2111.00050 has no
 * counterpart); they serve error-path tests and the roofline denominators of
 * the benchmark.  Conventions as in qb.h (status codes, void* streams).
 */
#ifndef QB_DIAG_H
#define QB_DIAG_H

#include "qb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Device status word of a space.  The kernels of a space record failed
 * device-side checks in one 32-bit word on the device, without faulting:
 *   bit 0  a gathered index fell outside its sector (the access was skipped or
 *          sent to row 0),
 *   bit 1  a ket's rank recomputed from its occupations disagreed with its index,
 *   bit 2  a resident sector did not fit its shared-memory buffers.
 * Every call that synchronises reads the word; a nonzero word is cleared and the
 * call returns QB_EINTERNAL.  qb_space_status first ORs set_bits into the word on
 * the host side (a device-to-host read, OR, host-to-device write, ordered on
 * `stream`; 0 leaves the word alone), then writes the word to *status (host, may
 * be NULL) without clearing it.  A nonzero set_bits lets a test exercise the error
 * path of the next call without any device fault.  Synchronises the stream. */
int qb_space_status(qb_space* space, int set_bits, int* status, void* stream);

/* FP64 fused multiply-add rate of the current GPU, for the roofline denominator
 * of FP64-equivalent work: a grid of 8 CTAs per SM of 256 threads, each running 8
 * independent DFMA chains of 2048 dependent operations, timed with CUDA events on
 * `stream` (best of `reps` >= 1 launches after one untimed launch).
 * *tflops (host) receives 2 x FMAs / second / 1e12.  Allocates and frees 2.5 MB
 * of device memory.  Synchronises the stream. */
int qb_measure_fp64_fma(int reps, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QB_DIAG_H */
