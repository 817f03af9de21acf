/*
 * fusedpr_diag.h -- diagnostics exported by libfusedpr.so beside the C ABI of
 * fusedpr.h.  They compute nothing of the method: a gather-rate probe that
 * measures the ceiling the sweep is held against, and a launch counter.
 * Same conventions as fusedpr.h (status codes, streams, no CPU fallback).
 */
#ifndef FUSEDPR_DIAG_H
#define FUSEDPR_DIAG_H

#include "fusedpr.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Diagnostic (no counterpart in the paper, computes nothing of the method):
 * *sink += sum over j < m of y[idx[j]], with the sweep's access pattern
 * (16-byte index loads kept out of L1, eight gathers in flight per lane, the
 * first `hot` entries of y read from shared memory, one 1024-thread block
 * per SM).  Timed by the caller, it gives the rate at which this device
 * serves the sweep's irregular gathers alone.
 *   idx   device int32 [m], 16-byte aligned (PR_ERR_INVALID_ARG otherwise);
 *         an entry outside [0, n) gathers y[0] instead
 *   y     device float [n];  hot: 0 <= hot <= min(n, 49152)
 *   sink  device float [1], accumulated with atomics
 * Returns without synchronising.
 */
pr_status pr_gather_probe(const int32_t *idx, int64_t m, const float *y, int32_t n, int32_t hot,
                          float *sink, void *stream);

/* Number of CUDA kernels the library has launched in this process so far
 * (each iteration of a device-side loop counts as one launch).  Diagnostics
 * only; no device work. */
uint64_t pr_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* FUSEDPR_DIAG_H */
