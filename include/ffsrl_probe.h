/*
 * ffsrl_probe.h - on-chip peak probes of libffsrl.so.
 *
 * The step kernel of the batched XPBD simulator is bound by shared-memory
 * bandwidth and FP32 issue, not by HBM: every env's positions stay in shared
 * memory for a whole step while the coloured constraint passes gather them
 * (FF-SRL, arXiv 2503.18616, Sec. III-A, Algorithm 1, run as colour
 * Gauss-Seidel). These two calls measure the device's own ceilings for those
 * resources, so that the kernel's fractions are taken against measured
 * numbers and not nominal ones. The paper has no counterpart: they are
 * measurement infrastructure.
 *
 * Both run on the current CUDA device, on their own stream, synchronously,
 * and allocate a small device buffer (freed before returning). Each launches
 * a warm-up and then `repeats` timed launches (CUDA events), and returns the
 * best rate. Return: 0 on success, FFSRL_E_INVAL (-1) for repeats < 1,
 * FFSRL_E_CUDA (-2) on a CUDA error; ffsrl_last_error() gives the message.
 */
#ifndef FFSRL_PROBE_H
#define FFSRL_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* FP32 fused multiply-add throughput: every thread of two 1024-thread CTAs
 * per SM runs eight independent FMA chains. *tflops = 2 x FMAs / time
 * (TFLOP/s), *ms = the best launch's duration. */
int ffsrl_probe_fp32(int32_t repeats, double* tflops, double* ms);

/* Shared-memory load bandwidth: every thread of two 1024-thread CTAs per SM
 * reads 16-byte words whose quarter-warp addresses cover whole 128-byte lines
 * (no bank conflicts). *gbs = bytes loaded / time (GB/s), *ms as above. */
int ffsrl_probe_smem(int32_t repeats, double* gbs, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* FFSRL_PROBE_H */
