/*
 * cqprobe — measurement probe that comes with the fastcq library (a separate
 * shared library, libcqprobe.so). It measures the FMA rates that bound the
 * FP64 and FP32 fast solves on the GPU it runs on; the paper has no counterpart.
 */
#ifndef CQPROBE_H
#define CQPROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sustained fused multiply-add rate of one precision (prec 0: FP64 DFMA, 1: FP32
 * FFMA): a grid of `blocks` x `threads` threads (32 <= threads <= 256, a multiple
 * of 32), each running 8 independent FMA chains for `iters` rounds, is launched
 * once to warm up and once timed with CUDA events on `stream` (synchronises it).
 * out_dev: caller-owned device buffer of blocks * threads doubles (prec 0) or
 * floats (prec 1) that receives the chains' sums. *flops_per_s_host = 2 * 8 *
 * iters * blocks * threads / time. Returns 0, -1 for invalid arguments, -3 for a
 * CUDA error. */
int cq_probe_fma_rate(int32_t prec, int32_t blocks, int32_t threads, int32_t iters, void *out_dev,
                      double *flops_per_s_host, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CQPROBE_H */
