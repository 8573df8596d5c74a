/*
 * tpc_probe.h -- measurement helper of libtpcgpu.so: arithmetic-throughput
 * probes that give the roofline denominators of the Kalman stages (binary32
 * and binary64 fused multiply-add rates of this GPU).  The paper has no
 * counterpart; the tracker never calls them.
 */
#ifndef TPC_PROBE_H
#define TPC_PROBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Enqueue one launch of `blocks` x `threads` threads, each running 8
 * independent chains of `iters` fused multiply-adds (x = x * a + b) in
 * binary32 (precision 32) or binary64 (precision 64), and writing one value
 * per block to `out` (device, `blocks` floats or doubles, caller-owned) so
 * that no work can be elided.  *flops (host) receives the flops the launch
 * executes (2 per multiply-add).  The caller times the launch (CUDA events on
 * `stream`).  Errors: TPC_ERR_ARG (precision not 32 or 64, blocks outside
 * [1, 2^20], threads outside [32, 1024] or not a multiple of 32, iters
 * outside [1, 2^24], null out or flops), TPC_ERR_CUDA. */
int tpc_probe_fma(int32_t precision, int32_t blocks, int32_t threads, int32_t iters, void *out, int64_t *flops,
                  void *stream);

#ifdef __cplusplus
}
#endif
#endif
