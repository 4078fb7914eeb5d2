/*
 * Measurement helpers of the mgpu library (not part of the matrix-element
 * method).
 */
#ifndef MGPU_BENCH_H
#define MGPU_BENCH_H

#ifdef __cplusplus
extern "C" {
#endif

/* FP64 fused multiply-add throughput of the current device.  Launches
 * `blocks` x 256 threads that each run `iters` rounds of 16 independent FMA
 * chains (no memory traffic), times `reps` launches with CUDA events on a
 * private stream after one warm-up, and writes the best rate in FP64 flops/s
 * (FMA = 2 flops) to *flops_out.  blocks <= 0 picks 8 per SM.  Returns 0 or
 * a negative mgpu status (MG_ERR_CUDA on a CUDA failure). */
int mg_probe_fp64_peak(int blocks, int iters, int reps, double *flops_out);

/* Test hook for the bounded waits of the tensor-core colour sum: every CTA's
 * operand barrier then expects extra_bytes more than its copies deliver, so
 * the wait runs out (about a second), the kernel records a timeout and
 * returns; mg_device_status reports MG_ERR_DEVICE_TIMEOUT.  0 disables. */
struct mg_process;
int mg_debug_inject_stall(struct mg_process *p, unsigned int extra_bytes);

/* Copies an internal buffer of the surrogate's last forward/backward pass to
 * the host as FP32 out[rows][cols] (padded widths): which = 0 activations of
 * layer input `layer` (0 = features), 1 pre-activations, 2 FP32 output
 * gradients of layer `layer`. */
struct mg_surrogate;
int mg_sur_debug_buffer(struct mg_surrogate *s, int which, int layer, int rows, float *out);

#ifdef __cplusplus
}
#endif
#endif
