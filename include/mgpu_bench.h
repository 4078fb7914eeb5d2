/*
 * Measurement helpers of the mgpu library (not part of the matrix-element
 * method).
 */
#ifndef MGPU_BENCH_H
#define MGPU_BENCH_H

#include <stdint.h>

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

/* Test hook for the jamp buffer of the diagram kernel (processes compiled
 * into the library): enable = 0 makes later calls on p update the jamps in
 * place in local memory instead of through FP64 reductions at L2 into the
 * per-process jamp buffer; 1 (the default) restores the buffer.  Both paths
 * form every jamp as the same sum in the same order, so their results are
 * bit-identical.  max_bytes > 0 replaces the buffer limit (24 GiB; an FP64
 * call whose buffer would exceed it runs as several launches of whole waves
 * of events, or of as many events as fit), 0 restores it.  Returns MG_OK or
 * MG_ERR_BAD_ARG (p NULL, max_bytes < 0). */
int mg_debug_jamp_buffer(struct mg_process *p, int enable, int64_t max_bytes);

/* The same test hook for the surrogate's tensor-core GEMMs: every later GEMM
 * launch of s makes its operand barrier expect extra_bytes more than its TMA
 * copies deliver, so the MMA thread's bounded wait runs out (about a second
 * per launch), the CTA records the timeout, frees its tensor memory and
 * returns; mg_sur_device_status then reports MG_ERR_DEVICE_TIMEOUT.  0
 * disables. */
struct mg_surrogate;
int mg_sur_debug_inject_stall(struct mg_surrogate *s, unsigned int extra_bytes);

/* Kernel timing of one process.  mg_set_kernel_timing(p, n) with n > 0
 * creates n CUDA event pairs; every later mg_sigmakin or mg_sigmakin_hel
 * call on p then records a pair on the caller's stream around each of its
 * kernel launches.  n = 0 switches timing off and destroys the
 * events.  mg_kernel_times waits for the last recorded event and writes per
 * kind (0 diagram kernel, 1 colour-sum kernel: the tensor-core one of the
 * mixed path or the FP64 one of a table-file process, 2 per-event sum) the summed device milliseconds ms_out[3] and the
 * launch counts launches_out[3] since the last reset; reset != 0 starts
 * over.  More than n launches between resets: MG_ERR_UNSUPPORTED (nothing
 * is reported).  Not thread-safe per process, like the other calls. */
int mg_set_kernel_timing(struct mg_process *p, int max_launches);
int mg_kernel_times(struct mg_process *p, int reset, double *ms_out, int *launches_out);

/* Number of kernel launches the library has issued since it was loaded
 * (every process and stream; the FP64 peak probe and replays of captured CUDA
 * graphs not included).  For counting the launches of a timed region. */
int mg_launch_count(unsigned long long *out);

/* Test hook for the tensor-core colour sum (mixed-precision processes): for
 * caller rows rows_dev[nrows][ncolor] (FP64, device; nrows a multiple of
 * 128), writes q8_dev[nrows / 8] = the sum over each 8 consecutive rows v of
 * v^T (D C) v, through the same BF16 splitting, tensor-core kernel (single
 * tile up to 128 flows, block-triangular above) and fixed-order sums as the
 * matrix-element path.  Allocates its workspace; synchronises. */
int mg_debug_colour_sum_rows(struct mg_process *p, const double *rows_dev, int64_t nrows,
                             double *q8_dev, void *stream);

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
