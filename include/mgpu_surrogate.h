/*
 * mgpu surrogate -- MLP estimate of log|M|^2 and the exact two-stage
 * unweighting it drives.  C ABI, same conventions as mgpu.h (device
 * pointers, asynchronous on `stream` unless stated, negative status on
 * error).
 *
 * The paper has no learned component (its "Summary and outlook" section
 * only names neural phase-space sampling, MadNIS, as future work); this
 * follows the published scheme of
 * rejection sampling with network weight estimates (Danziger, Janssen,
 * Schumann, Siegert, SciPost Phys. 12 (2022) 164), in which the exact matrix
 * element corrects every surrogate acceptance so the unweighted sample stays
 * exact:
 *   features  x = log(s_ij / s) for all particle pairs i < j (s = s_12),
 *             padded
 *   network   nin -> hidden (x nhidden, SiLU) -> 1, BF16 weights and
 *             activations, FP32 accumulation, FP32 master weights, Adam
 *   target    y = (log|M|^2 - mu) / sigma, MSE loss
 *   stage 1   keep u1 < w_hat / w_hat_max,  w_hat = exp(sigma f + mu) Phi
 *   stage 2   keep u2 < (w / w_hat) / r_max, w = |M|^2 Phi (exact, FP64)
 *   weight    max(1, w_hat / w_hat_max) * max(1, (w / w_hat) / r_max)
 */
#ifndef MGPU_SURROGATE_H
#define MGPU_SURROGATE_H

#include <stdint.h>

#include "mgpu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_surrogate mg_surrogate;

/* nin, hidden: multiples of 16 (nin >= number of pairs); nhidden >= 1;
 * bmax: rows per forward/backward chunk (multiple of 16, the training batch
 * limit).  Glorot-uniform weights from `seed`, zero biases.  Allocates its
 * device buffers (owned, freed by mg_sur_destroy). */
int mg_sur_create(int nin, int hidden, int nhidden, uint64_t seed, int bmax, mg_surrogate **out);
void mg_sur_destroy(mg_surrogate *s);

/* Parameters as FP32 host arrays [W_0 (out x in, row-major), b_0, W_1, b_1,
 * ...] without padding; *n = their number. */
int mg_sur_param_count(const mg_surrogate *s, int64_t *n);
int mg_sur_get_params(mg_surrogate *s, float *host);
int mg_sur_set_params(mg_surrogate *s, const float *host);
/* Gradients of the last mg_sur_loss_grad / training batch, same layout. */
int mg_sur_get_grads(mg_surrogate *s, float *host);

/* Target statistics mu, sigma of log(me_dev[0..n)), kept on the device. */
int mg_sur_fit_target(mg_surrogate *s, const double *me_dev, int64_t n, void *stream);
int mg_sur_get_target_stats(mg_surrogate *s, double *mu_sigma_host);

/* Forward + backward on one batch: momenta_dev[m][npar][4], standardised
 * targets y_dev[m] (FP32); m a multiple of 16, <= bmax.  *loss_out (host,
 * may be NULL; synchronises when given) = mean squared error. */
int mg_sur_loss_grad(mg_surrogate *s, const double *momenta_dev, int npar, const float *y_dev, int m,
                     double *loss_out, void *stream);
/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8) with the stored gradients. */
int mg_sur_adam(mg_surrogate *s, double lr, void *stream);
/* Training: `epochs` passes over the n events in order, full batches of
 * `batch` rows, targets log(me_dev) standardised with the fitted mu/sigma.
 * *last_epoch_loss (host, may be NULL) = mean batch loss of the last epoch. */
int mg_sur_train(mg_surrogate *s, const double *momenta_dev, int npar, const double *me_dev,
                 int64_t n, int epochs, int batch, double lr, void *stream, double *last_epoch_loss);
/* Predicted log|M|^2 (= sigma f + mu) for n events into logme_dev[n].
 * Asynchronous; a bounded wait of its tensor-core GEMMs that gave up is
 * reported by mg_sur_device_status or the next synchronising call. */
int mg_sur_predict(mg_surrogate *s, const double *momenta_dev, int npar, int64_t n,
                   double *logme_dev, void *stream);
/* Synchronises the stream; MG_ERR_DEVICE_TIMEOUT (and clears it) when a
 * bounded wait inside one of the surrogate's tensor-core GEMMs gave up since
 * the last check (its outputs are then not valid), MG_ERR_CUDA on a CUDA
 * error, else MG_OK.  mg_sur_train, mg_sur_loss_grad with a loss output and
 * mg_unweight2 make this check themselves. */
int mg_sur_device_status(mg_surrogate *s, void *stream);

/* Checkpoint / resume: weights, Adam state and target statistics in a
 * versioned binary file ("MGSUR001").  Load requires the same sizes. */
int mg_sur_save(mg_surrogate *s, const char *path);
int mg_sur_load(mg_surrogate *s, const char *path);

/* Two-stage unweighting of n candidates with process p (filtered, FP64 or
 * mixed): inputs momenta_dev[n][npar][4], phase-space weights phi_dev[n],
 * uniforms u1_dev[n], u2_dev[n]; outputs accept_dev[n] (0/1) and
 * weight_dev[n] (0 when rejected); *n_exact (host) = candidates whose exact
 * matrix element was evaluated (the stage-1 survivors, compacted in
 * candidate order).  Allocates its workspace per call; synchronises. */
int mg_unweight2(mg_process *p, mg_surrogate *s, const double *momenta_dev, const double *phi_dev,
                 const double *u1_dev, const double *u2_dev, int64_t n, double what_max,
                 double r_max, unsigned char *accept_dev, double *weight_dev, int64_t *n_exact,
                 void *stream);

#ifdef __cplusplus
}
#endif
#endif
