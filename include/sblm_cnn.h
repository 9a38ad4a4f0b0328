/*
 * sblm_cnn.h -- C ABI of the learned proposal that seeds the evolutionary fitter of sblm.h.
 *
 * The paper's fitter starts every population from uniform random genes (Appendix A,
 * "Initialisation"); Section 4.1 mentions a trained network only as a competing fitter. This
 * library adds a small 1D convolutional network, trained on the device on lightcurves that the
 * forward model of Section 2.2 generates, whose Gaussian outputs seed a chosen fraction of each
 * initial population. The EA and its exact chi^2 judge every seeded row; with no network the
 * fitter is the paper's (sblm_fit_batch).
 *
 * All conventions of sblm.h hold: host or device pointers (host ones are staged and the call
 * synchronises), `stream` a cudaStream_t as void*, errors returned as sblm_status with
 * sblm_last_error() describing them, buffers owned by the caller.
 *
 * Network (BF16 operands, FP32 accumulation on the tensor cores, FP32 master weights):
 *   input x [256 bins][2 channels]: asinh(10 (F / median - 1)) / 3 on bins with data, and the
 *   data mask (1 = the bin holds data), channels innermost;
 *   conv k=5 pad 2: 2->64 stride 1, 64->64 stride 2 (three times), each followed by the exact
 *   GELU x Phi(x); flatten position-major (2048); dense 2048->128, GELU; dense 128->12.
 *   Output [12]: means of the targets (t0', ln tE', u0, alpha / 2 pi, ln d, log10 q) then their
 *   log-variances, where t0' = (t0 - c) / h and tE' = tE / h for a curve observed on the window
 *   [c - h, c + h].
 *   Weights: one FP32 vector of sblm_cnn_num_params() values: per layer the weight matrix
 *   [fan_in][fan_out] (a convolution's row kk * C_in + c multiplies input position l * s + kk - 2,
 *   channel c) followed by its bias [fan_out], layers in order.
 *   Loss: Gaussian negative log-likelihood, mean over the batch of
 *   sum_j 0.5 ((y_j - mu_j)^2 exp(-s_j) + s_j).
 *
 * Random numbers: Philox4x64-10 as in the EA, with its own operator ids (counter word 1):
 * 7 initial weights, 8 training parameters, 9 training noise and masks, 10 seed rows.
 */
#ifndef SBLM_CNN_H
#define SBLM_CNN_H

#include "sblm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SBLM_CNN_BINS 256
#define SBLM_CNN_OUT 12

/* Training configuration; sblm_cnn_train_params_default() fills the values in brackets. */
typedef struct {
    int32_t batch;       /* curves per optimiser step [256], 1..4096 */
    int32_t n_steps;     /* length of the learning-rate schedule [4096] */
    int32_t warmup;      /* linear warm-up steps [200], >= 0 */
    int32_t precision;   /* forward model of the generator: SBLM_FP64/MIXED/FP32 [SBLM_FP32: FP32's
                            error near caustics is far below the noise of most training curves] */
    double lr;           /* peak learning rate [2e-3]; cosine decay to 0.1 lr at n_steps */
    double beta1;        /* [0.9] */
    double beta2;        /* [0.999] */
    double eps;          /* [1e-8] */
    double weight_decay; /* decoupled (AdamW) [1e-4] */
    double forced_frac;  /* fraction of training curves aimed through a caustic [0.1] */
    uint64_t seed;       /* Philox key word 0 of the generator [0] */
} sblm_cnn_train_params;

void sblm_cnn_train_params_default(sblm_cnn_train_params* p);

/* Number of FP32 weights of the network (326,156). */
int32_t sblm_cnn_num_params(void);

/*
 * Initial weights: every weight matrix but the last He-normal (standard deviation
 * sqrt(2 / fan_in)), the last 0.1 sqrt(1 / fan_in), biases zero. Weight p takes the cosine (p
 * even) or sine (p odd) Box-Muller deviate of Philox block (p >> 1, 7, 0, 0) under key (seed, 0).
 *   weights [sblm_cnn_num_params()] FP32, written.
 */
sblm_status sblm_cnn_init(float* weights, uint64_t seed, void* stream);

/*
 * One batch of training curves, as sblm_cnn_train draws it at optimiser step `step`. Curve i:
 * parameters in window units from the sweep priors (t0' U[-0.4, 0.4], tE' log-U[0.04, 1.5],
 * u0 U[0, 1], alpha U[0, 2 pi), d log-U[0.3, 3], log10 q U[-4, 0]); with probability forced_frac
 * the trajectory is re-aimed through a caustic point (a root of the critical quartic
 * e^{i phi} z^2 (z - d)^2 - (1 + q) z^2 + 2 d z - d^2 mapped by the lens equation) crossed at
 * t' U[-0.8, 0.8]; magnification at the 256 bin centres s_j = -1 + (2 j + 1) / 256 by the forward
 * model in `precision`; flux A (1 + sigma z_j) with sigma log-U[1e-4, 0.05] and z_j unit normal;
 * bins dropped with probability U[0, 0.7] and, half the time, a gap of up to 40% of the bins
 * (at least 16 bins are kept); then the input normalisation above.
 *   x [batch][256][2] FP32, y [batch][6] FP32 targets, theta [batch][6] FP64 parameters in
 *   window units (t0', tE', u0, alpha, d, q); theta may be NULL.
 * batch 1..4096, 0 <= forced_frac <= 1.
 */
sblm_status sblm_cnn_make_batch(uint64_t seed, int64_t step, int32_t batch, double forced_frac,
                                int32_t precision, float* x, float* y, double* theta, void* stream);

/*
 * Network inputs of observed lightcurves (concatenated as in sblm_fit_batch): each curve is
 * resampled to 256 bins over its own span [t_min, t_max] (inverse-variance weighted mean flux
 * per bin, summed in epoch order; bin j = floor((t - t_min) / (t_max - t_min) * 256), the last
 * epoch in bin 255) and normalised.
 *   x [n_lc][256][2] FP32; window [n_lc][2] FP64 = (c, h) = (midpoint, half span) of each curve.
 */
sblm_status sblm_cnn_bin(const double* t, const double* flux, const double* sigma,
                         const int64_t* offsets, int32_t n_lc, float* x, double* window,
                         void* stream);

/* Network outputs out [batch][12] FP32 for inputs x [batch][256][2]; batch >= 1. */
sblm_status sblm_cnn_forward(const float* weights, const float* x, int32_t batch, float* out,
                             void* stream);

/*
 * Loss and its gradient with respect to every weight, by the hand-written backward pass
 * (BF16 operands, FP32 accumulation; the reduction over the batch is split in a fixed order, so
 * repeated calls agree bit for bit).
 *   y [batch][6] targets; *loss (FP64, host or device); grad [sblm_cnn_num_params()] FP32.
 */
sblm_status sblm_cnn_loss_grad(const float* weights, const float* x, const float* y,
                               int32_t batch, double* loss, float* grad, void* stream);

/*
 * One AdamW step (decoupled weight decay, bias-corrected moments) at 1-based step t with the
 * learning rate of the schedule in *p, from a given gradient.
 *   weights [N] and adam_state [2 N] (first then second moments) FP32, updated in place.
 */
sblm_status sblm_cnn_adamw(float* weights, float* adam_state, const float* grad,
                           const sblm_cnn_train_params* p, int64_t t, void* stream);

/*
 * Train on the device: optimiser steps first_step .. first_step + n_run - 1 of the schedule in
 * *p, each drawing a fresh batch (sblm_cnn_make_batch at that step), running the forward and
 * backward passes and an AdamW step. The step's launches are captured once in a CUDA graph and
 * replayed. weights [N] and adam_state [2 N] are updated in place (zero adam_state before the
 * first step); loss_history [n_run] FP32 (may be NULL) receives each step's batch loss.
 */
sblm_status sblm_cnn_train(float* weights, float* adam_state, const sblm_cnn_train_params* p,
                           int64_t first_step, int32_t n_run, float* loss_history, void* stream);

/*
 * Seed rows from the network's outputs (draw round 0): row 0 of lightcurve l is the network's
 * mean; row r >= 1 draws y = mu + exp(s / 2) n with n six Box-Muller deviates of Philox blocks
 * (0, 10, r, 0..1) under key (seed, l). y is mapped to physical parameters with the curve's window
 * (t0 = c + h y0, tE = h e^{y1}, u0 = y2, alpha = 2 pi y3 wrapped to [0, 2 pi), d = e^{y4},
 * log10 q = y5) and encoded as genes over `bounds` (Eq. (EMMA-encoding)), clamped to [0, 1]; a
 * non-finite gene becomes 0.5.
 *   out [n_lc][12], window [n_lc][2]; genes [n_lc][n_seed][6] FP64.
 */
sblm_status sblm_cnn_propose(const float* out, const double* window, int32_t n_lc,
                             const sblm_bounds* bounds, int32_t n_seed, uint64_t seed,
                             double* genes, void* stream);

/*
 * sblm_fit_batch_tuned whose initial populations hold given rows: rows n_pop - n_seed .. n_pop - 1
 * of lightcurve l's first population are seed_genes[l][0 .. n_seed - 1] (genes in [0, 1]); the
 * other rows, and every restart, are the paper's random initialisation. 0 <= n_seed <= n_pop;
 * seed_genes may be NULL when n_seed = 0.
 */
sblm_status sblm_fit_batch_seeded(const double* t, const double* flux, const double* sigma,
                                  const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                  const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                  const double* seed_genes, int32_t n_seed, double* best_theta,
                                  double* best_chi2, void* stream);

/*
 * The proposal-seeded batched fit in one call: sblm_cnn_bin and sblm_cnn_forward on the device,
 * then the batched fit with n_seed = round(seed_frac * n_pop) proposal rows in place of the last
 * n_seed random rows of each first population: the rows of sblm_cnn_propose (seed =
 * params->seed). Restarts are the paper's random initialisation. weights NULL or seed_frac 0 gives
 * the paper's fitter. 0 <= seed_frac <= 1.
 */
sblm_status sblm_fit_batch_cnn(const double* t, const double* flux, const double* sigma,
                               const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                               const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                               const float* weights, double seed_frac, double* best_theta,
                               double* best_chi2, void* stream);

/*
 * sblm_fit_batch_cnn with the success monitor of sblm.h (sblm_batch_monitor; monitor may be
 * NULL, then this is sblm_fit_batch_cnn). The monitor's arrays follow the pointer rules of the
 * other arguments (host or device); first_gen is written when the call returns.
 */
sblm_status sblm_fit_batch_monitored(const double* t, const double* flux, const double* sigma,
                                     const int64_t* offsets, int32_t n_lc, const sblm_bounds* bounds,
                                     const sblm_ea_params* params, const sblm_batch_tuning* tuning,
                                     const float* weights, double seed_frac,
                                     const sblm_batch_monitor* monitor, double* best_theta,
                                     double* best_chi2, void* stream);

/*
 * Diagnostic of the tensor-core kernels' bounded waits (no counterpart in the paper): launches one
 * block whose wait on an mbarrier that nothing ever arrives on gives up after `polls` polls
 * (1 <= polls <= 2^20; each poll is one bounded mbarrier.try_wait), sets the device flag that a
 * tensor-core tile sets when it gives up, and maps it to a status exactly as the sblm_cnn_* calls
 * do. Expected result: SBLM_ETIMEOUT, with the flag cleared so that the next call starts clean.
 * No tensor memory is allocated and no MMA is issued. Synchronises `stream`.
 */
sblm_status sblm_cnn_selftest_timeout(int32_t polls, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SBLM_CNN_H */
