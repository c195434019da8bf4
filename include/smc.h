/*
 * smc.h - C ABI of libsmc, a GB300 (sm_103a) implementation of the data-annealed
 * Sequential Monte Carlo sampler for neural-network posteriors described in
 * "Investigating Batch Inference in a Sequential Monte Carlo Framework for
 * Neural Networks" (Millard, Murphy, Green, Maskell).
 *
 * The sampler keeps J particles theta_j (one weight vector of a network each)
 * with log-weights log w_j and targets, at iteration k,
 *     log pi_k(theta) = -|theta|^2 / (2 sigma^2) + sum_{i in D_k} c_i log p(y_i | theta)
 * where D_k is the data-annealed subset (Sec. 3: whole mini-batches appended to
 * a cumulatively growing subset), c_i = N / M_k for the fixed schedules
 * (Sec. 3, eq. approx-grad) and c_i in {1, beta_k} for smooth data annealing
 * (Sec. 3.1, eq. sda_initial_target and the annealed target after it).
 *
 * Conventions shared by every call
 *  - Status: every call returns smc_status.  A CUDA error or a device-side
 *    timeout makes the context sticky-failed: later calls return SMC_ESTATE
 *    until smc_destroy.  Nothing aborts, traps or exits the process.
 *  - Ownership: the context owns all device state.  Inputs are copied during
 *    the call; output buffers are caller-owned.  Pointer arguments are host
 *    pointers unless the argument or a flag says "device".
 *  - Streams: all work is enqueued on the stream given in smc_config (0 = the
 *    legacy default stream).  Calls that return statistics synchronise that
 *    stream before returning.
 *  - Threads: one context must not be used by two threads at once.
 *  - Parameter order: a particle's parameter vector ("canonical order") lists
 *    the parametric layers in order, each as W (row-major: dense [n_out][n_in],
 *    conv [c_out][c_in][k][k]) followed by b [n_out]; D is its length.  Arrays
 *    of particles are [J][D] row-major.
 */
#ifndef SMC_H
#define SMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SMC_ABI_VERSION 1

typedef struct smc_ctx smc_ctx;

typedef enum {
    SMC_OK = 0,
    SMC_EINVAL = 1,        /* bad argument or inconsistent model/config */
    SMC_ENOMEM = 2,        /* device or pinned-host allocation failed */
    SMC_ECUDA = 3,         /* a CUDA runtime/driver call failed */
    SMC_ESTATE = 4,        /* call out of order, or context already failed */
    SMC_ENUMERIC = 5,      /* every particle's log-weight is -inf or NaN */
    SMC_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
    SMC_EUNSUPPORTED = 7   /* valid request this library does not implement */
} smc_status;

enum { SMC_LAYER_DENSE = 0, SMC_LAYER_CONV = 1, SMC_LAYER_MAXPOOL2 = 2, SMC_LAYER_BNORM = 3 };
enum { SMC_ACT_TANH = 0, SMC_ACT_RELU = 1, SMC_ACT_IDENTITY = 2 };
enum { SMC_LIK_CATEGORICAL = 0, SMC_LIK_GAUSSIAN = 1 };
enum { SMC_PREC_FP32 = 0, SMC_PREC_BF16 = 1 };
enum { SMC_RESAMPLE_SYSTEMATIC = 0, SMC_RESAMPLE_MULTINOMIAL = 1 };
enum {
    SMC_SCHED_CONSTANT = 0, SMC_SCHED_FB = 1, SMC_SCHED_CTR = 2,
    SMC_SCHED_LINEAR = 3, SMC_SCHED_AUTOMATED = 4, SMC_SCHED_SDA = 5,
    /* Constant and CTR drawing a fresh mini-batch each iteration (Sec. 3.1
     * names this variant beside the cumulative ones): M_k rows starting at
     * row (k M_k) mod N of the annealed order, wrapping past N, so that
     * consecutive iterations walk through the data; once M_k = N the subset
     * is all rows from row 0. */
    SMC_SCHED_CONSTANT_FRESH = 6, SMC_SCHED_CTR_FRESH = 7
};
enum { SMC_PROPOSAL_PLAIN = 0, SMC_PROPOSAL_LEARNED = 1, SMC_PROPOSAL_EXPLORE = 2 };
#define SMC_LEARNED_NUM_PARAMS 706   /* 8-64-2 network: W1 [64][8], b1 [64], W2 [2][64], b2 [2] */

/* One layer.  DENSE: n_in -> n_out.  CONV: valid ksize x ksize cross-correlation,
 * stride 1, n_in = c_in channels -> n_out = c_out channels.  MAXPOOL2: 2x2 max
 * pool with stride 2 (n_in, n_out, ksize ignored).  BNORM: the batch
 * normalisation of Sec. 4's convolution-batchnorm blocks in its inference form
 * (fixed statistics): z = gamma_c a + beta_c per channel c of the input map (or
 * per feature after a dense layer), n_in = n_out = that channel count, its W
 * segment gamma [c] and its b segment beta [c]; it must follow a dense or conv
 * layer (SMC_EINVAL otherwise) and runs on the FP32 engine only (a BF16
 * context refuses the model with SMC_EUNSUPPORTED).  An
 * activation follows every parametric layer except the last and except a layer
 * followed by a BNORM layer (conv -> bnorm -> activation); the last layer
 * (dense or conv) gives the logits (categorical likelihood) or the mean
 * (Gaussian likelihood, n_out = 1). */
typedef struct { int32_t kind, n_in, n_out, ksize; } smc_layer;

typedef struct {
    int32_t version;           /* SMC_ABI_VERSION */
    int32_t n_layers;
    const smc_layer* layers;   /* host array of n_layers, copied */
    int32_t in_c, in_h, in_w;  /* input shape (c, h, w); a feature vector is (d, 1, 1) */
    int32_t activation;        /* SMC_ACT_* */
    int32_t likelihood;        /* SMC_LIK_* */
    double prior_sigma;        /* q_0 = N(0, prior_sigma^2 I)  (eq. init_weight's q_0) */
    double noise_sigma;        /* Gaussian likelihood only */
} smc_model;

/* Training set: x [n][in_c*in_h*in_w] float32 in (c, h, w) order; y_class
 * int32 [n] (categorical) or y_value float32 [n] (Gaussian).  on_device != 0
 * means the pointers are device pointers.  The data are copied at smc_init. */
typedef struct {
    const float* x;
    const int32_t* y_class;
    const float* y_value;
    int64_t n;
    int32_t on_device;
} smc_data;

typedef struct {
    int32_t version;           /* SMC_ABI_VERSION */
    int32_t n_particles;       /* J >= 1 (<= 4096) */
    uint64_t seed;             /* keys the mini-batch order, prior draws, momenta, uniforms */
    int32_t precision;         /* SMC_PREC_FP32: all arithmetic FP32 (SIMT kernels).
                                  SMC_PREC_BF16: network contractions in BF16 on tcgen05
                                  tensor cores with FP32 accumulation (dense models only). */
    int32_t resampler;         /* SMC_RESAMPLE_* */
    int32_t scaled;            /* 1: c_i = N/M_k on the log-likelihood and gradient
                                     (eq. approx-grad); 0: c_i = 1 */
    int64_t chunk_rows;        /* rows per forward/backward chunk (0 = automatic) */
    void* stream;              /* cudaStream_t */
    int32_t timing;            /* 1: record per-kernel-family CUDA-event times */
} smc_config;

typedef struct {
    int32_t kind;              /* SMC_SCHED_* (Sec. 3.1) */
    int64_t C;                 /* initial subset size */
    int64_t kappa;             /* mini-batch increment */
    int32_t K;                 /* number of iterations (for the 0.9K switch) */
    int32_t k_start;           /* iteration to start at (0 normally) */
    double beta0;              /* SDA: initial temperature (0.1) */
    double beta_reinit;        /* SDA: temperature after an append (0.1) */
    double delta_s;            /* SDA: entropy increment Delta S (1) */
} smc_schedule;

typedef struct {
    double h;                  /* leapfrog step size (of the plain proposal) */
    int32_t S;                 /* leapfrog steps (S = 1: Langevin dynamics) */
    int32_t proposal;          /* SMC_PROPOSAL_PLAIN: M = I, step h.
                                  SMC_PROPOSAL_LEARNED: per-segment mass and step from the
                                    learned network (not in the paper); falls back to PLAIN for
                                    one iteration after a learned move left J_eff < J/10.
                                  SMC_PROPOSAL_EXPLORE: particles split into `groups` groups,
                                    group g > 0 moving with the network's proposal perturbed by
                                    explore_sigma N(0, 1) in log space; the best group (mean squared
                                    jump x group ESS / group size) becomes a training row. */
    int32_t groups;            /* EXPLORE: candidate groups (2..16) */
    int32_t pad_;
    double explore_sigma;      /* EXPLORE: perturbation scale */
} smc_step_params;

typedef struct {
    double ess;                /* J_eff after the call (eq. jeff) */
    double mean_logpi;         /* mean of log pi_k(theta_j) over particles */
    double beta;               /* temperature of the tempered block (1 for fixed schedules) */
    int64_t rows;              /* |D_k| */
    int32_t k;                 /* iteration index */
    int32_t n_nonfinite;       /* particles whose log pi was not finite (log w set to -inf) */
    int32_t grad_evals;        /* gradient evaluations over D_k made by the call */
    int32_t proposal_used;     /* SMC_PROPOSAL_* actually used (PLAIN after a fallback) */
    double h_used;             /* step of group 0 */
} smc_step_stats;

typedef struct {
    int32_t appended;          /* 1 if rows were added to the subset */
    int32_t k;                 /* new iteration index */
    int64_t rows;              /* |D_{k}| after the call */
    int64_t rows_full;         /* SDA: fully included rows (= rows for fixed schedules) */
    double beta;               /* SDA temperature after the call */
} smc_anneal_info;

/* ---------------------------------------------------------------- lifecycle */

/* Create a sampler.  Validates the model, copies the training set to the GPU in
 * the order of one Fisher-Yates permutation drawn from `seed` (Sec. 3:
 * mini-batches drawn without replacement; D_k is the first |D_k| rows of that
 * order), and draws theta_0 ~ q_0 = N(0, prior_sigma^2 I) (eq. init_weight) with
 * Philox4x32-10.  Errors: SMC_EINVAL (shape/arg), SMC_EUNSUPPORTED (BF16 with a
 * non-dense model), SMC_ENOMEM, SMC_ECUDA.  *out is NULL on error. */
smc_status smc_init(const smc_model* model, const smc_data* train,
                    const smc_config* cfg, smc_ctx** out);

/* Release all device and host resources.  NULL is ignored. */
void smc_destroy(smc_ctx* ctx);

/* Human-readable name of a status code (static storage). */
const char* smc_status_string(smc_status s);

/* Last error message recorded by a context (never NULL); with ctx = NULL, the
 * last error of a stateless entry point on the calling thread. */
const char* smc_last_error(const smc_ctx* ctx);

/* Parameter count D of one particle. */
int64_t smc_num_params(const smc_ctx* ctx);

/* --------------------------------------------------------- the SMC iteration */

/* Fix the annealing schedule (Sec. 3.1) and start at iteration k_start: set the
 * subset D_{k_start}, evaluate log pi_0 and its gradient at the current
 * particles and set log w_0 = log pi_0(theta) - log q_0(theta), i.e. the
 * coefficient-weighted log-likelihood (eq. init_weight); then normalise
 * (eq. normalise) and compute the ESS (eq. jeff).  `stats` may be NULL.
 * Errors: SMC_EINVAL (C < 1, kappa < 1, K < 1), SMC_ENUMERIC. */
smc_status smc_set_schedule(smc_ctx* ctx, const smc_schedule* sched, smc_step_stats* stats);

/* One move + reweight under the current target pi_k (Sec. 2.1):
 * P^0 ~ N(0, M); S leapfrog steps (eqs. mom_first, pos_update, mom_second);
 * log w += log pi_k(theta_k) - log pi_{k-1}(theta_{k-1}) - P_k' M^-1 P_k / 2
 *          + P^0' M^-1 P^0 / 2 (eq. weight_update_fp, reversed-momentum L-kernel);
 * normalise and ESS.  M = I for SMC_PROPOSAL_PLAIN; a per-layer diagonal mass and
 * step chosen by the learned proposal for SMC_PROPOSAL_LEARNED (not in the paper).
 * Errors: SMC_EINVAL (h < 0, S < 1), SMC_ENUMERIC, SMC_ETIMEOUT, SMC_ECUDA. */
smc_status smc_step(smc_ctx* ctx, const smc_step_params* p, smc_step_stats* stats);

/* Advance to the target of iteration k+1 (Sec. 3.1): fixed schedules compute
 * M_{k+1}; SDA updates beta from the weighted moments of Omega and Omega_hat
 * (eqs. beta_initial_data_k / beta_annealed_k) or, once beta has reached 1,
 * appends the next mini-batch and resets beta.  `info` may be NULL. */
smc_status smc_anneal_next(smc_ctx* ctx, smc_anneal_info* info);

/* Resample when J_eff < J/2 (Sec. 2) or when force != 0, then set every weight
 * to 1/J.  Systematic or multinomial per smc_config.resampler, computed on an
 * exact fixed-point cumulative sum of the normalised weights.  did_resample
 * may be NULL. */
smc_status smc_resample(smc_ctx* ctx, int32_t force, int32_t* did_resample);

/* Weighted posterior predictive (Sec. 2, E_pi[f] ~ sum_j w~_j f(theta_j)) with
 * f = softmax of the network's logits: probs_out[n][n_classes] (float32).
 * x_test [n][input] float32.  on_device: 1 if x_test and probs_out are device
 * pointers.  Categorical models only (SMC_EUNSUPPORTED otherwise). */
smc_status smc_posterior_predict(smc_ctx* ctx, const float* x_test, int64_t n,
                                 int32_t on_device, float* probs_out);

/* Replace training rows [row0, row0 + n) of the annealed order with host data
 * x [n][input], y [n] (stream-ordered copy through pinned staging).  Lets a
 * caller keep the training set in host memory and stream the subset each
 * iteration. */
smc_status smc_upload_rows(smc_ctx* ctx, int64_t row0, int64_t n,
                           const float* x, const int32_t* y_class, const float* y_value);

/* smc_upload_rows without a stall: the host-to-device copy is enqueued on the
 * context's own copy stream into a device staging buffer and the call returns
 * at once; the rows take effect at the next smc_set_schedule or
 * smc_anneal_next (in stream order, before that iteration's evaluations), so
 * a caller can upload iteration k+1's rows while iteration k computes.
 * x / y_class / y_value must stay valid and unchanged until that call has
 * returned; pinned memory makes the copy asynchronous.  Uploads apply in
 * call order, also when mixed with smc_upload_rows (which first applies
 * staged rows).
 * Like smc_upload_rows this moves data and does not change the target: the
 * rows are expected to carry the training set's values, and a cached
 * gradient or log pi is kept.  Errors: SMC_EINVAL (range), SMC_ENOMEM (the
 * first call allocates an N-row staging buffer), SMC_ECUDA. */
smc_status smc_upload_rows_async(smc_ctx* ctx, int64_t row0, int64_t n,
                                 const float* x, const int32_t* y_class, const float* y_value);

/* ------------------------------------------ learned proposal (not in the paper) */

/* Get (host out [SMC_LEARNED_NUM_PARAMS]) and/or set (host in) the proposal
 * network's FP32 parameters; either pointer may be NULL.  A new context holds
 * a network whose output layer is zero, i.e. the plain proposal. */
smc_status smc_learned_params(smc_ctx* ctx, float* get, const float* set);

/* Fit the network to the collected training rows by full-batch Adam (FP32,
 * hand-written backward pass on the GPU) for `epochs` epochs at rate lr;
 * *loss gets the mean squared error of the last epoch (may be NULL).
 * SMC_ESTATE when no rows were collected. */
smc_status smc_learned_train(smc_ctx* ctx, int32_t epochs, double lr, double* loss);

/* Number of collected training rows; features [n][8] and targets [n][2] copied
 * to host buffers when non-NULL (capacity given by *n_rows on input). */
smc_status smc_learned_data(smc_ctx* ctx, int64_t* n_rows, float* features, float* targets);
smc_status smc_learned_reset_data(smc_ctx* ctx);

/* Replace the collected training rows by host features [n][8] and targets
 * [n][2] (n <= 16384). */
smc_status smc_learned_load_data(smc_ctx* ctx, const float* features, const float* targets, int64_t n);

/* Features [n_seg][8], candidates [groups][n_seg + 1] (log inverse masses, then
 * log step multiplier) and scores [groups + 1] (last: index of the best group)
 * of the last learned / exploring step (host buffers, each may be NULL). */
smc_status smc_learned_last(smc_ctx* ctx, float* features, float* candidates, double* scores);

/* Number of parameter segments (one W and one b per parametric layer). */
int32_t smc_num_segments(const smc_ctx* ctx);

/* Loss and gradient of the proposal network's mean squared error for host
 * features [n][8], targets [n][2] and parameters [SMC_LEARNED_NUM_PARAMS],
 * computed by the library's training kernel (host outputs). */
smc_status smc_k_learned_loss_grad(const float* features, const float* targets, int64_t n, const float* params,
                                   float* grad, double* loss, void* stream);

/* ------------------------------------------------ state access (tests, tools) */

/* Copy particles [J][D] (canonical order, float32), log-weights [J] and the
 * cached log pi of the last evaluated target [J] to host buffers; any may be NULL. */
smc_status smc_get_state(smc_ctx* ctx, float* theta, double* logw, double* logpi);

/* Overwrite the particles from host [J][D]; invalidates the cached gradient.
 * logw / logpi (host [J]) may be NULL to leave them unchanged. */
smc_status smc_set_state(smc_ctx* ctx, const float* theta, const double* logw, const double* logpi);

/* Inject the standard-normal draws z [J][D] (host, canonical order) used for the
 * momentum of the next smc_step instead of Philox (P^0 = M^{1/2} z). */
smc_status smc_set_noise(smc_ctx* ctx, const float* z);

/* Inject resampling uniforms for the next smc_resample: 1 value (systematic) or
 * J values (multinomial), host, each in [0, 1). */
smc_status smc_set_uniforms(smc_ctx* ctx, const double* u, int32_t n);

/* ---- particle-sharded runs (several contexts, one per GPU, holding
 * consecutive particle ranges of one sampler; the normalisation and
 * resampling of Sec. 2 need all J weights, so a driver exchanges them between
 * the calls below).  The paper runs on one device and has no counterpart. */

/* Global index of this context's particle 0.  The prior and momentum draws of
 * particle j then use the Philox stream positions of global particle
 * first_particle + j, so G contexts with consecutive ranges draw exactly what
 * one context with all particles draws.  Redraws theta_0 (eq. init_weight) with
 * those positions; call before smc_set_schedule. */
smc_status smc_set_shard(smc_ctx* ctx, int64_t first_particle);

/* Draw n uniforms in [0, 1) from the context's resampling stream (host
 * SplitMix64; the stream smc_resample consumes; injected uniforms first).
 * Contexts with equal seeds draw equal values. */
smc_status smc_draw_uniforms(smc_ctx* ctx, int32_t n, double* u);

/* Install normalised weights w~ [J] (host; this context's slice of the global
 * weights, eq. normalise) and the global ESS (eq. jeff).  Used by SDA moments,
 * prediction and the next resampling decision. */
smc_status smc_set_weights(smc_ctx* ctx, const double* wn, double ess);

/* This context's partial SDA moments under its current weights (Sec. 3.1):
 * out[0..3] = sum_j w~_j Omega^_j, sum_j w~_j Omega^_j^2, sum_j w~_j Omega_j,
 * sum_j w~_j Omega_j Omega^_j, with Omega^ = -L_b and Omega = -L_a. */
smc_status smc_sda_partials(smc_ctx* ctx, double* out);

/* smc_anneal_next with the four SDA moments supplied (summed over all shards)
 * instead of computed from this context's particles; identical to
 * smc_anneal_next for the fixed schedules. */
smc_status smc_anneal_next_moments(smc_ctx* ctx, const double* moments, smc_anneal_info* info);

/* Checkpoint (the paper has no counterpart: run infrastructure).  Writes the
 * sampler's dynamic state to the file `path`: particles, raw and normalised
 * log-weights, cached log pi and its two log-likelihood sums, last ancestors,
 * the cached gradient (if valid), the schedule position and target (k, row
 * regions, coefficients, beta), the step counter that positions the momentum
 * stream, the host resampling-uniform stream, and the learned proposal
 * (parameters, Adam moments, collected training rows).  Model, data and
 * configuration are not stored; noise or uniforms injected but not yet
 * consumed are dropped.  SMC_EINVAL if the file cannot be written. */
smc_status smc_checkpoint(smc_ctx* ctx, const char* path);

/* Restore a checkpoint into a context created with the same model, data, J,
 * seed and precision (checked; SMC_EINVAL on a mismatch, another library
 * version or a truncated file; the context is unchanged when a header check
 * fails).  Continuing from the restored state reproduces the original run bit
 * for bit. */
smc_status smc_restore(smc_ctx* ctx, const char* path);

/* Evaluate, at the current particles and under the current target, log pi [J],
 * the gradient of the log-likelihood part sum_i c_i grad log p(y_i|theta)
 * [J][D] (canonical order, prior excluded) and the unweighted log-likelihood
 * sums over the fully weighted rows (la) and the tempered block (lb).  Host
 * outputs, each may be NULL. */
smc_status smc_eval(smc_ctx* ctx, double* logpi, float* grad_ll, double* la, double* lb);

/* Device-pointer forms for callers that keep the particles on the GPU (the
 * binding's torch.autograd.Function around the adjoint).  theta and grad are
 * [J][D] float32 in canonical order, logpi is [J] float64, all device memory
 * of the context's device; both calls only enqueue work on the context's
 * stream (no host synchronisation).  smc_set_state_device overwrites the
 * particles (log-weights and cached log pi unchanged) and invalidates the
 * cached gradient.  smc_eval_device evaluates, under the current target,
 * log pi(theta) (eq. approx-grad's estimate plus the prior, as in smc_eval) and
 * its full gradient grad log pi = sum_i c_i grad log p(y_i|theta) - theta /
 * sigma^2; either output may be NULL.  Errors: SMC_EINVAL (NULL context or
 * theta), SMC_ESTATE (before smc_set_schedule or after a failure), SMC_ECUDA. */
smc_status smc_set_state_device(smc_ctx* ctx, const float* theta_dev);
smc_status smc_eval_device(smc_ctx* ctx, double* logpi_dev, float* grad_dev);

/* The annealed row order (Sec. 3: mini-batches drawn without replacement):
 * perm[r] = index of the training row stored at position r, [n] int32 host. */
smc_status smc_get_permutation(smc_ctx* ctx, int32_t* perm);

/* Normalised weights [J] (host). */
smc_status smc_get_weights(smc_ctx* ctx, double* wn);

/* Ancestor indices [J] chosen by the last resampling (host). */
smc_status smc_get_ancestors(smc_ctx* ctx, int32_t* ancestors);

/* Kernel launches made by this context so far, and per-family CUDA-event times
 * in milliseconds (accumulated while smc_config.timing = 1).  Family order:
 * 0 first-layer forward GEMM, 1 head/adjoint, 2 first-layer weight-gradient GEMM,
 * 3 hidden-layer GEMMs, 4 leapfrog, 5 weights/normalise/ESS, 6 resample+gather,
 * 7 other network kernels (SIMT path), 8 partial reductions, 9 first-layer
 * forward GEMM with the head/adjoint fused into it, 10 adjoint GEMMs of
 * hidden layers (dZ_{l-1} = dZ_l W_l * act'), 11 weight-gradient GEMMs of
 * hidden layers (BF16 engine of deeper networks).  times may be NULL;
 * n_fam is the capacity of times. */
smc_status smc_get_counters(smc_ctx* ctx, int64_t* launches, double* times, int32_t n_fam,
                            int64_t* calls_per_family);
smc_status smc_reset_counters(smc_ctx* ctx);

/* ------------------------------------------ stateless kernels (device pointers) */

/* Normalise log-weights [J] (device) into wn [J] (device) and write J_eff to
 * *ess_dev (device, 1 double): eqs. normalise and jeff in FP64. */
smc_status smc_k_normalise(const double* logw_dev, int32_t J, double* wn_dev,
                           double* ess_dev, void* stream);

/* Ancestors [J] (device int32) from normalised weights wn [J] (device, FP64)
 * and uniforms u (host: 1 value for systematic, J for multinomial). */
smc_status smc_k_resample(const double* wn_dev, int32_t J, int32_t kind,
                          const double* u_host, int32_t* ancestors_dev, void* stream);

/* Same result as smc_k_resample, for callers that cannot allocate device
 * memory: code under an allocator that owns all device memory (a framework's
 * caching allocator that has reserved the GPU, where a cudaMalloc of its own
 * would fail or fragment the pool), or a loop that cannot afford the
 * device-wide synchronisation a cudaFree implies.  It calls no cudaMalloc,
 * cudaFree or allocating library routine; the uniforms are staged in a static
 * 32 KiB device array (4096 doubles) that every GPU loading the library keeps
 * until the process exits.  The paper has no counterpart: this is a service of
 * the library.  J above 4096 is rejected with SMC_EINVAL; smc_last_error(NULL)
 * then names the limit.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current), so make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's uniforms; calls that overlap on the GPU (different
 * streams, or threads) race on it, so serialise them.  The call synchronises
 * `stream` before returning.  Device pointers wn_dev / ancestors_dev as in
 * smc_k_resample; u_host is host memory. */
smc_status smc_k_resample_noalloc(const double* wn_dev, int32_t J, int32_t kind,
                                  const double* u_host, int32_t* ancestors_dev, void* stream);

/* n standard normals of the (seed, stream_id, iteration) Philox4x32-10 +
 * Box-Muller sequence starting at `offset` (device float32 out). */
smc_status smc_k_philox_normals(uint64_t seed, uint32_t stream_id, uint32_t iteration,
                                uint64_t offset, int64_t n, float* out_dev, void* stream);

/* Raw Philox4x32-10 blocks: out_dev [n][4] u32 for counters (q, 0, c2, c3),
 * q = 0..n-1, under key (k0, k1). */
smc_status smc_k_philox_u32(uint32_t k0, uint32_t k1, uint32_t c2, uint32_t c3,
                            int64_t n, uint32_t* out_dev, void* stream);

/* Failure-detection probe (no counterpart in the paper): launches one thread
 * that waits, through the same bounded device-side wait as the tensor-core
 * kernels (an mbarrier polled with a %globaltimer limit, here limit_ms), on an
 * mbarrier it completes itself only if `arrive` != 0.  Returns SMC_OK when the
 * phase completed and SMC_ETIMEOUT when the wait gave up; the GPU context stays
 * usable either way.  SMC_EINVAL unless 0 < limit_ms <= 10000. */
smc_status smc_k_wait_probe(double limit_ms, int32_t arrive, void* stream);

/* C[m][n] = sum_k A[m][k] B[n][k] on tcgen05 tensor cores: A [M][K] and B [N][K]
 * BF16 row-major with row pitches lda, ldb (elements, multiples of 8), C FP32
 * row-major with pitch ldc.  Device pointers.  K-tails and ragged M/N are
 * handled (TMA zero fill).  accumulate != 0 adds into C. */
smc_status smc_k_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb,
                           float* C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                           int32_t accumulate, void* stream);

/* Batched form of smc_k_gemm_bf16 on tcgen05 CTA pairs (the contraction of
 * the BF16 engine's hidden layers and weight gradients, Sec. 3 eq. approx-grad
 * summed over rows): for b = 0..batch-1
 *     C_b[m][n] = sum_k A_b[m][k] B_b[n][k]
 * with A_b's element (m, k) at A + b a_bstride + (a_mn_major ? k lda + m : m lda + k)
 * and B_b's element (n, k) at B + b b_bstride + (b_mn_major ? k ldb + n : n ldb + k)
 * (BF16 elements; a_bstride = 0 / b_bstride = 0: every batch reads the same
 * matrix), C_b[m][n] at C + b c_bstride + m ldc + n (FP32).  An MN-major
 * operand is read in place as the transpose of a row-major matrix, so
 * dW = dZ^T A over the rows of two [rows][width] arrays needs no transposed
 * copy.  Device pointers, 16-byte aligned; lda, ldb, a_bstride, b_bstride
 * multiples of 8 elements.  K tails and ragged M / N read zeros.
 * accumulate != 0 adds into C.  Synchronises `stream`.  Errors: SMC_EINVAL
 * (sizes, pitches, alignment), SMC_ENOMEM, SMC_ECUDA, SMC_ETIMEOUT. */
smc_status smc_k_gemm_bf16_batched(const void* A, int32_t a_mn_major, int64_t lda, int64_t a_bstride,
                                   const void* B, int32_t b_mn_major, int64_t ldb, int64_t b_bstride,
                                   float* C, int64_t ldc, int64_t c_bstride,
                                   int64_t M, int64_t N, int64_t K, int32_t batch,
                                   int32_t accumulate, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SMC_H */
