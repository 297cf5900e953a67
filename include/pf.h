/*
 * pf.h -- C ABI of the GB300 ensemble particle filter.
 *
 * The library runs the parallelisation scheme of Crisan, Miguez & Rios
 * (arXiv:1407.8071): M fully independent bootstrap particle filters
 * (Algorithm 1) with N_m particles each, on one GPU, and the average of their
 * estimates (Definition 1).  Every step of the filter runs in this library's
 * own sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: a pf_status.  Nothing aborts or prints; pf_last_error()
 *   gives a one-line description of the last failure on a context.
 * - Ownership: the caller owns every pointer it passes in.  Inputs are read
 *   (or copied) during the call, or, for asynchronous device work, before the
 *   work the call enqueues completes on the context's stream; no pointer is
 *   retained after a call returns unless stated.
 * - Host/device: an argument named h_* is host memory, d_* is device memory
 *   of the current CUDA device.  Unprefixed pointers are host memory.
 * - Streams: device work is enqueued on the context's stream (pf_set_stream;
 *   default: a stream the context creates).  Calls are asynchronous unless
 *   they return host data (pf_estimate, pf_get_*), which synchronise.
 * - Threads: a context is used by one host thread at a time.
 * - Errors are sticky per context: after PF_ECUDA or PF_ENUMERIC every further
 *   step returns PF_ESTATE until pf_destroy.
 * - Sizes: 1 <= M, 1 <= N_m <= 2^24, sum_m N_m * dx * 4 bytes must fit in
 *   device memory (else PF_ENOMEM).
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 * seed, counter (particle i, observation t, filter m, stream<<24 | block),
 * and Box-Muller normals from 24-bit uniforms; the stream ids are
 * 0 truth dynamics, 1 observation noise, 2 prior, 3 particle dynamics,
 * 4 resampling uniforms, 5 proposal noise, 6 other.
 */
#ifndef PF_GB300_PF_H
#define PF_GB300_PF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__) || defined(__clang__)
#define PF_API __attribute__((visibility("default")))
#else
#define PF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_ctx pf_ctx; /* opaque; owns all of its device memory */

typedef enum {
    PF_OK = 0,
    PF_EINVAL = 1,       /* invalid argument (NULL where required, size out of range, bad model) */
    PF_ENOMEM = 2,       /* device or host allocation failed                                      */
    PF_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed                           */
    PF_ENUMERIC = 4,     /* a filter's weights were all zero or not finite (pf_last_error names it) */
    PF_ETIMEOUT = 5,     /* a bounded device-side wait gave up                                    */
    PF_ESTATE = 6,       /* the context is in an error state, or the call is out of order         */
    PF_EUNSUPPORTED = 7  /* the model or option is not available in this build                    */
} pf_status;

typedef enum {
    PF_MODEL_LINEAR_GAUSSIAN = 0, /* dx in [1,4]; drift -A x; params = A (dx*dx, row-major)           */
    PF_MODEL_LORENZ63 = 1,        /* dx = 3; Sec. 4.1 eqs. eqDiscreteLorenz-1..3; params = (s, r, b)  */
    PF_MODEL_FHN_LATTICE = 2,     /* dx = 2 J^2, J even in [2,44]; Sec. 5.1 lattice, Rogers-McCulloch
                                     form; params = (a, b, c1, c2, d, D, stim_amp, stim_steps,
                                     stim_block); state = v-plane then w-plane, node = row*J + col   */
    PF_MODEL_FHN_PAPER = 3        /* dx = 3 J^2, J even in [2,44]; the paper's own lattice, eqs. eqUd,
                                     eqVd with the random stimulus of eqs. eqStimulusRegion-
                                     eqPsi_ijt; state = U-plane, V-plane, S-plane (sub-steps since
                                     the node's last stimulus event, capped at l0); 17 params:
                                     alpha_3..alpha_0 of p3, beta_0..beta_2, 1/D, forcing amplitude,
                                     forcing period and pulse width (sub-steps), forced columns,
                                     u-, u+, round(eps 2^24), stimulus amplitude, l0.  Noise only
                                     on U; the stimulus draws use Philox stream 6 (particles) / 7
                                     (pf_simulate's truth), block = sub-step index.               */
} pf_model_kind;

/* The Markov kernel tau_t (Sec. 2.2, eq. eqKernel): steps_per_obs Euler-
 * Maruyama sub-steps x <- x + dt f(x) + sigma_dyn sqrt(dt) z between two
 * observations.  params is copied. */
typedef struct {
    int32_t kind;          /* pf_model_kind                      */
    int32_t dx;            /* state dimension                    */
    int32_t J;             /* lattice side (FHN), else 0         */
    int32_t steps_per_obs; /* K >= 1                             */
    const double *params;  /* model constants, see pf_model_kind */
    int32_t n_params;
} pf_model;

/* The likelihood g_t^y (Sec. 2.2): y = x[idx] + sigma_obs * noise,
 * 1 <= dy <= 4096; idx is copied. */
typedef struct {
    int32_t dy;
    const int32_t *idx;
    double sigma_obs;
} pf_obs_op;

/* Prior tau_0 = N(x0_mean, sigma0^2 I) (Alg. 1 step 1) and the seed. x0_mean
 * (dx doubles) is copied. */
typedef struct {
    double sigma_dyn;
    const double *x0_mean;
    double sigma0;
    uint64_t seed;
} pf_noise;

typedef enum {
    PF_STAT_MEAN = 0,         /* (f, pi_t^N) with f = x[var]: post-resampling particle mean        */
    PF_STAT_LOG_EVIDENCE = 1, /* log G_t^N, eq. eqGtN (Gaussian constant included)                  */
    PF_STAT_ESS = 2,          /* (sum w)^2 / sum w^2 before resampling                               */
    PF_STAT_LOG_Z = 3,        /* log sum_i exp(l_i) of this step's log-weights (no constant)         */
    PF_STAT_FALLBACK = 4      /* 1 where the learned proposal fell back to the transition this step   */
} pf_stat_kind;

/* A statistic request.  kind = PF_STAT_MEAN uses var (0 <= var < dx, or -1 for
 * all dx variables).  per_filter = 0 asks for the ensemble average over the M
 * filters (Definition 1; for ESS / LOG_EVIDENCE / LOG_Z the plain average);
 * per_filter = 1 asks for the M per-filter values. */
typedef struct {
    int32_t kind;
    int32_t var;
    int32_t per_filter;
} pf_stat;

/* Optional allocator for context memory.  alloc returns NULL on failure;
 * free receives the pointer and size alloc returned.  stream is the
 * context's cudaStream_t. */
typedef void *(*pf_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*pf_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* --------------------------------------------------------------------- */
/* Context life cycle                                                    */
/* --------------------------------------------------------------------- */

/* Sets the allocator used by contexts created afterwards on this process
 * (NULL, NULL restores cudaMalloc / cudaFree).  Not thread-safe with
 * concurrent pf_create. */
PF_API pf_status pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void *user);

/* Creates M independent bootstrap filters with N[m] particles each for the
 * model, observation operator and noise given (Sec. 3.1: M independent
 * instances of Algorithm 1 on one observation record).  Draws the initial
 * particles (Alg. 1 step 1) on the device.  N has M entries.  On success *out
 * is a new context (destroy with pf_destroy); on failure *out is NULL.
 * Errors: PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_EUNSUPPORTED. */
PF_API pf_status pf_create(const pf_model *model, int32_t M, const int32_t *N, double dt, const pf_obs_op *obs,
                    const pf_noise *noise, pf_ctx **out);

/* Frees the context and its device memory.  NULL-safe.  Synchronises the
 * context's stream first. */
PF_API void pf_destroy(pf_ctx *ctx);

/* Last error text of a context (or, when ctx is NULL, of the last failed
 * pf_create or context-free call on this thread).  Valid until the next call
 * on that context. */
PF_API const char *pf_last_error(const pf_ctx *ctx);

/* Uses the caller's cudaStream_t for all later work of this context (NULL:
 * back to the context's own stream).  The stream must outlive its use. */
PF_API pf_status pf_set_stream(pf_ctx *ctx, void *stream);

/* --------------------------------------------------------------------- */
/* The hot path: one observation time of all M filters                   */
/* --------------------------------------------------------------------- */

/* One recursive step of Algorithm 1 for every particle of every filter:
 * propagation through tau_t and the weights w_t (step 2a), per-filter
 * normalisation in FP64 with the running G_t^N (eq. eqGtN), systematic
 * resampling (step 2b), and the per-filter and ensemble means (Definition 1).
 * h_obs: host FP32 observation y_t, dy values when obs_stride = 0 (one record
 * shared by every filter, Sec. 4.2), or M rows of obs_stride >= dy floats
 * (one record per filter).  Asynchronous; h_obs may be reused on return.
 * Errors: PF_EINVAL, PF_ECUDA, PF_ESTATE. */
PF_API pf_status pf_step(pf_ctx *ctx, const float *h_obs, int32_t obs_stride);

/* pf_step with the observation already in device memory (d_obs, same layout
 * as h_obs); d_obs must stay valid until the step completes on the stream. */
PF_API pf_status pf_step_device(pf_ctx *ctx, const float *d_obs, int32_t obs_stride);

/* pf_step_device launched without its CUDA graph, with CUDA events around
 * its two halves as a step runs them: h_ms[0] receives the device time of
 * the propagation and weighting (Alg. 1 step 2a), h_ms[1] that of the
 * resampling with the estimates (step 2b, Definition 1).  For measuring the
 * step; the filter advances exactly as with pf_step_device.  Synchronises.
 * Bootstrap filters only.  Errors: PF_EINVAL, PF_ESTATE, PF_EUNSUPPORTED,
 * PF_ECUDA. */
PF_API pf_status pf_step_timed(pf_ctx *ctx, const float *d_obs, int32_t obs_stride, float *h_ms);

/* The two halves of pf_step, for callers that inspect the weighted particles
 * between them: pf_propagate is step 2a (propagate + log-weights);
 * pf_resample is the normalisation, step 2b and the estimates.  A pf_step is
 * exactly pf_propagate followed by pf_resample.  pf_propagate_device takes the
 * observation from device memory like pf_step_device.  Out-of-order calls return
 * PF_ESTATE. */
PF_API pf_status pf_propagate(pf_ctx *ctx, const float *h_obs, int32_t obs_stride);
PF_API pf_status pf_propagate_device(pf_ctx *ctx, const float *d_obs, int32_t obs_stride);
PF_API pf_status pf_resample(pf_ctx *ctx);

/* Reads a statistic of the last completed step (synchronises).  out receives
 * 1 value (ensemble), dx values (MEAN with var = -1), M values (per_filter),
 * or M*dx values (MEAN, var = -1, per_filter; row-major [m][var]).
 * Errors: PF_EINVAL, PF_ECUDA, PF_ENUMERIC (a filter degenerated), PF_ESTATE
 * (no step completed yet). */
PF_API pf_status pf_estimate(pf_ctx *ctx, const pf_stat *stat, double *out);

/* The number of kernels one pf_step launches: the kernel nodes of the CUDA
 * graph the latest pf_step captured (a step is replayed from that graph).
 * Errors: PF_EINVAL, PF_ESTATE (no step captured yet: no pf_step, or a
 * recording context, whose steps are launched directly). */
PF_API pf_status pf_step_kernels(pf_ctx *ctx, int32_t *n);

/* The same values without waiting: enqueues their device-to-host copy on the
 * context's stream into h_out (host memory owned by the caller, pinned for a
 * truly asynchronous copy; same sizes and layout as pf_estimate), together
 * with a copy of the device error word, and returns.  h_out holds the values
 * once pf_estimate_wait has returned; steps enqueued after this call do not
 * disturb them, so a caller can enqueue step t+1 before reading step t.
 * Non-MEAN statistics are available per filter only (their M-average is
 * formed on the host by pf_estimate).  Errors: PF_EINVAL, PF_ESTATE,
 * PF_EUNSUPPORTED, PF_ECUDA. */
PF_API pf_status pf_estimate_async(pf_ctx *ctx, const pf_stat *stat, double *h_out);

/* Waits for the latest pf_estimate_async copy only (not for work enqueued
 * after it), then reports a degenerate filter (PF_ENUMERIC) or an expired
 * device wait (PF_ETIMEOUT) seen by the step it belongs to, as pf_estimate
 * does.  Errors: PF_EINVAL, PF_ESTATE (nothing enqueued), PF_ECUDA,
 * PF_ENUMERIC, PF_ETIMEOUT. */
PF_API pf_status pf_estimate_wait(pf_ctx *ctx);

/* Picks the launch schedule of this context's hot kernels by timing the
 * candidates on copies of its particles: for the lattice, nodes per thread and
 * particles per CTA (one particle per CTA up to as many as fit in 1024
 * threads), and for four (eight) nodes per thread whether the kernel is the
 * build for three or four (two or three) CTAs per SM; for every model, threads
 * per resampling tile
 * CTA (64, 128, 256 -- fewer threads and more CTAs for small filters).  The
 * choice is cached per (model, lattice side, K, dx, particle counts) for the
 * process, and reported in h_choice[0..2] (may be NULL): h_choice[0] particles
 * per lattice CTA (0 for the small models, which run one particle per thread),
 * h_choice[1] resampling threads, h_choice[2] lattice nodes per thread (2, 4
 * or 8; 1 for the small models).  The filter's state, statistics and step counter
 * are unchanged.
 * Synchronises; needs about one particle buffer of temporary device memory.
 * Errors: PF_ESTATE (between pf_propagate and pf_resample, or recording),
 * PF_ENOMEM, PF_ECUDA. */
PF_API pf_status pf_autotune(pf_ctx *ctx, int32_t *h_choice);

/* Switches the context between the bootstrap filter (on = 0, the default) and
 * the auxiliary particle filter of Pitt & Shephard (on = 1), the filter the
 * paper runs on its lattice (Sec. 5.3; the remark after Corollary 2 extends
 * the analysis to it).  Per observation t each filter then: predicts every
 * particle without noise over the K sub-steps (mu); resamples (systematic,
 * exact) with weights W_{t-1} g_t(mu); propagates the selected particles with
 * the transition; weights them by g_t(x) / g_t(mu_ancestor).  PF_STAT_MEAN is
 * then the weighted mean, PF_STAT_ESS the ESS of the second-stage weights, and
 * PF_STAT_LOG_EVIDENCE accumulates the unbiased estimate [sum W g(mu)] x
 * [(1/N) sum w].  pf_get_logw returns the second-stage log-weights; switching
 * on or pf_set_state makes them uniform.  Steps go through pf_step /
 * pf_step_device only (pf_propagate, pf_resample and pf_set_logw return
 * PF_EUNSUPPORTED), and the mode is not combined with the learned proposal
 * or tuple recording.  Synchronises.
 * Errors: PF_ESTATE, PF_EUNSUPPORTED, PF_ENOMEM. */
PF_API pf_status pf_set_auxiliary(pf_ctx *ctx, int32_t on);

/* Resampling only when it is needed: a filter resamples at step t only if its
 * effective sample size is below ess_threshold x N_m (0 <= ess_threshold <= 1;
 * any other value, e.g. -1 or 2, restores resampling at every step, Algorithm 1
 * as printed and the default).  Between resamplings a filter carries its log-
 * weights: its step's log-weights are the carried ones plus log g_t; log G_t
 * gains log sum exp(log-weights) - log sum exp(carried); PF_STAT_MEAN is the
 * mean under the carried weights (uniform right after a resampling);
 * PF_STAT_ESS is the ESS the decision was taken on.  pf_set_state makes the
 * carried weights uniform.  Steps go through pf_step / pf_step_device only;
 * not combined with the auxiliary filter, the learned proposal or recording.
 * Synchronises.  Errors: PF_EINVAL (NaN), PF_ESTATE, PF_EUNSUPPORTED, PF_ENOMEM. */
PF_API pf_status pf_set_resampling(pf_ctx *ctx, double ess_threshold);

/* Sets the launch schedule explicitly (0 in any field: the default):
 * nodes_per_thread 2, 4 or 8 for the lattice kernels (4 and 8 where J
 * is divisible by them),
 * particles_per_cta >= 1 for the lattice (clamped to what fits in 1024
 * threads), resample_threads 64, 128 or 256 (at least an eighth of the
 * largest tile, min(N_m, 1024): a tile CTA takes 4 particles per thread, or 8
 * where 4 do not cover the tile).  Results do not depend on the schedule
 * (particles and ancestors bit for bit; FP64 estimates to summation order).
 * Synchronises.  Errors: PF_EINVAL, PF_ESTATE. */
PF_API pf_status pf_set_schedule(pf_ctx *ctx, int32_t nodes_per_thread, int32_t particles_per_cta,
                                 int32_t resample_threads);

/* Failure injection from the host, for testing a caller's error handling
 * without faulting the GPU: writes the context's device error word as a
 * failed bounded device wait (code = PF_ETIMEOUT) or a filter whose weights
 * all vanished (code = PF_ENUMERIC, naming `filter`) would have written it,
 * behind the work already on the context's stream (synchronises).  The next
 * pf_estimate or pf_estimate_wait then returns that code and the context
 * refuses further steps (PF_ESTATE), exactly as after the real failure.  The
 * paper has no counterpart (its analysis assumes exact arithmetic).
 * Errors: PF_EINVAL (another code, filter out of range), PF_ECUDA. */
PF_API pf_status pf_inject_error(pf_ctx *ctx, int32_t code, int32_t filter);

/* Definition 1's average over the M filters, from per-filter estimates held
 * on the host (the form a caller that splits the filters over several
 * processes gathers): h_out[s] = (sum_m h_est[m * n_stat + s]) / M for
 * s < n_stat.  h_est: M x n_stat doubles, row-major [m][s] (host);
 * h_out: n_stat doubles (host).  The sum over m is exact (a fixed-point
 * accumulator spanning the binary64 range) and rounded once to the nearest
 * double, so the result does not depend on the order of the filters or on how
 * they were split; the division by M is one IEEE rounding.  A NaN, or
 * infinities of both signs, give NaN.  Host code only: no device, no stream.
 * Errors: PF_EINVAL. */
PF_API pf_status pf_ensemble_average(int32_t M, int32_t n_stat, const double *h_est, double *h_out);

/* --------------------------------------------------------------------- */
/* Inspection and state transfer (synchronous; for tests and checkpoints) */
/* --------------------------------------------------------------------- */

/* Number of completed observation steps t (0 after pf_create). */
PF_API pf_status pf_get_time(const pf_ctx *ctx, int32_t *t);

/* Copies the current particles to/from host FP32 memory laid out as
 * [sum_m N_m][dx], filter after filter, particle-major.  After pf_propagate
 * they are the weighted particles x-bar_t; after pf_resample / pf_step the
 * resampled x_t.  pf_set_state also sets the step counter to t (so the next
 * step draws the random numbers of observation t + 1): a checkpoint resumes
 * bit-identically. */
PF_API pf_status pf_get_state(pf_ctx *ctx, float *h_x);
PF_API pf_status pf_set_state(pf_ctx *ctx, const float *h_x, int32_t t);

/* FP32 log-weights l_i = log g_t(x-bar_i) without the Gaussian constant, after
 * pf_propagate (sum N_m values).  pf_set_logw replaces them (before
 * pf_resample). */
PF_API pf_status pf_get_logw(pf_ctx *ctx, float *h_l);
PF_API pf_status pf_set_logw(pf_ctx *ctx, const float *h_l);

/* Filter-local ancestor indices a_i of the last resampling (sum N_m int32). */
PF_API pf_status pf_get_ancestors(pf_ctx *ctx, int32_t *h_a);

/* --------------------------------------------------------------------- */
/* Stateless building blocks (device pointers; enqueued on `stream`)      */
/* --------------------------------------------------------------------- */

/* Philox4x32-10 of n counters: d_ctr and d_out are n x 4 uint32. */
PF_API pf_status pf_rng_philox(int64_t n, const uint32_t *d_ctr, uint32_t key0, uint32_t key1, uint32_t *d_out,
                        void *stream);

/* Four FP32 Box-Muller normals per counter (key = seed): d_z is n x 4. */
PF_API pf_status pf_rng_normals(int64_t n, const uint32_t *d_ctr, uint64_t seed, float *d_z, void *stream);

/* A keyed pseudo-random permutation of [0, n): d_perm[i] = pi(i) (n int64,
 * device).  pi is four rounds of (add a key word, multiply by an odd
 * constant, xor-shift) on the integers below the next power of two >= n, each
 * a bijection there, keyed by the Philox4x32-10 block (0, 0, 0, stream 6)
 * under `seed`, and cycle-walked into [0, n) -- a bijection of [0, n) that
 * every element evaluates on its own (no sort).  Used to shuffle training
 * batches.  Errors: PF_EINVAL, PF_ECUDA. */
PF_API pf_status pf_permutation(int64_t n, uint64_t seed, int64_t *d_perm, void *stream);

/* Bytes of device scratch pf_systematic_resample needs for M filters with
 * `total` particles in all. */
PF_API size_t pf_systematic_scratch_bytes(int32_t M, int64_t total);

/* Systematic resampling of M filters (Algorithm 1 step 2b, systematic form)
 * from unnormalised FP64 weights w in [0, 1] and one uniform u_m in [0, 1)
 * per filter.  Definition (exact, reproducible bit for bit):
 * L = ceil(log2 N_m), q_k = floor(w_k 2^(52-L)) (an integer below 2^53),
 * C_k = q_0 + ... + q_k (exact), U = floor(u_m 2^32), and
 * a_i = min{k : C_k > (i + U 2^-32) C_{N-1} / N_m} in exact arithmetic (the
 * device compares C_k N 2^32 with (i 2^32 + U) C_{N-1} in 128-bit integers).
 * h_N: the M particle counts (host); the filters' weights sit contiguously in
 * d_w, filter after filter (sum N_m doubles), and each filter's largest
 * weight should be 1 so that its quantised total is positive.
 * d_u: M doubles.  d_anc receives sum N_m filter-local indices.
 * d_scratch: caller-owned device scratch of at least
 * pf_systematic_scratch_bytes(M, sum N_m) bytes, 256-byte aligned; it may be
 * reused once the call's work completes on `stream`.  The call synchronises
 * `stream` once to upload its launch plan, then enqueues three kernels.
 * Errors: PF_EINVAL, PF_ECUDA. */
PF_API pf_status pf_systematic_resample(int32_t M, const int32_t *h_N, const double *d_w, const double *d_u,
                                 int32_t *d_anc, void *d_scratch, size_t scratch_bytes, void *stream);

/* --------------------------------------------------------------------- */
/* Learned proposal network (growth direction)                            */
/* --------------------------------------------------------------------- */

/* The network of the learned proposal: 51 inputs (5x5 patches of v and w
 * around an observed lattice node, row-major, mirrored at the lattice edge,
 * then y at the node) -> 128 -> 128 -> 4 outputs (o_mu_v, o_mu_w, o_s_v,
 * o_s_w), exact GELU between layers.  Parameters: PF_MLP_PARAMS FP32 values,
 * W1 (128 x 51), b1 (128), W2 (128 x 128), b2 (128), W3 (4 x 128), b3 (4),
 * row-major.  The kernels use bfloat16 operands on the tensor cores and FP32
 * accumulation.  At the observed nodes the last Euler-Maruyama sub-step before
 * an observation is then drawn from q = N(m + h o_mu, (h exp(clip(o_s,-3,3)))^2)
 * with h = sigma_dyn sqrt(dt) and m the transition mean; the weights carry
 * p g / q (the paper's analysis covers such importance functions, Sec. 6
 * footnote). */
#define PF_MLP_PARAMS 23684

/* Forward pass of `rows` FP32 input rows (rows x 51, device) -> d_out
 * (rows x 4, device).  d_theta: PF_MLP_PARAMS FP32 values on the device. */
PF_API pf_status pf_mlp_forward(int64_t rows, const float *d_in, const float *d_theta, float *d_out, void *stream);

/* The same network evaluated on lattice states, its input rows built on the
 * device from the states inside the kernel (the form the filter runs: the
 * fifth-generation tensor cores, tcgen05 with accumulators in tensor memory,
 * and an erf approximation with |error| <= 1.5e-7 in the GELU).  J: lattice
 * side (2..44); d_x: P particles of 2 J^2 FP32 (v-plane, then w-plane);
 * h_obs_idx: dy node indices in [0, J^2) (host, copied); d_y: dy FP32
 * observations shared by all particles; d_theta: PF_MLP_PARAMS FP32 values;
 * d_out: (P dy) x 4 FP32, row p dy + j for particle p and observed node j.
 * All device pointers; enqueued on `stream` with stream-ordered temporaries.
 * Errors: PF_EINVAL, PF_ENOMEM, PF_ECUDA. */
PF_API pf_status pf_proposal_forward(int32_t J, int64_t P, const float *d_x, int32_t dy, const int32_t *h_obs_idx,
                                     const float *d_y, const float *d_theta, float *d_out, void *stream);

/* Training state on the device: FP32 master parameters and Adam moments
 * (beta1 0.9, beta2 0.999, eps 1e-8), workspace for batches up to max_batch
 * rows.  h_theta: initial parameters (copied). */
typedef struct pf_mlp_trainer pf_mlp_trainer;
PF_API pf_status pf_mlp_trainer_create(const float *h_theta, int32_t n_params, int64_t max_batch,
                                       pf_mlp_trainer **out);
/* One step on a batch: d_X (batch x 51 inputs) and d_R (batch x 2 standardised
 * residuals r = (x'_target - m) / h) on the device.  Loss: the mean over rows
 * of sum_c (r_c - o_mu_c)^2 / (2 e^{2 s_c}) + s_c, s_c = clip(o_s_c, -3, 3).
 * lr > 0 takes an Adam step; lr = 0 only computes the gradient.  h_grad
 * (PF_MLP_PARAMS floats) and h_loss may be NULL; when either is given the
 * call synchronises `stream`.  Deterministic (fixed-order reductions). */
PF_API pf_status pf_mlp_train_step(pf_mlp_trainer *tr, int64_t batch, const float *d_X, const float *d_R, float lr,
                                   float *h_grad, double *h_loss, void *stream);
/* pf_mlp_train_step on a shuffled mini-batch gathered by the library: the
 * rows pi(first), ..., pi(first + batch - 1) of d_X (n x 51) and d_R (n x 2),
 * with pi the keyed permutation of [0, n) that pf_permutation(n, perm_seed)
 * gives.  An epoch of shuffled batches takes one seed and first = 0, batch,
 * 2 batch, ...  Requires first + batch <= n.  Errors: PF_EINVAL, PF_ECUDA. */
PF_API pf_status pf_mlp_train_step_shuffled(pf_mlp_trainer *tr, int64_t n, const float *d_X, const float *d_R,
                                            int64_t batch, int64_t first, uint64_t perm_seed, float lr,
                                            float *h_grad, double *h_loss, void *stream);
/* Copies the current parameters to host memory (synchronous). */
PF_API pf_status pf_mlp_trainer_get(pf_mlp_trainer *tr, float *h_theta);
/* NULL-safe. */
PF_API void pf_mlp_trainer_destroy(pf_mlp_trainer *tr);

/* Turns the learned proposal on for a lattice context (h_theta: PF_MLP_PARAMS
 * FP32 network parameters, copied) or off (h_theta = NULL).  Each step then
 * draws the last sub-step at the observed nodes from q (see above) with the
 * transition's own normals, weights by g p / q, and falls back to the
 * transition for a filter whose ESS under q is below ess_frac N (the
 * PF_STAT_FALLBACK statistic reports it).  A zero output layer reproduces the
 * bootstrap filter exactly.  Synchronises.  Errors: PF_EINVAL,
 * PF_EUNSUPPORTED (not a lattice), PF_ENOMEM, PF_ESTATE. */
PF_API pf_status pf_set_proposal(pf_ctx *ctx, const float *h_theta, int32_t n_params, double ess_frac);

/* How much of each observation interval the learned proposal acts on: the
 * last `span` Euler-Maruyama sub-steps (1 <= span <= steps_per_obs; default 1,
 * the last sub-step).  The network is evaluated once per interval, on the
 * state before the first of them and y; at each of them the observed nodes
 * draw from N(m + h o_mu, (h e^{clip(o_s)})^2) with that sub-step's normal and
 * transition mean m, and the weights carry g times the product over the span
 * of p / q.  Only a span of one has a fallback to the transition (its
 * candidate comes from the same state); for longer spans ess_frac is
 * ignored.  Tuple recording builds its network inputs from the state before
 * the span, with the residual of the last sub-step as the target.  Spans
 * above one need J divisible by 4.  Synchronises.  Errors: PF_EINVAL,
 * PF_EUNSUPPORTED, PF_ESTATE. */
PF_API pf_status pf_set_proposal_span(pf_ctx *ctx, int32_t span);

/* Records training tuples for the proposal network during the following
 * steps (lattice contexts): for every resampled particle whose filter-local
 * index is a multiple of `stride` and every observed node, the 51 network
 * inputs of its ancestor before the last sub-step (d_X, rows of 51 floats) and
 * the standardised residual (x_t - m) / h of its node (d_R, rows of 2 floats).
 * d_X and d_R are caller-owned device buffers of `capacity` rows that must
 * stay valid while recording is on; tuples past capacity are dropped.  Steps
 * taken while recording are launched without a CUDA graph.  d_X = NULL stops
 * recording.  Synchronises. */
PF_API pf_status pf_record_tuples(pf_ctx *ctx, float *d_X, float *d_R, int64_t capacity, int32_t stride);
/* Rows written so far by the current recording (at most its capacity). */
PF_API pf_status pf_recorded_tuples(const pf_ctx *ctx, int64_t *count);

/* Systematic resampling that allocates nothing.  Some callers cannot call
 * cudaMalloc when they resample -- host frameworks that own every device
 * allocation, real-time loops with a fixed memory budget, where an allocation
 * could fail or stall -- and cannot hand over scratch either.  This variant of
 * pf_systematic_resample takes the same arguments minus the scratch, and uses
 * a device array built into the library instead (about 3.3 MB, held by every
 * GPU that loads the library until the process exits).
 * The paper has no counterpart; it is a convenience of this library.
 * Limits: M <= PF_NOALLOC_MAX_FILTERS and sum N_m <= PF_NOALLOC_MAX_PARTICLES,
 * else PF_EINVAL (message in pf_last_error(NULL)).
 * Each call looks the array's address up on the current device, which must be
 * the device of `stream` and of the pointers.  The first call on a device also
 * loads the array there (the library's device code is loaded on first use), so
 * that first call should come before any stream capture.
 * Every call on a device shares the one array, which keeps the previous call's
 * contents: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The call calls no
 * cudaMalloc, cudaFree or allocating routine; like pf_systematic_resample it
 * synchronises `stream` once to upload its plan.  Results are identical to
 * pf_systematic_resample's.
 * Errors: PF_EINVAL, PF_ECUDA. */
#define PF_NOALLOC_MAX_FILTERS 1024
#define PF_NOALLOC_MAX_PARTICLES 262144
PF_API pf_status pf_systematic_resample_noalloc(int32_t M, const int32_t *h_N, const double *d_w, const double *d_u,
                                                int32_t *d_anc, void *stream);

/* Self-test of the failure detection of bounded device waits.  Every wait of
 * this library's kernels on another agent (the tensor cores' completion
 * barriers) is bounded by the GPU's global timer; a wait that runs out sets
 * the error word the host turns into PF_ETIMEOUT instead of hanging the GPU.
 * This call runs one such wait, with a 20 ms limit, on a barrier of its own:
 * arrive != 0 completes the barrier first (the wait succeeds: PF_OK); arrive
 * == 0 leaves it incomplete, so nothing can end the wait but its limit
 * (PF_ETIMEOUT, message in pf_last_error(NULL)).  Either way no work is in
 * flight when the wait gives up, the kernel returns, and the device and every
 * context stay usable.  stream: a CUDA stream of the current device, or NULL.
 * Synchronises the stream.  Errors: PF_ECUDA.  The paper has no counterpart;
 * it checks this library's own error path. */
PF_API pf_status pf_probe_bounded_wait(int32_t arrive, void *stream);

/* --------------------------------------------------------------------- */
/* Synthetic records                                                      */
/* --------------------------------------------------------------------- */

/* Simulates the hidden state and a T-step observation record on the device
 * in FP64 with the stream-0 (dynamics) and stream-1 (observation noise)
 * random numbers of `record` (counter word 2).  init_random = 0 starts at
 * x0_mean, 1 draws X_0 from the prior with stream 6.  h_x: (T+1) x dx
 * doubles (X_0 .. X_T at observation times); h_y: T x dy floats (may be
 * NULL).  Synchronous.  Errors: PF_EINVAL, PF_ENOMEM, PF_ECUDA. */
PF_API pf_status pf_simulate(const pf_model *model, double dt, const pf_obs_op *obs, const pf_noise *noise, int32_t T,
                      int32_t record, int32_t init_random, double *h_x, float *h_y);

/* Library version string. */
PF_API const char *pf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PF_GB300_PF_H */
