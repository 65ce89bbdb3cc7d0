/*
 * tsmc.h -- C ABI of the B300 transdimensional SMC library (libtsmc.so).
 *
 * Method: Demasi & Del Pozzo, "Massively parallel transdimensional sampling
 * with data assimilation".  A population of particles (k, theta_k) moves from
 * the prior (or from a previous posterior) to the posterior through tempered
 * bridges (Sec. 2, Eqs. prior_bridge / reuse_bridge); each stage reweights
 * (Eq. incremental_weight), picks beta by ESS bisection (Eqs. ess, ess_target),
 * resamples and mutates with a mixture of NUTS and reversible-jump birth/death
 * kernels (Eq. kernel_mixture, Sec. 3.1-3.2, Sec. 4).
 *
 * Conventions
 *   - Every pointer argument named *_dev is CUDA device memory of the current
 *     device; *_host is host memory.  The caller owns every buffer.  The
 *     library never allocates device memory: all state lives in the workspace
 *     the caller passes to tsmc_create.
 *   - Coordinates z are FP64, row-major [n_problems * P][kmax][D], unconstrained
 *     (logit) coordinates, or positions on a circle for the parameters set in
 *     tsmc_config.wrap_mask; D = 3 (pulse: A, t0, w), 4 (sinusoid: A, f, fdot,
 *     phi0), 1 (linear-amplitude test model).  Rows k >= K_p are ignored on
 *     input and written as zero.
 *   - Particle index = problem * P + local index.
 *   - All calls are ordered on the stream given to tsmc_create.  Calls that
 *     return host values synchronise that stream; the others are asynchronous.
 *   - Errors: argument errors return TSMC_EINVAL synchronously; CUDA launch
 *     errors return TSMC_ECUDA.  A non-finite target density is not an error
 *     (it means probability zero: the move is rejected / the subtree diverges).
 *     A particle whose coordinates give a non-finite likelihood or Gauss-Newton
 *     diagonal (a NaN coordinate) is left out of the metric and gets weight zero
 *     at the next reweighting, so resampling drops it.
 *     tsmc_last_error gives a one-line message for the last failure.
 *   - One context per host thread; contexts are independent.
 */
#ifndef TSMC_H
#define TSMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TSMC_OK = 0,
  TSMC_EINVAL = -1,     /* bad argument (sizes, null pointers, non-finite data) */
  TSMC_ENOMEM = -2,     /* workspace smaller than tsmc_workspace_bytes */
  TSMC_ECUDA = -3,      /* a CUDA call or kernel launch failed */
  TSMC_ENONFINITE = -4, /* non-finite value in host data */
  TSMC_ETIMEOUT = -5,   /* reserved: a bounded device wait ran out */
  TSMC_ESTATE = -6      /* call out of order (e.g. moves before data) */
} tsmc_status;

typedef enum { TSMC_PULSE = 0, TSMC_SINUSOID = 1, TSMC_PULSE_LINAMP = 2 } tsmc_model;
typedef enum { TSMC_FP64 = 0, TSMC_MIXED = 1 } tsmc_precision;
typedef enum { TSMC_SCHED_ROUNDS = 0, TSMC_SCHED_MIXTURE = 1 } tsmc_schedule;

typedef struct {
  int32_t model;          /* tsmc_model */
  int32_t precision;      /* tsmc_precision: FP64 everywhere, or FP32 templates/residuals */
  int32_t schedule;       /* ROUNDS: each round one RJ move then one NUTS transition;
                             MIXTURE: each round each particle draws NUTS/birth/death
                             with p_nuts/p_birth/p_death (Eq. kernel_mixture) */
  int32_t n_problems;     /* independent data sets sharing one launch */
  int32_t particles;      /* P, particles per problem */
  int32_t kmax;           /* maximum component count (LINAMP: the fixed count) */
  int32_t n_mut;          /* mutation rounds per stage */
  int32_t max_depth;      /* NUTS maximum tree depth (<= 10) */
  double alpha;           /* ESS target fraction, Eq. ess_target */
  double p_nuts, p_birth, p_death;  /* Eq. kernel_mixture; p_birth=p_death=0.5 in ROUNDS */
  double amp_mean, amp_sd;          /* LINAMP Gaussian amplitude prior */
  uint64_t seed;          /* Philox4x64-10 key word 0 (word 1 = problem_base + problem index) */
  int32_t threads;        /* threads per particle block (32..256, multiple of 32); 0: default
                             (64 for TSMC_PULSE on TSMC_MIXED; else 128) */
  int32_t samples_per_thread;  /* mixed path register tile: 0 (default 32), 16 or 32 */
  int32_t pulse_window;   /* mixed pulse path: 1 skips every (component, 32-thread sample
                             range) pair where |t - t0| > 6 w throughout, i.e. all template
                             terms < 2^-26 A (under the FP32 resolution of A); 0 evaluates
                             every component on every sample.  FP64 path: always 0. */
  int32_t kmin;           /* minimum component count: K prior U{kmin..kmax} (0 <= kmin <= kmax;
                             LINAMP: ignored, K is kmax) */
  int32_t birth_proposal; /* 0: births drawn from the prior (Sec. 4, the paper's method);
                             1: from the population mixture described at
                             tsmc_build_birth_proposal (Sec. 6 suggestion).  LINAMP: ignored */
  double birth_prior_weight;  /* eps in (0, 1] of that mixture (used when birth_proposal = 1) */
  int32_t channels;       /* 0 or 1: one data channel.  2 (TSMC_SINUSOID only): the two
                             noise-orthogonal channels A and E of Sec. 5.2; each problem's
                             data are channel A's samples then channel E's (same times,
                             2 x a multiple of 32 samples), channel c sees
                             response[2c] A cos(phi(t) + response[2c+1]).  With a flat PSD S
                             the frequency-domain likelihood of eq. gw_likelihood equals this
                             time-domain one with sigma^2 = S / (2 dt) (Parseval; DC and
                             Nyquist bins aside).  No tsmc_assimilate for two channels. */
  double response[4];     /* channels = 2: (r_A, delta_A, r_E, delta_E), r_c > 0 */
  int32_t problem_base;   /* >= 0: Philox key word 1 of problem b is problem_base + b.  A
                             process that owns problems [a, a + n) of a larger set of
                             independent problems sets it to a and draws exactly the random
                             numbers a context over the whole set draws for them (sharding
                             across GPUs needs no exchange); 0 for a single context */
  int32_t fused_rounds;   /* mixed path, tsmc_run_stage: 0 (default) launches the birth/death
                             and NUTS kernels once per round; 1 runs the n_mut rounds of a
                             stage in one persistent launch (each block takes the next
                             particle, longest first, and runs all its rounds, so no block
                             idles behind the deepest trees at the end of a round).  Both give
                             the same results bit for bit; on the pulse and band workloads the
                             fused kernel computed 8% fewer component*samples per second.  The
                             FP64 path always launches per round. */
  int32_t particles_global; /* 0: the context holds each problem's whole population.  Else
                               the particles of each problem are sharded across processes
                               (see the calls for a sharded population below): the whole population
                               has particles_global particles per problem and this context
                               holds particles [particle_base, particle_base + particles) */
  int32_t particle_base;  /* global index of the context's first particle (Philox counter
                             word 0 = particle_base + local index), 0 unless sharded */
  uint32_t wrap_mask;     /* bit d set: parameter d is periodic on [lo_d, hi_d), a phase such
                             as the sinusoid phi0 ~ U[0, 2 pi) of Sec. 5.2 (bit 3):
                             theta = lo + (hi - lo)(z - floor z), so z lives on a circle, its
                             prior density is flat (log prior 0, no gradient or curvature),
                             prior draws and births take z = u in (0, 1), and every NUTS
                             transition leaves the coordinate reduced to z - floor z.  0: every
                             parameter uses the logit map.  Bits at or above the model's D, a
                             bit also set in a problem's logmask (tsmc_set_problem), the LINAMP
                             model and birth_proposal = 1 (whose kernel density is not
                             periodic) give TSMC_EINVAL */
} tsmc_config;

/* Opaque context: created by tsmc_create, released by tsmc_destroy. */
typedef struct tsmc_ctx tsmc_ctx;

/* Workspace size for a configuration and per-problem sample capacities
 * n_capacity_host[n_problems] (the largest N each problem will hold, including
 * assimilated samples; both channels' samples for channels = 2).  Each capacity must be
 * in [1, 2^24]: sample indices are exact in FP32 and fit 32-bit arithmetic in the
 * sample loops; otherwise TSMC_EINVAL.  The workspace must be 256-byte aligned device
 * memory. */
tsmc_status tsmc_workspace_bytes(const tsmc_config* cfg, const int64_t* n_capacity_host,
                                 size_t* bytes);

/* Creates a context over a caller-owned workspace; cuda_stream is a cudaStream_t
 * (NULL: legacy default stream).  The context keeps pointers into the workspace,
 * which must outlive it. */
tsmc_status tsmc_create(const tsmc_config* cfg, const int64_t* n_capacity_host,
                        void* workspace_dev, size_t bytes, void* cuda_stream, tsmc_ctx** ctx_out);
tsmc_status tsmc_destroy(tsmc_ctx* ctx);
const char* tsmc_last_error(const tsmc_ctx* ctx);

/* Data of one problem: samples d_n (host FP64, n <= capacity) on the grid
 * t_n = t_origin + n*dt with white noise sigma; per-parameter prior bounds
 * lo/hi (theta = lo + (hi-lo) s(z), or log-uniform where bit d of logmask is
 * set).  All samples count as new (n1 = 0).  Copies to the device. */
tsmc_status tsmc_set_problem(tsmc_ctx* ctx, int32_t problem, const double* d_host, int64_t n,
                             double t_origin, double dt, double sigma, const double* lo_host,
                             const double* hi_host, uint32_t logmask);

/* LINAMP only: fixed (t0, w) per component, host [kmax][2]. */
tsmc_status tsmc_set_fixed_components(tsmc_ctx* ctx, const double* tw_host);

/* Prior start (Sec. 4 step 1): K ~ U{kmin..kmax}, z ~ logistic (theta from its prior;
 * z ~ U(0, 1) for a periodic parameter); beta = 0, log Z = 0, step size
 * eps_0 = 0.5 (kmax D)^(-1/4), unit metric. */
tsmc_status tsmc_init_population(tsmc_ctx* ctx);

/* Posterior start / resume: population from device arrays, beta and log Z per problem. */
tsmc_status tsmc_set_population(tsmc_ctx* ctx, const double* z_dev, const int32_t* K_dev,
                                const double* beta_host, const double* logz_host);
/* Copies the population out (any output may be NULL). */
tsmc_status tsmc_get_population(tsmc_ctx* ctx, double* z_dev, int32_t* K_dev, double* ll_old_dev,
                                double* ll_new_dev);

/* Batched logL + adjoint gradient (hot path) over caller arrays for all
 * n_problems*P particles, each with its own K_p and its problem's data:
 *   r_n = d_n - sum_{k<K} h(t_n; theta_k)
 *   ll_old = -1/2 sum_{n<n1} r_n^2/sigma^2, ll_new = -1/2 sum_{n>=n1} r_n^2/sigma^2
 *   logp = ll_old + beta_p * ll_new + log prior(z)
 *   grad = d logp / dz   ([P][kmax][D], zero rows beyond K)
 *   fisher = per-particle sum over components of the Gauss-Newton diagonal
 *            sum_n c_n (dh/dz_d)^2/sigma^2 + prior curvature, [P][D]
 * beta_dev[n_problems] (NULL: the context's current beta).  Any output may be NULL
 * except ll_new_dev; grad and fisher cost a second pass over the samples. */
tsmc_status tsmc_eval_logl_grad(tsmc_ctx* ctx, const double* z_dev, const int32_t* K_dev,
                                const double* beta_dev, double* ll_old_dev, double* ll_new_dev,
                                double* logp_dev, double* grad_dev, double* fisher_dev);

/* Reversible-jump birth/death move on the context population (Sec. 3.1):
 * birth proposes one component from its prior, death removes a uniform one;
 * log alpha = dL_c + log p_death - log p_birth (birth) or its mirror (death),
 * dL_c from the incremental change (r.h - h.h/2)/sigma^2 (birth) or
 * -(r.h + h.h/2)/sigma^2 (death) with per-sample temperatures.  Random numbers
 * use (stage, round).  outcome_dev[P_total] (nullable): 0 no move, 1/2 birth/death
 * accepted, -1/-2 rejected. */
tsmc_status tsmc_rj_move(tsmc_ctx* ctx, int32_t stage, int32_t round, int32_t* outcome_dev);

/* One NUTS transition per particle (Sec. 3.2) with the context's step size and
 * diagonal metric.  acc_dev (mean min(1, e^{H0-H}) over leaves), nleaf_dev,
 * flags_dev (bit0 divergence, bits 8-15 depth) are nullable [P_total] outputs. */
tsmc_status tsmc_nuts_move(tsmc_ctx* ctx, int32_t stage, int32_t round, double* acc_dev,
                           int32_t* nleaf_dev, int32_t* flags_dev);

/* Step size and inverse diagonal metric per problem: eps_host[n_problems],
 * minv_host[n_problems][D]. */
tsmc_status tsmc_set_kernel_params(tsmc_ctx* ctx, const double* eps_host, const double* minv_host);
tsmc_status tsmc_get_kernel_params(tsmc_ctx* ctx, double* eps_host, double* minv_host);

/* Population birth proposal (Sec. 6: the particles of each SMC stage approximate its
 * tempered distribution, so that distribution can propose births).  In z coordinates
 *   q(z) = eps prior_z(z) + (1 - eps)/m sum_i N(z; c_i, diag(h^2)),
 * prior_z the standard logistic density per parameter, eps = birth_prior_weight, the
 * m = 256 centres c_i components drawn uniformly (with replacement) over all components of
 * the population, h_d = sd_d (4/(D+2))^(1/(D+4)) m^(-1/(D+4)) (normal-reference rule on the
 * centres, at least 1e-3).  Births then carry log prior_z(z_new) - log q(z_new) and deaths
 * log q(z_j) - log prior_z(z_j) in their acceptance.  With birth_proposal = 1,
 * tsmc_run_stage builds it after resampling from the resampled population; this call
 * builds it now from the context population with the given stage number in the random
 * stream (stream-ordered; EINVAL for LINAMP or stage < 0).  Until a build, every problem's
 * proposal is the prior. */
tsmc_status tsmc_build_birth_proposal(tsmc_ctx* ctx, int32_t stage);

/* The proposal of one problem into host out[n]: out[0] = m (0: none built or no
 * components), out[1..4] = h, out[5 ..] = centres [256][D] row-major.  n >= 5 + 256 D,
 * else EINVAL.  Synchronises the context stream. */
tsmc_status tsmc_get_birth_proposal(tsmc_ctx* ctx, int32_t problem, double* out_host, int64_t n);

/* Metric from the population (Sec. 3.2, mass matrix = Hessian of -log target):
 * minv_d = 1 / max(1e-8, mean over particles and active components of the
 * Gauss-Newton diagonal at the current beta; particles with a non-finite diagonal
 * are left out). */
tsmc_status tsmc_update_metric(tsmc_ctx* ctx);

/* Choose beta by ESS bisection, reweight (evidence increment) and resample
 * systematically (Sec. 2 steps 1-2).  Systematic resampling runs on weights quantised
 * to integers, round(exp(logw - max) 2^S) with S = 52 - ceil(log2 P), whose prefix sums
 * are exact; ancestor i is the first j with C_j > min((i + U) / P C_P, C_P - 1).  Host
 * outputs (nullable) [n_problems]; with all three NULL the call does not synchronise. */
tsmc_status tsmc_temper_reweight_resample(tsmc_ctx* ctx, int32_t stage, double* beta_host,
                                          double* logz_host, double* ess_host);
/* Current beta, log Z and last ESS per problem (host [n_problems], nullable);
 * synchronises the stream. */
tsmc_status tsmc_get_state(tsmc_ctx* ctx, double* beta_host, double* logz_host, double* ess_host);

/* Ancestors of the last resampling, [P_total] local indices (test access). */
tsmc_status tsmc_get_ancestors(tsmc_ctx* ctx, int32_t* anc_dev);

/* One whole stage: temper/reweight/resample, metric, n_mut mutation rounds,
 * step-size update eps <- eps exp(mean_acc - 0.8) clamped to [1e-4, 2].
 * Problems already at beta = 1 before the stage are skipped.  Host outputs
 * (nullable) [n_problems]; with all three NULL the call does not synchronise
 * (stages can be queued back to back).  Uses a CUDA graph for the mutation rounds
 * when use_graph != 0 and the stream is not the legacy default stream. */
tsmc_status tsmc_run_stage(tsmc_ctx* ctx, int32_t stage, int32_t use_graph, double* beta_host,
                           double* logz_host, double* ess_host);

/* Data assimilation (Eq. reuse_bridge, Sec. 5.1-5.2 posterior start): append
 * n_new samples to a problem, mark them new (n1 = old n), recompute each
 * particle's logL on the new samples and restart that problem's beta at 0.
 * The evidence accumulator restarts at 0 (it then estimates log Z(d2)/Z(d1)).
 * The bridge starts from the posterior of the samples held so far: a problem whose
 * beta is below 1 is refused with TSMC_ESTATE (nothing changes).  Other problems keep
 * their state.  Synchronises the stream. */
tsmc_status tsmc_assimilate(tsmc_ctx* ctx, int32_t problem, const double* d_new_host, int64_t n_new);

/* Philox4x64-10 (the library's random stream) on the device: out_dev[4*i..4*i+3]
 * = Philox(ctr_dev[4*i..4*i+3], {key0, key1}) for i < n. */
tsmc_status tsmc_philox(tsmc_ctx* ctx, const uint64_t* ctr_dev, uint64_t key0, uint64_t key1,
                        int64_t n, uint64_t* out_dev);

/* Statistics (no counterpart in the paper's method; measurement support):
 * cs_evals_host[4] = component*sample logL+grad evaluations done by this context's
 * kernels: [0] batched evaluations with a gradient and [1] NUTS (every leaf plus the
 * initial point), each the sum of K_p * N_b per evaluation; [2] and [3] the same
 * evaluations counting only the component*samples actually computed (less than
 * [0], [1] when pulse_window skips the far tails).  launches_host = kernels launched.
 * reset != 0 zeroes both after reading.  Synchronises the stream. */
tsmc_status tsmc_counters(tsmc_ctx* ctx, uint64_t* cs_evals_host, int64_t* launches_host,
                          int32_t reset);

/* Per-kernel-class event timing of eager launches (graphs are not used while it is
 * on).  Classes: 0 eval, 1 rj, 2 nuts, 3 temper, 4 resample, 5 gather, 6 metric,
 * 7 other.  tsmc_profile_read fills launches_host[8] and ms_host[8] (device time
 * between events recorded on the context stream around each launch) and
 * synchronises the stream; reset != 0 forgets the records.  enable > 1 also
 * creates that many events up front (two per recorded launch). */
tsmc_status tsmc_profile(tsmc_ctx* ctx, int32_t enable);
tsmc_status tsmc_profile_read(tsmc_ctx* ctx, int64_t* launches_host, double* ms_host, int32_t reset);

/* A population sharded across processes (Sec. 6: moves are independent per particle, the
 * reweighting, ESS and resampling are the global steps).  Each process holds a block of every
 * problem's particles in a context with particles_global and particle_base set, draws the
 * random numbers of those global particle indices, and joins the others with its own
 * collectives; a stage is:
 *   1. all-gather every shard's ll_new (tsmc_get_population) into ell [n_problems][P_global]
 *      in global particle order;
 *   2. tsmc_temper_resample_global: every process picks the same beta by ESS bisection,
 *      adds the same evidence increment and draws the same systematic ancestors anc
 *      [n_problems][P_global] (global indices) from the whole population;
 *   3. exchange particles so that each process holds rows anc[i] for its own i, then
 *      tsmc_load_population;
 *   4. tsmc_metric_sums, all-reduce (sum) the [n_problems][5] sums, tsmc_metric_apply;
 *   5. tsmc_mutation_rounds, all-reduce (sum) the [n_problems][2] acceptance statistics,
 *      tsmc_eps_update_apply.
 * With particles_global set, tsmc_run_stage and tsmc_temper_reweight_resample refuse with
 * TSMC_ESTATE, and births from the population proposal are not available (EINVAL at create).
 * All five calls are asynchronous on the context stream; device arrays as stated. */
tsmc_status tsmc_temper_resample_global(tsmc_ctx* ctx, int32_t stage, const double* ell_dev,
                                        int32_t* anc_dev);
/* Replaces the context's particles (z [P_total][kmax][D], K, ll_old, ll_new on the device)
 * and keeps beta, log Z, step size and metric; K outside [0, kmax] is clamped by the
 * kernels. */
tsmc_status tsmc_load_population(tsmc_ctx* ctx, const double* z_dev, const int32_t* K_dev,
                                 const double* ll_old_dev, const double* ll_new_dev);
/* Population sums of the metric over the context's particles, sums_dev [n_problems][5]:
 * per parameter the sum of the particles' Gauss-Newton sums, then the sum of K (particles
 * with a non-finite diagonal left out). */
tsmc_status tsmc_metric_sums(tsmc_ctx* ctx, double* sums_dev);
/* Metric from (all-reduced) sums: minv_d = 1 / max(1e-8, sum_d / sum K). */
tsmc_status tsmc_metric_apply(tsmc_ctx* ctx, const double* sums_dev);
/* The n_mut mutation rounds of a stage with the current step size and metric; writes the
 * stage's acceptance statistics (sum over moved particles of the acceptance statistic,
 * their number) per problem into stats_dev [n_problems][2]. */
tsmc_status tsmc_mutation_rounds(tsmc_ctx* ctx, int32_t stage, double* stats_dev);
/* Step-size update eps <- eps exp(sum / count - 0.8), clamped to [1e-4, 2], from
 * (all-reduced) statistics [n_problems][2]. */
tsmc_status tsmc_eps_update_apply(tsmc_ctx* ctx, const double* stats_dev);

/* Systematic resampling without any device allocation and without a context.
 *
 * The paper has no counterpart: this is a packaging variant of the resampling
 * step of tsmc_temper_reweight_resample for callers that cannot allocate device
 * memory and cannot hold a caller-sized workspace -- e.g. code running while a
 * stream is being captured into a CUDA graph (a cudaMalloc there breaks the
 * capture), host frameworks that hand all device memory to their own pool at
 * start-up, or latency-bound loops that must not take cudaMalloc's implicit
 * device synchronisation.  The caller still owns the input and output buffers.
 *
 *   logw_dev       [n_problems * particles] FP64 log-weights (any finite shift)
 *   ancestors_dev  [n_problems * particles] int32 output, local indices per problem:
 *                  a_i = min{j : C_j > min((i + U) / P C_P, C_P - 1)}, C the exact
 *                  integer prefix sums of round(exp(logw - max) 2^S), S = 52 -
 *                  ceil(log2 P), U from Philox key (seed, problem), counter
 *                  (0, stage, purpose 7, 0) -- the same draw and arithmetic as the
 *                  context path, so the results are identical.
 *   cuda_stream    cudaStream_t the kernel is launched on (NULL: legacy stream).
 *
 * Limits: n_problems * particles <= 65536 and n_problems <= 256; larger sizes are
 * rejected with TSMC_EINVAL (message in tsmc_last_error(NULL)).  The scratch is a
 * fixed 512 KB file-scope device array (plus 256 all-zero problem descriptors)
 * that every GPU which loads the library keeps until the process exits.  The
 * first call on a device looks up the arrays' device addresses
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Every call shares the same scratch and the kernel
 * overwrites it before reading it; calls whose kernels overlap on the GPU (for
 * example on two streams) race on it.  Asynchronous: no synchronisation. */
tsmc_status tsmc_resample_systematic_static(const double* logw_dev, int32_t n_problems,
                                            int32_t particles, uint64_t seed, int32_t stage,
                                            int32_t* ancestors_dev, void* cuda_stream);

/* Waits for the stream; returns TSMC_ECUDA with a message on an asynchronous error. */
tsmc_status tsmc_sync(tsmc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
