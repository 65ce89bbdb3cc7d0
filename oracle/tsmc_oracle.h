/*
 * tsmc_oracle.h -- the oracle: a plain, single-threaded FP64 CPU statement of
 * the transdimensional SMC method (Demasi & Del Pozzo, "Massively parallel
 * transdimensional sampling with data assimilation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; both sides implement
 * Philox4x64-10 from its published definition (Salmon et al., SC'11).
 *
 * Conventions (shared by specification only, not by code):
 *   z      particle coordinates, row-major [kmax][D], unconstrained (logit) space
 *   K      active component count; rows k >= K are ignored on input, zero on output
 *   c_n    per-sample temperature: 1 for n < n1 (already-assimilated samples), beta otherwise
 *   ll_old = -1/2 sum_{n<n1} r_n^2 / sigma^2,  ll_new = -1/2 sum_{n>=n1} r_n^2 / sigma^2
 *   logp   = ll_old + beta*ll_new + log prior density of z (fixed K)
 */
#ifndef TSMC_ORACLE_H
#define TSMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PULSE = 0, ORC_SINUSOID = 1, ORC_PULSE_LINAMP = 2 };
enum { ORC_SCHED_ROUNDS = 0, ORC_SCHED_MIXTURE = 1 };

/* Philox stream purposes; counter = {particle, stage, (round<<4)|purpose, index},
 * key = {seed, problem}. */
enum {
  ORC_PU_INIT = 0, ORC_PU_MOMENTUM = 1, ORC_PU_DIRECTION = 2, ORC_PU_LEAF = 3,
  ORC_PU_TOP = 4, ORC_PU_RJ = 5, ORC_PU_RJPARAM = 6, ORC_PU_RESAMPLE = 7,
  ORC_PU_MOVETYPE = 8, ORC_PU_KDE = 9
};

typedef struct {
  int32_t model;          /* ORC_PULSE / ORC_SINUSOID / ORC_PULSE_LINAMP */
  int32_t D;              /* parameters per component: 3 / 4 / 1 */
  int32_t kmax;           /* maximum component count (fixed K for LINAMP) */
  int32_t kmin;           /* minimum component count of the K prior (0 <= kmin <= kmax) */
  int32_t birth_proposal; /* 0: births from the prior; 1: population mixture (orc_kde) */
  double birth_prior_weight;      /* epsilon: prior weight of the population mixture */
  int32_t channels;       /* sinusoid: 1, or 2 data channels (A, E) */
  double resp[4];         /* two channels: (r_A, delta_A, r_E, delta_E), channel c sees
                             r_c A cos(phi(t) + delta_c) */
  int32_t n_mut;          /* mutation rounds per stage */
  int32_t max_depth;      /* NUTS maximum tree depth */
  int32_t schedule;       /* ORC_SCHED_ROUNDS or ORC_SCHED_MIXTURE */
  double alpha;           /* ESS target fraction */
  double p_nuts, p_birth, p_death;
  double lo[4], hi[4];    /* per-parameter prior bounds */
  uint32_t logmask;       /* bit d set: parameter d is log-uniform */
  double amp_mean, amp_sd;        /* LINAMP Gaussian amplitude prior */
  const double* fixed_tw;         /* LINAMP: [kmax][2] fixed (t0, w) */
  uint64_t seed;
  uint32_t wrapmask;      /* bit d set: parameter d is periodic on [lo, hi) (a phase) */
} orc_cfg;

typedef struct {
  const double* d;        /* samples d_n, n < n */
  int64_t n;              /* number of samples in use */
  int64_t n1;             /* first not-yet-assimilated sample (0: prior start) */
  double t_origin, dt;    /* t_n = t_origin + n*dt */
  double sigma;           /* white-noise standard deviation */
} orc_data;

/* Population birth proposal (the paper's suggestion for future work, Sec. 6: the
 * particles approximate each tempered distribution, so it can serve as the proposal):
 * q(z) = eps * prior_z(z) + (1 - eps) / m * sum_i N(z; c_i, diag(h^2)) in z coordinates. */
#define ORC_KDE_M 256
typedef struct {
  int32_t m;                      /* centres in use (0: the proposal is the prior) */
  double h[4];                    /* bandwidth per parameter type */
  double c[ORC_KDE_M * 4];        /* centres [m][D] */
} orc_kde;

void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
double orc_u01(uint64_t x);

/* z -> theta map and its derivative for one parameter of type d */
void orc_z_to_theta(const orc_cfg* c, int d, double z, double* theta, double* dtheta_dz);
double orc_z_from_u01(const orc_cfg* c, int d, double u);   /* z whose theta is the u-quantile */

/* single template and its parameter derivatives at time t (component k for LINAMP) */
double orc_template(const orc_cfg* c, int k, const double* theta, double t, double* dh);
/* the same in data channel ch (two-channel sinusoids: response r_ch, delta_ch) */
double orc_template_ch(const orc_cfg* c, int k, const double* theta, double t, int ch,
                       double* dh);

/* logL parts, tempered log target and its gradient for one particle */
void orc_logl_grad(const orc_cfg* c, const orc_data* dat, const double* z, int32_t K, double beta,
                   double* ll_old, double* ll_new, double* logp, double* grad,
                   double* gscale, double* fisher);

/* same over P particles; outputs are per particle, grad/gscale/fisher [P][kmax][D] (nullable) */
void orc_logl_grad_batch(const orc_cfg* c, const orc_data* dat, const double* z, const int32_t* K,
                         int32_t P, double beta, double* ll_old, double* ll_new, double* logp,
                         double* grad, double* gscale, double* fisher);

void orc_init_population(const orc_cfg* c, int32_t problem, int32_t P, double* z, int32_t* K);

/* one reversible-jump birth/death move for every particle (or, in the mixture schedule,
 * for the particles whose move-type draw selects birth or death).
 * outcome[i]: 0 no RJ move this round, 1 birth accepted, 2 death accepted,
 *             -1 birth rejected, -2 death rejected */
void orc_rj_move(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t stage,
                 int32_t round, double beta, int32_t P, double* z, int32_t* K,
                 double* ll_old, double* ll_new, int32_t* outcome);

/* the same move with births proposed from q (kde != NULL and c->birth_proposal == 1) */
void orc_rj_move_q(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t stage,
                   int32_t round, double beta, int32_t P, double* z, int32_t* K,
                   double* ll_old, double* ll_new, int32_t* outcome, const orc_kde* kde);

/* centres: m = ORC_KDE_M components drawn uniformly (with replacement) over all
 * components of the population; bandwidth by the normal-reference rule */
void orc_kde_build(const orc_cfg* c, int32_t problem, int32_t stage, int32_t P,
                   const double* z, const int32_t* K, orc_kde* kde);
double orc_log_prior_z(const orc_cfg* c, const double* z);     /* one component, D values */
double orc_kde_logq(const orc_cfg* c, const orc_kde* kde, const double* z);

/* one NUTS transition per particle with step size eps and diagonal inverse metric
 * minv[D] (per parameter type).  acc_stat[i] mean min(1,exp(H0-H)) over leaves,
 * n_leaf[i] leapfrog count (0: particle not moved), flags[i] bit0 diverged,
 * bits 8..15 final tree depth */
void orc_nuts_move(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t stage,
                   int32_t round, double beta, double eps, const double* minv, int32_t P,
                   double* z, const int32_t* K, double* ll_old, double* ll_new,
                   double* acc_stat, int32_t* n_leaf, int32_t* flags);

/* one leapfrog step of size eps (negative: backwards) */
void orc_leapfrog(const orc_cfg* c, const orc_data* dat, int32_t K, double beta, double eps,
                  const double* minv, double* z, double* p, double* grad, double* logp);

/* adaptive tempering: beta_new from ESS(delta) = alpha*P by bisection; logw = delta*ell;
 * logz_inc = LSE(logw) - log P; ess = ESS at the chosen delta */
void orc_temper(int32_t P, const double* ell, double alpha, double beta, double* beta_new,
                double* logz_inc, double* ess, double* logw);

/* systematic resampling: ancestors[i] for i < P */
int32_t orc_resample_scale(int32_t P);
void orc_resample(const orc_cfg* c, int32_t problem, int32_t stage, int32_t P,
                  const double* logw, int32_t* ancestors);

/* inverse diagonal metric per parameter type from the population's Gauss-Newton Hessian */
void orc_metric(const orc_cfg* c, const orc_data* dat, const double* z, const int32_t* K,
                int32_t P, double beta, double* minv);

double orc_eps_update(double eps, double mean_acc);
double orc_eps_initial(const orc_cfg* c);

/* one full SMC run (prior start when init_prior != 0, otherwise posterior start from the
 * given population with dat->n1 marking the new samples).  Per-stage diagnostics go to
 * beta_hist/logz_hist/ess_hist (length max_stages, nullable). Returns the stage count. */
int32_t orc_smc_run(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t P,
                    int32_t init_prior, int32_t stage0, int32_t max_stages, double* eps_io,
                    double* z, int32_t* K, double* ll_old, double* ll_new, double* logz,
                    double* beta_hist, double* logz_hist, double* ess_hist);

#ifdef __cplusplus
}
#endif
#endif
