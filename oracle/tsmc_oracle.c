/*
 * tsmc_oracle.c -- the oracle: plain single-threaded FP64 statement of the
 * transdimensional SMC method of Demasi & Del Pozzo.  TEST INFRASTRUCTURE:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Compile with -ffp-contract=off so that every expression rounds as written.
 * No blocking, fusion or reordering beyond the definitions cited per function.
 *
 * Parity status: every function below is pinned by the CPU tests (numpy's
 * Philox, Richardson finite-difference gradients, closed-form evidence of a
 * linear-Gaussian model, brute-force K posterior, prior invariance of the RJ
 * kernel, leapfrog reversibility, textbook ESS/resampling identities).
 */
#include "tsmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x64-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3" (SC'11): multipliers, Weyl key increments and the round.  */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    __uint128_t p0 = (__uint128_t)M0 * x0;
    __uint128_t p1 = (__uint128_t)M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 53 random bits mapped to the open interval (0,1): (x>>11)*2^-53 + 2^-54 */
double orc_u01(uint64_t x) { return (double)(x >> 11) * 0x1p-53 + 0x1p-54; }

static void draw(const orc_cfg* c, int32_t problem, uint64_t particle, int32_t stage,
                 int32_t round, int32_t purpose, uint64_t index, uint64_t out[4]) {
  uint64_t ctr[4] = {particle, (uint64_t)(uint32_t)stage,
                     ((uint64_t)(uint32_t)round << 4) | (uint64_t)purpose, index};
  uint64_t key[2] = {c->seed, (uint64_t)(uint32_t)problem};
  orc_philox(ctr, key, out);
}

/* Box-Muller: the m-th standard normal of a stream; call m/4 gives two pairs */
static double draw_normal(const orc_cfg* c, int32_t problem, uint64_t particle, int32_t stage,
                          int32_t round, int32_t purpose, uint64_t m) {
  uint64_t w[4];
  draw(c, problem, particle, stage, round, purpose, m / 4, w);
  int pair = (int)((m % 4) / 2);
  double ua = orc_u01(w[2 * pair]), ub = orc_u01(w[2 * pair + 1]);
  double rad = sqrt(-2.0 * log(ua));
  double ang = 2.0 * M_PI * ub;
  return (m % 2 == 0) ? rad * cos(ang) : rad * sin(ang);
}

/* ------------------------------------------------------------------------- */
/* Neumaier compensated summation                                             */
/* ------------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nval(const nsum* a) { return a->s + a->c; }

static double logaddexp(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  double m = a > b ? a : b;
  return m + log1p(exp(-fabs(a - b)));
}

/* ------------------------------------------------------------------------- */
/* Parameterisation.  Uniform prior on [lo,hi]: theta = lo + (hi-lo) s(z),    */
/* s the logistic function; log-uniform: log theta = log lo + (log hi-log lo) */
/* s(z).  Either way the prior density of z is the logistic density           */
/* s(z)(1-s(z)), with d/dz log = 1 - 2 s(z) and -d2/dz2 log = 2 s(1-s).        */
/* Periodic parameters (wrapmask; a phase, uniform on [lo, hi) with lo and hi */
/* the same point of the circle): theta = lo + (hi-lo) (z - floor z), so z    */
/* lives on the circle R/Z, the prior density of z is 1 per period (log 0)    */
/* and has no gradient or curvature.                                          */
/* LINAMP (linear-Gaussian test model): identity map, A ~ N(amp_mean, sd^2).  */
/* The paper samples in BlackJAX's unconstrained space (Sec. 4) and does not  */
/* state the map; this is the reading used throughout.                        */
/* ------------------------------------------------------------------------- */
static double logistic(double z) {
  if (z >= 0) return 1.0 / (1.0 + exp(-z));
  double e = exp(z);
  return e / (1.0 + e);
}

/* z of parameter d whose theta is the prior quantile u in (0, 1): logit(u), or u itself
 * for a periodic parameter */
double orc_z_from_u01(const orc_cfg* c, int d, double u) {
  if (c->wrapmask & (1u << d)) return u;
  return log(u) - log1p(-u);
}

void orc_z_to_theta(const orc_cfg* c, int d, double z, double* theta, double* dtheta_dz) {
  if (c->model == ORC_PULSE_LINAMP) { *theta = z; *dtheta_dz = 1.0; return; }
  if (c->wrapmask & (1u << d)) {
    *theta = c->lo[d] + (c->hi[d] - c->lo[d]) * (z - floor(z));
    *dtheta_dz = c->hi[d] - c->lo[d];
    return;
  }
  double s = logistic(z);
  double ds = s * (1.0 - s);
  if (c->logmask & (1u << d)) {
    double llo = log(c->lo[d]), lhi = log(c->hi[d]);
    double th = exp(llo + (lhi - llo) * s);
    *theta = th;
    *dtheta_dz = th * (lhi - llo) * ds;
  } else {
    *theta = c->lo[d] + (c->hi[d] - c->lo[d]) * s;
    *dtheta_dz = (c->hi[d] - c->lo[d]) * ds;
  }
}

/* log prior density of one coordinate, its z-gradient and curvature */
static void log_prior_1(const orc_cfg* c, int d, double z, double* lp, double* g,
                        double* curv) {
  if (c->model != ORC_PULSE_LINAMP && (c->wrapmask & (1u << d))) {
    *lp = 0.0; *g = 0.0; *curv = 0.0;
    return;
  }
  if (c->model == ORC_PULSE_LINAMP) {
    double sd = c->amp_sd, dz = (z - c->amp_mean) / sd;
    *lp = -0.5 * dz * dz - log(sd) - 0.5 * log(2.0 * M_PI);
    *g = -(z - c->amp_mean) / (sd * sd);
    *curv = 1.0 / (sd * sd);
    return;
  }
  double a = fabs(z);
  *lp = -a - 2.0 * log1p(exp(-a));
  double s = logistic(z);
  *g = 1.0 - 2.0 * s;
  *curv = 2.0 * s * (1.0 - s);
}

/* ------------------------------------------------------------------------- */
/* Templates.  Gaussian pulse h = A exp(-(t-t0)^2/(2w^2)); quasi-monochromatic */
/* sinusoid h = A cos(2 pi f t + pi fdot t^2 + phi0) with the phase evaluated  */
/* in the fixed order ((2pi f) t + (pi fdot)(t t)) + phi0.                     */
/* Pulses: the toy model of Sec. 5.1; sinusoids: the Galactic-binary signal   */
/* of Sec. 5.2 without the detector response.                                 */
/* ------------------------------------------------------------------------- */
double orc_template(const orc_cfg* c, int k, const double* th, double t, double* dh) {
  if (c->model == ORC_PULSE || c->model == ORC_PULSE_LINAMP) {
    double A = th[0], t0, w;
    if (c->model == ORC_PULSE) { t0 = th[1]; w = th[2]; }
    else { t0 = c->fixed_tw[2 * k]; w = c->fixed_tw[2 * k + 1]; }
    double u = (t - t0) / w;
    double g = exp(-0.5 * u * u);
    if (dh) {
      dh[0] = g;
      if (c->model == ORC_PULSE) {
        dh[1] = A * g * u / w;
        dh[2] = A * g * u * u / w;
      }
    }
    return A * g;
  }
  /* sinusoid: (A, f, fdot, phi0) */
  double A = th[0], f = th[1], fd = th[2], p0 = th[3];
  double phi = ((2.0 * M_PI * f) * t + (M_PI * fd) * (t * t)) + p0;
  double cph = cos(phi), sph = sin(phi);
  if (dh) {
    dh[0] = cph;
    dh[1] = -A * sph * (2.0 * M_PI * t);
    dh[2] = -A * sph * (M_PI * (t * t));
    dh[3] = -A * sph;
  }
  return A * cph;
}

/* Two data channels (Sec. 5.2: the noise-orthogonal channels A and E): with a */
/* simplified response, channel ch sees r_ch A cos(phi(t) + delta_ch).        */
double orc_template_ch(const orc_cfg* c, int k, const double* th, double t, int ch,
                       double* dh) {
  if (c->channels != 2) return orc_template(c, k, th, t, dh);
  const double r = c->resp[2 * ch], dl = c->resp[2 * ch + 1];
  double thc[4] = {r * th[0], th[1], th[2], th[3] + dl};
  const double h = orc_template(c, k, thc, t, dh);
  if (dh) dh[0] = r * dh[0];
  return h;
}

/* ------------------------------------------------------------------------- */
/* Likelihood (white Gaussian noise, time domain):                            */
/*   r_n = d_n - sum_{k<K} h(t_n; theta_k)                                     */
/*   logL_c = -1/2 sum_n c_n r_n^2 / sigma^2, c_n = 1 (n<n1) or beta (n>=n1)    */
/* i.e. the tempered prior bridge (beta on all samples, n1=0) and the reuse    */
/* bridge for appended samples (old samples untempered).  Adjoint gradient     */
/* dlogL_c/dtheta_kd = sum_n c_n r_n dh_k/dtheta_d / sigma^2, chain rule to z. */
/* gscale: the same sums of absolute terms (conditioning scale for tests).    */
/* fisher: Gauss-Newton diagonal sum_n c_n (dh/dz)^2/sigma^2 + prior curvature.*/
/* Sec. 2: the bridges Eq. prior_bridge and Eq. reuse_bridge; the noise model */
/* is Eq. gw_likelihood of Sec. 5.2 with a flat PSD, in the time domain.      */
/* ------------------------------------------------------------------------- */
#define ORC_MAXKD 256
void orc_logl_grad(const orc_cfg* c, const orc_data* dat, const double* z, int32_t K, double beta,
                   double* ll_old, double* ll_new, double* logp, double* grad,
                   double* gscale, double* fisher) {
  const int D = c->D;
  const int KD = K * D;
  double theta[ORC_MAXKD], dth[ORC_MAXKD];
  double lprior = 0.0, pg[ORC_MAXKD], pc[ORC_MAXKD];
  for (int i = 0; i < KD; ++i) {
    orc_z_to_theta(c, i % D, z[i], &theta[i], &dth[i]);
    double lp;
    log_prior_1(c, (int)(i % D), z[i], &lp, &pg[i], &pc[i]);
    lprior += lp;
  }
  nsum s_old = {0, 0}, s_new = {0, 0};
  nsum gacc[ORC_MAXKD];
  double aacc[ORC_MAXKD], facc[ORC_MAXKD];
  for (int i = 0; i < KD; ++i) { gacc[i].s = gacc[i].c = 0; aacc[i] = 0; facc[i] = 0; }
  double dh[4];
  /* two channels: samples [0, n/2) are channel A, [n/2, n) channel E, same times */
  const int64_t nc = c->channels == 2 ? dat->n / 2 : dat->n;
  for (int64_t n = 0; n < dat->n; ++n) {
    const int ch = (int)(n / nc);
    double t = dat->t_origin + (double)(n - ch * nc) * dat->dt;
    double hs = 0.0;
    for (int k = 0; k < K; ++k) hs += orc_template_ch(c, k, &theta[k * D], t, ch, NULL);
    double r = dat->d[n] - hs;
    double cn = (n < dat->n1) ? 1.0 : beta;
    if (n < dat->n1) nadd(&s_old, r * r); else nadd(&s_new, r * r);
    for (int k = 0; k < K; ++k) {
      orc_template_ch(c, k, &theta[k * D], t, ch, dh);
      for (int d = 0; d < D; ++d) {
        double term = cn * r * dh[d];
        nadd(&gacc[k * D + d], term);
        aacc[k * D + d] += fabs(term);
        facc[k * D + d] += cn * dh[d] * dh[d];
      }
    }
  }
  double is2 = 1.0 / (dat->sigma * dat->sigma);
  double lo = -0.5 * nval(&s_old) * is2, ln = -0.5 * nval(&s_new) * is2;
  if (ll_old) *ll_old = lo;
  if (ll_new) *ll_new = ln;
  if (logp) *logp = lo + beta * ln + lprior;
  const int KDmax = c->kmax * D;
  for (int i = 0; i < KDmax; ++i) {
    if (i < KD) {
      if (grad) grad[i] = nval(&gacc[i]) * is2 * dth[i] + pg[i];
      if (gscale) gscale[i] = aacc[i] * is2 * fabs(dth[i]) + fabs(pg[i]);
      if (fisher) fisher[i] = facc[i] * is2 * dth[i] * dth[i] + pc[i];
    } else {
      if (grad) grad[i] = 0.0;
      if (gscale) gscale[i] = 0.0;
      if (fisher) fisher[i] = 0.0;
    }
  }
}

void orc_logl_grad_batch(const orc_cfg* c, const orc_data* dat, const double* z, const int32_t* K,
                         int32_t P, double beta, double* ll_old, double* ll_new, double* logp,
                         double* grad, double* gscale, double* fisher) {
  const int64_t stride = (int64_t)c->kmax * c->D;
  for (int32_t i = 0; i < P; ++i) {
    orc_logl_grad(c, dat, z + i * stride, K[i], beta, ll_old ? ll_old + i : NULL,
                  ll_new ? ll_new + i : NULL, logp ? logp + i : NULL,
                  grad ? grad + i * stride : NULL, gscale ? gscale + i * stride : NULL,
                  fisher ? fisher + i * stride : NULL);
  }
}

/* ------------------------------------------------------------------------- */
/* Population initialisation (prior start): K ~ U{kmin..kmax}, each coordinate*/
/* z = logit(u) (so theta ~ its uniform / log-uniform prior); LINAMP: K fixed */
/* at kmax and A = amp_mean + amp_sd * normal.                                */
/* The prior start of Sec. 4 (particles drawn from the prior at beta = 0).    */
/* ------------------------------------------------------------------------- */
void orc_init_population(const orc_cfg* c, int32_t problem, int32_t P, double* z, int32_t* K) {
  const int D = c->D;
  const int64_t stride = (int64_t)c->kmax * D;
  for (int32_t i = 0; i < P; ++i) {
    uint64_t w[4];
    double* zi = z + i * stride;
    for (int64_t j = 0; j < stride; ++j) zi[j] = 0.0;
    if (c->model == ORC_PULSE_LINAMP) {
      K[i] = c->kmax;
      for (int j = 0; j < c->kmax; ++j)
        zi[j] = c->amp_mean + c->amp_sd * draw_normal(c, problem, i, 0, 0, ORC_PU_INIT, 4 + j);
      continue;
    }
    draw(c, problem, i, 0, 0, ORC_PU_INIT, 0, w);
    int32_t k = c->kmin + (int32_t)floor(orc_u01(w[0]) * (double)(c->kmax - c->kmin + 1));
    if (k > c->kmax) k = c->kmax;
    K[i] = k;
    for (int j = 0; j < k * D; ++j) {
      draw(c, problem, i, 0, 0, ORC_PU_INIT, 1 + j / 4, w);
      zi[j] = orc_z_from_u01(c, j % D, orc_u01(w[j % 4]));
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Reversible-jump birth/death (nested append/remove map, unit Jacobian).      */
/* Birth draws the new component from its prior, which cancels the prior      */
/* factor; death removes a uniformly chosen component, whose 1/(K+1) cancels   */
/* the label combinatorics.  With the incremental likelihood change            */
/*   birth: dL = sum_n c_n (r_n h_n - h_n^2/2)/sigma^2                          */
/*   death: dL = -sum_n c_n (r_n h_n + h_n^2/2)/sigma^2                         */
/* log alpha_birth = dL + log p(K+1) - log p(K) + log p_death - log p_birth,   */
/* log alpha_death = dL + log p(K-1) - log p(K) + log p_birth - log p_death;   */
/* p(K) uniform on {kmin..kmax} so the K-prior terms vanish inside the support.*/
/* Birth at kmax and death at kmin are rejected.  Acceptance iff log u < log a.*/
/* Sec. 3.1, Eq. rj_acceptance.                                               */
/* ------------------------------------------------------------------------- */
void orc_rj_move_q(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t stage,
                   int32_t round, double beta, int32_t P, double* z, int32_t* K,
                   double* ll_old, double* ll_new, int32_t* outcome, const orc_kde* kde) {
  const int D = c->D;
  const int64_t stride = (int64_t)c->kmax * D;
  const int use_q = kde != NULL && c->birth_proposal == 1;
  for (int32_t i = 0; i < P; ++i) {
    outcome[i] = 0;
    if (c->model == ORC_PULSE_LINAMP) continue;
    double* zi = z + i * stride;
    uint64_t w[4];
    int birth;
    draw(c, problem, i, stage, round, ORC_PU_RJ, 0, w);
    if (c->schedule == ORC_SCHED_MIXTURE) {
      uint64_t m[4];
      draw(c, problem, i, stage, round, ORC_PU_MOVETYPE, 0, m);
      double um = orc_u01(m[0]);
      if (um < c->p_nuts) continue;
      birth = um < c->p_nuts + c->p_birth;
    } else {
      birth = orc_u01(w[0]) < c->p_birth / (c->p_birth + c->p_death);
    }
    int32_t k = K[i];
    if (birth && k >= c->kmax) { outcome[i] = -1; continue; }
    if (!birth && k <= c->kmin) { outcome[i] = -2; continue; }
    /* the component that is added or removed, in theta space */
    double th_new[4], th_all[ORC_MAXKD], tmp;
    int32_t j = 0;
    for (int q = 0; q < k * D; ++q) orc_z_to_theta(c, q % D, zi[q], &th_all[q], &tmp);
    double znew[4];
    if (birth) {
      uint64_t pw[4], mw[4];
      draw(c, problem, i, stage, round, ORC_PU_RJPARAM, 0, pw);
      draw(c, problem, i, stage, round, ORC_PU_RJPARAM, 2, mw);
      if (use_q && kde->m > 0 && orc_u01(mw[0]) >= c->birth_prior_weight) {
        /* from the population mixture: centre q, then a normal step of width h */
        int32_t q = (int32_t)floor(orc_u01(mw[1]) * (double)kde->m);
        if (q >= kde->m) q = kde->m - 1;
        for (int d = 0; d < D; ++d)
          znew[d] = kde->c[q * D + d] +
                    kde->h[d] * draw_normal(c, problem, i, stage, round, ORC_PU_RJPARAM, 4 + d);
      } else {
        for (int d = 0; d < D; ++d) znew[d] = orc_z_from_u01(c, d, orc_u01(pw[d]));
      }
      for (int d = 0; d < D; ++d) orc_z_to_theta(c, d, znew[d], &th_new[d], &tmp);
    } else {
      j = (int32_t)floor(orc_u01(w[2]) * (double)k);
      if (j >= k) j = k - 1;
      for (int d = 0; d < D; ++d) th_new[d] = th_all[j * D + d];
    }
    nsum a_old = {0, 0}, a_new = {0, 0};
    const int64_t nc = c->channels == 2 ? dat->n / 2 : dat->n;
    for (int64_t n = 0; n < dat->n; ++n) {
      const int ch = (int)(n / nc);
      double t = dat->t_origin + (double)(n - ch * nc) * dat->dt;
      double hs = 0.0;
      for (int q = 0; q < k; ++q) hs += orc_template_ch(c, q, &th_all[q * D], t, ch, NULL);
      double r = dat->d[n] - hs;
      double h = orc_template_ch(c, birth ? k : j, th_new, t, ch, NULL);
      double term = birth ? (r * h - 0.5 * h * h) : -(r * h + 0.5 * h * h);
      if (n < dat->n1) nadd(&a_old, term); else nadd(&a_new, term);
    }
    double is2 = 1.0 / (dat->sigma * dat->sigma);
    double d_old = nval(&a_old) * is2, d_new = nval(&a_new) * is2;
    double dl = d_old + beta * d_new;
    double log_alpha = birth ? dl + log(c->p_death) - log(c->p_birth)
                             : dl + log(c->p_birth) - log(c->p_death);
    if (use_q) {   /* the proposal no longer cancels the prior of the component */
      if (birth) log_alpha += orc_log_prior_z(c, znew) - orc_kde_logq(c, kde, znew);
      else log_alpha += orc_kde_logq(c, kde, zi + j * D) - orc_log_prior_z(c, zi + j * D);
    }
    double u = orc_u01(w[1]);
    if (log(u) < log_alpha) {
      if (birth) {
        for (int d = 0; d < D; ++d) zi[k * D + d] = znew[d];
        K[i] = k + 1;
        outcome[i] = 1;
      } else {
        for (int d = 0; d < D; ++d) {
          zi[j * D + d] = zi[(k - 1) * D + d];
          zi[(k - 1) * D + d] = 0.0;
        }
        K[i] = k - 1;
        outcome[i] = 2;
      }
      ll_old[i] += d_old;
      ll_new[i] += d_new;
    } else {
      outcome[i] = birth ? -1 : -2;
    }
  }
}

void orc_rj_move(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t stage,
                 int32_t round, double beta, int32_t P, double* z, int32_t* K,
                 double* ll_old, double* ll_new, int32_t* outcome) {
  orc_rj_move_q(c, dat, problem, stage, round, beta, P, z, K, ll_old, ll_new, outcome, NULL);
}

/* ------------------------------------------------------------------------- */
/* Population birth proposal (Sec. 6: the particles of each stage approximate  */
/* its tempered distribution, which can serve as the birth proposal).         */
/* In z coordinates every parameter's prior is the standard logistic density, */
/*   log prior_z(z) = sum_d ( -|z_d| - 2 log(1 + e^{-|z_d|}) ).                */
/* The proposal mixes it with a Gaussian kernel density estimate:             */
/*   q(z) = eps prior_z(z) + (1 - eps)/m sum_i prod_d N(z_d; c_id, h_d^2),     */
/* whose m centres are components drawn uniformly, with replacement, over all */
/* components of the population (draw i: particle slot i of purpose KDE, the  */
/* stage, round 0), and h_d = sd_d (4/(D+2))^(1/(D+4)) m^(-1/(D+4)) (the      */
/* normal-reference rule, sd_d the sample deviation of the centres; at least  */
/* 1e-3).  The weight eps keeps q positive wherever the prior is.             */
/* ------------------------------------------------------------------------- */
double orc_log_prior_z(const orc_cfg* c, const double* z) {
  double s = 0.0;
  for (int d = 0; d < c->D; ++d) {
    if (c->wrapmask & (1u << d)) continue;   /* periodic: density 1 per period */
    const double a = fabs(z[d]);
    s += -a - 2.0 * log1p(exp(-a));
  }
  return s;
}

double orc_kde_logq(const orc_cfg* c, const orc_kde* kde, const double* z) {
  const int D = c->D;
  const double lp = orc_log_prior_z(c, z);
  if (kde->m == 0 || c->birth_prior_weight >= 1.0) return lp;
  /* terms of the mixture, then log-sum-exp in index order */
  double t[ORC_KDE_M + 1];
  t[0] = log(c->birth_prior_weight) + lp;
  const double lw = log((1.0 - c->birth_prior_weight) / (double)kde->m);
  for (int i = 0; i < kde->m; ++i) {
    double e = lw;
    for (int d = 0; d < D; ++d) {
      const double u = (z[d] - kde->c[i * D + d]) / kde->h[d];
      e += -0.5 * u * u - log(kde->h[d]) - 0.5 * log(2.0 * M_PI);
    }
    t[i + 1] = e;
  }
  double mx = t[0];
  for (int i = 1; i <= kde->m; ++i) if (t[i] > mx) mx = t[i];
  double sum = 0.0;
  for (int i = 0; i <= kde->m; ++i) sum += exp(t[i] - mx);
  return mx + log(sum);
}

void orc_kde_build(const orc_cfg* c, int32_t problem, int32_t stage, int32_t P,
                   const double* z, const int32_t* K, orc_kde* kde) {
  const int D = c->D;
  const int64_t stride = (int64_t)c->kmax * D;
  int64_t total = 0;
  for (int32_t i = 0; i < P; ++i) total += K[i];
  kde->m = 0;
  for (int d = 0; d < 4; ++d) kde->h[d] = 1.0;
  if (total == 0) return;
  kde->m = ORC_KDE_M;
  for (int32_t i = 0; i < ORC_KDE_M; ++i) {
    uint64_t w[4];
    draw(c, problem, (uint64_t)i, stage, 0, ORC_PU_KDE, 0, w);
    int64_t q = (int64_t)floor(orc_u01(w[0]) * (double)total);
    if (q >= total) q = total - 1;
    int32_t p = 0;          /* the particle holding component number q */
    int64_t before = 0;
    while (before + K[p] <= q) { before += K[p]; ++p; }
    const int64_t j = q - before;
    for (int d = 0; d < D; ++d) kde->c[i * D + d] = z[p * stride + j * D + d];
  }
  const double f = pow(4.0 / (double)(D + 2), 1.0 / (double)(D + 4)) *
                   pow((double)ORC_KDE_M, -1.0 / (double)(D + 4));
  for (int d = 0; d < D; ++d) {
    double mean = 0.0;
    for (int i = 0; i < ORC_KDE_M; ++i) mean += kde->c[i * D + d];
    mean /= (double)ORC_KDE_M;
    double var = 0.0;
    for (int i = 0; i < ORC_KDE_M; ++i) {
      const double e = kde->c[i * D + d] - mean;
      var += e * e;
    }
    var /= (double)(ORC_KDE_M - 1);
    double h = sqrt(var) * f;
    kde->h[d] = h < 1e-3 ? 1e-3 : h;
  }
}

/* ------------------------------------------------------------------------- */
/* Hamiltonian dynamics: H = -logp(z) + 1/2 p^T M^-1 p with diagonal M,        */
/* leapfrog p += eps/2 grad; z += eps M^-1 p; grad'; p += eps/2 grad'.         */
/* Sec. 3.2.                                                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
  const orc_cfg* c; const orc_data* dat; int32_t K; double beta;
  double ll_old, ll_new;
} target_ctx;

static double eval_target(target_ctx* tc, const double* z, double* grad) {
  double lo, ln, lp;
  orc_logl_grad(tc->c, tc->dat, z, tc->K, tc->beta, &lo, &ln, &lp, grad, NULL, NULL);
  tc->ll_old = lo; tc->ll_new = ln;
  return lp;
}

static void leapfrog_tc(target_ctx* tc, double eps, const double* minv, double* z, double* p,
                        double* grad, double* logp) {
  const int D = tc->c->D, n = tc->K * D;
  double gfull[ORC_MAXKD];
  for (int i = 0; i < n; ++i) p[i] = p[i] + 0.5 * eps * grad[i];
  for (int i = 0; i < n; ++i) z[i] = z[i] + eps * minv[i % D] * p[i];
  *logp = eval_target(tc, z, gfull);
  for (int i = 0; i < n; ++i) grad[i] = gfull[i];
  for (int i = 0; i < n; ++i) p[i] = p[i] + 0.5 * eps * grad[i];
}

void orc_leapfrog(const orc_cfg* c, const orc_data* dat, int32_t K, double beta, double eps,
                  const double* minv, double* z, double* p, double* grad, double* logp) {
  target_ctx tc = {c, dat, K, beta, 0, 0};
  leapfrog_tc(&tc, eps, minv, z, p, grad, logp);
}

static double kinetic(int n, int D, const double* minv, const double* p) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += minv[i % D] * p[i] * p[i];
  return 0.5 * s;
}

static double dot_minv(int n, int D, const double* minv, const double* rho, const double* p) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += rho[i] * (minv[i % D] * p[i]);
  return s;
}

/* ------------------------------------------------------------------------- */
/* NUTS transition (No-U-Turn sampler, Hoffman & Gelman 2014, with multinomial */
/* trajectory sampling and the generalised U-turn criterion of Betancourt     */
/* 2017).  Trajectory doubles up to max_depth times in a random direction.     */
/* Inside a new subtree leaves are selected by progressive multinomial         */
/* sampling (leaf replaces the candidate w.p. w_leaf / W_subtree); the subtree */
/* candidate replaces the trajectory candidate w.p. min(1, W_sub / W_old)      */
/* (biased progressive sampling).  Every sub-subtree of size 2^m >= 2 that     */
/* completes inside the new subtree is checked for a U-turn                    */
/* (rho . M^-1 p_end <= 0 at either end, rho = momentum sum over it); a subtree */
/* that turns or diverges (H - H0 > 1000 or non-finite) is discarded and the   */
/* transition stops.  After merging, the whole trajectory is checked the same  */
/* way.  Random numbers: direction (index = depth), leaf selection (index =    */
/* leaf number in the transition), top-level selection (index = depth),       */
/* momentum (normal m of the stream).                                          */
/* Sec. 3.2 (the paper uses BlackJAX's NUTS without stating its variant).     */
/* ------------------------------------------------------------------------- */
#define ORC_MAXDEPTH 10
void orc_nuts_move(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t stage,
                   int32_t round, double beta, double eps, const double* minv, int32_t P,
                   double* z, const int32_t* K, double* ll_old, double* ll_new,
                   double* acc_stat, int32_t* n_leaf_out, int32_t* flags) {
  const int D = c->D;
  const int64_t stride = (int64_t)c->kmax * D;
  for (int32_t i = 0; i < P; ++i) {
    acc_stat[i] = 0.0; n_leaf_out[i] = 0; flags[i] = 0;
    if (c->schedule == ORC_SCHED_MIXTURE) {
      uint64_t m[4];
      draw(c, problem, i, stage, round, ORC_PU_MOVETYPE, 0, m);
      if (!(orc_u01(m[0]) < c->p_nuts)) continue;
    }
    const int n = K[i] * D;
    if (n == 0) continue;
    double* zi = z + i * stride;
    target_ctx tc = {c, dat, K[i], beta, 0, 0};
    double g0[ORC_MAXKD], p0[ORC_MAXKD];
    double logp0 = eval_target(&tc, zi, g0);
    double cand_lo = tc.ll_old, cand_ln = tc.ll_new;
    for (int q = 0; q < n; ++q)
      p0[q] = sqrt(1.0 / minv[q % D]) *
              draw_normal(c, problem, i, stage, round, ORC_PU_MOMENTUM, (uint64_t)q);
    const double H0 = -logp0 + kinetic(n, D, minv, p0);
    double zL[ORC_MAXKD], pL[ORC_MAXKD], gL[ORC_MAXKD];
    double zR[ORC_MAXKD], pR[ORC_MAXKD], gR[ORC_MAXKD];
    double zc[ORC_MAXKD], rho[ORC_MAXKD];
    memcpy(zL, zi, n * sizeof(double)); memcpy(zR, zi, n * sizeof(double));
    memcpy(pL, p0, n * sizeof(double)); memcpy(pR, p0, n * sizeof(double));
    memcpy(gL, g0, n * sizeof(double)); memcpy(gR, g0, n * sizeof(double));
    memcpy(zc, zi, n * sizeof(double)); memcpy(rho, p0, n * sizeof(double));
    double logW = -H0;
    double sum_acc = 0.0;
    int leaves = 0, diverged = 0, depth_done = 0;
    for (int depth = 0; depth < c->max_depth; ++depth) {
      uint64_t w[4];
      draw(c, problem, i, stage, round, ORC_PU_DIRECTION, (uint64_t)depth, w);
      const int dir = orc_u01(w[0]) < 0.5 ? -1 : 1;
      double z1[ORC_MAXKD], p1[ORC_MAXKD], g1[ORC_MAXKD], lp1;
      if (dir > 0) { memcpy(z1, zR, n * 8); memcpy(p1, pR, n * 8); memcpy(g1, gR, n * 8); }
      else { memcpy(z1, zL, n * 8); memcpy(p1, pL, n * 8); memcpy(g1, gL, n * 8); }
      double sub_logW = -INFINITY, sub_rho[ORC_MAXKD];
      double sub_z[ORC_MAXKD], sub_lo = 0, sub_ln = 0;
      double ck_p[ORC_MAXDEPTH][ORC_MAXKD], ck_rho[ORC_MAXDEPTH][ORC_MAXKD];
      for (int q = 0; q < n; ++q) sub_rho[q] = 0.0;
      int valid = 1;
      const int nsub = 1 << depth;
      for (int l = 0; l < nsub; ++l) {
        leapfrog_tc(&tc, dir * eps, minv, z1, p1, g1, &lp1);
        const double lo_ = tc.ll_old, ln_ = tc.ll_new;
        const double H = -lp1 + kinetic(n, D, minv, p1);
        const int leaf_id = (nsub - 1) + l;
        ++leaves;
        if (isfinite(H)) { double a = exp(H0 - H); sum_acc += a < 1.0 ? a : 1.0; }
        if (!isfinite(H) || H - H0 > 1000.0) { valid = 0; diverged = 1; break; }
        const double lw = -H;
        const double new_logW = logaddexp(sub_logW, lw);
        int take = (l == 0);
        if (!take) {
          uint64_t lwv[4];
          draw(c, problem, i, stage, round, ORC_PU_LEAF, (uint64_t)leaf_id, lwv);
          take = orc_u01(lwv[0]) < exp(lw - new_logW);
        }
        if (take) { memcpy(sub_z, z1, n * 8); sub_lo = lo_; sub_ln = ln_; }
        sub_logW = new_logW;
        /* checkpoints at starts of aligned sub-subtrees, then U-turn checks at their ends */
        for (int m = 1; m <= depth; ++m) {
          if (l % (1 << m) == 0) {
            memcpy(ck_p[m], p1, n * 8);
            memcpy(ck_rho[m], sub_rho, n * 8);
          }
        }
        for (int q = 0; q < n; ++q) sub_rho[q] += p1[q];
        for (int m = 1; m <= depth && valid; ++m) {
          if ((l + 1) % (1 << m) == 0) {
            double seg[ORC_MAXKD];
            for (int q = 0; q < n; ++q) seg[q] = sub_rho[q] - ck_rho[m][q];
            if (dot_minv(n, D, minv, seg, ck_p[m]) <= 0.0 ||
                dot_minv(n, D, minv, seg, p1) <= 0.0)
              valid = 0;
          }
        }
        if (!valid) break;
      }
      if (!valid) break;
      if (dir > 0) { memcpy(zR, z1, n * 8); memcpy(pR, p1, n * 8); memcpy(gR, g1, n * 8); }
      else { memcpy(zL, z1, n * 8); memcpy(pL, p1, n * 8); memcpy(gL, g1, n * 8); }
      draw(c, problem, i, stage, round, ORC_PU_TOP, (uint64_t)depth, w);
      if (orc_u01(w[0]) < exp(sub_logW - logW)) {
        memcpy(zc, sub_z, n * 8); cand_lo = sub_lo; cand_ln = sub_ln;
      }
      logW = logaddexp(logW, sub_logW);
      for (int q = 0; q < n; ++q) rho[q] += sub_rho[q];
      depth_done = depth + 1;
      if (dot_minv(n, D, minv, rho, pL) <= 0.0 || dot_minv(n, D, minv, rho, pR) <= 0.0) break;
    }
    memcpy(zi, zc, n * 8);
    /* periodic coordinates leave the transition reduced to one period, z - floor(z), so
       that positions stay small (the state on the circle is the same) */
    for (int q = 0; q < n; ++q)
      if (c->wrapmask & (1u << (q % D))) zi[q] -= floor(zi[q]);
    ll_old[i] = cand_lo; ll_new[i] = cand_ln;
    acc_stat[i] = leaves > 0 ? sum_acc / leaves : 0.0;
    n_leaf_out[i] = leaves;
    flags[i] = diverged | (depth_done << 8);
  }
}

/* ------------------------------------------------------------------------- */
/* Adaptive tempering.  Incremental weights w_i = L_i^(beta'-beta) (previous   */
/* weights uniform after resampling); ESS = (sum w)^2 / sum w^2 evaluated as   */
/* exp(2 LSE(delta ell) - LSE(2 delta ell)); solve ESS = alpha P by bisection  */
/* on delta in (0, 1-beta], keeping the lower end so that ESS >= alpha P;      */
/* evidence increment log(1/P sum w_i) = LSE(delta ell) - log P.               */
/* Sec. 2: Eq. incremental_weight, Eq. ess, Eq. ess_target and the evidence   */
/* ratio that follows them.                                                   */
/* ------------------------------------------------------------------------- */
static double lse_scaled(int32_t P, const double* ell, double s) {
  double m = -INFINITY;
  for (int32_t i = 0; i < P; ++i) { double v = s * ell[i]; if (v > m) m = v; }
  if (m == -INFINITY) return -INFINITY;
  nsum acc = {0, 0};
  for (int32_t i = 0; i < P; ++i) nadd(&acc, exp(s * ell[i] - m));
  return m + log(nval(&acc));
}

static double ess_of(int32_t P, const double* ell, double delta) {
  return exp(2.0 * lse_scaled(P, ell, delta) - lse_scaled(P, ell, 2.0 * delta));
}

void orc_temper(int32_t P, const double* ell, double alpha, double beta, double* beta_new,
                double* logz_inc, double* ess, double* logw) {
  const double target = alpha * (double)P;
  const double dmax = 1.0 - beta;
  double delta;
  int to_one = 0;
  if (ess_of(P, ell, dmax) >= target) {
    delta = dmax; to_one = 1;
  } else {
    double lo = 0.0, hi = dmax;
    for (int it = 0; it < 100; ++it) {
      if (hi - lo < 1e-14) break;
      double mid = 0.5 * (lo + hi);
      if (ess_of(P, ell, mid) >= target) lo = mid; else hi = mid;
    }
    delta = lo > 0.0 ? lo : hi;
  }
  *beta_new = to_one ? 1.0 : beta + delta;
  for (int32_t i = 0; i < P; ++i) logw[i] = delta * ell[i];
  *logz_inc = lse_scaled(P, ell, delta) - log((double)P);
  *ess = ess_of(P, ell, delta);
}

/* ------------------------------------------------------------------------- */
/* Systematic resampling, the resampling step of Sec. 2 (its scheme is not    */
/* stated there).  The weights are quantised to integers,                      */
/*   W_i = round(exp(logw_i - max) 2^S),  S = 52 - ceil(log2 P),               */
/* so that every inclusive prefix sum C_j is an exact integer <= 2^52 (a     */
/* weight below 2^-(S+1) of the largest counts as zero).  One U ~ (0,1) per    */
/* (problem, stage); with t_i = (i + U) / P C_P, at most C_P - 1, the          */
/* ancestor is a_i = min{j : C_j > t_i}.                                       */
/* ------------------------------------------------------------------------- */
int32_t orc_resample_scale(int32_t P) {
  int32_t S = 52;
  for (int64_t q = 1; q < (int64_t)P; q <<= 1) --S;
  return S;
}

void orc_resample(const orc_cfg* c, int32_t problem, int32_t stage, int32_t P,
                  const double* logw, int32_t* ancestors) {
  double m = -INFINITY;
  for (int32_t i = 0; i < P; ++i) if (logw[i] > m) m = logw[i];
  const int32_t S = orc_resample_scale(P);
  int64_t* C = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
  int64_t run = 0;
  for (int32_t i = 0; i < P; ++i) {
    run += (int64_t)llrint(ldexp(exp(logw[i] - m), S));
    C[i] = run;
  }
  uint64_t w[4];
  draw(c, problem, 0, stage, 0, ORC_PU_RESAMPLE, 0, w);
  const double U = orc_u01(w[0]);
  const double total = (double)C[P - 1];
  int32_t j = 0;
  for (int32_t i = 0; i < P; ++i) {
    double target = ((double)i + U) / (double)P * total;
    if (target > total - 1.0) target = total - 1.0;
    while (j < P - 1 && !((double)C[j] > target)) ++j;
    ancestors[i] = j;
  }
  free(C);
}

/* ------------------------------------------------------------------------- */
/* Metric: the mass matrix is the Hessian of the negative log target, read as  */
/* the population mean (over particles and active components) of the          */
/* Gauss-Newton diagonal per parameter type, floored at 1e-8; minv = 1/M.      */
/* Step size: eps <- eps exp(mean_acc - 0.8), clamped to [1e-4, 2];            */
/* eps_0 = 0.5 (kmax D)^(-1/4).                                                */
/* Sec. 3.2 (mass matrix); the step-size rule is not stated in the paper.     */
/* ------------------------------------------------------------------------- */
void orc_metric(const orc_cfg* c, const orc_data* dat, const double* z, const int32_t* K,
                int32_t P, double beta, double* minv) {
  const int D = c->D;
  const int64_t stride = (int64_t)c->kmax * D;
  double* fis = (double*)malloc(sizeof(double) * (size_t)stride);
  double sum[4] = {0, 0, 0, 0};
  int64_t cnt = 0;
  for (int32_t i = 0; i < P; ++i) {
    if (K[i] == 0) continue;
    orc_logl_grad(c, dat, z + i * stride, K[i], beta, NULL, NULL, NULL, NULL, NULL, fis);
    for (int k = 0; k < K[i]; ++k)
      for (int d = 0; d < D; ++d) sum[d] += fis[k * D + d];
    cnt += K[i];
  }
  for (int d = 0; d < D; ++d) {
    double h = cnt > 0 ? sum[d] / (double)cnt : 1.0;
    if (!(h > 1e-8)) h = 1e-8;
    minv[d] = 1.0 / h;
  }
  free(fis);
}

double orc_eps_update(double eps, double mean_acc) {
  double e = eps * exp(mean_acc - 0.8);
  if (e < 1e-4) e = 1e-4;
  if (e > 2.0) e = 2.0;
  return e;
}

double orc_eps_initial(const orc_cfg* c) { return 0.5 * pow((double)(c->kmax * c->D), -0.25); }

/* ------------------------------------------------------------------------- */
/* One SMC run: [init] -> repeat { choose beta (ESS), reweight (evidence),     */
/* resample, metric, n_mut rounds of mutation } until beta = 1.  Rounds        */
/* schedule: each round one RJ move then one NUTS transition; mixture          */
/* schedule: each round every particle draws NUTS / birth / death.             */
/* Sec. 4; the mixture is Eq. kernel_mixture of Sec. 3 with the weights of    */
/* Sec. 5.1.                                                                  */
/* ------------------------------------------------------------------------- */
int32_t orc_smc_run(const orc_cfg* c, const orc_data* dat, int32_t problem, int32_t P,
                    int32_t init_prior, int32_t stage0, int32_t max_stages, double* eps_io,
                    double* z, int32_t* K, double* ll_old, double* ll_new, double* logz,
                    double* beta_hist, double* logz_hist, double* ess_hist) {
  const int D = c->D;
  const int64_t stride = (int64_t)c->kmax * D;
  if (init_prior) orc_init_population(c, problem, P, z, K);
  orc_logl_grad_batch(c, dat, z, K, P, 0.0, ll_old, ll_new, NULL, NULL, NULL, NULL);
  double* logw = (double*)malloc(sizeof(double) * (size_t)P);
  int32_t* anc = (int32_t*)malloc(sizeof(int32_t) * (size_t)P);
  double* z2 = (double*)malloc(sizeof(double) * (size_t)(P * stride));
  int32_t* K2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)P);
  double* lo2 = (double*)malloc(sizeof(double) * (size_t)P);
  double* ln2 = (double*)malloc(sizeof(double) * (size_t)P);
  double* acc = (double*)malloc(sizeof(double) * (size_t)P);
  int32_t* nl = (int32_t*)malloc(sizeof(int32_t) * (size_t)P);
  int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)P);
  double beta = 0.0, eps = *eps_io, minv[4];
  orc_kde* kde = (c->birth_proposal == 1 && c->model != ORC_PULSE_LINAMP)
                     ? (orc_kde*)malloc(sizeof(orc_kde)) : NULL;
  *logz = 0.0;
  int32_t s = 0;
  for (; s < max_stages && beta < 1.0; ++s) {
    const int32_t stage = stage0 + s;
    double bnew, inc, ess;
    orc_temper(P, ll_new, c->alpha, beta, &bnew, &inc, &ess, logw);
    beta = bnew;
    *logz += inc;
    orc_resample(c, problem, stage, P, logw, anc);
    for (int32_t i = 0; i < P; ++i) {
      int32_t a = anc[i];
      memcpy(z2 + i * stride, z + a * stride, sizeof(double) * (size_t)stride);
      K2[i] = K[a]; lo2[i] = ll_old[a]; ln2[i] = ll_new[a];
    }
    memcpy(z, z2, sizeof(double) * (size_t)(P * stride));
    memcpy(K, K2, sizeof(int32_t) * (size_t)P);
    memcpy(ll_old, lo2, sizeof(double) * (size_t)P);
    memcpy(ll_new, ln2, sizeof(double) * (size_t)P);
    orc_metric(c, dat, z, K, P, beta, minv);
    if (kde) orc_kde_build(c, problem, stage, P, z, K, kde);
    double acc_sum = 0.0;
    int64_t acc_n = 0;
    for (int32_t r = 0; r < c->n_mut; ++r) {
      orc_rj_move_q(c, dat, problem, stage, r, beta, P, z, K, ll_old, ll_new, fl, kde);
      orc_nuts_move(c, dat, problem, stage, r, beta, eps, minv, P, z, K, ll_old, ll_new, acc,
                    nl, fl);
      for (int32_t i = 0; i < P; ++i) if (nl[i] > 0) { acc_sum += acc[i]; ++acc_n; }
    }
    if (acc_n > 0) eps = orc_eps_update(eps, acc_sum / (double)acc_n);
    if (beta_hist) beta_hist[s] = beta;
    if (logz_hist) logz_hist[s] = *logz;
    if (ess_hist) ess_hist[s] = ess;
  }
  *eps_io = eps;
  free(logw); free(anc); free(z2); free(K2); free(lo2); free(ln2); free(acc); free(nl); free(fl);
  free(kde);
  return s;
}
