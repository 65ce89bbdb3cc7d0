// api.cu -- host side of libtsmc: the C ABI of include/tsmc.h over a
// caller-owned device workspace, kernel dispatch and the stage driver.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "../../include/tsmc.h"

using namespace tsmc;

// the context behind the opaque tsmc_ctx handle
struct tsmc_ctx {
  tsmc_config cfg{};
  int D = 0, kd = 0, T = 0, R = 32;
  int64_t Ptot = 0;
  cudaStream_t stream = nullptr;
  std::vector<ProbDev> probs_host;
  std::vector<int64_t> cap, off;
  std::vector<char> has_data;
  bool tw_set = false, pop_ready = false;
  // device buffers (carved from the workspace)
  ProbDev* probs = nullptr;
  double* d64 = nullptr;
  float* d32 = nullptr;
  double *z = nullptr, *z2 = nullptr;
  int32_t *K = nullptr, *K2 = nullptr;
  double *llo = nullptr, *llo2 = nullptr, *lln = nullptr, *lln2 = nullptr;
  double *logw = nullptr, *cw = nullptr;
  int32_t* anc = nullptr;
  double* acc = nullptr;
  int32_t *nleaf = nullptr, *flags = nullptr, *outcome = nullptr;
  double* fis = nullptr;
  double *beta = nullptr, *logz = nullptr, *ess = nullptr, *eps = nullptr, *minv = nullptr;
  double* stats = nullptr;
  int32_t* stage = nullptr;
  double* tw = nullptr;
  double* host_out = nullptr;  // pinned? plain host staging for small reads
  unsigned long long* cs_count = nullptr;
  int32_t* order = nullptr;      // [Ptot] launch order of particle blocks
  int32_t* order_hist = nullptr; // [kOrderBuckets] bucket counts / offsets (scratch)
  double* kde = nullptr;         // [n_problems][kKdeStride] population birth proposals
  int32_t* kcum = nullptr;       // [Ptot] prefix counts of K (scratch of the proposal build)
  unsigned int* next = nullptr;  // work counter of the persistent mutation launch
  double* msums = nullptr;       // [n_problems][5] population sums of the metric
  int64_t Pg = 0;                // particles per problem of the whole (sharded) population
  int mut_grid = 0;              // resident blocks of the persistent mutation kernel
  double nmax = 1.0;             // largest problem capacity (cost normalisation)
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  int64_t graph_kernels = 0;
  int64_t launches = 0;          // kernels launched by this context
  bool capturing = false;
  // optional per-kernel-class event timing (eager launches only)
  bool profiling = false;
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::string err;
};

namespace {

using Ctx = tsmc_ctx;

enum KClass { KC_EVAL = 0, KC_RJ = 1, KC_NUTS = 2, KC_TEMPER = 3, KC_RESAMPLE = 4, KC_GATHER = 5,
              KC_METRIC = 6, KC_OTHER = 7, KC_N = 8 };

thread_local std::string g_err;

tsmc_status fail(Ctx* c, tsmc_status st, const std::string& msg) {
  if (c) c->err = msg; else g_err = msg;
  return st;
}

tsmc_status cuda_check(Ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TSMC_OK;
  return fail(c, TSMC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TRY_CUDA(c, call) do { tsmc_status _s = cuda_check((c), (call), #call); if (_s != TSMC_OK) return _s; } while (0)
#define TRY(call) do { tsmc_status _s = (call); if (_s != TSMC_OK) return _s; } while (0)

int model_dim(int m) { return m == TSMC_SINUSOID ? 4 : (m == TSMC_PULSE ? 3 : 1); }

// workspace layout (every buffer 256-byte aligned)
struct Layout {
  size_t total = 0;
  size_t take(size_t bytes) {
    const size_t o = total;
    total += (bytes + 255) & ~size_t(255);
    return o;
  }
};

struct Offsets {
  size_t probs, d64, d32, z, z2, K, K2, llo, llo2, lln, lln2, logw, cw, anc, acc, nleaf, flags,
      outcome, fis, beta, logz, ess, eps, minv, stats, stage, tw, cs, order, order_hist, kde,
      kcum, next, msums;
};

tsmc_status check_cfg(const tsmc_config* cfg) {
  if (!cfg) return TSMC_EINVAL;
  if (cfg->model < 0 || cfg->model > 2 || cfg->precision < 0 || cfg->precision > 1) return TSMC_EINVAL;
  if (cfg->n_problems <= 0 || cfg->particles <= 0 || cfg->kmax < 1 || cfg->kmax > kMaxK) return TSMC_EINVAL;
  if (cfg->kmin < 0 || cfg->kmin > cfg->kmax) return TSMC_EINVAL;
  if (cfg->max_depth < 1 || cfg->max_depth > kMaxDepth || cfg->n_mut < 0) return TSMC_EINVAL;
  if (!(cfg->alpha > 0.0 && cfg->alpha <= 1.0)) return TSMC_EINVAL;
  if (cfg->schedule == TSMC_SCHED_ROUNDS && !(cfg->p_birth > 0.0 && cfg->p_death > 0.0)) return TSMC_EINVAL;
  if (cfg->threads != 0 && (cfg->threads < 32 || cfg->threads > 256 || cfg->threads % 32)) return TSMC_EINVAL;
  if (cfg->samples_per_thread != 0 && cfg->samples_per_thread != 16 && cfg->samples_per_thread != 32) return TSMC_EINVAL;
  if (cfg->pulse_window != 0 && cfg->pulse_window != 1) return TSMC_EINVAL;
  if (cfg->birth_proposal != 0 && cfg->birth_proposal != 1) return TSMC_EINVAL;
  if (cfg->birth_proposal == 1 && !(cfg->birth_prior_weight > 0.0 && cfg->birth_prior_weight <= 1.0))
    return TSMC_EINVAL;
  if (cfg->channels < 0 || cfg->channels > 2) return TSMC_EINVAL;
  if (cfg->problem_base < 0 || (int64_t)cfg->problem_base + cfg->n_problems > INT32_MAX)
    return TSMC_EINVAL;
  if (cfg->fused_rounds != 0 && cfg->fused_rounds != 1) return TSMC_EINVAL;
  if (cfg->particles_global != 0) {
    if (cfg->particles_global < cfg->particles || cfg->particle_base < 0 ||
        (int64_t)cfg->particle_base + cfg->particles > cfg->particles_global)
      return TSMC_EINVAL;
    // the population birth proposal would be built from one shard only
    if (cfg->birth_proposal == 1) return TSMC_EINVAL;
  } else if (cfg->particle_base != 0) {
    return TSMC_EINVAL;
  }
  if (cfg->channels == 2) {
    if (cfg->model != TSMC_SINUSOID) return TSMC_EINVAL;
    for (int q = 0; q < 4; ++q)
      if (!std::isfinite(cfg->response[q])) return TSMC_EINVAL;
    if (!(cfg->response[0] > 0.0) || !(cfg->response[2] > 0.0)) return TSMC_EINVAL;
  }
  if (cfg->wrap_mask != 0) {
    if (cfg->model == TSMC_PULSE_LINAMP || cfg->birth_proposal == 1) return TSMC_EINVAL;
    if (cfg->wrap_mask >> model_dim(cfg->model)) return TSMC_EINVAL;
  }
  return TSMC_OK;
}

Offsets plan(const tsmc_config* cfg, const int64_t* cap, Layout& L) {
  Offsets o{};
  const int D = model_dim(cfg->model);
  const int64_t Ptot = (int64_t)cfg->n_problems * cfg->particles;
  const int64_t kd = (int64_t)cfg->kmax * D;
  int64_t ncap = 0;
  for (int p = 0; p < cfg->n_problems; ++p) ncap += (cap[p] + 63) / 64 * 64;
  o.probs = L.take(sizeof(ProbDev) * cfg->n_problems);
  o.d64 = L.take(sizeof(double) * ncap);
  o.d32 = L.take(sizeof(float) * ncap);
  o.z = L.take(sizeof(double) * Ptot * kd);
  o.z2 = L.take(sizeof(double) * Ptot * kd);
  o.K = L.take(sizeof(int32_t) * Ptot);
  o.K2 = L.take(sizeof(int32_t) * Ptot);
  o.llo = L.take(sizeof(double) * Ptot);
  o.llo2 = L.take(sizeof(double) * Ptot);
  o.lln = L.take(sizeof(double) * Ptot);
  o.lln2 = L.take(sizeof(double) * Ptot);
  // log-weights, prefix sums and ancestors cover the whole population when it is sharded
  const int64_t Pw = (int64_t)cfg->n_problems *
                     std::max<int64_t>(cfg->particles, cfg->particles_global);
  o.logw = L.take(sizeof(double) * Pw);
  o.cw = L.take(sizeof(double) * Pw);
  o.anc = L.take(sizeof(int32_t) * Pw);
  const int64_t rows = std::max<int64_t>(1, cfg->n_mut);   // per-round rows of the fused stage
  o.acc = L.take(sizeof(double) * Ptot * rows);
  o.nleaf = L.take(sizeof(int32_t) * Ptot * rows);
  o.flags = L.take(sizeof(int32_t) * Ptot * rows);
  o.outcome = L.take(sizeof(int32_t) * Ptot);
  o.fis = L.take(sizeof(double) * Ptot * D);
  o.beta = L.take(sizeof(double) * cfg->n_problems);
  o.logz = L.take(sizeof(double) * cfg->n_problems);
  o.ess = L.take(sizeof(double) * cfg->n_problems);
  o.eps = L.take(sizeof(double) * cfg->n_problems);
  o.minv = L.take(sizeof(double) * 4 * cfg->n_problems);
  o.stats = L.take(sizeof(double) * 2 * cfg->n_problems);
  o.stage = L.take(sizeof(int32_t) * 4);
  o.tw = L.take(sizeof(double) * 2 * cfg->kmax);
  o.cs = L.take(sizeof(unsigned long long) * 4);   // nominal / computed x batched / NUTS
  o.order = L.take(sizeof(int32_t) * Ptot);
  o.order_hist = L.take(sizeof(int32_t) * kOrderBuckets);
  o.kde = L.take(sizeof(double) * kKdeStride * cfg->n_problems);
  o.kcum = L.take(sizeof(int32_t) * Ptot);
  o.next = L.take(sizeof(unsigned int) * 4);
  o.msums = L.take(sizeof(double) * 5 * cfg->n_problems);
  return o;
}

KParams kparams(Ctx* c) {
  KParams kp;
  kp.probs = c->probs;
  kp.n_problems = c->cfg.n_problems;
  kp.P = c->cfg.particles;
  kp.kmax = c->cfg.kmax;
  kp.kmin = c->cfg.kmin;
  kp.D = c->D;
  kp.model = c->cfg.model;
  kp.schedule = c->cfg.schedule;
  kp.max_depth = c->cfg.max_depth;
  kp.n_mut = c->cfg.n_mut;
  kp.p_nuts = c->cfg.p_nuts;
  kp.p_birth = c->cfg.p_birth;
  kp.p_death = c->cfg.p_death;
  kp.birth_proposal = (c->cfg.birth_proposal == 1 && c->cfg.model != TSMC_PULSE_LINAMP) ? 1 : 0;
  kp.birth_eps = c->cfg.birth_prior_weight;
  kp.kde = c->kde;
  kp.pa.model = c->cfg.model;
  kp.pa.amp_mean = c->cfg.amp_mean;
  kp.pa.amp_sd = c->cfg.amp_sd;
  kp.pa.window = (c->cfg.precision == TSMC_MIXED && c->cfg.pulse_window) ? 1 : 0;
  kp.seed = c->cfg.seed;
  kp.prob_base = c->cfg.problem_base;
  kp.particle_base = c->cfg.particle_base;
  kp.tw = c->tw;
  kp.z = c->z;
  kp.K = c->K;
  kp.ll_old = c->llo;
  kp.ll_new = c->lln;
  kp.beta = c->beta;
  kp.eps = c->eps;
  kp.minv = c->minv;
  kp.stage = c->stage;
  kp.cs_count = c->cs_count;
  kp.order = nullptr;
  return kp;
}

SmemPlan smem_plan(Ctx* c, bool fisher, int depth) {
  SmemPlan sp;
  sp.kd = c->kd;
  sp.kmax = c->cfg.kmax;
  sp.nw = c->T / 32;
  sp.depth = depth;
  sp.fisher = fisher;
  sp.nch = c->cfg.channels == 2 ? 2 : 1;
  return sp;
}

// Dynamic shared memory above 48 KB needs an opt-in per kernel; it is granted once per
// kernel variant, up to the device limit, before any launch (and before graph capture).
int g_smem_optin = 0;

// The particle kernels also prefer the largest shared-memory carveout of the unified
// L1/shared array: measured on the pulse workload (N = 16384, K_max = 40), the NUTS
// kernel with 26 KB per block ran 5% slower with the driver's default carveout (which
// keeps more L1: the FP32 samples then hit L1 instead of L2) than with the maximum one.
template <typename F>
tsmc_status allow_smem(Ctx* c, F* fn) {
  if (!g_smem_optin) {
    int dev = 0;
    TRY_CUDA(c, cudaGetDevice(&dev));
    TRY_CUDA(c, cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  }
  TRY_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared));
  return cuda_check(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            g_smem_optin - 2048),
                    "cudaFuncSetAttribute");
}

template <typename F>
tsmc_status launch_prep(Ctx* c, F* fn, size_t smem) {
  (void)fn;
  if ((int)smem > g_smem_optin - 2048) return fail(c, TSMC_EINVAL, "particle block needs too much shared memory");
  return TSMC_OK;
}

template <int MODEL, int PREC, int R>
tsmc_status prep_t(Ctx* c) {
  TRY(allow_smem(c, &k_eval<MODEL, PREC, R, true, true>));
  TRY(allow_smem(c, &k_eval<MODEL, PREC, R, true, false>));
  TRY(allow_smem(c, &k_eval<MODEL, PREC, R, false, false>));
  TRY(allow_smem(c, &k_rj<MODEL, PREC, R>));
  if constexpr (PREC == FP64) {
    TRY(allow_smem(c, &k_nuts<MODEL, PREC, R>));
  } else {
    TRY(allow_smem(c, &k_nuts_mixed<MODEL, R>));
    TRY(allow_smem(c, &k_mutate_mixed<MODEL, R>));
    // resident blocks of the persistent mutation kernel (more would only start once the
    // counter is spent; fewer would leave SM slots empty)
    SmemPlan sp = smem_plan(c, false, c->cfg.max_depth);
    const size_t sm = std::max(sp.nuts_mixed_kernel_bytes(), sp.rj_kernel_bytes());
    int per_sm = 0, dev = 0, n_sm = 0;
    TRY_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mutate_mixed<MODEL, R>,
                                                              c->T, sm));
    TRY_CUDA(c, cudaGetDevice(&dev));
    TRY_CUDA(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    c->mut_grid = std::max(1, per_sm) * n_sm;
  }
  return TSMC_OK;
}

cudaEvent_t pooled_event(Ctx* c) {
  if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// called before a kernel launch: starts its timing record when profiling
void pre(Ctx* c, int cls) {
  if (c->profiling && !c->capturing) {
    Ctx::Rec r{cls, pooled_event(c), pooled_event(c)};
    cudaEventRecord(r.a, c->stream);
    c->recs.push_back(r);
  }
}

// called after a kernel launch: error check, launch count, end of the timing record
tsmc_status post(Ctx* c, const char* what) {
  tsmc_status st = cuda_check(c, cudaGetLastError(), what);
  if (c->capturing) ++c->graph_kernels; else ++c->launches;
  if (c->profiling && !c->capturing && !c->recs.empty()) cudaEventRecord(c->recs.back().b, c->stream);
  return st;
}

tsmc_status last_launch(Ctx* c, const char* what) { return post(c, what); }

// longest-first order of the particle blocks for population K (device array)
tsmc_status build_order(Ctx* c, const int32_t* K) {
  TRY_CUDA(c, cudaMemsetAsync(c->order_hist, 0, sizeof(int32_t) * kOrderBuckets, c->stream));
  const unsigned nb = (unsigned)((c->Ptot + 255) / 256);
  pre(c, KC_OTHER);
  k_order_count<<<nb, 256, 0, c->stream>>>(K, c->probs, c->cfg.particles, c->cfg.kmax, c->nmax,
                                           c->Ptot, c->order_hist);
  TRY(post(c, "k_order_count"));
  pre(c, KC_OTHER);
  k_order_scan<<<1, kOrderBuckets, 0, c->stream>>>(c->order_hist);
  TRY(post(c, "k_order_scan"));
  pre(c, KC_OTHER);
  k_order_scatter<<<nb, 256, 0, c->stream>>>(K, c->probs, c->cfg.particles, c->cfg.kmax, c->nmax,
                                             c->Ptot, c->order_hist, c->order);
  return post(c, "k_order_scatter");
}

// ---- dispatch on (model, precision, samples per thread) ----
template <int MODEL, int PREC, int R>
tsmc_status eval_launch_t(Ctx* c, const EvalIO& io, bool grad, bool fisher) {
  TRY(build_order(c, io.K));
  KParams kp = kparams(c);
  kp.order = c->order;
  SmemPlan sp = smem_plan(c, fisher, 0);
  const size_t sm = sp.eval_kernel_bytes();
  const dim3 grid((unsigned)c->Ptot), block(c->T);
  if (fisher) {
    auto fn = &k_eval<MODEL, PREC, R, true, true>;
    TRY(launch_prep(c, fn, sm));
    pre(c, KC_EVAL);
    fn<<<grid, block, sm, c->stream>>>(kp, io, sp);
  } else if (grad) {
    auto fn = &k_eval<MODEL, PREC, R, true, false>;
    TRY(launch_prep(c, fn, sm));
    pre(c, KC_EVAL);
    fn<<<grid, block, sm, c->stream>>>(kp, io, sp);
  } else {
    auto fn = &k_eval<MODEL, PREC, R, false, false>;
    TRY(launch_prep(c, fn, sm));
    pre(c, KC_EVAL);
    fn<<<grid, block, sm, c->stream>>>(kp, io, sp);
  }
  return last_launch(c, "k_eval");
}

template <int MODEL, int PREC, int R>
tsmc_status rj_launch_t(Ctx* c, int round, int32_t* outcome) {
  KParams kp = kparams(c);
  SmemPlan sp = smem_plan(c, false, 0);
  const size_t sm = sp.rj_kernel_bytes();
  auto fn = &k_rj<MODEL, PREC, R>;
  TRY(launch_prep(c, fn, sm));
  pre(c, KC_RJ);
  fn<<<(unsigned)c->Ptot, c->T, sm, c->stream>>>(kp, round, outcome, sp);
  return last_launch(c, "k_rj");
}

template <int MODEL, int PREC, int R>
tsmc_status nuts_launch_t(Ctx* c, int round, NutsOut out) {
  TRY(build_order(c, c->K));
  KParams kp = kparams(c);
  kp.order = c->order;
  SmemPlan sp = smem_plan(c, false, c->cfg.max_depth);
  if constexpr (PREC == FP64) {
    const size_t sm = sp.nuts_kernel_bytes();
    auto fn = &k_nuts<MODEL, PREC, R>;
    TRY(launch_prep(c, fn, sm));
    pre(c, KC_NUTS);
    fn<<<(unsigned)c->Ptot, c->T, sm, c->stream>>>(kp, round, out, sp);
    return last_launch(c, "k_nuts");
  } else {
    const size_t sm = sp.nuts_mixed_kernel_bytes();
    auto fn = &k_nuts_mixed<MODEL, R>;
    TRY(launch_prep(c, fn, sm));
    pre(c, KC_NUTS);
    fn<<<(unsigned)c->Ptot, c->T, sm, c->stream>>>(kp, round, out, sp);
    return last_launch(c, "k_nuts_mixed");
  }
}

template <int MODEL, int PREC, int R>
tsmc_status mutate_launch_t(Ctx* c, int) {
  if constexpr (PREC != MIXED) {
    return fail(c, TSMC_EINVAL, "the fused mutation launch is a mixed-path kernel");
  } else {
    TRY(build_order(c, c->K));
    KParams kp = kparams(c);
    kp.order = c->order;
    SmemPlan sp = smem_plan(c, false, c->cfg.max_depth);
    const size_t sm = std::max(sp.nuts_mixed_kernel_bytes(), sp.rj_kernel_bytes());
    auto fn = &k_mutate_mixed<MODEL, R>;
    TRY(launch_prep(c, fn, sm));
    TRY_CUDA(c, cudaMemsetAsync(c->next, 0, sizeof(unsigned int), c->stream));
    const int grid = (int)std::min<int64_t>(c->mut_grid, c->Ptot);
    pre(c, KC_NUTS);
    fn<<<grid, c->T, sm, c->stream>>>(kp, c->cfg.n_mut, MutOut{c->outcome, c->acc, c->nleaf,
                                                                c->flags},
                                      sp, c->next, c->cfg.model != TSMC_PULSE_LINAMP ? 1 : 0);
    return last_launch(c, "k_mutate_mixed");
  }
}

#define DISPATCH(FN, ...)                                                                 \
  do {                                                                                    \
    const int m_ = c->cfg.model, p_ = c->cfg.precision;                                   \
    if (p_ == TSMC_FP64) {                                                                \
      if (m_ == TSMC_PULSE) return FN<PULSE, FP64, 8>(c, __VA_ARGS__);                    \
      if (m_ == TSMC_SINUSOID) return FN<SINUSOID, FP64, 8>(c, __VA_ARGS__);              \
      return FN<PULSE_LINAMP, FP64, 8>(c, __VA_ARGS__);                                   \
    }                                                                                     \
    if (c->R == 16) {                                                                     \
      if (m_ == TSMC_PULSE) return FN<PULSE, MIXED, 16>(c, __VA_ARGS__);                  \
      if (m_ == TSMC_SINUSOID) return FN<SINUSOID, MIXED, 16>(c, __VA_ARGS__);            \
      return FN<PULSE_LINAMP, MIXED, 16>(c, __VA_ARGS__);                                 \
    }                                                                                     \
    if (m_ == TSMC_PULSE) return FN<PULSE, MIXED, 32>(c, __VA_ARGS__);                    \
    if (m_ == TSMC_SINUSOID) return FN<SINUSOID, MIXED, 32>(c, __VA_ARGS__);              \
    return FN<PULSE_LINAMP, MIXED, 32>(c, __VA_ARGS__);                                   \
  } while (0)

template <int MODEL, int PREC, int R>
tsmc_status prep_launch_t(Ctx* c, int) { return prep_t<MODEL, PREC, R>(c); }
tsmc_status prep_launch(Ctx* c) { DISPATCH(prep_launch_t, 0); }

tsmc_status eval_launch(Ctx* c, const EvalIO& io, bool grad, bool fisher) {
  DISPATCH(eval_launch_t, io, grad, fisher);
}
tsmc_status rj_launch(Ctx* c, int round, int32_t* outcome) { DISPATCH(rj_launch_t, round, outcome); }
tsmc_status nuts_launch(Ctx* c, int round, NutsOut out) { DISPATCH(nuts_launch_t, round, out); }
tsmc_status mutate_launch(Ctx* c) { DISPATCH(mutate_launch_t, 0); }

tsmc_status require_ready(Ctx* c) {
  for (int p = 0; p < c->cfg.n_problems; ++p)
    if (!c->has_data[p]) return fail(c, TSMC_ESTATE, "problem data not set");
  if (c->cfg.model == TSMC_PULSE_LINAMP && !c->tw_set)
    return fail(c, TSMC_ESTATE, "fixed components not set");
  return TSMC_OK;
}

// every descriptor (resets the device-side done flags to the host copies)
tsmc_status upload_probs(Ctx* c) {
  return cuda_check(c, cudaMemcpyAsync(c->probs, c->probs_host.data(),
                                       sizeof(ProbDev) * c->probs_host.size(),
                                       cudaMemcpyHostToDevice, c->stream),
                    "upload problem descriptors");
}

// one descriptor: the other problems keep their device state (k_temper sets done on the
// device when a problem reaches beta = 1, and the host copies do not follow it)
tsmc_status upload_prob(Ctx* c, int problem) {
  return cuda_check(c, cudaMemcpyAsync(c->probs + problem, &c->probs_host[problem],
                                       sizeof(ProbDev), cudaMemcpyHostToDevice, c->stream),
                    "upload problem descriptor");
}

tsmc_status sync_stream(Ctx* c) {
  return cuda_check(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
}

// refresh ll_old / ll_new of the context population at the current beta
tsmc_status refresh_ll(Ctx* c) {
  EvalIO io{c->z, c->K, c->beta, c->llo, c->lln, nullptr, nullptr, nullptr};
  return eval_launch(c, io, false, false);
}

tsmc_status set_stage(Ctx* c, int stage) {
  pre(c, KC_OTHER);
  k_set_int<<<1, 1, 0, c->stream>>>(c->stage, stage);
  return last_launch(c, "k_set_int");
}

// mutation part of a stage: metric, n_mut rounds, step size (graph-capturable)
// population birth proposal from the context population (stage_arg < 0: device counter)
tsmc_status kde_launch(Ctx* c, int stage_arg) {
  const int D = c->D;
  const double factor = std::pow(4.0 / (double)(D + 2), 1.0 / (double)(D + 4)) *
                        std::pow((double)kKdeM, -1.0 / (double)(D + 4));
  pre(c, KC_OTHER);
  k_kde_build<<<c->cfg.n_problems, 256, 0, c->stream>>>(kparams(c), c->kcum, c->kde, factor,
                                                         stage_arg);
  return last_launch(c, "k_kde_build");
}

// population sums of the metric (a Gauss-Newton evaluation of the context population)
tsmc_status metric_sums_launch(Ctx* c, double* sums) {
  EvalIO io{c->z, c->K, c->beta, c->llo, c->lln, nullptr, nullptr, c->fis};
  TRY(eval_launch(c, io, true, true));
  pre(c, KC_METRIC);
  k_metric_sums<<<c->cfg.n_problems, 256, 0, c->stream>>>(c->fis, c->K, c->probs,
                                                           c->cfg.particles, c->D, sums);
  return last_launch(c, "k_metric_sums");
}

tsmc_status metric_apply_launch(Ctx* c, const double* sums) {
  const int np = c->cfg.n_problems;
  pre(c, KC_METRIC);
  k_metric_apply<<<(np + 127) / 128, 128, 0, c->stream>>>(sums, c->probs, np, c->D, c->minv);
  return last_launch(c, "k_metric_apply");
}

// the n_mut mutation rounds of a stage (statistics accumulate in c->stats)
tsmc_status rounds_body(Ctx* c);

tsmc_status mutation_body(Ctx* c) {
  const int np = c->cfg.n_problems;
  TRY(metric_sums_launch(c, c->msums));
  TRY(metric_apply_launch(c, c->msums));
  TRY(rounds_body(c));
  pre(c, KC_OTHER);
  k_eps_update<<<(np + 127) / 128, 128, 0, c->stream>>>(c->probs, c->stats, c->eps, np);
  return last_launch(c, "k_eps_update");
}

tsmc_status rounds_body(Ctx* c) {
  const int np = c->cfg.n_problems, P = c->cfg.particles;
  if (c->cfg.birth_proposal == 1 && c->cfg.model != TSMC_PULSE_LINAMP) TRY(kde_launch(c, -1));
  if (c->cfg.precision == TSMC_MIXED && c->cfg.fused_rounds == 1 && c->cfg.n_mut > 0) {
    // every round of every particle in one persistent launch (see k_mutate_mixed)
    TRY(mutate_launch(c));
    pre(c, KC_OTHER);
    k_round_stats_all<<<np, 256, 0, c->stream>>>(c->acc, c->nleaf, c->probs, P, c->Ptot,
                                                 c->cfg.n_mut, c->stats);
    TRY(last_launch(c, "k_round_stats_all"));
  } else {
    for (int r = 0; r < c->cfg.n_mut; ++r) {
      if (c->cfg.model != TSMC_PULSE_LINAMP) TRY(rj_launch(c, r, c->outcome));
      TRY(nuts_launch(c, r, NutsOut{c->acc, c->nleaf, c->flags}));
      pre(c, KC_OTHER);
      k_round_stats<<<np, 256, 0, c->stream>>>(c->acc, c->nleaf, c->probs, P, c->stats);
      TRY(last_launch(c, "k_round_stats"));
    }
  }
  return TSMC_OK;
}

tsmc_status temper_resample(Ctx* c, int stage) {
  const int np = c->cfg.n_problems, P = c->cfg.particles;
  TemperIO tio{c->lln, c->logw, c->beta, c->logz, c->ess, c->probs, c->cfg.alpha};
  const int tt = P >= 1024 ? 1024 : ((P + 31) / 32) * 32;
  pre(c, KC_TEMPER);
  if (c->cfg.precision == TSMC_MIXED) {   // FP32 bisection passes; prefix-sum buffer as scratch
    k_temper_mixed<<<np, tt, 0, c->stream>>>(tio, P, reinterpret_cast<float*>(c->cw));
    TRY(last_launch(c, "k_temper_mixed"));
  } else {
    k_temper<<<np, tt, 0, c->stream>>>(tio, P);
    TRY(last_launch(c, "k_temper"));
  }
  pre(c, KC_RESAMPLE);
  k_resample<<<np, tt, 0, c->stream>>>(c->logw, reinterpret_cast<long long*>(c->cw), c->anc,
                                       c->probs, c->cfg.seed, stage, P, c->cfg.problem_base);
  TRY(last_launch(c, "k_resample"));
  const int64_t work = c->Ptot * (c->kd + 1);
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, 148 * 16);
  pre(c, KC_GATHER);
  k_gather<<<blocks, 256, 0, c->stream>>>(c->anc, c->probs, P, c->kd, c->z, c->K, c->llo, c->lln,
                                          c->z2, c->K2, c->llo2, c->lln2, c->Ptot);
  TRY(last_launch(c, "k_gather"));
  TRY_CUDA(c, cudaMemcpyAsync(c->z, c->z2, sizeof(double) * c->Ptot * c->kd,
                              cudaMemcpyDeviceToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->K, c->K2, sizeof(int32_t) * c->Ptot, cudaMemcpyDeviceToDevice,
                              c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->llo, c->llo2, sizeof(double) * c->Ptot, cudaMemcpyDeviceToDevice,
                              c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->lln, c->lln2, sizeof(double) * c->Ptot, cudaMemcpyDeviceToDevice,
                              c->stream));
  return TSMC_OK;
}

tsmc_status read_problem_scalars(Ctx* c, double* beta_h, double* logz_h, double* ess_h) {
  const int np = c->cfg.n_problems;
  if (!beta_h && !logz_h && !ess_h) return TSMC_OK;   // nothing to read: stay asynchronous
  if (beta_h) TRY_CUDA(c, cudaMemcpyAsync(beta_h, c->beta, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
  if (logz_h) TRY_CUDA(c, cudaMemcpyAsync(logz_h, c->logz, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
  if (ess_h) TRY_CUDA(c, cudaMemcpyAsync(ess_h, c->ess, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
  return sync_stream(c);
}

float2 split_df(double x) {   // x = hi + lo with hi the FP32 rounding of x
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

bool all_finite(const double* a, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

tsmc_status tsmc_workspace_bytes(const tsmc_config* cfg, const int64_t* cap, size_t* bytes) {
  if (check_cfg(cfg) != TSMC_OK || !cap || !bytes) return fail(nullptr, TSMC_EINVAL, "bad config");
  for (int p = 0; p < cfg->n_problems; ++p)
    if (cap[p] <= 0 || cap[p] > (int64_t(1) << 24)) return fail(nullptr, TSMC_EINVAL, "bad capacity");
  Layout L;
  plan(cfg, cap, L);
  *bytes = L.total;
  return TSMC_OK;
}

tsmc_status tsmc_create(const tsmc_config* cfg, const int64_t* cap, void* ws, size_t bytes,
                        void* stream, tsmc_ctx** out) {
  if (!out) return fail(nullptr, TSMC_EINVAL, "null output");
  size_t need = 0;
  TRY(tsmc_workspace_bytes(cfg, cap, &need));
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return fail(nullptr, TSMC_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < need) return fail(nullptr, TSMC_ENOMEM, "workspace too small");
  Ctx* c = new Ctx();
  c->cfg = *cfg;
  c->D = model_dim(cfg->model);
  c->kd = cfg->kmax * c->D;
  c->Ptot = (int64_t)cfg->n_problems * cfg->particles;
  // default block: 128 threads; on the mixed path 64 for pulses (eight resident two-warp
  // blocks per SM at 26 KB of shared memory and <= 128 registers: more particles in flight
  // while one block runs its serial per-leaf work, and the 16 warp ranges of 1024 samples
  // of N = 16384 split evenly; five 96-thread blocks ran the NUTS rounds 6% slower)
  c->T = cfg->threads ? cfg->threads
         : cfg->precision != TSMC_MIXED ? 128
         : cfg->model == TSMC_PULSE ? 64 : 128;
  c->R = cfg->samples_per_thread ? cfg->samples_per_thread : 32;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  Offsets o = plan(cfg, cap, L);
  char* b = static_cast<char*>(ws);
  c->probs = reinterpret_cast<ProbDev*>(b + o.probs);
  c->d64 = reinterpret_cast<double*>(b + o.d64);
  c->d32 = reinterpret_cast<float*>(b + o.d32);
  c->z = reinterpret_cast<double*>(b + o.z);
  c->z2 = reinterpret_cast<double*>(b + o.z2);
  c->K = reinterpret_cast<int32_t*>(b + o.K);
  c->K2 = reinterpret_cast<int32_t*>(b + o.K2);
  c->llo = reinterpret_cast<double*>(b + o.llo);
  c->llo2 = reinterpret_cast<double*>(b + o.llo2);
  c->lln = reinterpret_cast<double*>(b + o.lln);
  c->lln2 = reinterpret_cast<double*>(b + o.lln2);
  c->logw = reinterpret_cast<double*>(b + o.logw);
  c->cw = reinterpret_cast<double*>(b + o.cw);
  c->anc = reinterpret_cast<int32_t*>(b + o.anc);
  c->acc = reinterpret_cast<double*>(b + o.acc);
  c->nleaf = reinterpret_cast<int32_t*>(b + o.nleaf);
  c->flags = reinterpret_cast<int32_t*>(b + o.flags);
  c->outcome = reinterpret_cast<int32_t*>(b + o.outcome);
  c->fis = reinterpret_cast<double*>(b + o.fis);
  c->beta = reinterpret_cast<double*>(b + o.beta);
  c->logz = reinterpret_cast<double*>(b + o.logz);
  c->ess = reinterpret_cast<double*>(b + o.ess);
  c->eps = reinterpret_cast<double*>(b + o.eps);
  c->minv = reinterpret_cast<double*>(b + o.minv);
  c->stats = reinterpret_cast<double*>(b + o.stats);
  c->stage = reinterpret_cast<int32_t*>(b + o.stage);
  c->tw = reinterpret_cast<double*>(b + o.tw);
  c->cs_count = reinterpret_cast<unsigned long long*>(b + o.cs);
  c->order = reinterpret_cast<int32_t*>(b + o.order);
  c->order_hist = reinterpret_cast<int32_t*>(b + o.order_hist);
  c->kde = reinterpret_cast<double*>(b + o.kde);
  c->kcum = reinterpret_cast<int32_t*>(b + o.kcum);
  c->next = reinterpret_cast<unsigned int*>(b + o.next);
  c->msums = reinterpret_cast<double*>(b + o.msums);
  c->Pg = std::max<int64_t>(cfg->particles, cfg->particles_global);
  for (int p = 0; p < cfg->n_problems; ++p) c->nmax = std::max(c->nmax, (double)cap[p]);
  c->cap.assign(cap, cap + cfg->n_problems);
  c->off.resize(cfg->n_problems);
  int64_t acc = 0;
  for (int p = 0; p < cfg->n_problems; ++p) { c->off[p] = acc; acc += (cap[p] + 63) / 64 * 64; }
  c->probs_host.assign(cfg->n_problems, ProbDev{});
  c->has_data.assign(cfg->n_problems, 0);
  for (int p = 0; p < cfg->n_problems; ++p) {
    ProbDev& pd = c->probs_host[p];
    pd.d64 = c->d64 + c->off[p];
    pd.d32 = c->d32 + c->off[p];
    pd.cap = cap[p];
  }
  // zero the state and scratch so every buffer starts defined
  cudaError_t e = cudaMemsetAsync(ws, 0, L.total, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    g_err = std::string("workspace clear: ") + cudaGetErrorString(e);
    delete c;
    return TSMC_ECUDA;
  }
  if (prep_launch(c) != TSMC_OK) {
    g_err = c->err;
    delete c;
    return TSMC_ECUDA;
  }
  *out = c;
  return TSMC_OK;
}

tsmc_status tsmc_destroy(tsmc_ctx* ctx) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (const Ctx::Rec& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  delete c;
  return TSMC_OK;
}

const char* tsmc_last_error(const tsmc_ctx* ctx) {
  const Ctx* c = ctx;
  return c ? c->err.c_str() : g_err.c_str();
}

tsmc_status tsmc_set_problem(tsmc_ctx* ctx, int32_t problem, const double* d_host, int64_t n,
                             double t_origin, double dt, double sigma, const double* lo,
                             const double* hi, uint32_t logmask) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (problem < 0 || problem >= c->cfg.n_problems) return fail(c, TSMC_EINVAL, "problem index out of range");
  if (!d_host || n <= 0 || n > c->cap[problem]) return fail(c, TSMC_EINVAL, "bad sample count");
  if (!(sigma > 0.0) || !std::isfinite(dt) || !std::isfinite(t_origin) || !std::isfinite(sigma))
    return fail(c, TSMC_EINVAL, "bad grid or noise level");
  if (!all_finite(d_host, n)) return fail(c, TSMC_ENONFINITE, "non-finite data");
  if (c->cfg.channels == 2 && (n % 64 != 0))
    return fail(c, TSMC_EINVAL, "two-channel data need 2 x (a multiple of 32) samples");
  ProbDev& pd = c->probs_host[problem];
  pd.n = n;
  pd.n1 = 0;
  pd.t_origin = t_origin;
  pd.dt = dt;
  pd.sigma = sigma;
  pd.inv_s2 = 1.0 / (sigma * sigma);
  if (logmask & c->cfg.wrap_mask)
    return fail(c, TSMC_EINVAL, "a periodic parameter cannot be log-uniform");
  pd.logmask = logmask;
  pd.wrapmask = c->cfg.wrap_mask;
  pd.done = 0;
  for (int d = 0; d < 4; ++d) {
    const bool used = d < c->D && c->cfg.model != TSMC_PULSE_LINAMP;
    pd.lo[d] = (used && lo) ? lo[d] : 0.0;
    pd.hi[d] = (used && hi) ? hi[d] : 1.0;
    if (used && (!lo || !hi || !(pd.hi[d] > pd.lo[d])))
      return fail(c, TSMC_EINVAL, "prior bounds must satisfy lo < hi");
    if (used && (logmask >> d & 1u) && !(pd.lo[d] > 0.0))
      return fail(c, TSMC_EINVAL, "log-uniform prior needs lo > 0");
    pd.llo[d] = (logmask >> d & 1u) ? std::log(pd.lo[d]) : 0.0;
    pd.lhi[d] = (logmask >> d & 1u) ? std::log(pd.hi[d]) : 0.0;
    const bool lg = logmask >> d & 1u;
    pd.f_off[d] = split_df(lg ? pd.llo[d] : pd.lo[d]);
    pd.f_span[d] = split_df(lg ? pd.lhi[d] - pd.llo[d] : pd.hi[d] - pd.lo[d]);
  }
  pd.f_to = split_df(t_origin);
  pd.f_dt = split_df(dt);
  pd.f_is2 = split_df(pd.inv_s2);
  pd.nch = c->cfg.channels == 2 ? 2 : 1;
  pd.nc = n / pd.nch;
  for (int q = 0; q < 4; ++q) {
    pd.resp[q] = pd.nch == 2 ? c->cfg.response[q] : (q % 2 == 0 ? 1.0 : 0.0);
    pd.f_resp[q] = (float)pd.resp[q];
  }
  TRY_CUDA(c, cudaMemcpyAsync(const_cast<double*>(pd.d64), d_host, sizeof(double) * n,
                              cudaMemcpyHostToDevice, c->stream));
  pre(c, KC_OTHER);
  k_to_f32<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, c->stream>>>(
      pd.d64, const_cast<float*>(pd.d32), n);
  TRY(last_launch(c, "k_to_f32"));
  TRY(upload_prob(c, problem));
  c->has_data[problem] = 1;
  return sync_stream(c);
}

tsmc_status tsmc_set_fixed_components(tsmc_ctx* ctx, const double* tw_host) {
  Ctx* c = ctx;
  if (!c || !tw_host) return TSMC_EINVAL;
  if (!all_finite(tw_host, 2 * c->cfg.kmax)) return fail(c, TSMC_ENONFINITE, "non-finite components");
  for (int k = 0; k < c->cfg.kmax; ++k)
    if (!(tw_host[2 * k + 1] > 0.0)) return fail(c, TSMC_EINVAL, "widths must be positive");
  TRY_CUDA(c, cudaMemcpyAsync(c->tw, tw_host, sizeof(double) * 2 * c->cfg.kmax,
                              cudaMemcpyHostToDevice, c->stream));
  c->tw_set = true;
  return sync_stream(c);
}

static tsmc_status reset_run_state(Ctx* c, const double* beta_h, const double* logz_h) {
  const int np = c->cfg.n_problems;
  std::vector<double> b(np, 0.0), lz(np, 0.0), eps(np), minv(4 * np, 1.0), st(2 * np, 0.0);
  const double e0 = 0.5 * std::pow((double)c->kd, -0.25);
  for (int p = 0; p < np; ++p) {
    eps[p] = e0;
    if (beta_h) b[p] = beta_h[p];
    if (logz_h) lz[p] = logz_h[p];
    c->probs_host[p].done = 0;
  }
  TRY(upload_probs(c));
  TRY_CUDA(c, cudaMemcpyAsync(c->beta, b.data(), sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->logz, lz.data(), sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->eps, eps.data(), sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->minv, minv.data(), sizeof(double) * 4 * np, cudaMemcpyHostToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->stats, st.data(), sizeof(double) * 2 * np, cudaMemcpyHostToDevice, c->stream));
  return sync_stream(c);
}

tsmc_status tsmc_init_population(tsmc_ctx* ctx) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  TRY(require_ready(c));
  TRY(reset_run_state(c, nullptr, nullptr));
  KParams kp = kparams(c);
  pre(c, KC_OTHER);
  k_init<<<(unsigned)((c->Ptot + 127) / 128), 128, 0, c->stream>>>(kp, c->Ptot);
  TRY(last_launch(c, "k_init"));
  TRY(refresh_ll(c));
  c->pop_ready = true;
  return sync_stream(c);
}

tsmc_status tsmc_set_population(tsmc_ctx* ctx, const double* z_dev, const int32_t* K_dev,
                                const double* beta_h, const double* logz_h) {
  Ctx* c = ctx;
  if (!c || !z_dev || !K_dev) return TSMC_EINVAL;
  TRY(require_ready(c));
  if (beta_h)
    for (int p = 0; p < c->cfg.n_problems; ++p)
      if (!(beta_h[p] >= 0.0 && beta_h[p] <= 1.0)) return fail(c, TSMC_EINVAL, "beta out of [0,1]");
  std::vector<int32_t> kh(c->Ptot);
  TRY_CUDA(c, cudaMemcpyAsync(kh.data(), K_dev, sizeof(int32_t) * c->Ptot, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_stream(c));
  for (int64_t i = 0; i < c->Ptot; ++i)
    if (kh[i] < 0 || kh[i] > c->cfg.kmax) return fail(c, TSMC_EINVAL, "K out of range");
  TRY(reset_run_state(c, beta_h, logz_h));
  TRY_CUDA(c, cudaMemcpyAsync(c->z, z_dev, sizeof(double) * c->Ptot * c->kd, cudaMemcpyDeviceToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->K, K_dev, sizeof(int32_t) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  TRY(refresh_ll(c));
  c->pop_ready = true;
  return sync_stream(c);
}

tsmc_status tsmc_get_population(tsmc_ctx* ctx, double* z_dev, int32_t* K_dev, double* llo_dev,
                                double* lln_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  if (z_dev) TRY_CUDA(c, cudaMemcpyAsync(z_dev, c->z, sizeof(double) * c->Ptot * c->kd, cudaMemcpyDeviceToDevice, c->stream));
  if (K_dev) TRY_CUDA(c, cudaMemcpyAsync(K_dev, c->K, sizeof(int32_t) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  if (llo_dev) TRY_CUDA(c, cudaMemcpyAsync(llo_dev, c->llo, sizeof(double) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  if (lln_dev) TRY_CUDA(c, cudaMemcpyAsync(lln_dev, c->lln, sizeof(double) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  return TSMC_OK;
}

tsmc_status tsmc_eval_logl_grad(tsmc_ctx* ctx, const double* z_dev, const int32_t* K_dev,
                                const double* beta_dev, double* llo_dev, double* lln_dev,
                                double* logp_dev, double* grad_dev, double* fis_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!z_dev || !K_dev || !lln_dev) return fail(c, TSMC_EINVAL, "null argument");
  TRY(require_ready(c));
  EvalIO io{z_dev, K_dev, beta_dev ? beta_dev : c->beta, llo_dev, lln_dev, logp_dev, grad_dev, fis_dev};
  return eval_launch(c, io, grad_dev != nullptr, fis_dev != nullptr);
}

tsmc_status tsmc_rj_move(tsmc_ctx* ctx, int32_t stage, int32_t round, int32_t* outcome_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  if (stage < 0 || round < 0 || round > 0x0FFFFFFF) return fail(c, TSMC_EINVAL, "bad stage/round");
  TRY(set_stage(c, stage));
  if (c->cfg.model == TSMC_PULSE_LINAMP) return TSMC_OK;
  return rj_launch(c, round, outcome_dev);
}

tsmc_status tsmc_nuts_move(tsmc_ctx* ctx, int32_t stage, int32_t round, double* acc_dev,
                           int32_t* nleaf_dev, int32_t* flags_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  if (stage < 0 || round < 0 || round > 0x0FFFFFFF) return fail(c, TSMC_EINVAL, "bad stage/round");
  TRY(set_stage(c, stage));
  return nuts_launch(c, round, NutsOut{acc_dev, nleaf_dev, flags_dev});
}

tsmc_status tsmc_set_kernel_params(tsmc_ctx* ctx, const double* eps_h, const double* minv_h) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  const int np = c->cfg.n_problems;
  if (eps_h) {
    for (int p = 0; p < np; ++p)
      if (!(eps_h[p] > 0.0) || !std::isfinite(eps_h[p])) return fail(c, TSMC_EINVAL, "eps must be positive");
    TRY_CUDA(c, cudaMemcpyAsync(c->eps, eps_h, sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
  }
  if (minv_h) {
    std::vector<double> m(4 * np, 1.0);
    for (int p = 0; p < np; ++p)
      for (int d = 0; d < c->D; ++d) {
        const double v = minv_h[p * c->D + d];
        if (!(v > 0.0) || !std::isfinite(v)) return fail(c, TSMC_EINVAL, "minv must be positive");
        m[4 * p + d] = v;
      }
    TRY_CUDA(c, cudaMemcpyAsync(c->minv, m.data(), sizeof(double) * 4 * np, cudaMemcpyHostToDevice, c->stream));
  }
  return sync_stream(c);
}

tsmc_status tsmc_build_birth_proposal(tsmc_ctx* ctx, int32_t stage) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (c->cfg.model == TSMC_PULSE_LINAMP || stage < 0)
    return fail(c, TSMC_EINVAL, "no birth proposal for this model or stage");
  return kde_launch(c, stage);
}

tsmc_status tsmc_get_birth_proposal(tsmc_ctx* ctx, int32_t problem, double* out_h, int64_t n) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!out_h || problem < 0 || problem >= c->cfg.n_problems || n < 5 + (int64_t)kKdeM * c->D)
    return fail(c, TSMC_EINVAL, "bad problem or output size");
  std::vector<double> v(kKdeStride);
  TRY_CUDA(c, cudaMemcpyAsync(v.data(), c->kde + (int64_t)problem * kKdeStride,
                              sizeof(double) * kKdeStride, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_stream(c));
  out_h[0] = v[0];
  for (int d = 0; d < 4; ++d) out_h[1 + d] = v[1 + d];
  for (int64_t i = 0; i < (int64_t)kKdeM * c->D; ++i) out_h[5 + i] = v[8 + i];
  return TSMC_OK;
}

tsmc_status tsmc_get_kernel_params(tsmc_ctx* ctx, double* eps_h, double* minv_h) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  const int np = c->cfg.n_problems;
  std::vector<double> m(4 * np);
  if (eps_h) TRY_CUDA(c, cudaMemcpyAsync(eps_h, c->eps, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(m.data(), c->minv, sizeof(double) * 4 * np, cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_stream(c));
  if (minv_h)
    for (int p = 0; p < np; ++p)
      for (int d = 0; d < c->D; ++d) minv_h[p * c->D + d] = m[4 * p + d];
  return TSMC_OK;
}

tsmc_status tsmc_update_metric(tsmc_ctx* ctx) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  TRY(metric_sums_launch(c, c->msums));
  return metric_apply_launch(c, c->msums);
}

tsmc_status tsmc_temper_reweight_resample(tsmc_ctx* ctx, int32_t stage, double* beta_h,
                                          double* logz_h, double* ess_h) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (c->Pg != c->cfg.particles)
    return fail(c, TSMC_ESTATE, "sharded population: use tsmc_temper_resample_global");
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  if (stage < 0) return fail(c, TSMC_EINVAL, "bad stage");
  TRY(temper_resample(c, stage));
  return read_problem_scalars(c, beta_h, logz_h, ess_h);
}

tsmc_status tsmc_get_state(tsmc_ctx* ctx, double* beta_h, double* logz_h, double* ess_h) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  TRY(read_problem_scalars(c, beta_h, logz_h, ess_h));
  return sync_stream(c);
}

tsmc_status tsmc_get_ancestors(tsmc_ctx* ctx, int32_t* anc_dev) {
  Ctx* c = ctx;
  if (!c || !anc_dev) return TSMC_EINVAL;
  TRY_CUDA(c, cudaMemcpyAsync(anc_dev, c->anc, sizeof(int32_t) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  return TSMC_OK;
}

tsmc_status tsmc_run_stage(tsmc_ctx* ctx, int32_t stage, int32_t use_graph, double* beta_h,
                           double* logz_h, double* ess_h) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (c->Pg != c->cfg.particles)
    return fail(c, TSMC_ESTATE, "sharded population: use tsmc_temper_resample_global");
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  if (stage < 0) return fail(c, TSMC_EINVAL, "bad stage");
  TRY(set_stage(c, stage));
  TRY(temper_resample(c, stage));
  if (use_graph && c->stream != nullptr && !c->profiling) {
    if (!c->graph_valid) {
      cudaGraph_t g = nullptr;
      TRY_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      c->capturing = true;
      c->graph_kernels = 0;
      tsmc_status st = mutation_body(c);
      c->capturing = false;
      cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (st != TSMC_OK) { if (g) cudaGraphDestroy(g); return st; }
      TRY(cuda_check(c, e, "cudaStreamEndCapture"));
      e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      TRY(cuda_check(c, e, "cudaGraphInstantiate"));
      c->graph_valid = true;
    }
    TRY_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
    c->launches += c->graph_kernels;
  } else {
    TRY(mutation_body(c));
  }
  return read_problem_scalars(c, beta_h, logz_h, ess_h);
}

tsmc_status tsmc_assimilate(tsmc_ctx* ctx, int32_t problem, const double* d_new, int64_t n_new) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (problem < 0 || problem >= c->cfg.n_problems) return fail(c, TSMC_EINVAL, "problem index out of range");
  if (!c->pop_ready || !c->has_data[problem]) return fail(c, TSMC_ESTATE, "no population");
  ProbDev& pd = c->probs_host[problem];
  if (!d_new || n_new <= 0 || pd.n + n_new > pd.cap) return fail(c, TSMC_EINVAL, "bad sample count");
  if (pd.nch == 2) return fail(c, TSMC_EINVAL, "two-channel problems take no appended samples");
  if (!all_finite(d_new, n_new)) return fail(c, TSMC_ENONFINITE, "non-finite data");
  // the reuse bridge (Eq. reuse_bridge) starts from the posterior of the samples held so
  // far: particles still tempered (beta < 1) would enter it with unit weight and no
  // importance correction
  double beta_now = 0.0;
  TRY_CUDA(c, cudaMemcpyAsync(&beta_now, c->beta + problem, sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
  TRY(sync_stream(c));
  if (!(beta_now >= 1.0))
    return fail(c, TSMC_ESTATE, "assimilate needs the posterior of the data held so far (beta = 1)");
  TRY_CUDA(c, cudaMemcpyAsync(const_cast<double*>(pd.d64) + pd.n, d_new, sizeof(double) * n_new,
                              cudaMemcpyHostToDevice, c->stream));
  pre(c, KC_OTHER);
  k_to_f32<<<(unsigned)std::min<int64_t>((n_new + 255) / 256, 1024), 256, 0, c->stream>>>(
      pd.d64 + pd.n, const_cast<float*>(pd.d32) + pd.n, n_new);
  TRY(last_launch(c, "k_to_f32"));
  pd.n1 = pd.n;
  pd.n += n_new;
  pd.done = 0;
  TRY(upload_prob(c, problem));
  const double zero = 0.0;
  TRY_CUDA(c, cudaMemcpyAsync(c->beta + problem, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->logz + problem, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TRY(refresh_ll(c));
  return sync_stream(c);
}

tsmc_status tsmc_philox(tsmc_ctx* ctx, const uint64_t* ctr_dev, uint64_t key0, uint64_t key1,
                        int64_t n, uint64_t* out_dev) {
  Ctx* c = ctx;
  if (!c || !ctr_dev || !out_dev || n < 0) return TSMC_EINVAL;
  if (n == 0) return TSMC_OK;
  pre(c, KC_OTHER);
  k_philox<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(ctr_dev, key0, key1, n, out_dev);
  return last_launch(c, "k_philox");
}

tsmc_status tsmc_counters(tsmc_ctx* ctx, uint64_t* cs_evals_host, int64_t* launches_host,
                          int32_t reset) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  unsigned long long v[4] = {0, 0, 0, 0};
  TRY_CUDA(c, cudaMemcpyAsync(v, c->cs_count, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
  TRY(sync_stream(c));
  if (cs_evals_host)
    for (int i = 0; i < 4; ++i) cs_evals_host[i] = (uint64_t)v[i];
  if (launches_host) *launches_host = c->launches;
  if (reset) {
    TRY_CUDA(c, cudaMemsetAsync(c->cs_count, 0, sizeof(v), c->stream));
    c->launches = 0;
    TRY(sync_stream(c));
  }
  return TSMC_OK;
}

tsmc_status tsmc_profile(tsmc_ctx* ctx, int32_t enable) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  c->profiling = enable != 0;
  // create the events up front: no driver object creation inside a timed region
  while (c->profiling && (int64_t)c->pool.size() < std::max<int64_t>(enable, 0)) {
    cudaEvent_t e = nullptr;
    TRY_CUDA(c, cudaEventCreate(&e));
    c->pool.push_back(e);
  }
  return TSMC_OK;
}

tsmc_status tsmc_profile_read(tsmc_ctx* ctx, int64_t* launches_host, double* ms_host, int32_t reset) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  TRY(sync_stream(c));
  std::vector<int64_t> n(KC_N, 0);
  std::vector<double> ms(KC_N, 0.0);
  for (const Ctx::Rec& r : c->recs) {
    float t = 0.f;
    TRY_CUDA(c, cudaEventElapsedTime(&t, r.a, r.b));
    n[r.cls] += 1;
    ms[r.cls] += (double)t;
  }
  for (int k = 0; k < KC_N; ++k) {
    if (launches_host) launches_host[k] = n[k];
    if (ms_host) ms_host[k] = ms[k];
  }
  if (reset) {
    for (const Ctx::Rec& r : c->recs) { c->pool.push_back(r.a); c->pool.push_back(r.b); }
    c->recs.clear();
  }
  return TSMC_OK;
}

// ---------------------------------------------------------------------------
// A population sharded across processes (tsmc_config.particles_global): the calls that
// take or give the population-wide quantities, so that the caller's collectives join the
// shards (see include/tsmc.h).
// ---------------------------------------------------------------------------
tsmc_status tsmc_temper_resample_global(tsmc_ctx* ctx, int32_t stage, const double* ell_dev,
                                        int32_t* anc_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!ell_dev || !anc_dev) return fail(c, TSMC_EINVAL, "null log-likelihoods or ancestors");
  if (stage < 0) return fail(c, TSMC_EINVAL, "bad stage");
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  const int np = c->cfg.n_problems;
  const int P = (int)c->Pg;
  TRY(set_stage(c, stage));
  TemperIO tio{ell_dev, c->logw, c->beta, c->logz, c->ess, c->probs, c->cfg.alpha};
  const int tt = P >= 1024 ? 1024 : ((P + 31) / 32) * 32;
  pre(c, KC_TEMPER);
  if (c->cfg.precision == TSMC_MIXED) {
    k_temper_mixed<<<np, tt, 0, c->stream>>>(tio, P, reinterpret_cast<float*>(c->cw));
    TRY(last_launch(c, "k_temper_mixed"));
  } else {
    k_temper<<<np, tt, 0, c->stream>>>(tio, P);
    TRY(last_launch(c, "k_temper"));
  }
  pre(c, KC_RESAMPLE);
  k_resample<<<np, tt, 0, c->stream>>>(c->logw, reinterpret_cast<long long*>(c->cw), anc_dev,
                                       c->probs, c->cfg.seed, stage, P, c->cfg.problem_base);
  return last_launch(c, "k_resample");
}

tsmc_status tsmc_load_population(tsmc_ctx* ctx, const double* z_dev, const int32_t* K_dev,
                                 const double* llo_dev, const double* lln_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!z_dev || !K_dev || !llo_dev || !lln_dev) return fail(c, TSMC_EINVAL, "null argument");
  TRY(require_ready(c));
  TRY_CUDA(c, cudaMemcpyAsync(c->z, z_dev, sizeof(double) * c->Ptot * c->kd, cudaMemcpyDeviceToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->K, K_dev, sizeof(int32_t) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->llo, llo_dev, sizeof(double) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  TRY_CUDA(c, cudaMemcpyAsync(c->lln, lln_dev, sizeof(double) * c->Ptot, cudaMemcpyDeviceToDevice, c->stream));
  c->pop_ready = true;
  return TSMC_OK;
}

tsmc_status tsmc_metric_sums(tsmc_ctx* ctx, double* sums_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!sums_dev) return fail(c, TSMC_EINVAL, "null sums");
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  return metric_sums_launch(c, sums_dev);
}

tsmc_status tsmc_metric_apply(tsmc_ctx* ctx, const double* sums_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!sums_dev) return fail(c, TSMC_EINVAL, "null sums");
  return metric_apply_launch(c, sums_dev);
}

tsmc_status tsmc_mutation_rounds(tsmc_ctx* ctx, int32_t stage, double* stats_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!stats_dev) return fail(c, TSMC_EINVAL, "null statistics");
  if (stage < 0) return fail(c, TSMC_EINVAL, "bad stage");
  if (!c->pop_ready) return fail(c, TSMC_ESTATE, "no population");
  const size_t nb = sizeof(double) * 2 * c->cfg.n_problems;
  TRY_CUDA(c, cudaMemsetAsync(c->stats, 0, nb, c->stream));
  TRY(set_stage(c, stage));
  TRY(rounds_body(c));
  TRY_CUDA(c, cudaMemcpyAsync(stats_dev, c->stats, nb, cudaMemcpyDeviceToDevice, c->stream));
  return cuda_check(c, cudaMemsetAsync(c->stats, 0, nb, c->stream), "clear statistics");
}

tsmc_status tsmc_eps_update_apply(tsmc_ctx* ctx, const double* stats_dev) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  if (!stats_dev) return fail(c, TSMC_EINVAL, "null statistics");
  const int np = c->cfg.n_problems;
  TRY_CUDA(c, cudaMemcpyAsync(c->stats, stats_dev, sizeof(double) * 2 * np,
                              cudaMemcpyDeviceToDevice, c->stream));
  pre(c, KC_OTHER);
  k_eps_update<<<(np + 127) / 128, 128, 0, c->stream>>>(c->probs, c->stats, c->eps, np);
  return last_launch(c, "k_eps_update");
}

// ---------------------------------------------------------------------------
// Allocation-free systematic resampling.  Scratch (the 64-bit prefix sums and a
// block of all-zero problem descriptors, i.e. no problem marked done) lives in
// file-scope device arrays that every GPU loading this library keeps until exit.
// ---------------------------------------------------------------------------
}  // extern "C"

#define TSMC_STATIC_MAX_PARTICLES 65536   /* n_problems * particles: 512 KB of 64-bit prefix sums */
#define TSMC_STATIC_MAX_PROBLEMS 256

static __device__ __align__(256) long long g_static_prefix[TSMC_STATIC_MAX_PARTICLES];
static __device__ __align__(256) ProbDev g_static_probs[TSMC_STATIC_MAX_PROBLEMS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
long long* g_static_prefix_dev[kMaxDevices] = {};
ProbDev* g_static_probs_dev[kMaxDevices] = {};

// device addresses of the static arrays for the current device (looked up once per device)
tsmc_status static_scratch(long long** prefix, ProbDev** probs) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, TSMC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, TSMC_EINVAL, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_prefix_dev[dev]) {
    void* a = nullptr;
    void* b = nullptr;
    e = cudaGetSymbolAddress(&a, g_static_prefix);
    if (e != cudaSuccess)
      return fail(nullptr, TSMC_ECUDA, std::string("cudaGetSymbolAddress(prefix): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&b, g_static_probs);
    if (e != cudaSuccess)
      return fail(nullptr, TSMC_ECUDA, std::string("cudaGetSymbolAddress(problems): ") + cudaGetErrorString(e));
    g_static_prefix_dev[dev] = static_cast<long long*>(a);
    g_static_probs_dev[dev] = static_cast<ProbDev*>(b);
  }
  *prefix = g_static_prefix_dev[dev];
  *probs = g_static_probs_dev[dev];
  return TSMC_OK;
}
}  // namespace

extern "C" {

tsmc_status tsmc_resample_systematic_static(const double* logw_dev, int32_t n_problems,
                                            int32_t particles, uint64_t seed, int32_t stage,
                                            int32_t* ancestors_dev, void* cuda_stream) {
  if (!logw_dev || !ancestors_dev) return fail(nullptr, TSMC_EINVAL, "null log-weights or ancestors");
  if (n_problems < 1 || particles < 1 || stage < 0)
    return fail(nullptr, TSMC_EINVAL, "need n_problems >= 1, particles >= 1, stage >= 0");
  if (n_problems > TSMC_STATIC_MAX_PROBLEMS)
    return fail(nullptr, TSMC_EINVAL, "n_problems above the static limit of 256");
  if ((int64_t)n_problems * particles > TSMC_STATIC_MAX_PARTICLES)
    return fail(nullptr, TSMC_EINVAL,
                "n_problems * particles above the static scratch limit of 65536");
  long long* prefix = nullptr;
  ProbDev* probs = nullptr;
  TRY(static_scratch(&prefix, &probs));
  const int tt = particles >= 1024 ? 1024 : ((particles + 31) / 32) * 32;
  k_resample<<<n_problems, tt, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(
      logw_dev, prefix, ancestors_dev, probs, seed, stage, particles, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, TSMC_ECUDA, std::string("k_resample: ") + cudaGetErrorString(e));
  return TSMC_OK;
}

tsmc_status tsmc_sync(tsmc_ctx* ctx) {
  Ctx* c = ctx;
  if (!c) return TSMC_EINVAL;
  return sync_stream(c);
}

}  // extern "C"
