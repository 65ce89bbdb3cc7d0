// kernels.cuh -- the sampler's kernels: batched evaluation, reversible-jump
// birth/death, NUTS transitions, prior initialisation, ESS tempering,
// systematic resampling and the population metric.
#pragma once
#include <type_traits>

#include "likelihood.cuh"

namespace tsmc {

// Everything a population kernel needs, passed by value.
struct KParams {
  const ProbDev* probs;
  int32_t n_problems, P, kmax, kmin, D, model, schedule, max_depth, n_mut;
  double p_nuts, p_birth, p_death;
  int32_t birth_proposal;    // 0: births from the prior; 1: population mixture (kde)
  double birth_eps;          // prior weight of the population mixture
  const double* kde;         // [n_problems][kKdeStride] population birth proposals
  PriorArgs pa;
  uint64_t seed;
  int32_t prob_base;         // Philox key word 1 = prob_base + problem index
  int64_t particle_base;     // Philox counter word 0 = particle_base + local particle index
  const double* tw;          // LINAMP fixed (t0, w), [kmax][2]
  double* z;                 // [Ptot][kmax][D]
  int32_t* K;                // [Ptot]
  double* ll_old;            // [Ptot]
  double* ll_new;            // [Ptot]
  const double* beta;        // [n_problems]
  const double* eps;         // [n_problems]
  const double* minv;        // [n_problems][4]
  const int32_t* stage;      // device stage counter (graph-stable)
  unsigned long long* cs_count;  // component*sample logL+grad evaluations (statistic)
  const int32_t* order;      // block -> particle (longest first), or null for identity
};

// Shared-memory carve for one particle block.
struct SmemPlan {
  int kd;          // kmax * D
  int kmax;        // component slots
  int nw;          // warps per block
  int depth;       // NUTS checkpoint levels (0 for non-NUTS kernels)
  bool fisher;
  int nch;         // data channels (mixed-path constants per channel)
  __host__ __device__ size_t eval_bytes() const {
    return sizeof(double) * (4 * (size_t)kd + (size_t)nw * kd * (fisher ? 2 : 1) + 128 + 8 + 64) +
           sizeof(float) * (size_t)kmax * NCF * nch + 32;
  }
  __host__ __device__ size_t nuts_bytes() const {
    return sizeof(double) * (size_t)kd * (14 + 2 * (size_t)(depth + 1));   // 8-byte slots
  }
  // mixed NUTS: 5 double-float position vectors, 9 FP32 vectors, 2 (depth + 1) FP32
  // checkpoint rows, and the leaf uniforms of the largest subtree
  __host__ __device__ size_t nuts_mixed_bytes() const {
    return sizeof(float2) * 5 * (size_t)kd + sizeof(float) * (size_t)kd * (9 + 2 * (size_t)(depth + 1)) +
           sizeof(float) * ((size_t)1 << (depth > 0 ? depth - 1 : 0)) + 16;
  }
  __host__ __device__ size_t nuts_mixed_kernel_bytes() const {
    return eval_bytes() + nuts_mixed_bytes() + 64;
  }
  // eval kernel: + gradient and Gauss-Newton staging; RJ: + proposal coordinates
  __host__ __device__ size_t eval_kernel_bytes() const {
    return eval_bytes() + 2 * sizeof(double) * (size_t)kd + 64;
  }
  __host__ __device__ size_t rj_kernel_bytes() const {
    return eval_bytes() + sizeof(double) * (size_t)(kd + 4) + 64;
  }
  __host__ __device__ size_t nuts_kernel_bytes() const { return eval_bytes() + nuts_bytes() + 64; }
};

__device__ __forceinline__ EvalSmem carve_eval(char*& p, const SmemPlan& sp, const double* tw) {
  EvalSmem sm;
  double* d = reinterpret_cast<double*>(p);
  sm.th = d; d += sp.kd;
  sm.dth = d; d += sp.kd;
  sm.pg = d; d += sp.kd;
  sm.pc = d; d += sp.kd;
  sm.wacc = d; d += (size_t)sp.nw * sp.kd;
  if (sp.fisher) { sm.wfis = d; d += (size_t)sp.nw * sp.kd; } else { sm.wfis = nullptr; }
  sm.red = d; d += 128;
  sm.scal = d; d += 8;
  sm.exptab = reinterpret_cast<float2*>(d); d += 64;
  if (reinterpret_cast<uintptr_t>(d) & 8) d += 1;   // float4 loads of the constants
  sm.cf = reinterpret_cast<float*>(d);
  sm.cfch = sp.kmax * NCF;
  p = reinterpret_cast<char*>(sm.cf + (size_t)sp.kmax * NCF * sp.nch);
  // keep 8-byte alignment for what follows
  p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
  sm.tw = tw;
  return sm;
}

// ---------------------------------------------------------------------------
// Batched evaluation: one block per particle (caller arrays).  The tempered likelihood
// of the bridges Eq. prior_bridge and Eq. reuse_bridge (Sec. 2) and its gradient.
// ---------------------------------------------------------------------------
struct EvalIO {
  const double* z; const int32_t* K; const double* beta;
  double* ll_old; double* ll_new; double* logp; double* grad; double* fis_sum;
};

// particle-block kernels: at most 256 threads; the register budget leaves room for 2
// (32 samples per thread) or 3 (16 samples per thread) resident blocks per SM
#define TSMC_PARTICLE_BOUNDS __launch_bounds__(256, (PREC == MIXED && R == 16) ? 3 : 2)

// The problem descriptor is copied to shared memory once per block: its fields are
// read where they are used instead of holding ~70 registers across the kernel.
__device__ __forceinline__ const ProbDev& stage_problem(const ProbDev* probs, int prob,
                                                        ProbDev& s) {
  static_assert(sizeof(ProbDev) % 8 == 0, "ProbDev is copied as 8-byte words");
  const uint64_t* src = reinterpret_cast<const uint64_t*>(probs + prob);
  uint64_t* dst = reinterpret_cast<uint64_t*>(&s);
  for (int i = threadIdx.x; i < (int)(sizeof(ProbDev) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return s;
}

template <int MODEL, int PREC, int R, bool GRAD, bool FISHER>
__global__ void TSMC_PARTICLE_BOUNDS k_eval(KParams kp, EvalIO io, SmemPlan sp) {
  extern __shared__ __align__(16) char smem[];
  constexpr int D = model_d<MODEL>();
  const int64_t gi = kp.order ? (int64_t)kp.order[blockIdx.x] : (int64_t)blockIdx.x;
  const int prob = (int)(gi / kp.P);
  __shared__ ProbDev s_pb;
  const ProbDev& pb = stage_problem(kp.probs, prob, s_pb);
  char* p = smem;
  EvalSmem sm = carve_eval(p, sp, kp.tw);
  double* gbuf = reinterpret_cast<double*>(p);   // [kd] gradient staging
  double* fbuf = gbuf + sp.kd;                  // [kd] Gauss-Newton staging
  const int K = min(max(io.K[gi], 0), kp.kmax);   // caller array: clamp to the slots
  const double beta = io.beta[prob];
  const double* z = io.z + gi * (int64_t)sp.kd;
  if (PREC == MIXED) init_block_tables(sm);
  __syncthreads();
  block_eval<MODEL, PREC, R, GRAD, FISHER>(pb, kp.pa, K, beta, z, sm, gbuf, fbuf);
  const int tid = threadIdx.x;
  if (tid == 0) {
    if (io.ll_old) io.ll_old[gi] = sm.scal[1];
    io.ll_new[gi] = sm.scal[2];
    if (io.logp) io.logp[gi] = sm.scal[0];
  }
  if (GRAD && io.grad) {
    double* g = io.grad + gi * (int64_t)sp.kd;
    for (int i = tid; i < sp.kd; i += blockDim.x) g[i] = i < K * D ? gbuf[i] : 0.0;
  }
  if (GRAD && tid == 0 && kp.cs_count) {   // slots 0 / 2: batched, nominal / computed
    atomicAdd(kp.cs_count, (unsigned long long)K * (unsigned long long)pb.n);
    atomicAdd(kp.cs_count + 2, (unsigned long long)sm.scal[3]);
  }
  if (FISHER && io.fis_sum) {
    if (tid < D) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += fbuf[k * D + tid];
      io.fis_sum[gi * D + tid] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Prior initialisation (the prior start of Sec. 4): one thread per particle.
// ---------------------------------------------------------------------------
__global__ void k_init(KParams kp, int64_t Ptot) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= Ptot) return;
  const int prob = (int)(gi / kp.P);
  const int pkey = prob + kp.prob_base;
  const uint64_t li = (uint64_t)(gi % kp.P) + (uint64_t)kp.particle_base;
  const int kd = kp.kmax * kp.D;
  double* z = kp.z + gi * kd;
  for (int j = 0; j < kd; ++j) z[j] = 0.0;
  if (kp.model == PULSE_LINAMP) {
    kp.K[gi] = kp.kmax;
    for (int j = 0; j < kp.kmax; ++j)
      z[j] = kp.pa.amp_mean +
             kp.pa.amp_sd * draw_normal(kp.seed, pkey, li, 0, 0, PU_INIT, 4 + (uint64_t)j);
    return;
  }
  Rand4 w = draw(kp.seed, pkey, li, 0, 0, PU_INIT, 0);
  int k = kp.kmin + (int)floor(__dmul_rn(u01(w.w[0]), (double)(kp.kmax - kp.kmin + 1)));
  if (k > kp.kmax) k = kp.kmax;
  kp.K[gi] = k;
  const uint32_t wrap = kp.probs[prob].wrapmask;
  for (int j = 0; j < k * kp.D; ++j) {
    if ((j & 3) == 0) w = draw(kp.seed, pkey, li, 0, 0, PU_INIT, 1 + (uint64_t)(j >> 2));
    const double u = u01(w.w[j & 3]);
    // theta at the prior quantile u: logit(u), or u itself on a periodic coordinate
    z[j] = (wrap >> (j % kp.D) & 1u) ? u : log(u) - log1p(-u);
  }
}

// ---------------------------------------------------------------------------
// Reversible-jump birth/death: one block per particle (Sec. 3.1 nested map,
// Eq. rj_acceptance).
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Population birth proposal (Sec. 6: the particles of a stage approximate its tempered
// distribution, so it can serve as the birth proposal).  In z coordinates every
// parameter's prior is the standard logistic density; the proposal is
//   q(z) = eps prior_z(z) + (1 - eps)/m sum_i prod_d N(z_d; c_id, h_d^2).
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ double log_prior_z(const double* z) {
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double a = fabs(z[d]);
    s += -a - 2.0 * log1p(exp(-a));
  }
  return s;
}

__device__ __forceinline__ double block_max1(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < nw; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// log q(z) for one component z[D]; all threads call it and all get the value
template <int D>
__device__ double kde_logq_block(const double* kde, const double* z, double eps, double* red) {
  const double lp = log_prior_z<D>(z);
  const int m = (int)kde[0];
  if (m == 0 || eps >= 1.0) return lp;
  const double lw = log((1.0 - eps) / (double)m);
  const double c2 = 0.5 * log(2.0 * kPi);
  auto term = [&](int i) {   // i = 0: the prior part; i >= 1: centre i - 1
    if (i == 0) return log(eps) + lp;
    double e = lw;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double h = kde[1 + d];
      const double u = (z[d] - kde[8 + (i - 1) * D + d]) / h;
      e += -0.5 * u * u - log(h) - c2;
    }
    return e;
  };
  double mx = -INFINITY;
  for (int i = threadIdx.x; i <= m; i += blockDim.x) mx = fmax(mx, term(i));
  mx = block_max1(mx, red);
  double v[1] = {0.0};
  for (int i = threadIdx.x; i <= m; i += blockDim.x) v[0] += exp(term(i) - mx);
  block_sum<1>(v, red);
  return mx + log(v[0]);
}

// one particle's move (all threads of the block call it; block-uniform exits)
template <int MODEL, int PREC, int R>
__device__ void rj_particle(const KParams& kp, int64_t gi, int round, int32_t* outcome,
                            const SmemPlan& sp) {
  extern __shared__ __align__(16) char smem[];
  constexpr int D = model_d<MODEL>();
  __shared__ int s_move;       // 0 none, 1 birth, 2 death
  __shared__ int s_j;
  __shared__ double s_u;
  __shared__ double s_znew[4];
  const int prob = (int)(gi / kp.P);
  const int pkey = prob + kp.prob_base;
  const uint64_t li = (uint64_t)(gi % kp.P) + (uint64_t)kp.particle_base;
  __shared__ ProbDev s_pb;
  const ProbDev& pb = stage_problem(kp.probs, prob, s_pb);
  if (pb.done) return;
  const int stage = *kp.stage;
  const int K = min(max(kp.K[gi], 0), kp.kmax);
  const int tid = threadIdx.x;
  if (tid == 0) {
    int move = 0;
    const Rand4 w = draw(kp.seed, pkey, li, stage, round, PU_RJ, 0);
    bool birth;
    bool active = kp.model != PULSE_LINAMP;
    if (active && kp.schedule == 1) {
      const Rand4 m = draw(kp.seed, pkey, li, stage, round, PU_MOVETYPE, 0);
      const double um = u01(m.w[0]);
      active = !(um < kp.p_nuts);
      birth = um < kp.p_nuts + kp.p_birth;
    } else {
      birth = u01(w.w[0]) < kp.p_birth / (kp.p_birth + kp.p_death);
    }
    int out = 0;
    if (active) {
      if (birth && K >= kp.kmax) out = -1;
      else if (!birth && K <= kp.kmin) out = -2;
      else move = birth ? 1 : 2;
    }
    if (move == 1) {
      const Rand4 pw = draw(kp.seed, pkey, li, stage, round, PU_RJPARAM, 0);
      const double* kde = kp.kde + (int64_t)prob * kKdeStride;
      const Rand4 mw = draw(kp.seed, pkey, li, stage, round, PU_RJPARAM, 2);
      const int m = kp.birth_proposal ? (int)kde[0] : 0;
      if (m > 0 && u01(mw.w[0]) >= kp.birth_eps) {
        // from the population mixture: a centre, then a normal step of width h
        int q = (int)floor(__dmul_rn(u01(mw.w[1]), (double)m));
        if (q >= m) q = m - 1;
        for (int d = 0; d < D; ++d)
          s_znew[d] = __dadd_rn(kde[8 + q * D + d],
                                __dmul_rn(kde[1 + d], draw_normal(kp.seed, pkey, li, stage, round,
                                                                  PU_RJPARAM, 4 + (uint64_t)d)));
      } else {
        for (int d = 0; d < D; ++d) {
          const double u = u01(pw.w[d]);
          s_znew[d] = (pb.wrapmask >> d & 1u) ? u : log(u) - log1p(-u);
        }
      }
    } else if (move == 2) {
      int j = (int)floor(__dmul_rn(u01(w.w[2]), (double)K));
      if (j >= K) j = K - 1;
      s_j = j;
    }
    s_u = u01(w.w[1]);
    s_move = move;
    if (move == 0 && outcome) outcome[gi] = out;
  }
  __syncthreads();
  const int move = s_move;
  if (move == 0) return;
  char* p = smem;
  EvalSmem sm = carve_eval(p, sp, kp.tw);
  double* zs = reinterpret_cast<double*>(p);    // [kd + D]
  const double* zg = kp.z + gi * (int64_t)sp.kd;
  if (PREC == MIXED) init_block_tables(sm);
  for (int i = tid; i < K * D; i += blockDim.x) zs[i] = zg[i];
  if (move == 1 && tid < D) zs[K * D + tid] = s_znew[tid];
  __syncthreads();
  // with the population proposal the component's prior no longer cancels:
  // birth + log prior_z(z_new) - log q(z_new), death + log q(z_j) - log prior_z(z_j)
  double qcorr = 0.0;
  if (kp.birth_proposal) {
    const double* zc = zs + (move == 1 ? K : s_j) * D;
    const double lq = kde_logq_block<D>(kp.kde + (int64_t)prob * kKdeStride, zc, kp.birth_eps,
                                        sm.red);
    const double lp = log_prior_z<D>(zc);
    qcorr = move == 1 ? lp - lq : lq - lp;
  }
  const int kp_idx = move == 1 ? K : s_j;      // index of the proposed component
  eval_setup<MODEL, PREC>(pb, kp.pa, move == 1 ? K + 1 : K, zs, sm);
  const int N = (int)pb.n, n1 = (int)pb.n1;   // < 2^24 samples
  double a_old = 0.0, a_new = 0.0;
  const int seg = blockDim.x * R;
  const int warp = tid >> 5;
  for (int base = 0; base < N; base += seg) {
    const int wfirst = base + warp * 32 * R;
    if (wfirst >= N) continue;
    const float wf = (float)wfirst, wl = (float)(wfirst + 32 * R - 1);
    const int m = base + tid * R;
    // two-channel sinusoids: the thread's channel and local sample index
    const int ch = (MODEL == SINUSOID && pb.nch == 2 && m >= (int)pb.nc) ? 1 : 0;
    const int ml = m - ch * (int)pb.nc;
    if (PREC == MIXED) {
      const float* cfb = sm.cf + ch * sm.cfch;
      const bool win = MODEL != SINUSOID && kp.pa.window;
      float cfp[NCF];
      load_cf(cfb + kp_idx * NCF, cfp);
      if (win && outside_support(cfp, wf, wl)) continue;   // proposal is zero here
      float r[R], hp[R];
#pragma unroll
      for (int j = 0; j < R; ++j) r[j] = (m + j < N) ? pb.d32[m + j] : 0.0f;
      const float mf = (float)ml;
      for (int k = 0; k < K; ++k) {
        float cf[NCF], h[R];
        load_cf(cfb + k * NCF, cf);
        if (win && outside_support(cf, wf, wl)) continue;
        mixed_vals<MODEL, R>(cf, mf, h);
#pragma unroll
        for (int j = 0; j < R; ++j) r[j] -= h[j];
      }
      mixed_vals<MODEL, R>(cfp, mf, hp);
      float so = 0.f, sn = 0.f;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int n = m + j;
        const float h = n < N ? hp[j] : 0.0f;
        const float t = move == 1 ? __fmaf_rn(-0.5f * h, h, r[j] * h)
                                  : -__fmaf_rn(0.5f * h, h, r[j] * h);
        if (n < n1) so += t; else sn += t;
      }
      a_old += (double)so;
      a_new += (double)sn;
    } else {
      double hs[R];
#pragma unroll
      for (int j = 0; j < R; ++j) hs[j] = 0.0;
      double thb[4], thpb[4];
      for (int k = 0; k < K; ++k) {
        const double* th = chan_theta<MODEL>(pb, ch, sm.th + k * D, thb);
        const double tw0 = MODEL == PULSE_LINAMP ? sm.tw[2 * k] : 0.0;
        const double tw1 = MODEL == PULSE_LINAMP ? sm.tw[2 * k + 1] : 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j)
          hs[j] = __dadd_rn(hs[j], fp64_val<MODEL>(th, tw0, tw1, time_of(pb, ml + j), nullptr));
      }
      const double* thp = chan_theta<MODEL>(pb, ch, sm.th + kp_idx * D, thpb);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int n = m + j;
        if (n >= N) continue;
        const double r = __dadd_rn(pb.d64[n], -hs[j]);
        const double h = fp64_val<MODEL>(thp, 0.0, 0.0, time_of(pb, ml + j), nullptr);
        const double rh = __dmul_rn(r, h), hh = __dmul_rn(__dmul_rn(0.5, h), h);
        const double t = move == 1 ? __dadd_rn(rh, -hh) : -__dadd_rn(rh, hh);
        if (n < n1) a_old += t; else a_new += t;
      }
    }
  }
  double v[2] = {a_old, a_new};
  block_sum<2>(v, sm.red);
  if (tid == 0) {
    const double d_old = v[0] * pb.inv_s2, d_new = v[1] * pb.inv_s2;
    const double beta = kp.beta[prob];
    const double dl = d_old + beta * d_new;
    const double la = (move == 1 ? dl + log(kp.p_death) - log(kp.p_birth)
                                 : dl + log(kp.p_birth) - log(kp.p_death)) + qcorr;
    int out;
    double* zw = kp.z + gi * (int64_t)sp.kd;
    if (log(s_u) < la) {
      if (move == 1) {
        for (int d = 0; d < D; ++d) zw[K * D + d] = s_znew[d];
        kp.K[gi] = K + 1;
        out = 1;
      } else {
        const int j = s_j;
        for (int d = 0; d < D; ++d) {
          zw[j * D + d] = zw[(K - 1) * D + d];
          zw[(K - 1) * D + d] = 0.0;
        }
        kp.K[gi] = K - 1;
        out = 2;
      }
      kp.ll_old[gi] += d_old;
      kp.ll_new[gi] += d_new;
    } else {
      out = move == 1 ? -1 : -2;
    }
    if (outcome) outcome[gi] = out;
  }
}

template <int MODEL, int PREC, int R>
__global__ void TSMC_PARTICLE_BOUNDS k_rj(KParams kp, int round, int32_t* outcome, SmemPlan sp) {
  const int64_t gi = kp.order ? (int64_t)kp.order[blockIdx.x] : (int64_t)blockIdx.x;
  rj_particle<MODEL, PREC, R>(kp, gi, round, outcome, sp);
}

// ---------------------------------------------------------------------------
// Population birth proposal of one problem per block (256 threads): m = kKdeM centres
// drawn uniformly, with replacement, over all components of the population (draw i:
// particle slot i of purpose PU_KDE, the stage, round 0), found by a binary search in
// the inclusive prefix sum of K; bandwidth h_d = sd_d * factor (factor =
// (4/(D+2))^(1/(D+4)) m^(-1/(D+4)) from the host), at least 1e-3, with the mean and
// deviation summed in centre order.  kcum: [n_problems][P] int32 scratch.
// ---------------------------------------------------------------------------
__global__ void k_kde_build(KParams kp, int32_t* kcum, double* kde_out, double factor,
                            int stage_arg) {
  __shared__ int32_t s_part[256];
  const int prob = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  if (kp.probs[prob].done) return;
  const int stage = stage_arg >= 0 ? stage_arg : *kp.stage;
  const int P = kp.P, D = kp.D;
  const int32_t* K = kp.K + (int64_t)prob * P;
  int32_t* cum = kcum + (int64_t)prob * P;
  double* out = kde_out + (int64_t)prob * kKdeStride;
  const int chunk = (P + T - 1) / T, lo = min(P, tid * chunk), hi = min(P, lo + chunk);
  int32_t local = 0;
  for (int i = lo; i < hi; ++i) local += K[i];
  s_part[tid] = local;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {   // inclusive scan of the per-thread sums
    const int32_t v = tid >= o ? s_part[tid - o] : 0;
    __syncthreads();
    s_part[tid] += v;
    __syncthreads();
  }
  int32_t run = tid > 0 ? s_part[tid - 1] : 0;
  for (int i = lo; i < hi; ++i) {
    run += K[i];
    cum[i] = run;
  }
  const int32_t total = s_part[T - 1];
  __syncthreads();
  if (total == 0) {
    if (tid == 0) {
      out[0] = 0.0;
      for (int d = 0; d < 4; ++d) out[1 + d] = 1.0;
    }
    return;
  }
  const int64_t kd = (int64_t)kp.kmax * D;
  for (int i = tid; i < kKdeM; i += T) {
    const Rand4 w = draw(kp.seed, prob + kp.prob_base, (uint64_t)i, stage, 0, PU_KDE, 0);
    int32_t q = (int32_t)floor(__dmul_rn(u01(w.w[0]), (double)total));
    if (q >= total) q = total - 1;
    int a = 0, b = P - 1;   // first particle whose inclusive count exceeds q
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (cum[mid] > q) b = mid; else a = mid + 1;
    }
    const int j = q - (cum[a] - K[a]);
    const double* zp = kp.z + ((int64_t)prob * P + a) * kd + (int64_t)j * D;
    for (int d = 0; d < D; ++d) out[8 + i * D + d] = zp[d];
  }
  __syncthreads();
  if (tid < D) {
    const int d = tid;
    double mean = 0.0;
    for (int i = 0; i < kKdeM; ++i) mean = __dadd_rn(mean, out[8 + i * D + d]);
    mean = __ddiv_rn(mean, (double)kKdeM);
    double var = 0.0;
    for (int i = 0; i < kKdeM; ++i) {
      const double e = __dsub_rn(out[8 + i * D + d], mean);
      var = __dadd_rn(var, __dmul_rn(e, e));
    }
    var = __ddiv_rn(var, (double)(kKdeM - 1));
    const double h = __dmul_rn(__dsqrt_rn(var), factor);
    out[1 + d] = h < 1e-3 ? 1e-3 : h;
  }
  if (tid == 0) out[0] = (double)kKdeM;
}

// ---------------------------------------------------------------------------
// NUTS transition (Sec. 3.2): one block per particle.  Warps 0 and 1 run the tree
// logic on the (K*D)-vectors in shared memory; every leapfrog calls the block-wide
// evaluation.  Control values are broadcast through shared memory.  k_nuts is the FP64
// path (control in FP64, the oracle's arithmetic); k_nuts_mixed the mixed path.
// ---------------------------------------------------------------------------
struct NutsOut { double* acc; int32_t* nleaf; int32_t* flags; };

// Tree-control arithmetic of k_nuts: FP64 (bit-level agreement with the oracle).
__device__ __forceinline__ double ct_exp(double x) { return exp(x); }
__device__ __forceinline__ double ct_log1p(double x) { return log1p(x); }

template <typename CT>
__device__ __forceinline__ double lae(double a, double b) {   // log(e^a + e^b)
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = a > b ? a : b;
  return m + (double)ct_log1p(ct_exp((CT)(-fabs(a - b))));
}

template <typename CT>
__device__ __forceinline__ CT momentum_normal(uint64_t seed, int problem, uint64_t particle,
                                              int stage, int round, uint64_t m);
template <>
__device__ __forceinline__ double momentum_normal<double>(uint64_t seed, int problem,
                                                          uint64_t particle, int stage,
                                                          int round, uint64_t m) {
  return draw_normal(seed, problem, particle, stage, round, PU_MOMENTUM, m);
}

template <typename CT>
__device__ __forceinline__ CT warp_dot_minv(const CT* a, const CT* b, const CT* minv, int n,
                                            int D) {
  CT s = 0;
  for (int i = threadIdx.x & 31; i < n; i += 32) s += a[i] * (minv[i % D] * b[i]);
  return warp_sum(s);
}

template <int MODEL, int PREC, int R>
__global__ void TSMC_PARTICLE_BOUNDS k_nuts(KParams kp, int round, NutsOut out, SmemPlan sp) {
  static_assert(PREC == FP64, "the mixed path runs k_nuts_mixed");
  using CT = double;
  extern __shared__ __align__(16) char smem[];
  constexpr int D = model_d<MODEL>();
  __shared__ int s_flag[8];
  __shared__ double s_ctl[8];
  __shared__ CT s_minv[4];
  __shared__ double s_uleaf;   // uniform of the next leaf's multinomial choice
  const int64_t gi = kp.order ? (int64_t)kp.order[blockIdx.x] : (int64_t)blockIdx.x;
  const int prob = (int)(gi / kp.P);
  const int pkey = prob + kp.prob_base;
  const uint64_t li = (uint64_t)(gi % kp.P) + (uint64_t)kp.particle_base;
  __shared__ ProbDev s_pb;
  const ProbDev& pb = stage_problem(kp.probs, prob, s_pb);
  if (pb.done) return;
  const int stage = *kp.stage;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = min(max(kp.K[gi], 0), kp.kmax);
  const int n = K * D;
  bool run = n > 0;
  if (kp.schedule == 1) {
    const Rand4 m = draw(kp.seed, pkey, li, stage, round, PU_MOVETYPE, 0);
    run = run && (u01(m.w[0]) < kp.p_nuts);
  }
  if (!run) {
    if (tid == 0) {
      if (out.acc) out.acc[gi] = 0.0;
      if (out.nleaf) out.nleaf[gi] = 0;
      if (out.flags) out.flags[gi] = 0;
    }
    return;
  }
  char* p = smem;
  EvalSmem sm = carve_eval(p, sp, kp.tw);
  const int kd = sp.kd;
  // positions (FP64) and the evaluation's gradient output (CT, in an 8-byte slot)
  double* vd = reinterpret_cast<double*>(p);
  double *zc = vd, *z1 = vd + kd, *zL = vd + 2 * kd, *zR = vd + 3 * kd, *sz = vd + 4 * kd;
  CT* g1 = reinterpret_cast<CT*>(vd + 5 * kd);
  // momenta, gradients at the ends, momentum sums and checkpoints (CT), one slot of
  // 8 bytes per element each so the layout does not depend on CT
  CT* vc = reinterpret_cast<CT*>(vd + 6 * kd);
  const int st = (int)(sizeof(double) / sizeof(CT)) * kd;   // CT elements per slot
  CT *p1 = vc, *pL = vc + st, *pR = vc + 2 * st, *gL = vc + 3 * st, *gR = vc + 4 * st;
  CT *rho = vc + 5 * st, *srho = vc + 6 * st;
  CT* p1n = vc + 7 * st;                       // next momentum (swapped with p1 per leaf)
  CT* ckp = vc + 8 * st;                       // [(depth+1)][kd] CT
  CT* ckr = ckp + (size_t)(sp.depth + 1) * kd;
  const double beta = kp.beta[prob];
  const double eps = kp.eps[prob];
  if (tid < 4) s_minv[tid] = (CT)kp.minv[4 * prob + tid];
  const CT* minv = s_minv;
  const double* zg = kp.z + gi * (int64_t)kd;
  for (int i = tid; i < n; i += blockDim.x) { zc[i] = zg[i]; z1[i] = zg[i]; }
  __syncthreads();
  double cs_done = 0.0;   // component*samples computed (thread 0)
  // The evaluation has one call site: iteration l = -1 evaluates the initial point,
  // then the leaves l = 0 .. 2^depth - 1 of each subtree follow in order.
  // Scalar tree state lives in shared memory and is touched by lane 0 of warp 0
  // (s_flag[6] by lane 0 of the U-turn warp); decisions reach the other lanes by
  // shuffles, the other warps by s_flag.
  // s_ctl: 0 H0, 1 logW, 2 sum_acc, 3 cand_lo, 4 cand_ln, 5 sub_logW, 6 sub_lo, 7 sub_ln
  // s_flag: 0 leaf valid (energy), 1 stop, 2 direction, 3 leaves, 4 diverged, 5 depth done,
  //         6 no U-turn inside the subtree
  int depth = 0, l = -1;
  double de = 0.0;
  CT de_c = 0;
  for (;;) {
    const int nsub = 1 << depth;
    if (l == 0) {   // a new subtree: direction, and the trajectory end it grows from
      if (warp == 0) {
        int dir = 0;
        if (lane == 0) {
          const Rand4 w = draw(kp.seed, pkey, li, stage, round, PU_DIRECTION, (uint64_t)depth);
          dir = u01(w.w[0]) < 0.5 ? -1 : 1;
          s_ctl[5] = -INFINITY;
          s_flag[0] = 1;
          s_flag[2] = dir;
        }
        dir = __shfl_sync(0xffffffffu, dir, 0);
        const double* zs0 = dir > 0 ? zR : zL;
        const CT *ps0 = dir > 0 ? pR : pL, *gs0 = dir > 0 ? gR : gL;
        for (int i = lane; i < n; i += 32) {
          z1[i] = zs0[i]; p1[i] = ps0[i]; g1[i] = gs0[i]; srho[i] = 0;
        }
      }
      __syncthreads();
      de = s_flag[2] * eps;
      de_c = (CT)de;
    }
    if (l >= 0) {   // leapfrog: half step in momentum, full step in position
      if (warp == 0) {
        for (int i = lane; i < n; i += 32) {
          const CT ph = p1[i] + (CT)0.5 * de_c * g1[i];
          p1[i] = ph;
          z1[i] = z1[i] + de * (double)minv[i % D] * (double)ph;
        }
      }
      if (l > 0 && tid == blockDim.x - 1) {   // the leaf's uniform, off the control path
        const Rand4 w = draw(kp.seed, pkey, li, stage, round, PU_LEAF,
                             (uint64_t)((nsub - 1) + l));
        s_uleaf = u01(w.w[0]);
      }
      __syncthreads();
    }
    block_eval<MODEL, PREC, R, true, false, CT>(pb, kp.pa, K, beta, z1, sm, g1, nullptr);
    if (tid == 0) cs_done += sm.scal[3];
    if (l < 0) {   // initial point: momentum, H0 and both trajectory ends
      if (warp == 0) {
        for (int i = lane; i < n; i += 32) {
          const CT pm = sqrt((CT)1 / minv[i % D]) *
                        momentum_normal<CT>(kp.seed, pkey, li, stage, round, (uint64_t)i);
          pL[i] = pm; pR[i] = pm; rho[i] = pm;
          zL[i] = zc[i]; zR[i] = zc[i];
          gL[i] = g1[i]; gR[i] = g1[i];
        }
        __syncwarp();
        CT kin = 0;
        for (int i = lane; i < n; i += 32) kin += minv[i % D] * pL[i] * pL[i];
        kin = warp_sum(kin);
        if (lane == 0) {
          const double H0 = -sm.scal[0] + 0.5 * (double)kin;
          s_ctl[0] = H0;
          s_ctl[1] = -H0;
          s_ctl[2] = 0.0;
          s_ctl[3] = sm.scal[1];
          s_ctl[4] = sm.scal[2];
          s_flag[3] = 0; s_flag[4] = 0; s_flag[5] = 0;
        }
      }
      if (kp.max_depth <= 0) break;
      l = 0;
      continue;
    }
    // ---- leaf: momentum half step p' = p + eps/2 grad.  Warp 0: energy and the
    // multinomial choice; warp uw (1, or 0 after it in a one-warp block): p' into the
    // other momentum buffer, checkpoints and the U-turn checks of the subtrees the
    // leaf closes.  Divergence or a U-turn ends the transition, so the U-turn state
    // written on a divergent leaf is never read. ----
    const int uw = blockDim.x > 32 ? 1 : 0;
    if (warp == 0) {
      CT kin = 0;
      for (int i = lane; i < n; i += 32) {
        const CT pn = p1[i] + (CT)0.5 * de_c * g1[i];
        kin += minv[i % D] * pn * pn;
      }
      kin = warp_sum(kin);
      const double H = -sm.scal[0] + 0.5 * (double)kin;
      const double H0 = s_ctl[0];
      int ok = 1, take = 0;
      if (lane == 0) {
        s_flag[3] += 1;
        if (isfinite(H)) {
          const double a = (double)ct_exp((CT)(H0 - H));
          s_ctl[2] += a < 1.0 ? a : 1.0;
        }
        if (!isfinite(H) || H - H0 > 1000.0) {
          ok = 0;
          s_flag[4] = 1;
        } else {
          const double lw = -H;
          const double nl = lae<CT>(s_ctl[5], lw);
          take = (l == 0);
          if (!take) take = s_uleaf < (double)ct_exp((CT)(lw - nl));
          if (take) { s_ctl[6] = sm.scal[1]; s_ctl[7] = sm.scal[2]; }
          s_ctl[5] = nl;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      take = __shfl_sync(0xffffffffu, take, 0);
      if (ok && take)
        for (int i = lane; i < n; i += 32) sz[i] = z1[i];
      if (lane == 0) s_flag[0] = ok;
    }
    if (warp == uw) {
      for (int i = lane; i < n; i += 32) p1n[i] = p1[i] + (CT)0.5 * de_c * g1[i];
      for (int mm = 1; mm <= depth; ++mm) {
        if ((l & ((1 << mm) - 1)) == 0) {
          for (int i = lane; i < n; i += 32) {
            ckp[mm * kd + i] = p1n[i];
            ckr[mm * kd + i] = srho[i];
          }
        }
      }
      for (int i = lane; i < n; i += 32) srho[i] += p1n[i];
      __syncwarp();
      int uok = 1;
      for (int mm = 1; mm <= depth && uok; ++mm) {
        if (((l + 1) & ((1 << mm) - 1)) == 0) {
          CT s1 = 0, s2 = 0;
          for (int i = lane; i < n; i += 32) {
            const CT seg = srho[i] - ckr[mm * kd + i];
            const CT mi = minv[i % D];
            s1 += seg * (mi * ckp[mm * kd + i]);
            s2 += seg * (mi * p1n[i]);
          }
          s1 = warp_sum(s1);
          s2 = warp_sum(s2);
          if (s1 <= 0 || s2 <= 0) uok = 0;
        }
      }
      if (lane == 0) s_flag[6] = uok;
    }
    __syncthreads();
    {
      CT* t = p1; p1 = p1n; p1n = t;   // p1 now holds p'
    }
    if (s_flag[0] == 0 || s_flag[6] == 0) break;   // divergence or a U-turn inside the subtree
    if (++l < nsub) continue;
    // ---- subtree complete: merge it into the trajectory ----
    if (warp == 0) {
      const int dir = s_flag[2];
      double* ze = dir > 0 ? zR : zL;
      CT *pe = dir > 0 ? pR : pL, *ge = dir > 0 ? gR : gL;
      for (int i = lane; i < n; i += 32) { ze[i] = z1[i]; pe[i] = p1[i]; ge[i] = g1[i]; }
      int take = 0;
      if (lane == 0) {
        const Rand4 w = draw(kp.seed, pkey, li, stage, round, PU_TOP, (uint64_t)depth);
        take = u01(w.w[0]) < (double)ct_exp((CT)(s_ctl[5] - s_ctl[1]));
        if (take) { s_ctl[3] = s_ctl[6]; s_ctl[4] = s_ctl[7]; }
        s_ctl[1] = lae<CT>(s_ctl[1], s_ctl[5]);
        s_flag[5] = depth + 1;
      }
      take = __shfl_sync(0xffffffffu, take, 0);
      if (take)
        for (int i = lane; i < n; i += 32) zc[i] = sz[i];
      for (int i = lane; i < n; i += 32) rho[i] += srho[i];
      __syncwarp();
      const CT dl = warp_dot_minv<CT>(rho, pL, minv, n, D);
      const CT dr = warp_dot_minv<CT>(rho, pR, minv, n, D);
      if (lane == 0) s_flag[1] = (dl <= 0 || dr <= 0) ? 1 : 0;
    }
    __syncthreads();
    if (s_flag[1]) break;            // U-turn of the whole trajectory
    if (++depth >= kp.max_depth) break;
    l = 0;
  }
  if (warp == 0) {
    double* zw = kp.z + gi * (int64_t)kd;
    // periodic coordinates leave the transition reduced to one period
    for (int i = lane; i < n; i += 32)
      zw[i] = (pb.wrapmask >> (i % D) & 1u) ? __dadd_rn(zc[i], -floor(zc[i])) : zc[i];
    if (lane == 0) {
      const int leaves = s_flag[3];
      kp.ll_old[gi] = s_ctl[3];
      kp.ll_new[gi] = s_ctl[4];
      if (out.acc) out.acc[gi] = leaves > 0 ? s_ctl[2] / leaves : 0.0;
      if (out.nleaf) out.nleaf[gi] = leaves;
      if (out.flags) out.flags[gi] = s_flag[4] | (s_flag[5] << 8);
      if (kp.cs_count) {  // slots 1 / 3: NUTS (initial point + every leaf), nominal / computed
        atomicAdd(kp.cs_count + 1, (unsigned long long)n / D * (unsigned long long)pb.n *
                                       (unsigned long long)(leaves + 1));
        atomicAdd(kp.cs_count + 3, (unsigned long long)cs_done);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// NUTS transition on the mixed path (Sec. 3.2): the tree of k_nuts (same moves, same
// random stream) with no FP64 instruction per leaf.  Every FP64 warp instruction holds a
// sub-partition's FP64 unit for tens of cycles on this part, and the per-leaf phases
// that run beside the sample loop (setup, block totals, tree control) sit on each leaf's
// critical path, so: positions are double-float pairs (converted from and to FP64 once per
// transition), the energies H and the log-weights double-float, momenta, U-turn sums,
// acceptance statistics and the probabilities compared with uniforms FP32, uniforms 24-bit.
// The uniforms of a subtree's leaves are drawn in parallel when the subtree starts, the
// direction bits and top-level uniforms of every depth when the transition starts.
// ---------------------------------------------------------------------------
// 24 random bits to the open interval (0, 1): ((x >> 40) + 1/2) 2^-24
__device__ __forceinline__ float u01f(uint64_t x) {
  return __fmaf_rn((float)(uint32_t)(x >> 40), 0x1p-24f, 0x1p-25f);
}
__device__ __forceinline__ bool df_gt(DF a, DF b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
// a + b for a double-float a and a float b (a non-finite a gives the plain sum)
__device__ __forceinline__ DF df_add_f(DF a, float b) {
  if (!isfinite(a.hi)) return DF{a.hi + b, 0.f};
  const DF s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
// a - b rounded to FP32 (finite a, b)
__device__ __forceinline__ float df_sub_f(DF a, DF b) { return df_add(a, df_neg(b)).hi; }
// log(e^a + e^b) of double-float log-weights (hi = -inf: weight zero)
__device__ __forceinline__ DF df_lae(DF a, DF b) {
  if (a.hi == -INFINITY) return b;
  if (b.hi == -INFINITY) return a;
  const bool ab = df_gt(a, b);
  const DF m = ab ? a : b, o = ab ? b : a;
  return df_add_f(m, log1pf(expf(df_sub_f(o, m))));
}
// m-th standard normal of the momentum stream: the Box-Muller pairing of draw_normal, in FP32
// from 24-bit uniforms
__device__ __forceinline__ float momentum_normal_f(uint64_t seed, int problem, uint64_t particle,
                                                   int stage, int round, uint64_t m) {
  const Rand4 r = draw(seed, problem, particle, stage, round, PU_MOMENTUM, m >> 2);
  const int pair = (int)((m & 3) >> 1);
  const float ua = u01f(r.w[2 * pair]), ub = u01f(r.w[2 * pair + 1]);
  const float rad = sqrtf(-2.0f * logf(ua));
  float sn, cs;
  sincospif(2.0f * ub, &sn, &cs);
  return (m & 1) ? rad * sn : rad * cs;
}

// one particle's transition (all threads of the block call it; block-uniform exits)
template <int MODEL, int R>
__device__ void nuts_particle_mixed(const KParams& kp, int64_t gi, int round, NutsOut out,
                                    const SmemPlan& sp) {
  extern __shared__ __align__(16) char smem[];
  constexpr int D = model_d<MODEL>();
  __shared__ int s_flag[8];
  // 0 H0, 1 log W of the trajectory, 3/4 ll_old/ll_new of the chosen point, 5 log W of the
  // current subtree, 6/7 ll_old/ll_new of its candidate
  __shared__ DF s_ctl[8];
  __shared__ float s_acc;                 // sum over leaves of min(1, e^{H0 - H})
  __shared__ float s_minv[4];
  __shared__ int s_dir[kMaxDepth];
  __shared__ float s_utop[kMaxDepth];
  const int prob = (int)(gi / kp.P);
  const int pkey = prob + kp.prob_base;
  const uint64_t li = (uint64_t)(gi % kp.P) + (uint64_t)kp.particle_base;
  __shared__ ProbDev s_pb;
  const ProbDev& pb = stage_problem(kp.probs, prob, s_pb);
  if (pb.done) return;
  const int stage = *kp.stage;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = min(max(kp.K[gi], 0), kp.kmax);
  const int n = K * D;
  bool run = n > 0;
  if (kp.schedule == 1) {
    const Rand4 m = draw(kp.seed, pkey, li, stage, round, PU_MOVETYPE, 0);
    run = run && (u01(m.w[0]) < kp.p_nuts);
  }
  if (!run) {
    if (tid == 0) {
      if (out.acc) out.acc[gi] = 0.0;
      if (out.nleaf) out.nleaf[gi] = 0;
      if (out.flags) out.flags[gi] = 0;
    }
    return;
  }
  char* p = smem;
  EvalSmem sm = carve_eval(p, sp, kp.tw);
  const int kd = sp.kd;
  float2* vz = reinterpret_cast<float2*>(p);
  float2 *zc = vz, *z1 = vz + kd, *zL = vz + 2 * kd, *zR = vz + 3 * kd, *sz = vz + 4 * kd;
  float* vf = reinterpret_cast<float*>(vz + 5 * kd);
  float *g1 = vf, *p1 = vf + kd, *pL = vf + 2 * kd, *pR = vf + 3 * kd, *gL = vf + 4 * kd;
  float *gR = vf + 5 * kd, *rho = vf + 6 * kd, *srho = vf + 7 * kd;
  float* p1n = vf + 8 * kd;                        // next momentum (swapped with p1 per leaf)
  float* ckp = vf + 9 * kd;                        // [(depth+1)][kd]
  float* ckr = ckp + (size_t)(sp.depth + 1) * kd;
  float* uleaf = ckr + (size_t)(sp.depth + 1) * kd;   // leaf uniforms of the current subtree
  const double beta = kp.beta[prob];
  const DF beta_df = to_df(beta);
  const float eps_f = (float)kp.eps[prob];
  if (tid < 4) s_minv[tid] = (float)kp.minv[4 * prob + tid];
  const float* minv = s_minv;
  const double* zg = kp.z + gi * (int64_t)kd;
  init_block_tables(sm);
  for (int i = tid; i < n; i += blockDim.x) {
    const DF v = to_df(zg[i]);
    zc[i] = make_float2(v.hi, v.lo);
    z1[i] = zc[i];
  }
  if (tid < kp.max_depth) {   // direction (u01 < 1/2 <=> top bit clear) and top uniform per depth
    const Rand4 w = draw(kp.seed, pkey, li, stage, round, PU_DIRECTION, (uint64_t)tid);
    s_dir[tid] = (w.w[0] >> 63) ? 1 : -1;
    const Rand4 t = draw(kp.seed, pkey, li, stage, round, PU_TOP, (uint64_t)tid);
    s_utop[tid] = u01f(t.w[0]);
  }
  __syncthreads();
  unsigned long long cs_done = 0;   // component*samples computed (thread 0)
  // one evaluation call site: iteration l = -1 evaluates the initial point, then the leaves
  // l = 0 .. 2^depth - 1 of each subtree follow in order (see k_nuts for the flags)
  int depth = 0, l = -1;
  float de_c = 0.f;
  bool moved = false;   // the transition's point changed (read by warp 0)
  for (;;) {
    const int nsub = 1 << depth;
    if (l == 0) {   // a new subtree: its leaves' uniforms, and the end it grows from
      for (int q = tid + 1; q < nsub; q += blockDim.x) {
        const Rand4 w = draw(kp.seed, pkey, li, stage, round, PU_LEAF, (uint64_t)((nsub - 1) + q));
        uleaf[q] = u01f(w.w[0]);
      }
      const int dir = s_dir[depth];
      if (warp == 0) {
        if (lane == 0) {
          s_ctl[5] = DF{-INFINITY, 0.f};
          s_flag[0] = 1;
        }
        const float2* zs0 = dir > 0 ? zR : zL;
        const float *ps0 = dir > 0 ? pR : pL, *gs0 = dir > 0 ? gR : gL;
        for (int i = lane; i < n; i += 32) {
          z1[i] = zs0[i]; p1[i] = ps0[i]; g1[i] = gs0[i]; srho[i] = 0.f;
        }
      }
      __syncthreads();
      de_c = dir > 0 ? eps_f : -eps_f;
    }
    {
      // leapfrog (l >= 0): half step in momentum and full step in position, element by
      // element inside the evaluation's setup
      const LeapPre<float2> leap{p1, g1, z1, minv, de_c};
      block_eval_mixed<MODEL, R, true, false, float, false, float2>(
          pb, kp.pa, K, beta, z1, sm, g1, nullptr, l >= 0 ? &leap : nullptr, beta_df);
    }
    if (tid == 0) cs_done += (unsigned long long)*sm.scalc();
    const float* f = sm.scalf();
    const DF logp{f[0], f[1]};
    if (l < 0) {   // initial point: momentum, H0 and both trajectory ends
      if (warp == 0) {
        for (int i = lane; i < n; i += 32) {
          const float pm = sqrtf(1.0f / minv[i % D]) *
                           momentum_normal_f(kp.seed, pkey, li, stage, round, (uint64_t)i);
          pL[i] = pm; pR[i] = pm; rho[i] = pm;
          zL[i] = zc[i]; zR[i] = zc[i];
          gL[i] = g1[i]; gR[i] = g1[i];
        }
        __syncwarp();
        float kin = 0.f;
        for (int i = lane; i < n; i += 32) kin += minv[i % D] * pL[i] * pL[i];
        kin = warp_sum(kin);
        if (lane == 0) {
          const DF H0 = df_add_f(df_neg(logp), 0.5f * kin);
          s_ctl[0] = H0;
          s_ctl[1] = df_neg(H0);
          s_acc = 0.f;
          s_ctl[3] = DF{f[2], f[3]};
          s_ctl[4] = DF{f[4], f[5]};
          s_flag[3] = 0; s_flag[4] = 0; s_flag[5] = 0;
        }
      }
      if (kp.max_depth <= 0) break;
      l = 0;
      continue;
    }
    // ---- leaf: warp 0 energy and multinomial choice; warp uw momentum, checkpoints and
    // U-turn checks of the subtrees the leaf closes (as in k_nuts) ----
    const int uw = blockDim.x > 32 ? 1 : 0;
    if (warp == 0) {
      float kin = 0.f;
      for (int i = lane; i < n; i += 32) {
        const float pn = p1[i] + 0.5f * de_c * g1[i];
        kin += minv[i % D] * pn * pn;
      }
      kin = warp_sum(kin);
      const DF H = df_add_f(df_neg(logp), 0.5f * kin);
      int ok = 1, take = 0;
      if (lane == 0) {
        s_flag[3] += 1;
        const bool fin = isfinite(H.hi) && isfinite(H.lo);
        const float dH = fin ? df_sub_f(H, s_ctl[0]) : INFINITY;   // H - H0
        if (fin) {
          const float a = expf(-dH);
          s_acc += a < 1.0f ? a : 1.0f;
        }
        if (!fin || dH > 1000.0f) {
          ok = 0;
          s_flag[4] = 1;
        } else {
          const DF lw = df_neg(H);
          const DF nl = df_lae(s_ctl[5], lw);
          take = (l == 0);
          if (!take) take = uleaf[l] < expf(df_sub_f(lw, nl));
          if (take) { s_ctl[6] = DF{f[2], f[3]}; s_ctl[7] = DF{f[4], f[5]}; }
          s_ctl[5] = nl;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      take = __shfl_sync(0xffffffffu, take, 0);
      if (ok && take)
        for (int i = lane; i < n; i += 32) sz[i] = z1[i];
      if (lane == 0) s_flag[0] = ok;
    }
    if (warp == uw) {
      for (int i = lane; i < n; i += 32) p1n[i] = p1[i] + 0.5f * de_c * g1[i];
      for (int mm = 1; mm <= depth; ++mm) {
        if ((l & ((1 << mm) - 1)) == 0) {
          for (int i = lane; i < n; i += 32) {
            ckp[mm * kd + i] = p1n[i];
            ckr[mm * kd + i] = srho[i];
          }
        }
      }
      for (int i = lane; i < n; i += 32) srho[i] += p1n[i];
      __syncwarp();
      int uok = 1;
      for (int mm = 1; mm <= depth && uok; ++mm) {
        if (((l + 1) & ((1 << mm) - 1)) == 0) {
          float s1 = 0.f, s2 = 0.f;
          for (int i = lane; i < n; i += 32) {
            const float seg = srho[i] - ckr[mm * kd + i];
            const float mi = minv[i % D];
            s1 += seg * (mi * ckp[mm * kd + i]);
            s2 += seg * (mi * p1n[i]);
          }
          s1 = warp_sum(s1);
          s2 = warp_sum(s2);
          if (s1 <= 0.f || s2 <= 0.f) uok = 0;
        }
      }
      if (lane == 0) s_flag[6] = uok;
    }
    __syncthreads();
    {
      float* t = p1; p1 = p1n; p1n = t;   // p1 now holds p'
    }
    if (s_flag[0] == 0 || s_flag[6] == 0) break;   // divergence or a U-turn inside the subtree
    if (++l < nsub) continue;
    // ---- subtree complete: merge it into the trajectory ----
    if (warp == 0) {
      const int dir = s_dir[depth];
      float2* ze = dir > 0 ? zR : zL;
      float *pe = dir > 0 ? pR : pL, *ge = dir > 0 ? gR : gL;
      for (int i = lane; i < n; i += 32) { ze[i] = z1[i]; pe[i] = p1[i]; ge[i] = g1[i]; }
      int take = 0;
      if (lane == 0) {
        take = s_utop[depth] < expf(df_sub_f(s_ctl[5], s_ctl[1]));
        if (take) { s_ctl[3] = s_ctl[6]; s_ctl[4] = s_ctl[7]; }
        s_ctl[1] = df_lae(s_ctl[1], s_ctl[5]);
        s_flag[5] = depth + 1;
      }
      take = __shfl_sync(0xffffffffu, take, 0);
      if (take) {
        moved = true;
        for (int i = lane; i < n; i += 32) zc[i] = sz[i];
      }
      for (int i = lane; i < n; i += 32) rho[i] += srho[i];
      __syncwarp();
      const float dl = warp_dot_minv<float>(rho, pL, minv, n, D);
      const float dr = warp_dot_minv<float>(rho, pR, minv, n, D);
      if (lane == 0) s_flag[1] = (dl <= 0.f || dr <= 0.f) ? 1 : 0;
    }
    __syncthreads();
    if (s_flag[1]) break;            // U-turn of the whole trajectory
    if (++depth >= kp.max_depth) break;
    l = 0;
  }
  if (warp == 0) {
    // an unmoved particle keeps its FP64 coordinates exactly; periodic coordinates leave
    // the transition reduced to one period either way
    double* zw = kp.z + gi * (int64_t)kd;
    const uint32_t wm = pb.wrapmask;
    if (moved) {
      for (int i = lane; i < n; i += 32) zw[i] = to_double(zc[i]);
    }
    if (wm) {
      __syncwarp();
      for (int i = lane; i < n; i += 32)
        if (wm >> (i % D) & 1u) zw[i] = __dadd_rn(zw[i], -floor(zw[i]));
    }
    if (lane == 0) {
      const int leaves = s_flag[3];
      kp.ll_old[gi] = df_to_double(s_ctl[3]);
      kp.ll_new[gi] = df_to_double(s_ctl[4]);
      if (out.acc) out.acc[gi] = leaves > 0 ? (double)s_acc / leaves : 0.0;
      if (out.nleaf) out.nleaf[gi] = leaves;
      if (out.flags) out.flags[gi] = s_flag[4] | (s_flag[5] << 8);
      if (kp.cs_count) {  // slots 1 / 3: NUTS (initial point + every leaf), nominal / computed
        atomicAdd(kp.cs_count + 1, (unsigned long long)n / D * (unsigned long long)pb.n *
                                       (unsigned long long)(leaves + 1));
        atomicAdd(kp.cs_count + 3, cs_done);
      }
    }
  }
}

template <int MODEL, int R>
__global__ void __launch_bounds__(256, 2) k_nuts_mixed(KParams kp, int round, NutsOut out,
                                                         SmemPlan sp) {
  const int64_t gi = kp.order ? (int64_t)kp.order[blockIdx.x] : (int64_t)blockIdx.x;
  nuts_particle_mixed<MODEL, R>(kp, gi, round, out, sp);
}

// ---------------------------------------------------------------------------
// The mutation rounds of a stage in one persistent launch (mixed path): within a stage the
// step size, the metric and the birth proposal are fixed, so a particle's rounds (birth /
// death, then a NUTS transition, n_mut times) depend on no other particle.  Each block
// takes the next particle from a counter, in the longest-first order, and runs all its
// rounds; a block whose particle finishes early takes another one instead of idling at
// the end of a per-round launch behind the deepest trees.  Blocks never wait on one another
// (the counter is their only shared state), so any grid size is safe; the host launches as
// many blocks as are resident at once.  Per-round outputs go to [round][particle] rows.
// Opt-in (tsmc_config.fused_rounds): with longest-first ordering the per-round launches
// keep their slots busy to within a few percent, and this larger kernel computes ~8% fewer
// component*samples per second than the separate ones on the pulse and band workloads.
// ---------------------------------------------------------------------------
struct MutOut {
  int32_t* outcome;   // [Ptot] birth/death outcome of the last round
  double* acc;        // [n_rounds][Ptot]
  int32_t* nleaf;     // [n_rounds][Ptot]
  int32_t* flags;     // [n_rounds][Ptot]
};

template <int MODEL, int R>
__global__ void __launch_bounds__(256, 2) k_mutate_mixed(KParams kp, int n_rounds, MutOut mo,
                                                           SmemPlan sp, unsigned int* next,
                                                           int rj) {
  __shared__ unsigned int s_item;
  const unsigned int total = (unsigned int)(kp.n_problems * kp.P);
  const int64_t Ptot = (int64_t)total;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1u);
    __syncthreads();
    const unsigned int item = s_item;
    __syncthreads();   // every thread has read s_item before it is written again
    if (item >= total) return;
    const int64_t gi = kp.order ? (int64_t)kp.order[item] : (int64_t)item;
    for (int r = 0; r < n_rounds; ++r) {
      if (rj) {
        rj_particle<MODEL, MIXED, R>(kp, gi, r, mo.outcome, sp);
        __syncthreads();
      }
      NutsOut no{mo.acc + r * Ptot, mo.nleaf + r * Ptot, mo.flags + r * Ptot};
      nuts_particle_mixed<MODEL, R>(kp, gi, r, no, sp);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Adaptive tempering (Sec. 2, Eqs. incremental_weight, ess and ess_target; one block
// per problem): ESS(delta) = (sum x)^2 / sum x^2 with
// x_i = exp(delta (ell_i - max ell)); bisection for ESS = alpha P on (0, 1-beta].
// ---------------------------------------------------------------------------
struct TemperIO {
  const double* ell;   // ll_new [Ptot]
  double* logw;        // [Ptot]
  double* beta;        // [n_problems] in/out
  double* logz;        // [n_problems] in/out
  double* ess;         // [n_problems]
  ProbDev* probs;      // done flags
  double alpha;
};

__device__ void ess_sums(const double* ell, int P, double m, double delta, double* red,
                         double& s1, double& s2) {
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double e = ell[i];
    const double x = isfinite(e) ? exp(delta * (e - m)) : 0.0;
    v[0] += x;
    v[1] += x * x;
  }
  block_sum<2>(v, red);
  s1 = v[0];
  s2 = v[1];
}

__global__ void __launch_bounds__(1024) k_temper(TemperIO io, int P) {
  __shared__ double red[128];
  __shared__ double s_m;
  const int prob = blockIdx.x;
  const double* ell = io.ell + (int64_t)prob * P;
  double* logw = io.logw + (int64_t)prob * P;
  const double beta = io.beta[prob];
  if (beta >= 1.0) {
    if (threadIdx.x == 0) io.probs[prob].done = 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) logw[i] = 0.0;
    return;
  }
  double mx = -INFINITY;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double e = ell[i];
    if (isfinite(e) && e > mx) mx = e;
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    s_m = m;
  }
  __syncthreads();
  const double m = s_m;
  const double target = io.alpha * (double)P;
  const double dmax = 1.0 - beta;
  double s1, s2;
  ess_sums(ell, P, m, dmax, red, s1, s2);
  double delta;
  bool to_one = false;
  if (s1 * s1 / s2 >= target) {
    delta = dmax;
    to_one = true;
  } else {
    double lo = 0.0, hi = dmax;
    for (int it = 0; it < 100; ++it) {
      if (hi - lo < 1e-14) break;
      const double mid = 0.5 * (lo + hi);
      ess_sums(ell, P, m, mid, red, s1, s2);
      if (s1 * s1 / s2 >= target) lo = mid; else hi = mid;
    }
    delta = lo > 0.0 ? lo : hi;
    ess_sums(ell, P, m, delta, red, s1, s2);
  }
  // a particle whose likelihood is not finite has zero weight, as in the ESS sums
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double e = ell[i];
    logw[i] = isfinite(e) ? delta * e : -INFINITY;
  }
  if (threadIdx.x == 0) {
    io.beta[prob] = to_one ? 1.0 : beta + delta;
    io.logz[prob] += (delta * m + log(s1)) - log((double)P);
    io.ess[prob] = s1 * s1 / s2;
  }
}

// Mixed path: the ESS of each bisection pass in FP32 from d_i = ell_i - max (stored once
// as FP32), x_i = 2^(delta d_i log2 e); the chosen delta then gets one FP64 pass for
// the ESS, the log-weights and the evidence increment, as above.
__device__ void ess_sums_f32(const float* d, int P, float delta, float* redf, float& s1,
                             float& s2) {
  float a = 0.f, b = 0.f;
  const float k = delta * 1.44269504088896341f;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const float x = exp2f(k * d[i]);
    a += x;
    b = __fmaf_rn(x, x, b);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) { redf[warp] = a; redf[32 + warp] = b; }
  __syncthreads();
  a = 0.f; b = 0.f;
  for (int w = 0; w < nw; ++w) { a += redf[w]; b += redf[32 + w]; }
  s1 = a;
  s2 = b;
}

__global__ void __launch_bounds__(1024) k_temper_mixed(TemperIO io, int P, float* dscratch) {
  __shared__ double red[128];
  __shared__ float redf[64];
  __shared__ double s_m;
  const int prob = blockIdx.x;
  const double* ell = io.ell + (int64_t)prob * P;
  double* logw = io.logw + (int64_t)prob * P;
  float* d = dscratch + (int64_t)prob * P;
  const double beta = io.beta[prob];
  if (beta >= 1.0) {
    if (threadIdx.x == 0) io.probs[prob].done = 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) logw[i] = 0.0;
    return;
  }
  double mx = -INFINITY;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double e = ell[i];
    if (isfinite(e) && e > mx) mx = e;
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    s_m = m;
  }
  __syncthreads();
  const double m = s_m;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double e = ell[i];
    d[i] = isfinite(e) ? (float)(e - m) : -INFINITY;
  }
  __syncthreads();
  const double target = io.alpha * (double)P;
  const double dmax = 1.0 - beta;
  float a, b;
  ess_sums_f32(d, P, (float)dmax, redf, a, b);
  double delta;
  bool to_one = false;
  if ((double)a * (double)a / (double)b >= target) {
    delta = dmax;
    to_one = true;
  } else {
    double lo = 0.0, hi = dmax;
    for (int it = 0; it < 100; ++it) {
      if (hi - lo < 1e-14) break;
      const double mid = 0.5 * (lo + hi);
      ess_sums_f32(d, P, (float)mid, redf, a, b);
      if ((double)a * (double)a / (double)b >= target) lo = mid; else hi = mid;
    }
    delta = lo > 0.0 ? lo : hi;
  }
  double s1, s2;
  ess_sums(ell, P, m, delta, red, s1, s2);
  // a particle whose likelihood is not finite has zero weight, as in the ESS sums
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double e = ell[i];
    logw[i] = isfinite(e) ? delta * e : -INFINITY;
  }
  if (threadIdx.x == 0) {
    io.beta[prob] = to_one ? 1.0 : beta + delta;
    io.logz[prob] += (delta * m + log(s1)) - log((double)P);
    io.ess[prob] = s1 * s1 / s2;
  }
}

// ---------------------------------------------------------------------------
// Systematic resampling (the resampling step of Sec. 2; one block per problem) on
// quantised weights: W_i = round(exp(logw_i - max) 2^S), S = 52 - ceil(log2 P), so the
// inclusive prefix sums C_j are exact integers (at most 2^52) whatever the summation
// order, and a_i = min{j : C_j > t_i}, t_i = min((i + U) / P C_P, C_P - 1), U from Philox.
// The ancestors are therefore the same bit for bit on any summation schedule.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int resample_scale(int P) {
  int S = 52;
  for (long long q = 1; q < (long long)P; q <<= 1) --S;
  return S;
}

__global__ void __launch_bounds__(1024) k_resample(const double* logw_all, long long* cw_all,
                                                   int32_t* anc_all, const ProbDev* probs,
                                                   uint64_t seed, int stage, int P,
                                                   int prob_base) {
  __shared__ double red[32];
  __shared__ long long s_carry[33];
  __shared__ double s_m;
  const int prob = blockIdx.x;
  if (probs[prob].done) return;
  const double* logw = logw_all + (int64_t)prob * P;
  long long* C = cw_all + (int64_t)prob * P;
  int32_t* anc = anc_all + (int64_t)prob * P;
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double mx = -INFINITY;
  for (int i = tid; i < P; i += T) mx = logw[i] > mx ? logw[i] : mx;
  mx = warp_max(mx);
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = -INFINITY;
    for (int w = 0; w < (T >> 5); ++w) m = red[w] > m ? red[w] : m;
    s_m = m;
  }
  __syncthreads();
  const double m = s_m;
  const double scale = ldexp(1.0, resample_scale(P));   // exact power of two
  // contiguous chunk per thread, sequential local scan, then block exclusive scan
  const int chunk = (P + T - 1) / T;
  const int b = tid * chunk, e = min(P, b + chunk);
  long long run = 0;
  for (int i = b; i < e; ++i) {
    const double w = exp(__dadd_rn(logw[i], -m));
    run += w > 0.0 ? __double2ll_rn(__dmul_rn(w, scale)) : 0ll;   // NaN, 0: no weight
    C[i] = run;
  }
  long long x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  long long excl = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) excl = 0;
  if (lane == 31) s_carry[warp] = x;
  __syncthreads();
  if (tid == 0) {
    long long c = 0;
    for (int w = 0; w < (T >> 5); ++w) { const long long t = s_carry[w]; s_carry[w] = c; c += t; }
    s_carry[32] = c;
  }
  __syncthreads();
  const long long off = s_carry[warp] + excl;
  for (int i = b; i < e; ++i) C[i] += off;
  __syncthreads();
  const double total = (double)C[P - 1];       // exact: at most 2^52
  const Rand4 w = draw(seed, prob + prob_base, 0, stage, 0, PU_RESAMPLE, 0);
  const double U = u01(w.w[0]);
  for (int i = tid; i < P; i += T) {
    double target = __dmul_rn(__ddiv_rn(__dadd_rn((double)i, U), (double)P), total);
    if (target > total - 1.0) target = total - 1.0;
    int lo = 0, hi = P - 1;    // first j with C_j > target (C_{P-1} = total > target)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((double)C[mid] > target) hi = mid; else lo = mid + 1;
    }
    anc[i] = lo;
  }
}

// gather the population rows of the ancestors into the alternate buffers
__global__ void k_gather(const int32_t* anc, const ProbDev* probs, int P, int kd,
                         const double* z, const int32_t* K, const double* lo, const double* ln,
                         double* z2, int32_t* K2, double* lo2, double* ln2, int64_t Ptot) {
  const int64_t total = Ptot * (kd + 1);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / (kd + 1);
    const int c = (int)(t % (kd + 1));
    const int prob = (int)(i / P);
    const int64_t src = probs[prob].done ? i : (int64_t)prob * P + anc[i];
    if (c < kd) z2[i * kd + c] = z[src * kd + c];
    else { K2[i] = K[src]; lo2[i] = lo[src]; ln2[i] = ln[src]; }
  }
}

// ---------------------------------------------------------------------------
// Metric (the mass matrix of Sec. 3.2) and step size (one block per problem)
// ---------------------------------------------------------------------------
// population sums of the metric per problem: sums[prob][0..3] = sum over particles of the
// per-particle Gauss-Newton sums, sums[prob][4] = sum of K (particles with a non-finite
// diagonal left out)
__global__ void k_metric_sums(const double* fis_sum, const int32_t* K, const ProbDev* probs, int P,
                              int D, double* sums) {
  __shared__ double red[160];
  const int prob = blockIdx.x;
  if (probs[prob].done) return;
  double v[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const int64_t g = (int64_t)prob * P + i;
    bool fin = true;
    for (int d = 0; d < D; ++d) fin = fin && isfinite(fis_sum[g * D + d]);
    if (!fin) continue;   // a particle with a non-finite coordinate has zero density
    for (int d = 0; d < D; ++d) v[d] += fis_sum[g * D + d];
    v[4] += (double)K[g];
  }
  block_sum<5>(v, red);
  if (threadIdx.x < 5) sums[5 * prob + threadIdx.x] = v[threadIdx.x];
}

// M^-1 from the population sums: minv_d = 1 / max(1e-8, sum_d / sum K)  (unit metric when
// no component exists)
__global__ void k_metric_apply(const double* sums, const ProbDev* probs, int n_problems, int D,
                               double* minv) {
  const int prob = blockIdx.x * blockDim.x + threadIdx.x;
  if (prob >= n_problems || probs[prob].done) return;
  const double* v = sums + 5 * prob;
  for (int d = 0; d < 4; ++d) {
    double h = (d < D && v[4] > 0.0) ? v[d] / v[4] : 1.0;
    if (!(h > 1e-8)) h = 1e-8;
    minv[4 * prob + d] = 1.0 / h;
  }
}

// acceptance statistics of n_rounds rounds stored as [round][Ptot] rows, added round by
// round in the order of k_round_stats (one launch instead of one per round)
__global__ void k_round_stats_all(const double* acc, const int32_t* nleaf, const ProbDev* probs,
                                  int P, int64_t Ptot, int n_rounds, double* stats) {
  __shared__ double red[64];
  const int prob = blockIdx.x;
  if (probs[prob].done) return;
  for (int r = 0; r < n_rounds; ++r) {
    double v[2] = {0, 0};
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      const int64_t g = r * Ptot + (int64_t)prob * P + i;
      if (nleaf[g] > 0) { v[0] += acc[g]; v[1] += 1.0; }
    }
    block_sum<2>(v, red);
    if (threadIdx.x == 0) { stats[2 * prob] += v[0]; stats[2 * prob + 1] += v[1]; }
  }
}

// per-round acceptance statistics: stats[prob] += (sum acc over moved, count)
__global__ void k_round_stats(const double* acc, const int32_t* nleaf, const ProbDev* probs,
                              int P, double* stats) {
  __shared__ double red[64];
  const int prob = blockIdx.x;
  if (probs[prob].done) return;
  double v[2] = {0, 0};
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const int64_t g = (int64_t)prob * P + i;
    if (nleaf[g] > 0) { v[0] += acc[g]; v[1] += 1.0; }
  }
  block_sum<2>(v, red);
  if (threadIdx.x == 0) { stats[2 * prob] += v[0]; stats[2 * prob + 1] += v[1]; }
}

__global__ void k_eps_update(const ProbDev* probs, double* stats, double* eps, int n_problems) {
  const int prob = blockIdx.x * blockDim.x + threadIdx.x;
  if (prob >= n_problems) return;
  if (!probs[prob].done && stats[2 * prob + 1] > 0.0) {
    double e = eps[prob] * exp(stats[2 * prob] / stats[2 * prob + 1] - 0.8);
    e = e < 1e-4 ? 1e-4 : (e > 2.0 ? 2.0 : e);
    eps[prob] = e;
  }
  stats[2 * prob] = 0.0;
  stats[2 * prob + 1] = 0.0;
}

// ---------------------------------------------------------------------------
// Longest-first launch order: particle blocks sorted by cost K_p * N_b (bucketed,
// descending) so the largest blocks start first and the last wave is short.
// ---------------------------------------------------------------------------
constexpr int kOrderBuckets = 1024;

__device__ __forceinline__ int order_key(const int32_t* K, const ProbDev* probs, int64_t i, int P,
                                         int kmax, double nmax) {
  const int prob = (int)(i / P);
  const int k = min(max(K[i], 0), kmax);
  const double cost = (double)k * (double)probs[prob].n / ((double)kmax * nmax);  // in [0, 1]
  const int b = min(kOrderBuckets - 1, (int)(cost * (kOrderBuckets - 1) + 0.5));
  return kOrderBuckets - 1 - b;   // ascending key = descending cost
}

__global__ void k_order_count(const int32_t* K, const ProbDev* probs, int P, int kmax, double nmax,
                              int64_t Ptot, int32_t* hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Ptot) atomicAdd(&hist[order_key(K, probs, i, P, kmax, nmax)], 1);
}

__global__ void k_order_scan(int32_t* hist) {   // one block of kOrderBuckets threads
  __shared__ int32_t s[kOrderBuckets];
  const int t = threadIdx.x;
  s[t] = hist[t];
  __syncthreads();
  for (int o = 1; o < kOrderBuckets; o <<= 1) {
    const int32_t v = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  hist[t] = t == 0 ? 0 : s[t - 1];   // exclusive offsets
}

__global__ void k_order_scatter(const int32_t* K, const ProbDev* probs, int P, int kmax,
                                double nmax, int64_t Ptot, int32_t* offsets, int32_t* order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Ptot) {
    const int pos = atomicAdd(&offsets[order_key(K, probs, i, P, kmax, nmax)], 1);
    order[pos] = (int32_t)i;
  }
}

__global__ void k_set_int(int32_t* p, int v) { *p = v; }

__global__ void k_to_f32(const double* a, float* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_philox(const uint64_t* ctr, uint64_t k0, uint64_t k1, int64_t n,
                         uint64_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Rand4 r = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
  for (int j = 0; j < 4; ++j) out[4 * i + j] = r.w[j];
}

}  // namespace tsmc
