// likelihood.cuh -- batched residual, Gaussian log-likelihood and adjoint gradient.
//
// One thread block evaluates one particle: its K active components against the
// N samples of its problem.  Threads own R consecutive samples of a segment of
// blockDim*R samples; the residual of a segment lives in registers.
//
//   forward  r_n = d_n - sum_{k<K} h(t_n; theta_k)                (Sec. 5, time domain)
//            ll_old/ll_new = -1/2 sum r_n^2/sigma^2 over n<n1 / n>=n1
//   adjoint  dlogL_c/dtheta_kd = sum_n c_n r_n dh_k/dtheta_d / sigma^2, c_n = 1 or beta
//            (tempered bridges, Eqs. prior_bridge and reuse_bridge)
//
// FP64 path: every template value computed directly per sample in the order
// the definition states (phase ((2pi f) t + (pi fdot)(t t)) + phi0).
// Mixed path: FP32 templates and residuals.  Pulses use an exact FP32 anchor
// v0 = (t - t0) sqrt(log2 e / 2)/w per 8 samples (double-float product of the
// sample index) and the multiplicative recurrence g_{j+1} = g_j q_j,
// q_{j+1} = q_j rho (rho = 2^(-2 delta^2)); sinusoids use a double-float phase
// anchor per thread, reduced mod 2pi with a three-part Cody-Waite split of 2pi,
// then a rotation recurrence.  Mixed-path sums: FP32 over a thread's samples, a warp
// tree, per-warp Kahan rows across segments and double-float block totals; the FP64
// path sums in FP64 (blocked pairwise).
#pragma once
#include "common.cuh"

namespace tsmc {

// ---------------------------------------------------------------------------
// coordinate map (logit -> prior range) and log prior density of z
// ---------------------------------------------------------------------------
struct PriorArgs {
  int model;
  int window;       // mixed pulse path: skip (component, warp range) pairs beyond |v| > 7
  double amp_mean, amp_sd;
};

__device__ __forceinline__ void coord(const ProbDev& pb, const PriorArgs& pa, int d, double z,
                                      double& th, double& dth, double& lp, double& pg,
                                      double& pc) {
  if (pa.model == PULSE_LINAMP) {
    const double sd = pa.amp_sd, dz = (z - pa.amp_mean) / sd;
    th = z; dth = 1.0;
    lp = -0.5 * dz * dz - log(sd) - 0.5 * log(kTwoPi);
    pg = -(z - pa.amp_mean) / (sd * sd);
    pc = 1.0 / (sd * sd);
    return;
  }
  if (pb.wrapmask & (1u << d)) {   // periodic: theta = lo + span (z - floor z), flat prior
    const double span = __dadd_rn(pb.hi[d], -pb.lo[d]);
    th = __dadd_rn(pb.lo[d], __dmul_rn(span, __dadd_rn(z, -floor(z))));
    dth = span;
    lp = 0.0; pg = 0.0; pc = 0.0;
    return;
  }
  const double s = logistic(z);
  const double ds = __dmul_rn(s, __dadd_rn(1.0, -s));
  if (pb.logmask & (1u << d)) {
    const double span = __dadd_rn(pb.lhi[d], -pb.llo[d]);
    th = exp(__dadd_rn(pb.llo[d], __dmul_rn(span, s)));
    dth = __dmul_rn(__dmul_rn(th, span), ds);
  } else {
    const double span = __dadd_rn(pb.hi[d], -pb.lo[d]);
    th = __dadd_rn(pb.lo[d], __dmul_rn(span, s));
    dth = __dmul_rn(span, ds);
  }
  const double a = fabs(z);
  lp = -a - 2.0 * log1p(exp(-a));
  pg = 1.0 - 2.0 * s;
  pc = 2.0 * s * (1.0 - s);
}

// ---------------------------------------------------------------------------
// FP32 helpers (hand-written PTX for the SFU approximations)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sina(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cosa(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// a + m * delta with a = a_hi + a_lo, delta = d_hi + d_lo (double-float); the product
// m * d_hi is split exactly with an FMA, so the result carries the error of one FP32
// rounding of the final value only.
__device__ __forceinline__ float dd_axpy(float a_hi, float a_lo, float d_hi, float d_lo, float m) {
  const float p = __fmul_rn(m, d_hi);
  const float e = __fmaf_rn(m, d_hi, -p);
  const float s = __fadd_rn(a_hi, p);
  const float lo = __fmaf_rn(m, d_lo, a_lo);
  return __fadd_rn(s, __fadd_rn(e, lo));
}

// 2pi = C1 + C2 + C3 (each the FP32 rounding of the remainder)
constexpr float kC1 = 6.2831854820251465f;
constexpr float kC2 = -1.7484555314695172e-07f;
constexpr float kC3 = -6.8604980400235275e-15f;
constexpr float kInv2Pi = 0.15915493667125702f;

// ---------------------------------------------------------------------------
// Per-component FP32 constants of the mixed path (NCF floats per component)
// ---------------------------------------------------------------------------
constexpr int NCF = 12;
constexpr double kLog2E = 1.4426950408889634074;
constexpr double kCu = 1.1774100225154746910;   // sqrt(2 ln 2): u = v * kCu

// Support window of the mixed pulse path: a (component, warp range) pair is skipped when
// |v| > kSupportV on the whole range, i.e. |t - t0| > 6 widths, where every term is below
// 2^-26 A (under the FP32 resolution of the amplitude, and far under the ~50 eps32
// relative error of the template recurrence).
constexpr float kSupportV = 5.1f;   // 6 sqrt(log2(e) / 2) = 5.096

// pulse: v = (t - t0) kappa, kappa = sqrt(log2(e)/2)/w, g = 2^(-v^2)
__device__ __forceinline__ void pulse_prep(double A, double t0, double w, const ProbDev& pb,
                                           float* cf) {
  const double kap = sqrt(0.5 * kLog2E) / w;
  const double a0 = (pb.t_origin - t0) * kap;
  const double del = pb.dt * kap;
  const float a_hi = (float)a0, d_hi = (float)del;
  cf[0] = (float)A;
  cf[1] = a_hi;
  cf[2] = (float)(a0 - (double)a_hi);
  cf[3] = d_hi;
  cf[4] = (float)(del - (double)d_hi);
  cf[5] = (float)exp2(-2.0 * del * del);
  cf[6] = (float)(2.0 * del);
  cf[7] = (float)(del * del);
  cf[8] = del > 0.5 ? 1.0f : 0.0f;   // coarse grid: evaluate every sample directly
}

// sinusoid: phi(n) = phi_o + Om n + Gam n^2 with phi_o the phase at t_origin,
// Om = 2pi (f + fdot t_origin) dt, Gam = pi fdot dt^2
__device__ __forceinline__ void sin_prep(double A, double f, double fd, double p0,
                                         const ProbDev& pb, float* cf) {
  const double to = pb.t_origin;
  double phi = ((kTwoPi * f) * to + (kPi * fd) * (to * to)) + p0;
  phi = remainder(phi, kTwoPi);
  const double om = (kTwoPi * f + kTwoPi * fd * to) * pb.dt;
  const float om_hi = (float)om;
  cf[0] = (float)A;
  cf[1] = (float)phi;
  cf[2] = om_hi;
  cf[3] = (float)(om - (double)om_hi);
  cf[4] = (float)(kPi * fd * pb.dt * pb.dt);
  double so, co;
  sincos(om, &so, &co);
  cf[5] = (float)co;
  cf[6] = (float)so;
}

__device__ __forceinline__ void sin_anchor(const float* cf, float m, float& c, float& s) {
  const float p = __fmul_rn(m, cf[2]);
  const float e = __fmaf_rn(m, cf[2], -p);
  const float kq = rintf(__fmul_rn(p, kInv2Pi));
  float r = __fmaf_rn(-kq, kC1, p);
  r = __fmaf_rn(-kq, kC2, r);
  r = __fmaf_rn(-kq, kC3, r);
  const float extra = __fadd_rn(e, __fmaf_rn(m, cf[3], __fmul_rn(cf[4], __fmul_rn(m, m))));
  r = __fadd_rn(__fadd_rn(r, extra), cf[1]);
  const float k2 = rintf(__fmul_rn(r, kInv2Pi));
  r = __fmaf_rn(-k2, kC1, r);
  r = __fmaf_rn(-k2, kC2, r);
  c = cosa(r);
  s = sina(r);
}

// template values of one component on the thread's R samples starting at index m
template <int MODEL, int R>
__device__ __forceinline__ void mixed_vals(const float* cf, float m, float (&h)[R]) {
  if (MODEL == SINUSOID) {
    float c, s;
    sin_anchor(cf, m, c, s);
    const float A = cf[0], rc = cf[5], rs = cf[6];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      h[j] = A * c;
      const float c2 = __fmaf_rn(c, rc, -s * rs);
      s = __fmaf_rn(s, rc, c * rs);
      c = c2;
    }
  } else {
    const float A = cf[0];
    const float v00 = dd_axpy(cf[1], cf[2], cf[3], cf[4], m);
    if (cf[8] != 0.0f) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float v = __fmaf_rn((float)j, cf[3], v00);
        h[j] = A * ex2a(-v * v);
      }
    } else {
#pragma unroll
      for (int c8 = 0; c8 < R / 8; ++c8) {
        const float v0 = __fmaf_rn((float)(8 * c8), cf[3], v00);
        float g = ex2a(-v0 * v0);
        float q = ex2a(fminf(-__fmaf_rn(v0, cf[6], cf[7]), 64.0f));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          h[8 * c8 + j] = A * g;
          g *= q;
          q *= cf[5];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Packed sample registers of the mixed likelihood loop.  A thread's R residuals
// are R/2 float2 pairs so that one packed FP32 instruction (FFMA2 / FMUL2 /
// FADD2 of the sm_100 family) advances two independent recurrences per issue
// slot.  Pair i, half h holds local sample pair_sample(i, h):
//   pulse:    (j, j + 8) inside each run of 16 samples: the two halves are two
//             8-sample chunks with their own anchors, stepped in lockstep; every
//             element sees exactly the operations of the scalar recurrence
//   sinusoid: (i, i + R/2): two rotation chains, each with its own phase anchor
// ---------------------------------------------------------------------------
template <int MODEL, int R>
__host__ __device__ constexpr int pair_sample(int i, int h) {
  return MODEL == SINUSOID ? i + h * (R / 2) : ((i >> 3) << 4) + (h << 3) + (i & 7);
}
template <int MODEL, int R>
__host__ __device__ constexpr int sample_pair(int s) {
  return MODEL == SINUSOID ? s % (R / 2) : ((s >> 4) << 3) + (s & 7);
}
template <int MODEL, int R>
__host__ __device__ constexpr int sample_half(int s) {
  return MODEL == SINUSOID ? s / (R / 2) : (s >> 3) & 1;
}
template <int MODEL, int R>
__device__ __forceinline__ float& slot(float2 (&r)[R / 2], int s) {
  return sample_half<MODEL, R>(s) ? r[sample_pair<MODEL, R>(s)].y
                                  : r[sample_pair<MODEL, R>(s)].x;
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// r -= h(t_{m+s}) for C components on the thread's R samples (packed pairs).
// Sinusoids take C = 2: the two components' rotation recurrences are interleaved
// for instruction-level parallelism, and every residual element still receives the
// first component's update before the second's (the order of two single calls).
// Pulses take C = 1 (the pulse kernels are issue-bound already).
template <int MODEL, int R, int C>
__device__ __forceinline__ void mixed_sub(const float (&cf)[C][NCF], float m, float2 (&r)[R / 2]) {
  static_assert(R % 16 == 0, "packed pulse chunks need R a multiple of 16");
  if constexpr (MODEL == SINUSOID) {
    float2 c[C], s[C], nA[C], rc[C], rs[C], nrs[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
      sin_anchor(cf[u], m, c[u].x, s[u].x);
      sin_anchor(cf[u], m + (float)(R / 2), c[u].y, s[u].y);
      nA[u] = f2(-cf[u][0]); rc[u] = f2(cf[u][5]); rs[u] = f2(cf[u][6]); nrs[u] = f2(-cf[u][6]);
    }
#pragma unroll
    for (int j = 0; j < R / 2; ++j) {
#pragma unroll
      for (int u = 0; u < C; ++u) r[j] = __ffma2_rn(nA[u], c[u], r[j]);
#pragma unroll
      for (int u = 0; u < C; ++u) {
        const float2 c2 = __ffma2_rn(c[u], rc[u], __fmul2_rn(s[u], nrs[u]));
        s[u] = __ffma2_rn(s[u], rc[u], __fmul2_rn(c[u], rs[u]));
        c[u] = c2;
      }
    }
  } else {
    static_assert(C == 1, "pulse components one at a time");
    const bool coarse = cf[0][8] != 0.0f;
    float2 nA[C], del[C], rho[C], v00[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
      nA[u] = f2(-cf[u][0]); del[u] = f2(cf[u][3]); rho[u] = f2(cf[u][5]);
      v00[u] = f2(dd_axpy(cf[u][1], cf[u][2], cf[u][3], cf[u][4], m));
    }
    if (coarse) {   // C == 1: direct evaluation of every sample
#pragma unroll
      for (int i = 0; i < R / 2; ++i) {
        const float2 v = __ffma2_rn(make_float2((float)pair_sample<MODEL, R>(i, 0),
                                                (float)pair_sample<MODEL, R>(i, 1)), del[0], v00[0]);
        r[i] = __ffma2_rn(nA[0], make_float2(ex2a(-v.x * v.x), ex2a(-v.y * v.y)), r[i]);
      }
      return;
    }
#pragma unroll
    for (int p = 0; p < R / 16; ++p) {
      float2 g[C], q[C];
#pragma unroll
      for (int u = 0; u < C; ++u) {
        const float2 v0 = __ffma2_rn(make_float2((float)(16 * p), (float)(16 * p + 8)), del[u],
                                     v00[u]);
        const float2 sq = __fmul2_rn(v0, v0);
        const float2 qa = __ffma2_rn(v0, f2(cf[u][6]), f2(cf[u][7]));
        g[u] = make_float2(ex2a(-sq.x), ex2a(-sq.y));
        q[u] = make_float2(ex2a(fminf(-qa.x, 64.0f)), ex2a(fminf(-qa.y, 64.0f)));
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int u = 0; u < C; ++u) r[8 * p + j] = __ffma2_rn(nA[u], g[u], r[8 * p + j]);
#pragma unroll
        for (int u = 0; u < C; ++u) {
          g[u] = __fmul2_rn(g[u], q[u]);
          q[u] = __fmul2_rn(q[u], rho[u]);
        }
      }
    }
  }
}

// adjoint partial sums of C components over the thread's samples
// (rc = c_n r_n / sigma^2, packed pairs as above); C as in mixed_sub
//   pulse:    s0 = sum rc g, s1 = sum rc g v, s2 = sum rc g v^2 (per 8-sample chunk from
//             running sums, combined with the chunk's end point)
//   sinusoid: s0 = sum rc cos, s1 = sum rc sin, s2 = sum rc sin n, s3 = sum rc sin n^2
template <int MODEL, int R, int C>
__device__ __forceinline__ void mixed_adj(const float (&cf)[C][NCF], float m,
                                          const float2 (&rc)[R / 2], float (&o)[C][4]) {
  if constexpr (MODEL == SINUSOID) {
    const float mh = m + (float)(R / 2);
    float2 c[C], s[C], rcs[C], rsn[C], nrsn[C], sc[C], u0[C], u1[C], u2[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
      sin_anchor(cf[u], m, c[u].x, s[u].x);
      sin_anchor(cf[u], mh, c[u].y, s[u].y);
      rcs[u] = f2(cf[u][5]); rsn[u] = f2(cf[u][6]); nrsn[u] = f2(-cf[u][6]);
      sc[u] = u0[u] = u1[u] = u2[u] = f2(0.f);
    }
#pragma unroll
    for (int j = 0; j < R / 2; ++j) {
#pragma unroll
      for (int u = 0; u < C; ++u) {
        sc[u] = __ffma2_rn(rc[j], c[u], sc[u]);
        const float2 p = __fmul2_rn(rc[j], s[u]);
        u0[u] = __fadd2_rn(u0[u], p);
        u1[u] = __ffma2_rn(p, f2((float)j), u1[u]);
        u2[u] = __ffma2_rn(p, f2((float)(j * j)), u2[u]);
        const float2 c2 = __ffma2_rn(c[u], rcs[u], __fmul2_rn(s[u], nrsn[u]));
        s[u] = __ffma2_rn(s[u], rcs[u], __fmul2_rn(c[u], rsn[u]));
        c[u] = c2;
      }
    }
#pragma unroll
    for (int u = 0; u < C; ++u) {
      o[u][0] = sc[u].x + sc[u].y;
      o[u][1] = u0[u].x + u0[u].y;
      o[u][2] = __fmaf_rn(m, u0[u].x, u1[u].x) + __fmaf_rn(mh, u0[u].y, u1[u].y);
      o[u][3] = __fmaf_rn(m, __fmaf_rn(m, u0[u].x, 2.0f * u1[u].x), u2[u].x) +
                __fmaf_rn(mh, __fmaf_rn(mh, u0[u].y, 2.0f * u1[u].y), u2[u].y);
    }
  } else {
    static_assert(C == 1, "pulse components one at a time");
    const bool coarse = cf[0][8] != 0.0f;
    float2 del[C], rho[C], v00[C];
    float2 s0[C], s1[C], s2[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
      del[u] = f2(cf[u][3]); rho[u] = f2(cf[u][5]);
      v00[u] = f2(dd_axpy(cf[u][1], cf[u][2], cf[u][3], cf[u][4], m));
      s0[u] = s1[u] = s2[u] = f2(0.f);
    }
    if (coarse) {   // C == 1
      float2 a0 = f2(0.f), a1 = f2(0.f), a2 = f2(0.f);
#pragma unroll
      for (int i = 0; i < R / 2; ++i) {
        const float2 v = __ffma2_rn(make_float2((float)pair_sample<MODEL, R>(i, 0),
                                                (float)pair_sample<MODEL, R>(i, 1)), del[0], v00[0]);
        const float2 p = __fmul2_rn(rc[i], make_float2(ex2a(-v.x * v.x), ex2a(-v.y * v.y)));
        a0 = __fadd2_rn(a0, p);
        a1 = __ffma2_rn(p, v, a1);
        a2 = __ffma2_rn(__fmul2_rn(p, v), v, a2);
      }
      o[0][0] = a0.x + a0.y; o[0][1] = a1.x + a1.y; o[0][2] = a2.x + a2.y; o[0][3] = 0.f;
      return;
    }
    const float2 ndel = f2(-cf[0][3]), del2 = f2(cf[0][7]);
#pragma unroll
    for (int p = 0; p < R / 16; ++p) {
      float2 v0[C], g[C], q[C], c[C], e[C], fs[C];
#pragma unroll
      for (int u = 0; u < C; ++u) {
        v0[u] = __ffma2_rn(make_float2((float)(16 * p), (float)(16 * p + 8)), del[u], v00[u]);
        const float2 sq = __fmul2_rn(v0[u], v0[u]);
        const float2 qa = __ffma2_rn(v0[u], f2(cf[u][6]), f2(cf[u][7]));
        g[u] = make_float2(ex2a(-sq.x), ex2a(-sq.y));
        q[u] = make_float2(ex2a(fminf(-qa.x, 64.0f)), ex2a(fminf(-qa.y, 64.0f)));
      }
      // running sums over the chunk with p_j = rc_j g_j: c_k = sum_{j<=k} p_j,
      // e_k = sum_{m<=k} c_m, f_k = sum_{m<=k} e_m, so that at its end c = sum p,
      // e = sum (8 - j) p and f = sum (8 - j)(9 - j)/2 p (five packed operations per step
      // and no per-step constants)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int u = 0; u < C; ++u) {
          if (j == 0) {
            c[u] = __fmul2_rn(rc[8 * p], g[u]);
            e[u] = c[u];
            fs[u] = c[u];
          } else {
            c[u] = __ffma2_rn(rc[8 * p + j], g[u], c[u]);
            e[u] = __fadd2_rn(e[u], c[u]);
            fs[u] = __fadd2_rn(fs[u], e[u]);
          }
          g[u] = __fmul2_rn(g[u], q[u]);
          q[u] = __fmul2_rn(q[u], rho[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < C; ++u) {
        // with w = 8 - j and V = v0 + 8 del (v one past the chunk): v = V - del w, so
        // sum p v = V c - del e;  sum p v^2 = V (V c - 2 del e) + del^2 (2 f - e), with
        // V c - 2 del e formed as (sum p v) - del e; the chunk sums are kept per half of
        // the packed pair and the two halves added at the end
        const float2 V = __ffma2_rn(f2(8.0f), del[u], v0[u]);
        const float2 ne = __fmul2_rn(ndel, e[u]);
        const float2 c1 = __ffma2_rn(V, c[u], ne);
        const float2 w2 = __ffma2_rn(f2(2.0f), fs[u], make_float2(-e[u].x, -e[u].y));
        const float2 c2 = __ffma2_rn(V, __fadd2_rn(c1, ne), __fmul2_rn(del2, w2));
        s0[u] = __fadd2_rn(s0[u], c[u]);
        s1[u] = __fadd2_rn(s1[u], c1);
        s2[u] = __fadd2_rn(s2[u], c2);
      }
    }
#pragma unroll
    for (int u = 0; u < C; ++u) {
      o[u][0] = s0[u].x + s0[u].y; o[u][1] = s1[u].x + s1[u].y; o[u][2] = s2[u].x + s2[u].y;
      o[u][3] = 0.f;
    }
  }
}

// Gauss-Newton partial sums (metric only): cw = c_n / sigma^2 (0 for padding)
//   pulse: (sum cw g^2, sum cw g^2 v^2, sum cw g^2 v^4); sinusoid: (sum cw cos^2,
//   sum cw sin^2 t^2, sum cw sin^2 t^4, sum cw sin^2) with t in FP32
template <int MODEL, int R>
__device__ __forceinline__ void mixed_fis(const float* cf, float m, const float (&cw)[R],
                                          float t_o, float dt, float (&o)[4]) {
  o[0] = o[1] = o[2] = o[3] = 0.f;
  if (MODEL == SINUSOID) {
    float c, s;
    sin_anchor(cf, m, c, s);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float t = __fmaf_rn(m + (float)j, dt, t_o);
      const float s2 = cw[j] * s * s, t2 = t * t;
      o[0] = __fmaf_rn(cw[j] * c, c, o[0]);
      o[1] = __fmaf_rn(s2, t2, o[1]);
      o[2] = __fmaf_rn(s2 * t2, t2, o[2]);
      o[3] += s2;
      const float c2 = __fmaf_rn(c, cf[5], -s * cf[6]);
      s = __fmaf_rn(s, cf[5], c * cf[6]);
      c = c2;
    }
  } else {
    const float v00 = dd_axpy(cf[1], cf[2], cf[3], cf[4], m);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float v = __fmaf_rn((float)j, cf[3], v00);
      const float g = ex2a(-v * v);
      const float a = cw[j] * g * g, v2 = v * v;
      o[0] += a;
      o[1] = __fmaf_rn(a, v2, o[1]);
      o[2] = __fmaf_rn(a * v2, v2, o[2]);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 templates (direct, in the defining order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double time_of(const ProbDev& pb, int64_t n) {
  return __dadd_rn(pb.t_origin, __dmul_rn((double)n, pb.dt));
}

template <int MODEL>
__device__ __forceinline__ double fp64_val(const double* th, double tw0, double tw1, double t,
                                           double* dh) {
  if (MODEL == SINUSOID) {
    const double A = th[0], f = th[1], fd = th[2], p0 = th[3];
    const double phi = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(kTwoPi, f), t),
                                           __dmul_rn(__dmul_rn(kPi, fd), __dmul_rn(t, t))),
                                 p0);
    double sph, cph;
    sincos(phi, &sph, &cph);
    if (dh) {
      const double mas = __dmul_rn(-A, sph);
      dh[0] = cph;
      dh[1] = __dmul_rn(mas, __dmul_rn(kTwoPi, t));
      dh[2] = __dmul_rn(mas, __dmul_rn(kPi, __dmul_rn(t, t)));
      dh[3] = mas;
    }
    return __dmul_rn(A, cph);
  } else {
    const double A = th[0];
    const double t0 = MODEL == PULSE ? th[1] : tw0;
    const double w = MODEL == PULSE ? th[2] : tw1;
    const double u = __ddiv_rn(__dadd_rn(t, -t0), w);
    const double g = exp(__dmul_rn(__dmul_rn(-0.5, u), u));
    if (dh) {
      dh[0] = g;
      if (MODEL == PULSE) {
        const double ag = __dmul_rn(A, g);
        dh[1] = __ddiv_rn(__dmul_rn(ag, u), w);
        dh[2] = __ddiv_rn(__dmul_rn(__dmul_rn(ag, u), u), w);
      }
    }
    return __dmul_rn(A, g);
  }
}

template <int MODEL>
__host__ __device__ constexpr int model_d() { return MODEL == SINUSOID ? 4 : (MODEL == PULSE ? 3 : 1); }

// ---------------------------------------------------------------------------
// Shared-memory scratch of one block evaluation
// ---------------------------------------------------------------------------
struct EvalSmem {
  double* th;     // [KDmax] theta
  double* dth;    // [KDmax] dtheta/dz
  double* pg;     // [KDmax] prior gradient
  double* pc;     // [KDmax] prior curvature
  float* cf;      // [channels][kmax][NCF] mixed-path constants
  int cfch;       // floats between the constant sets of two channels
  double* wacc;   // [nwarps][KDmax] per-warp gradient slot sums
  double* wfis;   // [nwarps][KDmax] per-warp Gauss-Newton slot sums
  double* red;    // [32*4] reduction scratch
  double* scal;   // [8]: logp, ll_old, ll_new, component*samples computed; [4..7] see scalf
  const double* tw;  // LINAMP fixed (t0, w) [kmax][2] (global)
  float2* exptab;    // mixed path: 2^(j/64), j < 64, as double-float (filled per block)
  // mixed path: FP32 views of the same storage
  __device__ float* fth() const { return reinterpret_cast<float*>(th); }
  __device__ float* fdth() const { return reinterpret_cast<float*>(dth); }
  __device__ float* fpg() const { return reinterpret_cast<float*>(pg); }
  __device__ float* fpc() const { return reinterpret_cast<float*>(pc); }
  __device__ float2* wacc2() const { return reinterpret_cast<float2*>(wacc); }
  __device__ float2* wfis2() const { return reinterpret_cast<float2*>(wfis); }
  // double-float totals of the mixed NUTS evaluation (scal[4..7]): logp, ll_old, ll_new as
  // hi/lo pairs, then the component*samples computed as an int
  __device__ float* scalf() const { return reinterpret_cast<float*>(scal + 4); }
  __device__ int* scalc() const { return reinterpret_cast<int*>(scal + 4) + 6; }
};

// ---------------------------------------------------------------------------
// double-float (hi + lo) arithmetic in FP32: error-free TwoSum (Knuth)
// ---------------------------------------------------------------------------
struct DF { float hi, lo; };

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s.hi, e);
  return DF{h, __fsub_rn(e, __fsub_rn(h, s.hi))};
}

__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

__device__ __forceinline__ double df_to_double(DF v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ DF df_from(float2 v) { return DF{v.x, v.y}; }

__device__ __forceinline__ DF quick_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return quick_two_sum(p, e);
}

__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
  return quick_two_sum(p, e);
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// fractional part of a double-float coordinate, in [0, 1); a non-finite coordinate gives 0
// (an FP64 coordinate beyond 2^52 has no fractional part either)
__device__ __forceinline__ DF df_frac(DF z) {
  if (!isfinite(z.hi)) return DF{0.f, 0.f};
  DF f = two_sum(z.hi - floorf(z.hi), z.lo);   // the first difference is exact
  if (f.hi < 0.f) f = df_add(f, DF{1.f, 0.f});
  else if (f.hi >= 1.f) f = df_add(f, DF{-1.f, 0.f});
  return f;
}

// 1 / a (a > 0): FP32 reciprocal refined by one Newton step in double-float
__device__ __forceinline__ DF df_recip(DF a) {
  const float q = __frcp_rn(a.hi);
  // residual 1 - a q, exact for the hi part by FMA
  const float r = __fsub_rn(__fmaf_rn(-a.hi, q, 1.0f), __fmul_rn(a.lo, q));
  return quick_two_sum(q, __fmul_rn(q, r));
}

// 2^(j/64), j < 64, as double-float, into shared memory (threads 0..63 of the block)
__device__ __forceinline__ void fill_exp_table(float2* tab) {
  if (threadIdx.x < 64) {
    const double v = exp2((double)threadIdx.x / 64.0);
    const float hi = (float)v;
    tab[threadIdx.x] = make_float2(hi, (float)(v - (double)hi));
  }
}

// per-block tables of the mixed path, at kernel start (before the first __syncthreads):
// the 2^(j/64) table and cleared active-component masks (every evaluation leaves them
// cleared again)
__device__ __forceinline__ void init_block_tables(EvalSmem& sm) {
  fill_exp_table(sm.exptab);
}

// e^x as double-float for x in [-80, 80], FP32 arithmetic only (table-driven method of
// Tang, ACM TOMS 15(2), 1989): x = n ln2/64 + r with n integer and |r| <= ln2/128,
// e^x = 2^(n div 64) 2^((n mod 64)/64) e^r, e^r from its Taylor series to r^5.
// Relative error ~1e-12.
__device__ __forceinline__ DF df_exp(DF x, const float2* tab) {
  if (x.hi < -80.0f) x = DF{-80.0f, 0.0f};     // e^-80 ~ 1.8e-35: below every use here
  if (x.hi > 80.0f) x = DF{80.0f, 0.0f};
  const float n = rintf(__fmul_rn(x.hi, 92.3324813842773438f));   // 64 / ln 2 (FP32)
  // ln2/64 = L1 + L2 + L3, L1 with 11 significant bits so n * L1 is exact for |n| < 2^13
  constexpr float L1 = 0.01082611083984375f;               // 0x1.62cp-7
  constexpr float L2 = 4.313856607041089e-06f;
  constexpr float L3 = -2.0164562565278682e-13f;
  const float r1 = __fmaf_rn(-n, L1, x.hi);                // exact
  const float p2 = __fmul_rn(n, L2);
  DF r = two_sum(r1, -p2);
  r.lo = __fadd_rn(r.lo, __fsub_rn(x.lo, __fmaf_rn(n, L2, -p2)));
  r.lo = __fsub_rn(r.lo, __fmul_rn(n, L3));
  r = quick_two_sum(r.hi, r.lo);
  const float rh = r.hi;
  // e^r - 1 = r + r^2 (1/2 + r (1/6 + r (1/24 + r / 120)))
  float q = __fmaf_rn(rh, 1.0f / 120.0f, 1.0f / 24.0f);
  q = __fmaf_rn(rh, q, 1.0f / 6.0f);
  q = __fmaf_rn(rh, q, 0.5f);
  q = __fmul_rn(__fmul_rn(rh, rh), q);
  DF em1 = df_add(r, DF{q, 0.0f});
  DF er = df_add(DF{1.0f, 0.0f}, em1);
  const int ni = (int)n;
  const int j = ni & 63;
  const int k = (ni - j) / 64;   // floor division (ni - j is a multiple of 64)
  DF v = df_mul(df_from(tab[j]), er);
  return DF{ldexpf(v.hi, k), ldexpf(v.lo, k)};
}

// theta of parameter d from an FP64 coordinate, as double-float (uniform or log-uniform
// map), with s(z) and 1 - s(z) both from e^{-|z|}; also returns dtheta/dz in FP32
struct Coord32 { float th, dth, lp, pg, pc; };

// theta in double-float from a double-float coordinate z; with pr != nullptr also the log
// prior density of z and its first two derivatives (lp, pg, pc of Coord32) from the same
// e^{-|z|} and 1/(1+e)
template <bool WRAP = true>
__device__ __forceinline__ DF theta_df(const ProbDev& pb, int d, DF z, const float2* tab,
                                       float& dth, Coord32* pr = nullptr) {
  if constexpr (WRAP) {
    if (pb.wrapmask & (1u << d)) {   // periodic, flat prior
      if (pr) { pr->lp = 0.f; pr->pg = 0.f; pr->pc = 0.f; }
      const DF span = df_from(pb.f_span[d]);
      dth = span.hi;
      return df_add(df_from(pb.f_off[d]), df_mul(span, df_frac(z)));
    }
  }
  const bool pos = z.hi >= 0.f;
  const DF az = pos ? z : df_neg(z);
  const DF e = df_exp(df_neg(az), tab);              // e^{-|z|}
  const DF q = df_recip(df_add(DF{1.0f, 0.0f}, e));  // 1 / (1 + e)
  const DF eq = df_mul(e, q);
  const DF s = pos ? q : eq;                         // s(z)
  const float ds = __fmul_rn(q.hi, eq.hi);           // s (1 - s)
  if (pr) {
    // 1 - 2 s = -+(1 - e) q: 1 - e in double-float keeps the prior gradient's relative
    // precision near z = 0, where (1 - s) - s would cancel to an absolute FP32 error
    const float om = df_add(DF{1.0f, 0.0f}, df_neg(e)).hi;
    pr->lp = -az.hi - 2.f * log1pf(e.hi);
    pr->pg = (pos ? -om : om) * q.hi;
    pr->pc = 2.f * ds;
  }
  const DF span = df_from(pb.f_span[d]);
  DF th = df_add(df_from(pb.f_off[d]), df_mul(span, s));
  if (pb.logmask & (1u << d)) {
    th = df_exp(th, tab);
    dth = th.hi * span.hi * ds;
  } else {
    dth = span.hi * ds;
  }
  return th;
}

template <int MODEL>
__device__ __forceinline__ void finish_component(int prec, const double* th, const double* S,
                                                 const ProbDev& pb, double* g) {
  // S: slot sums (already scaled by 1/sigma^2 and c_n); g: dlogL/dtheta
  if (prec == FP64) {
    for (int d = 0; d < model_d<MODEL>(); ++d) g[d] = S[d];
    return;
  }
  if (MODEL == SINUSOID) {
    const double A = th[0], to = pb.t_origin, dt = pb.dt;
    g[0] = S[0];
    g[1] = -A * kTwoPi * (to * S[1] + dt * S[2]);
    g[2] = -A * kPi * (to * to * S[1] + 2.0 * to * dt * S[2] + dt * dt * S[3]);
    g[3] = -A * S[1];
  } else if (MODEL == PULSE) {
    const double aw = th[0] / th[2];
    g[0] = S[0];
    g[1] = aw * kCu * S[1];
    g[2] = aw * kCu * kCu * S[2];
  } else {
    g[0] = S[0];
  }
}

template <int MODEL>
__device__ __forceinline__ void finish_fisher(int prec, const double* th, const double* F,
                                              double* f) {
  if (prec == FP64) {
    for (int d = 0; d < model_d<MODEL>(); ++d) f[d] = F[d];
    return;
  }
  if (MODEL == SINUSOID) {
    const double A2 = th[0] * th[0];
    f[0] = F[0];
    f[1] = A2 * kTwoPi * kTwoPi * F[1];
    f[2] = A2 * kPi * kPi * F[2];
    f[3] = A2 * F[3];
  } else if (MODEL == PULSE) {
    const double aw = th[0] / th[2];
    f[0] = F[0];
    f[1] = aw * aw * kCu * kCu * F[1];
    f[2] = aw * aw * kCu * kCu * kCu * kCu * F[2];
  } else {
    f[0] = F[0];
  }
}

// ---------------------------------------------------------------------------
// FP32 coordinate map (mixed path; parameters whose FP32 rounding stays far
// below the path's tolerance: amplitudes, widths, frequency derivative, phase)
// ---------------------------------------------------------------------------

// WRAP = false: the problem has no periodic parameter (the branch is compiled out)
template <bool WRAP = true>
__device__ __forceinline__ Coord32 coord32(const ProbDev& pb, const PriorArgs& pa, int d, DF zz) {
  const float z = zz.hi;
  Coord32 c;
  if constexpr (WRAP) {
    if (pa.model != PULSE_LINAMP && (pb.wrapmask & (1u << d))) {   // periodic, flat prior
      const DF f = df_frac(zz);
      c.th = pb.f_off[d].x + pb.f_span[d].x * (f.hi + f.lo);
      c.dth = pb.f_span[d].x;
      c.lp = 0.f; c.pg = 0.f; c.pc = 0.f;
      return c;
    }
  }
  if (pa.model == PULSE_LINAMP) {
    const float sd = (float)pa.amp_sd, dz = (z - (float)pa.amp_mean) / sd;
    c.th = z; c.dth = 1.f;
    c.lp = -0.5f * dz * dz - logf(sd) - 0.918938533204673f;
    c.pg = -dz / sd;
    c.pc = 1.f / (sd * sd);
    return c;
  }
  // s and 1 - s both from e^{-|z|}: s (1 - s) keeps full FP32 relative precision at
  // large |z|, where forming 1 - s by subtraction would cancel
  const float a = fabsf(z);
  const float e = expf(-a);
  const float om = -expm1f(-a);      // 1 - e, no cancellation near z = 0
  const float q = 1.f / (1.f + e);
  const float s = z >= 0.f ? q : e * q;
  const float sc = z >= 0.f ? e * q : q;
  const float ds = s * sc;
  const float off = pb.f_off[d].x, span = pb.f_span[d].x;   // FP32 roundings of the bounds
  if (pb.logmask & (1u << d)) {
    c.th = expf(off + span * s);
    c.dth = c.th * span * ds;
  } else {
    c.th = off + span * s;
    c.dth = span * ds;
  }
  c.lp = -a - 2.f * log1pf(e);
  c.pg = (z >= 0.f ? -om : om) * q;   // 1 - 2 s with full relative precision
  c.pc = 2.f * ds;
  return c;
}

// theta and dtheta/dz in FP64 for the parameters that set where a template sits
// (pulse centre and width, sinusoid frequency): their FP32 rounding, or the FP32
// rounding of the log-space argument of a log-uniform map, would move the template
// by more than the path's tolerance (tails of narrow pulses, far end of the grid).
template <bool WRAP = true>
__device__ __forceinline__ double theta64(const ProbDev& pb, int d, double z, double& dth) {
  if constexpr (WRAP) {
    if (pb.wrapmask & (1u << d)) {
      const double span = pb.hi[d] - pb.lo[d];
      dth = span;
      return pb.lo[d] + span * (z - floor(z));
    }
  }
  const double e = exp(-fabs(z));
  const double q = 1.0 / (1.0 + e);
  const double s = z >= 0.0 ? q : e * q;
  const double ds = s * (z >= 0.0 ? e * q : q);
  if (pb.logmask & (1u << d)) {
    const double span = pb.lhi[d] - pb.llo[d];
    const double th = exp(pb.llo[d] + span * s);
    dth = th * span * ds;
    return th;
  }
  const double span = pb.hi[d] - pb.lo[d];
  dth = span * ds;
  return pb.lo[d] + span * s;
}

// pulse constants from the FP64 centre and width: kappa rounded once to FP32 and used
// for both a0 and delta, so v = (t - t0) kappa keeps its relative precision
__device__ __forceinline__ void pulse_prep32(float A, double t0, double w, const ProbDev& pb,
                                             float* cf) {
  const float kap = __fdiv_rn(0.849321800288019f, (float)w);    // sqrt(log2(e)/2) / w
  const double a0 = (pb.t_origin - t0) * (double)kap;
  const double del = pb.dt * (double)kap;
  const float a_hi = (float)a0, d_hi = (float)del;
  cf[0] = A;
  cf[1] = a_hi;
  cf[2] = (float)(a0 - (double)a_hi);
  cf[3] = d_hi;
  cf[4] = (float)(del - (double)d_hi);
  cf[5] = exp2f(-2.f * d_hi * d_hi);
  cf[6] = 2.f * d_hi;
  cf[7] = d_hi * d_hi;
  cf[8] = del > 0.5 ? 1.0f : 0.0f;   // coarse grid: evaluate every sample directly
  // support in sample index: |v| <= kSupportV; a0 + n del = v
  const float idel = __frcp_rn(d_hi);
  cf[9] = fmaxf(floorf((-kSupportV - a_hi) * idel) - 2.0f, -1.0e30f);
  cf[10] = fminf(ceilf((kSupportV - a_hi) * idel) + 2.0f, 1.0e30f);
}

// warp-uniform: the component has no term above 2^-26 A on samples [first, last]
// (sample indices as FP32, exact below 2^24; converted once per segment)
__device__ __forceinline__ bool outside_support(const float* cf, float first, float last) {
  return last < cf[9] || first > cf[10];
}

__device__ __forceinline__ void pulse_prep_df(float A, DF t0, float w, const ProbDev& pb,
                                              float* cf) {
  const float kap = __fdiv_rn(0.849321800288019f, w);    // sqrt(log2(e)/2) / w
  const DF a0 = df_mul_f(df_add(df_from(pb.f_to), df_neg(t0)), kap);
  const DF del = df_mul_f(df_from(pb.f_dt), kap);
  cf[0] = A;
  cf[1] = a0.hi;
  cf[2] = a0.lo;
  cf[3] = del.hi;
  cf[4] = del.lo;
  cf[5] = exp2f(-2.f * del.hi * del.hi);
  cf[6] = 2.f * del.hi;
  cf[7] = del.hi * del.hi;
  cf[8] = del.hi > 0.5f ? 1.0f : 0.0f;
  const float idel = __frcp_rn(del.hi);
  cf[9] = fmaxf(floorf((-kSupportV - a0.hi) * idel) - 2.0f, -1.0e30f);
  cf[10] = fminf(ceilf((kSupportV - a0.hi) * idel) + 2.0f, 1.0e30f);
}

__device__ __forceinline__ void sin_prep32(float A, double f, float fd, float p0,
                                           const ProbDev& pb, float* cf) {
  const double to = pb.t_origin;
  float phi = p0;
  if (to != 0.0) {
    double ph = ((kTwoPi * f) * to + (kPi * (double)fd) * (to * to)) + (double)p0;
    phi = (float)remainder(ph, kTwoPi);
  }
  const double om = (kTwoPi * f + kTwoPi * (double)fd * to) * pb.dt;
  const float om_hi = (float)om;
  cf[0] = A;
  cf[1] = phi;
  cf[2] = om_hi;
  cf[3] = (float)(om - (double)om_hi);
  cf[4] = (float)(kPi * (double)fd * pb.dt * pb.dt);
  float so, co;
  sincosf(om_hi, &so, &co);
  cf[5] = co;
  cf[6] = so;
}

// ---------------------------------------------------------------------------
// Per-component setup: theta, Jacobians, prior terms and path constants.
// Must be called by all threads; ends with __syncthreads.  Returns the thread's
// share of the log prior (summed by the caller's block reduction).
// ---------------------------------------------------------------------------
template <int MODEL, int PREC>
__device__ double eval_setup_any(const ProbDev& pb, const PriorArgs& pa, int K, const double* z,
                                 EvalSmem& sm) {
  constexpr int D = model_d<MODEL>();
  double lp_sum = 0.0;
  for (int i = threadIdx.x; i < K * D; i += blockDim.x) {
    double th, dth, lp, pg, pc;
    coord(pb, pa, i % D, z[i], th, dth, lp, pg, pc);
    sm.th[i] = th; sm.dth[i] = dth; sm.pg[i] = pg; sm.pc[i] = pc;
    lp_sum += lp;
  }
  __syncthreads();
  return lp_sum;
}

// Kahan step in FP32 (explicit rounding: no reassociation or contraction)
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Warp totals of o[0..3], one value per group of 8 lanes: on return lane l holds the
// total of o[l >> 3].  Each total uses the pairing of the butterfly tree (offsets 16,
// 8, 4, 2, 1), so it equals warp_sum(o[v]) bit for bit, in 6 shuffles instead of 20.
__device__ __forceinline__ float warp_sum4_split(const float (&o)[4], int lane) {
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
  float k0 = b4 ? o[2] : o[0];
  float k1 = b4 ? o[3] : o[1];
  const float s0 = b4 ? o[0] : o[2];
  const float s1 = b4 ? o[1] : o[3];
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  float k = b3 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, b3 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// adds the warp totals of o[0..D-1] for component k to the warp's shared Kahan row
// acc[k*D + d] = (sum, compensation)
template <int D>
__device__ __forceinline__ void warp_accumulate(const float (&o)[4], int lane, int k,
                                                float2* acc) {
  if (D == 1) {
    const float v = warp_sum(o[0]);
    if (lane == 0) {
      float2 a = acc[k];
      kahan_add(a.x, a.y, v);
      acc[k] = a;
    }
  } else {
    const float v = warp_sum4_split(o, lane);
    const int d = lane >> 3;
    if ((lane & 7) == 0 && d < D) {
      float2 a = acc[k * D + d];
      kahan_add(a.x, a.y, v);
      acc[k * D + d] = a;
    }
  }
}

// Warp totals of two components' partial sums a[0..3], b[0..3], one value per group of 4
// lanes: on return lane l holds the total of (l & 16 ? b : a)[(l >> 2) & 3].  Each total
// again uses the pairing of the butterfly tree, so it equals warp_sum of that value bit
// for bit, in 9 shuffles instead of the 12 of two warp_sum4_split calls.
__device__ __forceinline__ float warp_sum8_split(const float (&a)[4], const float (&b)[4],
                                                 int lane) {
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
  float k[4];
#pragma unroll
  for (int v = 0; v < 4; ++v)
    k[v] = (b4 ? b[v] : a[v]) + __shfl_xor_sync(0xffffffffu, b4 ? a[v] : b[v], 16);
  float h0 = b3 ? k[2] : k[0], h1 = b3 ? k[3] : k[1];
  h0 += __shfl_xor_sync(0xffffffffu, b3 ? k[0] : k[2], 8);
  h1 += __shfl_xor_sync(0xffffffffu, b3 ? k[1] : k[3], 8);
  float t = b2 ? h1 : h0;
  t += __shfl_xor_sync(0xffffffffu, b2 ? h0 : h1, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// warp_accumulate for two components ka != kb at once (the same sums, row by row, as two
// warp_accumulate calls, with one reduction's latency instead of two)
template <int D>
__device__ __forceinline__ void warp_accumulate2(const float (&oa)[4], const float (&ob)[4],
                                                 int lane, int ka, int kb, float2* acc) {
  if (D == 1) {
    const bool b4 = (lane & 16) != 0;
    float t = (b4 ? ob[0] : oa[0]) + __shfl_xor_sync(0xffffffffu, b4 ? oa[0] : ob[0], 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((lane & 15) == 0) {
      const int k = b4 ? kb : ka;
      float2 a = acc[k];
      kahan_add(a.x, a.y, t);
      acc[k] = a;
    }
  } else {
    const float t = warp_sum8_split(oa, ob, lane);
    const int d = (lane >> 2) & 3;
    if ((lane & 3) == 0 && d < D) {
      const int i = (lane & 16 ? kb : ka) * D + d;
      float2 a = acc[i];
      kahan_add(a.x, a.y, t);
      acc[i] = a;
    }
  }
}

__device__ __forceinline__ void load_cf(const float* cf, float (&o)[NCF]) {
  const float4* c4 = reinterpret_cast<const float4*>(cf);
#pragma unroll
  for (int q = 0; q < NCF / 4; ++q) {
    const float4 v = c4[q];
    o[4 * q] = v.x; o[4 * q + 1] = v.y; o[4 * q + 2] = v.z; o[4 * q + 3] = v.w;
  }
}

// ---------------------------------------------------------------------------
// Block evaluation of one particle.  All threads call it.  Writes
//   sm.scal[0..3] = logp, ll_old, ll_new, component*samples computed
//   (visible to all threads on return)
//   grad_out[K*D] = dlogp/dz  (if GRAD; may alias shared memory)
//   fis_out[K*D]  = Gauss-Newton diagonal + prior curvature per element (if FISHER)
// R: samples per thread per segment (multiple of 8).
// Mixed path: per-lane slot sums and per-thread energies are FP32 with Kahan
// compensation across segments; the cross-warp totals are FP64.
// ---------------------------------------------------------------------------
// FP64 parameters of a component as seen in data channel ch (two-channel sinusoids:
// amplitude r_ch A, phase offset delta_ch); other models and one channel: th itself
template <int MODEL>
__device__ __forceinline__ const double* chan_theta(const ProbDev& pb, int ch, const double* th,
                                                    double* buf) {
  if (MODEL != SINUSOID || pb.nch != 2) return th;
  buf[0] = __dmul_rn(pb.resp[2 * ch], th[0]);
  buf[1] = th[1];
  buf[2] = th[2];
  buf[3] = __dadd_rn(th[3], pb.resp[2 * ch + 1]);
  return buf;
}

template <int MODEL, int PREC, int R, bool GRAD, bool FISHER>
__device__ void block_eval_fp64(const ProbDev& pb, const PriorArgs& pa, int K, double beta,
                                const double* z, EvalSmem& sm, double* grad_out,
                                double* fis_out) {
  constexpr int D = model_d<MODEL>();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  const double lp_sum = eval_setup_any<MODEL, PREC>(pb, pa, K, z, sm);

  const int64_t N = pb.n, n1 = pb.n1;
  double acc_old = 0.0, acc_new = 0.0;
  // per-lane slot sums for components k = lane (slot 0) and lane + 32 (slot 1)
  double ga[2][4], fa[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int d = 0; d < 4; ++d) ga[q][d] = fa[q][d] = 0.0;
  double done = 0.0;   // component*samples computed by this thread
  const int64_t seg = (int64_t)blockDim.x * R;
  for (int64_t base = 0; base < N; base += seg) {
    const int64_t wfirst = base + (int64_t)warp * 32 * R;
    if (wfirst >= N) continue;  // whole warp past the end (warp-uniform)
    const int64_t m = base + (int64_t)tid * R;
    const double mine = (double)(m < N ? (m + R <= N ? R : N - m) : 0);
    // two-channel sinusoids: the thread's channel and local sample index
    const int ch = (MODEL == SINUSOID && pb.nch == 2 && m >= pb.nc) ? 1 : 0;
    const int64_t ml = m - ch * pb.nc;
    double thb[4];
    double hs[R], r[R];
    done += mine * K;
#pragma unroll
    for (int j = 0; j < R; ++j) hs[j] = 0.0;
    for (int k = 0; k < K; ++k) {
      const double* th = chan_theta<MODEL>(pb, ch, sm.th + k * D, thb);
      const double tw0 = MODEL == PULSE_LINAMP ? sm.tw[2 * k] : 0.0;
      const double tw1 = MODEL == PULSE_LINAMP ? sm.tw[2 * k + 1] : 0.0;
#pragma unroll
      for (int j = 0; j < R; ++j)
        hs[j] = __dadd_rn(hs[j], fp64_val<MODEL>(th, tw0, tw1, time_of(pb, ml + j), nullptr));
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int64_t n = m + j;
      const bool valid = n < N, old = n < n1;
      const double rr = valid ? __dadd_rn(pb.d64[valid ? n : 0], -hs[j]) : 0.0;
      const double e = __dmul_rn(rr, rr);
      if (old) acc_old += e; else acc_new += e;
      r[j] = __dmul_rn(old ? 1.0 : beta, rr);   // c_n r_n (1/sigma^2 applied at the end)
    }
    if (GRAD || FISHER) {
      for (int k = 0; k < K; ++k) {
        const double* th = chan_theta<MODEL>(pb, ch, sm.th + k * D, thb);
        const double tw0 = MODEL == PULSE_LINAMP ? sm.tw[2 * k] : 0.0;
        const double tw1 = MODEL == PULSE_LINAMP ? sm.tw[2 * k + 1] : 0.0;
        double o[4] = {0, 0, 0, 0}, f[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < R; ++j) {
          double dh[4];
          fp64_val<MODEL>(th, tw0, tw1, time_of(pb, ml + j), dh);
          if (MODEL == SINUSOID && pb.nch == 2) dh[0] = __dmul_rn(pb.resp[2 * ch], dh[0]);
          const int64_t n = m + j;
          const double cn = n < N ? (n < n1 ? 1.0 : beta) : 0.0;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            o[d] += __dmul_rn(r[j], dh[d]);
            if (FISHER) f[d] += cn * dh[d] * dh[d];
          }
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
          if (GRAD) o[d] = warp_sum(o[d]);
          if (FISHER) f[d] = warp_sum(f[d]);
        }
        if (lane == (k & 31)) {
          const int q = k < 32 ? 0 : 1;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            if (q == 0) { ga[0][d] += o[d]; fa[0][d] += f[d]; }
            else { ga[1][d] += o[d]; fa[1][d] += f[d]; }
          }
        }
      }
    }
  }

  // ---- gradient / Gauss-Newton assembly: per-warp slots -> shared -> components ----
  if (GRAD || FISHER) {
    const int KDm = K * D;
    for (int k = lane; k < K; k += 32) {
      const int q = k < 32 ? 0 : 1;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (GRAD) sm.wacc[warp * KDm + k * D + d] = q == 0 ? ga[0][d] : ga[1][d];
        if (FISHER) sm.wfis[warp * KDm + k * D + d] = q == 0 ? fa[0][d] : fa[1][d];
      }
    }
    __syncthreads();
    const double is2 = pb.inv_s2;
    for (int k = tid; k < K; k += blockDim.x) {
      double S[4] = {0, 0, 0, 0}, F[4] = {0, 0, 0, 0}, g[4], f[4];
      for (int w = 0; w < nw; ++w) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          if (GRAD) S[d] += sm.wacc[w * KDm + k * D + d];
          if (FISHER) F[d] += sm.wfis[w * KDm + k * D + d];
        }
      }
      const double* th = sm.th + k * D;
      if (GRAD) {
        finish_component<MODEL>(PREC, th, S, pb, g);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int i = k * D + d;
          grad_out[i] = g[d] * is2 * sm.dth[i] + sm.pg[i];
        }
      }
      if (FISHER) {
        finish_fisher<MODEL>(PREC, th, F, f);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int i = k * D + d;
          fis_out[i] = f[d] * is2 * sm.dth[i] * sm.dth[i] + sm.pc[i];
        }
      }
    }
  }
  double v[4] = {acc_old, acc_new, lp_sum, done};
  block_sum<4>(v, sm.red);
  if (tid == 0) {
    const double lo = -0.5 * v[0] * pb.inv_s2, ln = -0.5 * v[1] * pb.inv_s2;
    sm.scal[0] = lo + beta * ln + v[2];
    sm.scal[1] = lo;
    sm.scal[2] = ln;
    sm.scal[3] = v[3];     // component*samples computed
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Mixed path: setup, evaluation and reductions in FP32 (double-float where a
// total needs more than 24 bits; pulse centre and width in double-float); FP64
// only for the sinusoid frequency map and phase constants and the final scalars.
// The serial parts run one thread per (component, parameter) where they can.
// ---------------------------------------------------------------------------
// Particle coordinates as FP64 (caller arrays) or double-float pairs (the mixed NUTS
// kernel's positions, updated without FP64 instructions)
__device__ __forceinline__ DF to_df(double z) {   // beyond the FP32 range: (+-inf, 0)
  const float h = (float)z;
  return DF{h, isfinite(h) ? (float)(z - (double)h) : 0.f};
}
__device__ __forceinline__ DF to_df(float2 z) { return DF{z.x, z.y}; }
__device__ __forceinline__ double to_double(double z) { return z; }
__device__ __forceinline__ double to_double(float2 z) { return (double)z.x + (double)z.y; }
// z += step, the leapfrog position step
__device__ __forceinline__ void pos_add(double& z, float step) { z = z + (double)step; }
__device__ __forceinline__ void pos_add(float2& z, float step) {
  if (!isfinite(z.x)) {   // a coordinate beyond the FP32 range stays where it is
    z.x += step;
    return;
  }
  const DF s = two_sum(z.x, step);
  const DF r = quick_two_sum(s.hi, __fadd_rn(s.lo, z.y));
  z = make_float2(r.hi, r.lo);
}

// Leapfrog step folded into the mixed setup (NUTS): element i's thread applies the
// momentum half step p_i += eps/2 g_i and the position step z_i += eps minv p_i before it
// maps z_i, with the arithmetic of the separate update (FP32 control; positions FP64 or
// double-float).
template <typename ZT>
struct LeapPre {
  float* p1;
  const float* g1;
  ZT* z1;
  const float* minv;
  float de_c;
};

// (1) of the mixed setup: one thread per (component, parameter), parameter-major over a
// component count padded to 32 so that every warp maps one parameter (no divergence
// between the maps of different parameters): element e -> group g = e / Kw, k = e % Kw.
// The group order starts at parameter 1 so that the amplitude's cheap map comes last: with
// two warps and three pulse parameters, centre and width (the double-float maps) fall on
// different warps.  WRAP = false for problems without periodic parameters.  Returns the
// thread's share of the log prior.
template <int MODEL, bool WRAP, typename ZT>
__device__ __forceinline__ float setup_elements(const ProbDev& pb, const PriorArgs& pa, int K,
                                                const ZT* z, EvalSmem& sm,
                                                const LeapPre<ZT>* leap) {
  constexpr int D = model_d<MODEL>();
  float lp = 0.f;
  float *th = sm.fth(), *dth = sm.fdth(), *pgv = sm.fpg(), *pcv = sm.fpc();
  float* th_lo = th + K * D;    // double-float low parts of the pulse centre and width
  const int Kw = (K + 31) & ~31;
  for (int e = threadIdx.x; e < D * Kw; e += blockDim.x) {
    const int grp = e / Kw, k = e - grp * Kw;
    const int d = grp + 1 < D ? grp + 1 : grp + 1 - D;
    if (k >= K) continue;
    const int i = k * D + d;
    if (leap) {
      const float ph = leap->p1[i] + 0.5f * leap->de_c * leap->g1[i];
      leap->p1[i] = ph;
      pos_add(leap->z1[i], leap->de_c * leap->minv[d] * ph);
    }
    const ZT zi = z[i];
    if (MODEL == PULSE && d > 0) {
      // centre and width to ~1e-12 relative in double-float (FP32 pipe, no FP64)
      Coord32 c;
      const DF t = theta_df<WRAP>(pb, d, to_df(zi), sm.exptab, c.dth, &c);
      th[i] = t.hi;
      th_lo[i] = t.lo;
      dth[i] = c.dth;
      pgv[i] = c.pg;
      pcv[i] = c.pc;
      lp += c.lp;
    } else {
      const Coord32 c = coord32<WRAP>(pb, pa, d, to_df(zi));
      th[i] = c.th;
      dth[i] = c.dth;
      pgv[i] = c.pg;
      pcv[i] = c.pc;
      lp += c.lp;
      if (MODEL == SINUSOID && d == 1) {   // frequency in FP64 for the phase constants
        double d1;
        sm.wacc[i / D] = theta64<WRAP>(pb, 1, to_double(zi), d1);   // scratch until the sample loop
        dth[i] = (float)d1;
      }
    }
  }
  return lp;
}

template <int MODEL, int R, typename ZT>
__device__ float eval_setup_mixed(const ProbDev& pb, const PriorArgs& pa, int K, const ZT* z,
                                  EvalSmem& sm, const LeapPre<ZT>* leap = nullptr) {
  constexpr int D = model_d<MODEL>();
  const float* th = sm.fth();
  const float* th_lo = th + K * D;   // double-float low parts of the pulse centre and width
  // (1) the coordinate maps (and the leapfrog position step), element by element
  const float lp = pb.wrapmask ? setup_elements<MODEL, true, ZT>(pb, pa, K, z, sm, leap)
                               : setup_elements<MODEL, false, ZT>(pb, pa, K, z, sm, leap);
  __syncthreads();
  // (2) one thread per component: path constants
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    float* cf = sm.cf + k * NCF;
    if (MODEL == SINUSOID) {
      if (pb.nch == 2) {   // channel c: amplitude r_c A, phase offset delta_c
        for (int ch = 0; ch < 2; ++ch)
          sin_prep32(pb.f_resp[2 * ch] * th[k * D], sm.wacc[k], th[k * D + 2],
                     th[k * D + 3] + pb.f_resp[2 * ch + 1], pb, cf + ch * sm.cfch);
      } else {
        sin_prep32(th[k * D], sm.wacc[k], th[k * D + 2], th[k * D + 3], pb, cf);
      }
    } else if (MODEL == PULSE) {
      const float A = th[k * D], w = th[k * D + 2];
      pulse_prep_df(A, DF{th[k * D + 1], th_lo[k * D + 1]}, w, pb, cf);
      cf[11] = A / w;                                 // gradient factor A / w
    } else {
      pulse_prep32(th[k * D], sm.tw[2 * k], sm.tw[2 * k + 1], pb, cf);
    }
  }
  __syncthreads();
  return lp;
}

// F64OUT: FP64 totals into sm.scal (logp, ll_old, ll_new, count); otherwise double-float
// totals into sm.scalf() (logp, ll_old, ll_new as hi/lo pairs) and the count into
// sm.scalc(), with no FP64 instruction (the mixed NUTS kernel).  beta_df: beta as
// double-float (used when !F64OUT).
template <int MODEL, int R, bool GRAD, bool FISHER, typename GT, bool F64OUT = true,
          typename ZT = double>
__device__ void block_eval_mixed(const ProbDev& pb, const PriorArgs& pa, int K, double beta,
                                 const ZT* z, EvalSmem& sm, GT* grad_out, double* fis_out,
                                 const LeapPre<ZT>* leap = nullptr, DF beta_df = DF{0.f, 0.f}) {
  constexpr int D = model_d<MODEL>();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  const float lp_t = eval_setup_mixed<MODEL, R, ZT>(pb, pa, K, z, sm, leap);

  // sample indices fit 32 bits (capacity < 2^24): no 64-bit integer work or
  // 64-bit conversions (which issue on the FP64 pipe) inside the sample loop
  const int N = (int)pb.n, n1 = (int)pb.n1;
  const float beta_f = (float)beta, inv_s2_f = (float)pb.inv_s2;
  float eo_s = 0.f, eo_c = 0.f, en_s = 0.f, en_c = 0.f;   // Kahan energies
  // per-warp Kahan rows (sum, compensation) of the component partial sums; only
  // this warp touches its rows until the barrier after the sample loop
  const int KDm = K * D;
  float2* const gacc = sm.wacc2() + warp * KDm;
  float2* const facc = FISHER ? sm.wfis2() + warp * KDm : nullptr;
  for (int i = lane; i < KDm; i += 32) {
    if (GRAD) gacc[i] = make_float2(0.f, 0.f);
    if (FISHER) facc[i] = make_float2(0.f, 0.f);
  }
  __syncwarp();
  const bool win = MODEL != SINUSOID && pa.window;
  int done = 0;   // component*samples this thread computed

  const int seg = blockDim.x * R;
  for (int base = 0; base < N; base += seg) {
    const int wfirst = base + warp * 32 * R;
    if (wfirst >= N) continue;  // whole warp past the end (warp-uniform)
    const int m = base + tid * R;
    const int mine = m < N ? (m + R <= N ? R : N - m) : 0;
    float2 r[R / 2];    // packed pairs (pair_sample layout)
    if (m + R <= N) {
      const float4* src = reinterpret_cast<const float4*>(pb.d32 + m);
#pragma unroll
      for (int q = 0; q < R / 4; ++q) {
        const float4 v = src[q];
        slot<MODEL, R>(r, 4 * q) = v.x;
        slot<MODEL, R>(r, 4 * q + 1) = v.y;
        slot<MODEL, R>(r, 4 * q + 2) = v.z;
        slot<MODEL, R>(r, 4 * q + 3) = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) slot<MODEL, R>(r, j) = (m + j < N) ? pb.d32[m + j] : 0.0f;
    }
    // two-channel sinusoids: the thread's channel (its R samples never straddle), its
    // local sample index and that channel's constants; r_c scales the adjoint sums
    const int ch = (MODEL == SINUSOID && pb.nch == 2 && m >= (int)pb.nc) ? 1 : 0;
    const float mf = (float)(m - ch * (int)pb.nc);
    const float* cfb = sm.cf + ch * sm.cfch;
    const float rch = pb.f_resp[2 * ch];
    // components active on this warp's range, ascending (all K without the window):
    // lanes test components lane and lane + 32 against the range's first and last sample
    // (the support bounds cf[9], cf[10] are whole sample indices)
    uint32_t act[2];
    if (win) {
      const float first = (float)wfirst, last = (float)min(wfirst + 32 * R - 1, N - 1);
      bool a0 = false, a1 = false;
      if (lane < K) a0 = !(last < sm.cf[lane * NCF + 9] || first > sm.cf[lane * NCF + 10]);
      if (lane + 32 < K)
        a1 = !(last < sm.cf[(lane + 32) * NCF + 9] || first > sm.cf[(lane + 32) * NCF + 10]);
      act[0] = __ballot_sync(0xffffffffu, a0);
      act[1] = __ballot_sync(0xffffffffu, a1);
    } else {
      act[0] = K >= 32 ? 0xffffffffu : ((1u << K) - 1u);
      act[1] = K >= 64 ? 0xffffffffu : (K > 32 ? ((1u << (K - 32)) - 1u) : 0u);
    }
    done += mine * (__popc(act[0]) + __popc(act[1]));
    // active components in ascending k (sinusoids two at a time)
    const unsigned long long act64 =
        (unsigned long long)act[0] | ((unsigned long long)act[1] << 32);
#pragma unroll 1
    for (unsigned long long bits = act64; bits;) {
      const int ka = __ffsll((long long)bits) - 1;
      bits &= bits - 1ull;
      if constexpr (MODEL == SINUSOID) {
        if (bits) {
          const int kb = __ffsll((long long)bits) - 1;
          bits &= bits - 1ull;
          float cf[2][NCF];
          load_cf(cfb + ka * NCF, cf[0]);
          load_cf(cfb + kb * NCF, cf[1]);
          mixed_sub<MODEL, R, 2>(cf, mf, r);
          continue;
        }
      }
      float cf[1][NCF];
      load_cf(cfb + ka * NCF, cf[0]);
      mixed_sub<MODEL, R, 1>(cf, mf, r);
    }
    // residual energy and the adjoint weights rc = c_n r_n / sigma^2
    float so = 0.f, sn = 0.f;
    if (m >= n1 && m + R <= N) {
      // every sample of the thread valid and new: packed products, two packed partial sums
      const float2 w = f2(beta_f * inv_s2_f);
      float2 acc0 = f2(0.f), acc1 = f2(0.f);
#pragma unroll
      for (int i = 0; i < R / 2; i += 2) {
        acc0 = __ffma2_rn(r[i], r[i], acc0);
        acc1 = __ffma2_rn(r[i + 1], r[i + 1], acc1);
        r[i] = __fmul2_rn(r[i], w);
        r[i + 1] = __fmul2_rn(r[i + 1], w);
      }
      sn = (acc0.x + acc0.y) + (acc1.x + acc1.y);
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) {     // sample order
        const int n = m + j;
        const bool valid = n < N, old = n < n1;
        float& rj = slot<MODEL, R>(r, j);
        const float rr = valid ? rj : 0.0f;
        const float e = rr * rr;
        if (old) so += e; else sn += e;
        rj = rr * (old ? inv_s2_f : beta_f * inv_s2_f);
      }
    }
    kahan_add(eo_s, eo_c, so);
    kahan_add(en_s, en_c, sn);
    if (GRAD) {
      // pulses: one component per pass, its partial sums held until the next component's
      // are ready and both reduced together; sinusoids: two components per pass
      int kp = -1;
      float op[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
      for (unsigned long long bits = act64; bits;) {
        const int ka = __ffsll((long long)bits) - 1;
        bits &= bits - 1ull;
        if constexpr (MODEL == SINUSOID) {
          if (bits) {
            const int kb = __ffsll((long long)bits) - 1;
            bits &= bits - 1ull;
            float cf[2][NCF], o[2][4];
            load_cf(cfb + ka * NCF, cf[0]);
            load_cf(cfb + kb * NCF, cf[1]);
            mixed_adj<MODEL, R, 2>(cf, mf, r, o);
            if (pb.nch == 2)
#pragma unroll
              for (int d = 0; d < 4; ++d) { o[0][d] *= rch; o[1][d] *= rch; }
            warp_accumulate2<D>(o[0], o[1], lane, ka, kb, gacc);
            continue;
          }
        }
        float cf[1][NCF], o[1][4];
        load_cf(cfb + ka * NCF, cf[0]);
        mixed_adj<MODEL, R, 1>(cf, mf, r, o);
        if (MODEL == SINUSOID && pb.nch == 2)
#pragma unroll
          for (int d = 0; d < 4; ++d) o[0][d] *= rch;
        if (MODEL == SINUSOID) {
          warp_accumulate<D>(o[0], lane, ka, gacc);
        } else if (kp < 0) {
          kp = ka;
#pragma unroll
          for (int d = 0; d < 4; ++d) op[d] = o[0][d];
        } else {
          warp_accumulate2<D>(op, o[0], lane, kp, ka, gacc);
          kp = -1;
        }
      }
      if (kp >= 0) warp_accumulate<D>(op, lane, kp, gacc);
    }
    if (FISHER) {
      float cw[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int n = m + j;
        cw[j] = n < N ? (n < n1 ? inv_s2_f : beta_f * inv_s2_f) : 0.0f;
      }
#pragma unroll 1
      for (int half = 0; half < 2; ++half)
      for (uint32_t bits = act[half]; bits; bits &= bits - 1u) {
        const int k = (half << 5) + __ffs(bits) - 1;
        float cf[NCF], o[4];
        load_cf(cfb + k * NCF, cf);
        mixed_fis<MODEL, R>(cf, mf, cw, (float)pb.t_origin, (float)pb.dt, o);
        if (MODEL == SINUSOID && pb.nch == 2)
#pragma unroll
          for (int d = 0; d < 4; ++d) o[d] *= rch * rch;
        warp_accumulate<D>(o, lane, k, facc);
      }
    }
  }

  // ---- block totals, part 1: warp totals of the energies, log prior and count,
  // taken before the barrier so they overlap the wait for the slowest warp ----
  DF e_o = warp_sum_df(DF{eo_s, -eo_c});
  DF e_n = warp_sum_df(DF{en_s, -en_c});
  DF e_p = warp_sum_df(DF{lp_t, 0.f});
  // a coordinate beyond the FP32 range has log prior -inf, which the double-float sum
  // would turn into NaN (inf - inf in its error term): such a warp takes the plain sum
  if (__any_sync(0xffffffffu, !isfinite(lp_t))) e_p = DF{warp_sum(lp_t), 0.f};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) done += __shfl_xor_sync(0xffffffffu, done, o);
  float* rf = reinterpret_cast<float*>(sm.red);
  int* ri = reinterpret_cast<int*>(rf + 6 * 32);
  if (lane == 0) {
    rf[warp * 6 + 0] = e_o.hi; rf[warp * 6 + 1] = e_o.lo;
    rf[warp * 6 + 2] = e_n.hi; rf[warp * 6 + 3] = e_n.lo;
    rf[warp * 6 + 4] = e_p.hi; rf[warp * 6 + 5] = e_p.lo;
    ri[warp] = done;
  }
  __syncthreads();
  // ---- per-warp Kahan rows (double-float: hi = s, lo = -c) -> gradient and metric,
  // one thread per (component, parameter) ----
  if (GRAD || FISHER) {
    const float* th = sm.fth();
    for (int i = tid; i < KDm; i += blockDim.x) {
      const int k = i / D, d = i - k * D;
      const float A = th[k * D];
      const float aw = MODEL == PULSE ? sm.cf[k * NCF + 11] : 0.f;   // A / w
      if (GRAD) {
        float g;
        if (MODEL == SINUSOID) {
          // t_n = t_origin + n dt: sum rc sin t = t_o S1 + dt S2, sum rc sin t^2 = ...
          DF S[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) S[v] = DF{0.f, 0.f};
          for (int w = 0; w < nw; ++w) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const float2 a = sm.wacc2()[w * KDm + k * D + v];
              S[v] = df_add(S[v], DF{a.x, -a.y});
            }
          }
          const double to = pb.t_origin, dt = pb.dt;
          if (d == 0) {
            g = S[0].hi + S[0].lo;
          } else if (d == 1) {
            const double s1 = df_to_double(S[1]), s2 = df_to_double(S[2]);
            g = (float)(-(double)A * kTwoPi * (to * s1 + dt * s2));
          } else if (d == 2) {
            const double s1 = df_to_double(S[1]), s2 = df_to_double(S[2]), s3 = df_to_double(S[3]);
            g = (float)(-(double)A * kPi * (to * to * s1 + 2.0 * to * dt * s2 + dt * dt * s3));
          } else {
            g = -A * (S[1].hi + S[1].lo);
          }
        } else {
          DF S{0.f, 0.f};
          for (int w = 0; w < nw; ++w) {
            const float2 a = sm.wacc2()[w * KDm + i];
            S = df_add(S, DF{a.x, -a.y});
          }
          const float c = MODEL == PULSE
                              ? (d == 0 ? 1.0f : (d == 1 ? aw * (float)kCu
                                                         : aw * (float)(kCu * kCu)))
                              : 1.0f;
          g = c * (S.hi + S.lo);
        }
        grad_out[i] = (GT)(g * sm.fdth()[i] + sm.fpg()[i]);
      }
      if (FISHER) {
        DF F{0.f, 0.f};
        for (int w = 0; w < nw; ++w) {
          const float2 a = sm.wfis2()[w * KDm + i];
          F = df_add(F, DF{a.x, -a.y});
        }
        float c = 1.0f;
        if (MODEL == SINUSOID) {
          const float A2 = A * A;
          c = d == 0 ? 1.0f : (d == 1 ? A2 * (float)(kTwoPi * kTwoPi)
                                      : (d == 2 ? A2 * (float)(kPi * kPi) : A2));
        } else if (MODEL == PULSE) {
          const float c2 = (float)(kCu * kCu);
          c = d == 0 ? 1.0f : (d == 1 ? aw * aw * c2 : aw * aw * c2 * c2);
        }
        const float f = c * (F.hi + F.lo);
        const float j = sm.fdth()[i];
        fis_out[i] = (double)(f * j * j + sm.fpc()[i]);
      }
    }
  }
  // ---- block totals, part 2: the last thread, beside the component loop ----
  if (tid == blockDim.x - 1) {
    DF a{0.f, 0.f}, b{0.f, 0.f}, c{0.f, 0.f};
    float cp = 0.f;   // plain sum of the log prior's warp totals (the non-finite case)
    long long cnt = 0;
    for (int w = 0; w < nw; ++w) {
      a = df_add(a, DF{rf[w * 6 + 0], rf[w * 6 + 1]});
      b = df_add(b, DF{rf[w * 6 + 2], rf[w * 6 + 3]});
      c = df_add(c, DF{rf[w * 6 + 4], rf[w * 6 + 5]});
      cp += rf[w * 6 + 4];
      cnt += ri[w];
    }
    if constexpr (F64OUT) {
      const double lo = -0.5 * df_to_double(a) * pb.inv_s2;
      const double ln = -0.5 * df_to_double(b) * pb.inv_s2;
      const double lp = isfinite(cp) ? df_to_double(c) : (double)cp;
      sm.scal[0] = lo + beta * ln + lp;
      sm.scal[1] = lo;
      sm.scal[2] = ln;
      sm.scal[3] = (double)cnt;
    } else {
      const DF nis{-0.5f * pb.f_is2.x, -0.5f * pb.f_is2.y};   // -1/(2 sigma^2), exact halving
      const DF lo = df_mul(a, nis), ln = df_mul(b, nis);
      DF lg = df_add(lo, df_mul(beta_df, ln));
      if (isfinite(cp) && isfinite(lg.hi)) lg = df_add(lg, c);
      else lg = DF{lg.hi + cp, 0.f};   // -inf log prior, or a NaN likelihood
      float* f = sm.scalf();
      f[0] = lg.hi; f[1] = lg.lo; f[2] = lo.hi; f[3] = lo.lo; f[4] = ln.hi; f[5] = ln.lo;
      *sm.scalc() = (int)cnt;
    }
  }
  __syncthreads();
}

// per-component setup for either path (all threads; ends with __syncthreads)
template <int MODEL, int PREC>
__device__ __forceinline__ double eval_setup(const ProbDev& pb, const PriorArgs& pa, int K,
                                             const double* z, EvalSmem& sm) {
  if constexpr (PREC == MIXED) return (double)eval_setup_mixed<MODEL, 32, double>(pb, pa, K, z, sm);
  else return eval_setup_any<MODEL, PREC>(pb, pa, K, z, sm);
}

// dispatcher: all threads call it; see block_eval_fp64 / block_eval_mixed
template <int MODEL, int PREC, int R, bool GRAD, bool FISHER, typename GT = double>
__device__ __forceinline__ void block_eval(const ProbDev& pb, const PriorArgs& pa, int K,
                                           double beta, const double* z, EvalSmem& sm,
                                           GT* grad_out, double* fis_out) {
  if constexpr (PREC == MIXED)
    block_eval_mixed<MODEL, R, GRAD, FISHER, GT>(pb, pa, K, beta, z, sm, grad_out, fis_out);
  else
    block_eval_fp64<MODEL, PREC, R, GRAD, FISHER>(pb, pa, K, beta, z, sm, grad_out, fis_out);
}

}  // namespace tsmc
