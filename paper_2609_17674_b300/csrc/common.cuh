// common.cuh -- device building blocks shared by every kernel of libtsmc:
// the Philox4x64-10 stream, problem descriptors and warp/block reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsmc {

constexpr double kPi = 3.141592653589793116;      // nearest double to pi
constexpr double kTwoPi = 2.0 * kPi;
constexpr int kMaxDepth = 10;                      // NUTS tree depth limit of the library
constexpr int kMaxK = 64;                          // component slots per particle (2 per lane)

enum Model { PULSE = 0, SINUSOID = 1, PULSE_LINAMP = 2 };
enum Prec { FP64 = 0, MIXED = 1 };
enum Purpose {
  PU_INIT = 0, PU_MOMENTUM = 1, PU_DIRECTION = 2, PU_LEAF = 3, PU_TOP = 4,
  PU_RJ = 5, PU_RJPARAM = 6, PU_RESAMPLE = 7, PU_MOVETYPE = 8, PU_KDE = 9
};

// Population birth proposal per problem (doubles): [0] m centres, [1..4] bandwidth h_d,
// [8 ..] centres [m][D] in z coordinates
constexpr int kKdeM = 256;
constexpr int kKdeStride = 8 + kKdeM * 4;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter layout of the
// sampler: {particle, stage, (round << 4) | purpose, index}; key {seed, problem}.
// ---------------------------------------------------------------------------
struct Rand4 { uint64_t w[4]; };

__device__ __forceinline__ Rand4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                        uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t a = 0xD2E7470EE14C6C93ull, b = 0xCA5A826395121157ull;
    const uint64_t lo_a = a * c0, hi_a = __umul64hi(a, c0);
    const uint64_t lo_b = b * c2, hi_b = __umul64hi(b, c2);
    const uint64_t n0 = hi_b ^ c1 ^ k0;
    const uint64_t n2 = hi_a ^ c3 ^ k1;
    c0 = n0; c1 = lo_b; c2 = n2; c3 = lo_a;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
  Rand4 r;
  r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
  return r;
}

// 53 bits to the open interval (0, 1): (x >> 11) 2^-53 + 2^-54
__device__ __forceinline__ double u01(uint64_t x) {
  return __dadd_rn(__dmul_rn((double)(x >> 11), 0x1p-53), 0x1p-54);
}

__device__ __forceinline__ Rand4 draw(uint64_t seed, int problem, uint64_t particle, int stage,
                                      int round, int purpose, uint64_t index) {
  return philox(particle, (uint64_t)(uint32_t)stage,
                ((uint64_t)(uint32_t)round << 4) | (uint64_t)purpose, index, seed,
                (uint64_t)(uint32_t)problem);
}

// m-th standard normal of a stream: Box-Muller on the pair (2j, 2j+1) of call m/4
__device__ __forceinline__ double draw_normal(uint64_t seed, int problem, uint64_t particle,
                                              int stage, int round, int purpose, uint64_t m) {
  const Rand4 r = draw(seed, problem, particle, stage, round, purpose, m >> 2);
  const int pair = (int)((m & 3) >> 1);
  const double ua = u01(r.w[2 * pair]), ub = u01(r.w[2 * pair + 1]);
  const double rad = sqrt(__dmul_rn(-2.0, log(ua)));
  const double ang = __dmul_rn(kTwoPi, ub);
  return (m & 1) ? __dmul_rn(rad, sin(ang)) : __dmul_rn(rad, cos(ang));
}

// ---------------------------------------------------------------------------
// Problem descriptor (device copy).  t_n = t_origin + n dt; samples n < n1 are
// already assimilated (temperature 1), samples n1 <= n < n are tempered by beta.
// ---------------------------------------------------------------------------
struct ProbDev {
  const double* d64;
  const float* d32;
  int64_t n, n1, cap;
  double t_origin, dt, sigma, inv_s2;
  double lo[4], hi[4], llo[4], lhi[4];
  uint32_t logmask;
  int32_t done;      // beta reached 1 in an earlier stage: skipped by stage kernels
  // double-float (hi, lo) copies for FP32 arithmetic on the mixed path:
  // t_origin, dt, and per parameter the map's offset and span (log-space if log-uniform)
  float2 f_to, f_dt, f_off[4], f_span[4];
  // sinusoids in two data channels (A, E): samples [0, nc) are channel A, [nc, 2 nc) channel
  // E at the same times; channel c sees resp[2c] A cos(phi(t) + resp[2c+1]).  nch = 1: one
  // channel, nc = n.
  int64_t nc;
  int32_t nch;
  uint32_t wrapmask; // bit d: parameter d periodic on [lo, hi): theta = lo + span (z - floor z)
  double resp[4];
  float f_resp[4];
  float2 f_is2;      // 1/sigma^2 as double-float
  float2 pad2_;
};

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Block-wide sum of NV doubles; every thread gets the totals.  red: >= 32*NV doubles
// of shared memory.  Summation order is fixed (deterministic).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * 32 + warp] = v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[i * 32 + w];
    v[i] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ double logaddexp(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = a > b ? a : b;
  return m + log1p(exp(-fabs(a - b)));
}

// logistic s(z) and the log of the logistic density s(1-s)
__device__ __forceinline__ double logistic(double z) {
  if (z >= 0.0) return 1.0 / (1.0 + exp(-z));
  const double e = exp(z);
  return e / (1.0 + e);
}

}  // namespace tsmc
