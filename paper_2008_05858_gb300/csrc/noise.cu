// Detector noise stage: photon and dark shot noise, pixel response non-uniformity, read-out
// noise and amplifier cross-talk added to a rendered frame (the last step of Sec. 2.2, which
// names these noises without formulas).  Per detector d of width W and pixel (r, c):
//
//   lam = max((1 + prnu z) S + dark, 0),  N ~ Poisson(lam),  M = N + xtalk N(r, W-1-c),
//   E = M + ron g,  ADU = clamp(floor(bias + E / gain + 1/2), 0, saturation),
//
// with z, g standard normals and the mirror pixel (r, W-1-c) read by the other amplifier of
// a two-output detector (the middle column of an odd width has none).  One thread owns one
// mirror pair q = r ceil(W/2) + c, so it reads both pixels, draws both counts and writes
// both results: in-place operation is safe and the cross-talk needs no second pass.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), a pure function of
// (key, counter), so the draws do not depend on the launch shape:
//   z pair: key = pattern seed, counter (q, d, 0, 0);   g pair: key = seed, counter (q, d, 0, 1);
//   counts of side s: key = seed, counters (q, d, i, 2 + s), trial i = 0, 1, ...
// Uniform u(a, b) = ((a >> 5) 2^26 + (b >> 6) + 1/2) 2^-53; normals by Box-Muller
// (rho = sqrt(-2 ln u(w0, w1)), phase 2 pi u(w2, w3), cos for the left pixel, sin for the
// right); Poisson by sequential inversion below lam = 10 and by Hormann's transformed
// rejection with squeeze (PTRS, 1993) from 10 up, one block per trial, at most 64 trials.
// Every decision is taken in FP64 with explicitly rounded operations (no contraction into
// FMA), so that a CPU restatement of the same definition draws the same integers.
#include <cstdint>

#include "e2e_kernels.h"

namespace e2e {

struct NoiseArgs {
  uint64_t seed, pattern_seed;
  double dark, prnu, ron, xtalk, gain, bias;
  int saturation, poisson;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 noise_block(uint64_t seed, uint32_t q, uint32_t d, uint32_t i, uint32_t stream) {
  return philox4x32_10(make_uint4(q, d, i, stream), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Uniform on (0, 1) from two words; every step is exact.
__device__ __forceinline__ double uni53(uint32_t a, uint32_t b) {
  return __dadd_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)), 0.5) *
         (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void normal_pair(uint64_t seed, uint32_t q, uint32_t d, uint32_t stream, double& left,
                                            double& right) {
  const uint4 w = noise_block(seed, q, d, 0, stream);
  const double rho = sqrt(__dmul_rn(-2.0, log(uni53(w.x, w.y))));
  const double ph = __dmul_rn(2.0 * 3.14159265358979323846, uni53(w.z, w.w));
  double s, c;
  sincos(ph, &s, &c);
  left = __dmul_rn(rho, c);
  right = __dmul_rn(rho, s);
}

__device__ double poisson_draw(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t side) {
  if (!(lam > 0.0)) return 0.0;
  if (lam < 10.0) {
    const uint4 w = noise_block(seed, q, d, 0, 2 + side);
    const double u = uni53(w.x, w.y);
    int k = 0;
    double p = exp(-lam), F = p;
    while (u > F && k < 200) {
      ++k;
      p = __dmul_rn(p, __ddiv_rn(lam, (double)k));
      F = __dadd_rn(F, p);
    }
    return (double)k;
  }
  const double slam = sqrt(lam), loglam = log(lam);
  const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
  const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
  const double invalpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dadd_rn(b, -3.4)));
  const double vr = __dadd_rn(0.9277, -__ddiv_rn(3.6224, __dadd_rn(b, -2.0)));
  for (uint32_t i = 0; i < 64; ++i) {
    const uint4 w = noise_block(seed, q, d, i, 2 + side);
    const double U = __dadd_rn(uni53(w.x, w.y), -0.5), V = uni53(w.z, w.w);
    const double us = __dadd_rn(0.5, -fabs(U));
    const double t = __dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b);
    const double k = floor(__dadd_rn(__dadd_rn(__dmul_rn(t, U), lam), 0.43));
    if (us >= 0.07 && V <= vr) return k;
    if (k < 0.0 || (us < 0.013 && V > us)) continue;
    const double lhs = __dadd_rn(__dadd_rn(log(V), log(invalpha)),
                                 -log(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
    const double rhs = __dadd_rn(__dadd_rn(-lam, __dmul_rn(k, loglam)), -lgamma(__dadd_rn(k, 1.0)));
    if (lhs <= rhs) return k;
  }
  return floor(__dadd_rn(lam, 0.5));
}

template <typename TI>
__device__ __forceinline__ double load_px(const TI* p) { return (double)*p; }

template <typename TO>
__device__ __forceinline__ void store_px(TO* p, double e, const NoiseArgs& a);

template <>
__device__ __forceinline__ void store_px<float>(float* p, double e, const NoiseArgs&) { *p = (float)e; }
template <>
__device__ __forceinline__ void store_px<double>(double* p, double e, const NoiseArgs&) { *p = e; }
template <>
__device__ __forceinline__ void store_px<uint16_t>(uint16_t* p, double e, const NoiseArgs& a) {
  double v = floor(__dadd_rn(__dadd_rn(a.bias, __ddiv_rn(e, a.gain)), 0.5));
  v = v < 0.0 ? 0.0 : v;
  v = v > (double)a.saturation ? (double)a.saturation : v;
  *p = (uint16_t)v;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_noise(const NoiseArgs a, const TI* __restrict__ src, int64_t src_pitch,
                                               TO* dst, int64_t dst_pitch, int H, int W, int det) {
  const int half = (W + 1) / 2;
  const int64_t n = (int64_t)H * half;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / half), c = (int)(t - (int64_t)r * half);
    const uint32_t q = (uint32_t)t;
    const int cm = W - 1 - c;
    const bool two = cm != c;
    const TI* srow = src + (int64_t)r * src_pitch;
    const double s0 = load_px(srow + c), s1 = two ? load_px(srow + cm) : 0.0;
    double z0, z1, g0, g1;
    normal_pair(a.pattern_seed, q, (uint32_t)det, 0, z0, z1);
    normal_pair(a.seed, q, (uint32_t)det, 1, g0, g1);
    double l0 = __dadd_rn(__dmul_rn(__dadd_rn(1.0, __dmul_rn(a.prnu, z0)), s0), a.dark);
    double l1 = __dadd_rn(__dmul_rn(__dadd_rn(1.0, __dmul_rn(a.prnu, z1)), s1), a.dark);
    l0 = l0 > 0.0 ? l0 : 0.0;
    l1 = l1 > 0.0 ? l1 : 0.0;
    const double n0 = a.poisson ? poisson_draw(l0, a.seed, q, (uint32_t)det, 0) : l0;
    const double n1 = (two && a.poisson) ? poisson_draw(l1, a.seed, q, (uint32_t)det, 1) : l1;
    const double m0 = two ? __dadd_rn(n0, __dmul_rn(a.xtalk, n1)) : __dadd_rn(n0, 0.0);
    const double m1 = __dadd_rn(n1, __dmul_rn(a.xtalk, n0));
    TO* drow = dst + (int64_t)r * dst_pitch;
    store_px(drow + c, __dadd_rn(m0, __dmul_rn(a.ron, g0)), a);
    if (two) store_px(drow + cm, __dadd_rn(m1, __dmul_rn(a.ron, g1)), a);
  }
}

template <typename TI, typename TO>
static cudaError_t launch_noise_t(const NoiseArgs& a, const void* src, int64_t sp, void* dst, int64_t dp, int H, int W,
                                  int det, cudaStream_t st) {
  const int64_t n = (int64_t)H * ((W + 1) / 2);
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_noise<TI, TO><<<(unsigned)blocks, 256, 0, st>>>(a, (const TI*)src, sp, (TO*)dst, dp, H, W, det);
  return cudaGetLastError();
}

cudaError_t launch_noise(uint64_t seed, uint64_t pattern_seed, double dark, double prnu, double ron, double xtalk,
                         double gain, double bias, int saturation, int poisson, int src_dtype, const void* src,
                         int64_t src_pitch, int dst_dtype, void* dst, int64_t dst_pitch, int H, int W, int det,
                         cudaStream_t st) {
  const NoiseArgs a{seed, pattern_seed, dark, prnu, ron, xtalk, gain, bias, saturation, poisson};
#define E2E_N(SI, TI, DI, TO) \
  if (src_dtype == SI && dst_dtype == DI) return launch_noise_t<TI, TO>(a, src, src_pitch, dst, dst_pitch, H, W, det, st);
  E2E_N(0, float, 0, float) E2E_N(0, float, 1, double) E2E_N(0, float, 2, uint16_t)
  E2E_N(1, double, 0, float) E2E_N(1, double, 1, double) E2E_N(1, double, 2, uint16_t)
#undef E2E_N
  return cudaErrorInvalidValue;
}

}  // namespace e2e
