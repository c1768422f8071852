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
// Every decision is the one FP64 arithmetic with explicitly rounded operations (no
// contraction into FMA) takes, so that a CPU restatement of the same definition draws the
// same integers.  The kernel reaches those decisions by filtered evaluation: it first
// computes each decided quantity in FP32 together with a bound on its distance from the FP64
// value; only when the FP32 value lies within that bound of the decision boundary (about one
// draw in 1e4 .. 1e5) does it redo the draw in FP64 (the functions below marked "exact").
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

// Exact FP64 Box-Muller pair.
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

// Exact FP64 draw: the definition, step by step.
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

// ------------------------------------------------------------------ FP32 filtered draws

// fl32 of the 53-bit uniform u = (2X + 1) 2^-54, X = (a >> 5) 2^26 + (b >> 6) (correctly
// rounded: one conversion of the exact integer), and fl32 of 1 - u.
__device__ __forceinline__ uint64_t uni53_num(uint32_t a, uint32_t b) {
  return ((((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6)) << 1) | 1ull;
}
__device__ __forceinline__ float uni53_f32(uint32_t a, uint32_t b) { return __ull2float_rn(uni53_num(a, b)) * 0x1p-54f; }
__device__ __forceinline__ float one_minus_uni53_f32(uint32_t a, uint32_t b) {
  return __ull2float_rn((1ull << 54) - uni53_num(a, b)) * 0x1p-54f;
}

// Box-Muller pair in FP32 and a bound eg on |g - g_exact| for both members: ln u from logf
// (u < 1/2) or log1pf(-(1 - u)) (u >= 1/2), each within 1 ulp of a correctly rounded
// argument; the phase from sincospif(2u) (1 ulp) with 2u exact.
__device__ __forceinline__ void normal_pair_f32(uint64_t seed, uint32_t q, uint32_t d, uint32_t stream, float& g0,
                                                float& g1, float& eg) {
  const uint4 w = noise_block(seed, q, d, 0, stream);
  const float u1 = uni53_f32(w.x, w.y);
  const float ln = u1 < 0.5f ? logf(u1) : log1pf(-one_minus_uni53_f32(w.x, w.y));
  const float rho = sqrtf(-2.f * ln);
  float s, c;
  sincospif(2.f * uni53_f32(w.z, w.w), &s, &c);
  g0 = rho * c;
  g1 = rho * s;
  eg = fmaf(rho, 1.5e-6f, 1e-7f);  // also covers a 2e-7 relative rounding of products with g
}

// Poisson draw with the exact function's integer result, from FP32 arithmetic whenever its
// error bound decides every comparison (see the file comment).
__device__ double poisson_filtered(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t side) {
  if (!(lam > 0.0)) return 0.0;
  const float l = __double2float_rn(lam);
  if (lam < 10.0) {
    // F_k in FP32: exp(-l) within 2 ulp, l within 2^-24 relative, each step within ~3 ulp:
    // |F32_k - F64_k| <= F (8.4e-7 + 2.4e-7 k); u within 2^-24 relative.  Bounds doubled.
    const uint4 w = noise_block(seed, q, d, 0, 2 + side);
    const float u = uni53_f32(w.x, w.y);
    float p = expf(-l), F = p;
    for (int k = 0; k < 200; ++k) {
      const float tol = fmaf(F, fmaf(1e-6f, (float)k, 4e-6f), fmaf(u, 2.5e-7f, 1e-12f));
      const float diff = u - F;
      if (diff > tol) {  // u > F_k: one more
        p = p * (l / (float)(k + 1));
        F = F + p;
        continue;
      }
      if (-diff > tol) return (double)k;      // u <= F_k
      return poisson_draw(lam, seed, q, d, side);  // too close to call
    }
    return 200.0;
  }
  // PTRS in FP32; k's final sum in FP64 (y + lam + 0.43), the rare slow acceptance in FP64
  const float sl = sqrtf(l);
  const float b = fmaf(2.53f, sl, 0.931f);
  const float a = fmaf(0.02483f, b, -0.059f);
  const float vr = 0.9277f - 3.6224f / (b - 2.f);
  double b64 = 0.0, a64 = 0.0, ia64 = 0.0, ll64 = 0.0;  // the exact constants, when needed
  // x = y + lam + 0.43 relative to Li = floor(lam): only the fraction enters the FP32 sum
  const double Li = floor(lam);
  const float lf = __double2float_rn(__dadd_rn(lam, -Li));
  for (uint32_t i = 0; i < 64; ++i) {
    const uint4 w = noise_block(seed, q, d, i, 2 + side);
    const float U = uni53_f32(w.x, w.y) - 0.5f, V = uni53_f32(w.z, w.w);
    const float us = 0.5f - fabsf(U);  // within 1.5e-7 of the exact us
    const float T = 2.f * a / us + b;
    const float y = T * U;
    const float yerr = fabsf(T) * fmaf(fabsf(U), fmaf(3e-7f, 1.f / us, 4e-6f), 2e-7f) + 1e-6f;
    const float xr = (y + lf) + 0.43f;
    const float xe = yerr + fmaf(fabsf(xr), 2.5e-7f, 1e-7f);
    const float kr = floorf(xr - xe);
    if (floorf(xr + xe) != kr) return poisson_draw(lam, seed, q, d, side);
    const double k = Li + (double)kr;
    // quick acceptance: us >= 0.07 && V <= vr
    const float mu = 3e-7f, mv = 8e-7f;
    const bool c1t = us - 0.07f > mu, c1f = 0.07f - us > mu, c2t = vr - V > mv, c2f = V - vr > mv;
    if (c1t && c2t) return k;
    if (!(c1f || c2f)) return poisson_draw(lam, seed, q, d, side);
    // rejection: k < 0 || (us < 0.013 && V > us)
    if (k < 0.0) continue;
    const bool d1t = 0.013f - us > mu, d1f = us - 0.013f > mu, d2t = V - us > mu, d2f = us - V > mu;
    if (d1t && d2t) continue;
    if (!(d1f || d2f)) return poisson_draw(lam, seed, q, d, side);
    // the slow acceptance test, exactly as the FP64 draw takes it
    if (b64 == 0.0) {
      const double slam = sqrt(lam);
      ll64 = log(lam);
      b64 = __dadd_rn(0.931, __dmul_rn(2.53, slam));
      a64 = __dadd_rn(-0.059, __dmul_rn(0.02483, b64));
      ia64 = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dadd_rn(b64, -3.4)));
    }
    const double U64 = __dadd_rn(uni53(w.x, w.y), -0.5), V64 = uni53(w.z, w.w);
    const double us64 = __dadd_rn(0.5, -fabs(U64));
    const double lhs = __dadd_rn(__dadd_rn(log(V64), log(ia64)),
                                 -log(__dadd_rn(__ddiv_rn(a64, __dmul_rn(us64, us64)), b64)));
    const double rhs = __dadd_rn(__dadd_rn(-lam, __dmul_rn(k, ll64)), -lgamma(__dadd_rn(k, 1.0)));
    if (lhs <= rhs) return k;
  }
  return floor(__dadd_rn(lam, 0.5));
}

// ------------------------------------------------------------------ kernels

// Pixel response R = 1 + prnu z of every pixel (FP64, the fixed pattern; computed once per
// model, pattern seed and prnu and kept by the library).
__global__ void __launch_bounds__(256) k_prnu_map(double* R, int H, int W, int det, uint64_t pattern_seed, double prnu) {
  const int half = (W + 1) / 2;
  const int64_t n = (int64_t)H * half;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / half), c = (int)(t - (int64_t)r * half);
    double z0, z1;
    normal_pair(pattern_seed, (uint32_t)t, (uint32_t)det, 0, z0, z1);
    R[(int64_t)r * W + c] = __dadd_rn(1.0, __dmul_rn(prnu, z0));
    if (W - 1 - c != c) R[(int64_t)r * W + (W - 1 - c)] = __dadd_rn(1.0, __dmul_rn(prnu, z1));
  }
}

template <typename TI>
__device__ __forceinline__ double load_px(const TI* p) { return (double)*p; }

// One thread per mirror pair.  TO = double: electrons in FP64 (exact read-out noise);
// float: electrons rounded to FP32 (FP32 read-out noise, within a few ulp of FP64);
// uint16_t: ADU, exact (filtered, FP64 read-out noise where the rounding is too close).
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_noise(const NoiseArgs a, const TI* __restrict__ src, int64_t src_pitch,
                                               const double* __restrict__ R, TO* dst, int64_t dst_pitch, int H, int W,
                                               int det) {
  const int half = (W + 1) / 2;
  const int64_t n = (int64_t)H * half;
  const float inv_gain = (float)(1.0 / a.gain);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / half), c = (int)(t - (int64_t)r * half);
    const uint32_t q = (uint32_t)t;
    const int cm = W - 1 - c;
    const bool two = cm != c;
    const TI* srow = src + (int64_t)r * src_pitch;
    const double s0 = load_px(srow + c), s1 = two ? load_px(srow + cm) : 0.0;
    const double R0 = R ? R[(int64_t)r * W + c] : 1.0, R1 = (R && two) ? R[(int64_t)r * W + cm] : 1.0;
    double l0 = __dadd_rn(__dmul_rn(R0, s0), a.dark), l1 = __dadd_rn(__dmul_rn(R1, s1), a.dark);
    l0 = l0 > 0.0 ? l0 : 0.0;
    l1 = l1 > 0.0 ? l1 : 0.0;
    const double n0 = a.poisson ? poisson_filtered(l0, a.seed, q, (uint32_t)det, 0) : l0;
    const double n1 = (two && a.poisson) ? poisson_filtered(l1, a.seed, q, (uint32_t)det, 1) : l1;
    TO* drow = dst + (int64_t)r * dst_pitch;
    if constexpr (sizeof(TO) == 8) {  // FP64 electrons: exact read-out noise
      double g0, g1;
      normal_pair(a.seed, q, (uint32_t)det, 1, g0, g1);
      const double m0 = two ? __dadd_rn(n0, __dmul_rn(a.xtalk, n1)) : __dadd_rn(n0, 0.0);
      drow[c] = (TO)__dadd_rn(m0, __dmul_rn(a.ron, g0));
      if (two) drow[cm] = (TO)__dadd_rn(__dadd_rn(n1, __dmul_rn(a.xtalk, n0)), __dmul_rn(a.ron, g1));
    } else {
      float g0, g1, eg;
      normal_pair_f32(a.seed, q, (uint32_t)det, 1, g0, g1, eg);
      const float ron = (float)a.ron, xt = (float)a.xtalk;
      const float e0 = fmaf(ron, g0, fmaf(xt, two ? (float)n1 : 0.f, (float)n0));
      const float e1 = fmaf(ron, g1, fmaf(xt, (float)n0, (float)n1));
      if constexpr (sizeof(TO) == 4) {
        drow[c] = (TO)e0;
        if (two) drow[cm] = (TO)e1;
      } else {  // ADU = clamp(floor((bias + E / gain) + 1/2)), decided exactly
        const float ig = inv_gain, bias = (float)a.bias;
        bool exact = false;
        float t[2] = {fmaf(e0, ig, bias) + 0.5f, fmaf(e1, ig, bias) + 0.5f};
        const float ee[2] = {e0, e1};
        float v[2];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const float xn = fabsf(xt) * (float)(s2 ? n0 : n1);
          const float mt = fmaf(fmaf(fabsf(ee[s2]), 4e-7f, fmaf(fabsf(ron), eg, xn * 2e-7f)), ig,
                                fmaf(fabsf(t[s2]), 4e-7f, 1e-6f));
          const float lo = floorf(t[s2] - mt);
          exact = exact || (lo != floorf(t[s2] + mt));
          v[s2] = lo;
        }
        if (exact) {  // too close to a rounding boundary: FP64 read-out noise, as the definition
          double g0d, g1d;
          normal_pair(a.seed, q, (uint32_t)det, 1, g0d, g1d);
          const double m0 = two ? __dadd_rn(n0, __dmul_rn(a.xtalk, n1)) : __dadd_rn(n0, 0.0);
          const double m1 = __dadd_rn(n1, __dmul_rn(a.xtalk, n0));
          // clamped to [-1, 65536] first: integers there are exact in FP32
          const double vd0 = floor(__dadd_rn(__dadd_rn(a.bias, __ddiv_rn(__dadd_rn(m0, __dmul_rn(a.ron, g0d)), a.gain)), 0.5));
          const double vd1 = floor(__dadd_rn(__dadd_rn(a.bias, __ddiv_rn(__dadd_rn(m1, __dmul_rn(a.ron, g1d)), a.gain)), 0.5));
          v[0] = (float)fmin(fmax(vd0, -1.0), 65536.0);
          v[1] = (float)fmin(fmax(vd1, -1.0), 65536.0);
        }
        const float sat = (float)a.saturation;
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) v[s2] = fminf(fmaxf(v[s2], 0.f), sat);
        drow[c] = (TO)v[0];
        if (two) drow[cm] = (TO)v[1];
      }
    }
  }
}

static int64_t noise_blocks(int64_t n) {
  int64_t blocks = (n + 255) / 256;
  return blocks > 152 * 16 ? 152 * 16 : blocks;
}

template <typename TI, typename TO>
static cudaError_t launch_noise_t(const NoiseArgs& a, const void* src, int64_t sp, const double* R, void* dst,
                                  int64_t dp, int H, int W, int det, cudaStream_t st) {
  const int64_t n = (int64_t)H * ((W + 1) / 2);
  if (n == 0) return cudaSuccess;
  k_noise<TI, TO><<<(unsigned)noise_blocks(n), 256, 0, st>>>(a, (const TI*)src, sp, R, (TO*)dst, dp, H, W, det);
  return cudaGetLastError();
}

cudaError_t launch_prnu_map(double* R, int H, int W, int det, uint64_t pattern_seed, double prnu, cudaStream_t st) {
  const int64_t n = (int64_t)H * ((W + 1) / 2);
  if (n == 0) return cudaSuccess;
  k_prnu_map<<<(unsigned)noise_blocks(n), 256, 0, st>>>(R, H, W, det, pattern_seed, prnu);
  return cudaGetLastError();
}

cudaError_t launch_noise(uint64_t seed, uint64_t pattern_seed, double dark, double prnu, double ron, double xtalk,
                         double gain, double bias, int saturation, int poisson, int src_dtype, const void* src,
                         int64_t src_pitch, const double* R, int dst_dtype, void* dst, int64_t dst_pitch, int H, int W,
                         int det, cudaStream_t st) {
  const NoiseArgs a{seed, pattern_seed, dark, prnu, ron, xtalk, gain, bias, saturation, poisson};
#define E2E_N(SI, TI, DI, TO) \
  if (src_dtype == SI && dst_dtype == DI)  \
    return launch_noise_t<TI, TO>(a, src, src_pitch, R, dst, dst_pitch, H, W, det, st);
  E2E_N(0, float, 0, float) E2E_N(0, float, 1, double) E2E_N(0, float, 2, uint16_t)
  E2E_N(1, double, 0, float) E2E_N(1, double, 1, double) E2E_N(1, double, 2, uint16_t)
#undef E2E_N
  return cudaErrorInvalidValue;
}

}  // namespace e2e
