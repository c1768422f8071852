// Counter-based random numbers of the detector-noise and photon kernels: Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, SC'11), 53-bit uniforms, Box-Muller normals and Poisson draws
// (sequential inversion below 10, Hormann's PTRS from 10 up).  Each sampler comes twice: an
// exact FP64 form (the definition, explicitly rounded, no FMA contraction), and an FP32 form
// that carries a bound on its distance from the exact one and falls back to it whenever a
// decision is too close to call, so both return the same integers.
#pragma once
#include <cstdint>

namespace e2e {

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

__device__ __forceinline__ uint4 rng_block(uint64_t seed, uint32_t q, uint32_t d, uint32_t i, uint32_t stream) {
  return philox4x32_10(make_uint4(q, d, i, stream), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Uniform on (0, 1) from two words; every step is exact.
__device__ __forceinline__ double uni53(uint32_t a, uint32_t b) {
  return __dadd_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)), 0.5) *
         (1.0 / 9007199254740992.0);
}

// Exact FP64 Box-Muller pair from block (q, d, i, stream).
__device__ __forceinline__ void normal_pair_ctr(uint64_t seed, uint32_t q, uint32_t d, uint32_t i, uint32_t stream,
                                                double& left, double& right) {
  const uint4 w = rng_block(seed, q, d, i, stream);
  const double rho = sqrt(__dmul_rn(-2.0, log(uni53(w.x, w.y))));
  const double ph = __dmul_rn(2.0 * 3.14159265358979323846, uni53(w.z, w.w));
  double s, c;
  sincos(ph, &s, &c);
  left = __dmul_rn(rho, c);
  right = __dmul_rn(rho, s);
}

__device__ __forceinline__ void normal_pair(uint64_t seed, uint32_t q, uint32_t d, uint32_t stream, double& left,
                                            double& right) {
  normal_pair_ctr(seed, q, d, 0, stream, left, right);
}

// Exact FP64 Poisson draw from blocks (q, d, trial, stream): the definition, step by step.
static __device__ double poisson_draw(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t stream) {
  if (!(lam > 0.0)) return 0.0;
  if (lam < 10.0) {
    const uint4 w = rng_block(seed, q, d, 0, stream);
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
    const uint4 w = rng_block(seed, q, d, i, stream);
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

// The 53-bit uniform u = A 2^-27 + (B + 1/2) 2^-53, A = a >> 5 (27 bits), B = b >> 6 (26 bits),
// in FP32 from two 32-bit conversions and two FMAs: the conversion of A, the conversion of B
// and each FMA round once, so |fl - u| <= 2^-23 u (+ a term below 2^-77).  And 1 - u, which
// has the same form with A' = 2^27 - 1 - A, B' = 2^26 - 1 - B, so it keeps its relative
// accuracy as u approaches 1.  (No 64-bit integer arithmetic: the FP32 samplers never touch
// the FP64 unit.)
__device__ __forceinline__ float uni53_parts_f32(uint32_t A, uint32_t B) {
  return fmaf(__uint2float_rn(A), 0x1p-27f, fmaf(__uint2float_rn(B), 0x1p-53f, 0x1p-54f));
}
__device__ __forceinline__ float uni53_f32(uint32_t a, uint32_t b) { return uni53_parts_f32(a >> 5, b >> 6); }
__device__ __forceinline__ float one_minus_uni53_f32(uint32_t a, uint32_t b) {
  return uni53_parts_f32(0x7FFFFFFu - (a >> 5), 0x3FFFFFFu - (b >> 6));
}

// Box-Muller pair in FP32 and a bound eg on |g - g_exact| for both members: ln u from logf
// (u < 1/2) or log1pf(-(1 - u)) (u >= 1/2), 1 ulp, of an argument within 2^-23 relative; the
// phase from sincospif(2u), 1 ulp, whose argument is within 2.4e-7 u of 2u (a phase error
// below 7.5e-7 rho in g).  Summed: |g - g_exact| < 1.1e-6 rho + 1e-7.
__device__ __forceinline__ void normal_pair_f32_ctr(uint64_t seed, uint32_t q, uint32_t d, uint32_t i,
                                                    uint32_t stream, float& g0, float& g1, float& eg) {
  const uint4 w = rng_block(seed, q, d, i, stream);
  const float u1 = uni53_f32(w.x, w.y);
  const float ln = u1 < 0.5f ? logf(u1) : log1pf(-one_minus_uni53_f32(w.x, w.y));
  const float rho = sqrtf(-2.f * ln);
  float s, c;
  sincospif(2.f * uni53_f32(w.z, w.w), &s, &c);
  g0 = rho * c;
  g1 = rho * s;
  eg = fmaf(rho, 2e-6f, 1e-7f);  // also covers a 2e-7 relative rounding of products with g
}

__device__ __forceinline__ void normal_pair_f32(uint64_t seed, uint32_t q, uint32_t d, uint32_t stream, float& g0,
                                                float& g1, float& eg) {
  normal_pair_f32_ctr(seed, q, d, 0, stream, g0, g1, eg);
}

// Poisson draw with the exact function's integer result, from FP32 arithmetic whenever its
// error bound decides every comparison (see the file comment).
// Sequential-inversion Poisson draw in FP32 for a mean l known to relative accuracy lrel:
// F_k within F (8.4e-7 + 2.4e-7 k) of the FP64 sums plus F (k + l) lrel for the mean's own
// error, u within 2^-23 relative; all bounds doubled.  Returns the count, or -1 when some
// comparison is too close to call (the caller then draws exactly).
static __device__ int inversion_f32(float l, float lrel, uint64_t seed, uint32_t q, uint32_t d, uint32_t stream) {
  const uint4 w = rng_block(seed, q, d, 0, stream);
  const float u = uni53_f32(w.x, w.y);
  float p = expf(-l), F = p;
  for (int k = 0; k < 200; ++k) {
    const float rel = fmaf(1e-6f, (float)k, 4e-6f) + 2.f * ((float)k + l) * lrel;
    const float tol = fmaf(F, rel, fmaf(u, 2.5e-7f, 1e-12f));
    const float diff = u - F;
    if (diff > tol) {  // u > F_k: one more
      p = p * (l / (float)(k + 1));
      F = F + p;
      continue;
    }
    if (-diff > tol) return k;  // u <= F_k
    return -1;
  }
  return 200;
}

static __device__ double poisson_filtered(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t stream) {
  if (!(lam > 0.0)) return 0.0;
  const float l = __double2float_rn(lam);
  if (lam < 10.0) {
    const int k = inversion_f32(l, 6e-8f, seed, q, d, stream);
    return k >= 0 ? (double)k : poisson_draw(lam, seed, q, d, stream);
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
    const uint4 w = rng_block(seed, q, d, i, stream);
    const float U = uni53_f32(w.x, w.y) - 0.5f, V = uni53_f32(w.z, w.w);
    const float us = 0.5f - fabsf(U);  // within 1.2e-7 of the exact us (u within 2^-23 u)
    const float T = 2.f * a / us + b;
    const float y = T * U;
    const float yerr = fabsf(T) * fmaf(fabsf(U), fmaf(3e-7f, 1.f / us, 4e-6f), 2e-7f) + 1e-6f;
    const float xr = (y + lf) + 0.43f;
    const float xe = yerr + fmaf(fabsf(xr), 2.5e-7f, 1e-7f);
    const float kr = floorf(xr - xe);
    if (floorf(xr + xe) != kr) return poisson_draw(lam, seed, q, d, stream);
    const double k = Li + (double)kr;
    // quick acceptance: us >= 0.07 && V <= vr
    const float mu = 3e-7f, mv = 8e-7f;
    const bool c1t = us - 0.07f > mu, c1f = 0.07f - us > mu, c2t = vr - V > mv, c2f = V - vr > mv;
    if (c1t && c2t) return k;
    if (!(c1f || c2f)) return poisson_draw(lam, seed, q, d, stream);
    // rejection: k < 0 || (us < 0.013 && V > us)
    if (k < 0.0) continue;
    const bool d1t = 0.013f - us > mu, d1f = us - 0.013f > mu, d2t = V - us > mu, d2f = us - V > mu;
    if (d1t && d2t) continue;
    if (!(d1f || d2f)) return poisson_draw(lam, seed, q, d, stream);
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

// ------------------------------------------------------------------ FP32 only (no FP64)
//
// The first pass of the noise stage decides draws in FP32 alone and defers the rest to an
// exact FP64 pass over a compacted list; these helpers return -1 for "too close to call".

// log of the Poisson pmf at k >= 0, -lam + k ln lam - lgamma(k + 1), for lam >= 10 given as
// Lf + frac (Lf an integer, frac in [0, 1)), and a bound on its error.  For n = k + 1 >= 10 the
// Stirling series in the well-conditioned form
//   -lam phi(x) + log1p(x) - ln(n)/2 - ln(2 pi)/2 - 1/(12n) + 1/(360n^3) - 1/(1260n^5),
//   x = (n - lam)/lam,  phi(x) = (1 + x) log1p(x) - x,
// (phi by its alternating series sum_j (-1)^j x^j / (j (j - 1)) for |x| < 1/4), which never
// subtracts terms of the size of lam; below, the direct form with lgammaf.
__device__ __forceinline__ float log_poisson_pmf_f32(float kr, float Lf, float frac, float& err) {
  const float lam = Lf + frac;
  const float n = Lf + kr + 1.f;  // k + 1, exact (integers below 2^24)
  if (n >= 10.f) {
    const float D = (kr + 1.f) - frac;  // n - lam, one rounding
    const float x = D / lam;
    float phi;
    if (fabsf(x) < 0.25f) {
      float t = -1.f / 132.f;  // j = 12
      t = fmaf(t, x, 1.f / 110.f);
      t = fmaf(t, x, -1.f / 90.f);
      t = fmaf(t, x, 1.f / 72.f);
      t = fmaf(t, x, -1.f / 56.f);
      t = fmaf(t, x, 1.f / 42.f);
      t = fmaf(t, x, -1.f / 30.f);
      t = fmaf(t, x, 1.f / 20.f);
      t = fmaf(t, x, -1.f / 12.f);
      t = fmaf(t, x, 1.f / 6.f);
      t = fmaf(t, -x, 0.5f);  // 1/2 - x/6 + x^2/12 - ...
      phi = x * x * t;
    } else {
      phi = fmaf(1.f + x, log1pf(x), -x);
    }
    const float in = 1.f / n, in2 = in * in;
    const float c = in * fmaf(in2, fmaf(in2, -1.f / 1260.f, 1.f / 360.f), -1.f / 12.f);  // -(1/12n - ...)
    const float lp = fmaf(-lam, phi, log1pf(x)) + fmaf(-0.5f, logf(n), -0.918938533f) + c;
    err = fmaf(2e-5f, fabsf(lam * phi), 2e-5f);
    return lp;
  }
  const float lp = fmaf(kr + Lf, logf(lam), -lam) - lgammaf(n);
  err = fmaf(1e-6f, lam + (kr + Lf) * fabsf(logf(lam)), 5e-5f);
  return lp;
}

// Hormann's PTRS in FP32 for lam = Lf + frac >= 10 known to le: the count, or -1 when a
// comparison (the floor that makes k, the quick acceptance, the rejection, the slow
// acceptance test) is too close to call, or 64 trials pass.
static __device__ int ptrs_f32(float Lf, float frac, float le, uint64_t seed, uint32_t q, uint32_t d,
                               uint32_t stream) {
  const float l = Lf + frac;
  const float sl = sqrtf(l);
  const float b = fmaf(2.53f, sl, 0.931f);
  const float a = fmaf(0.02483f, b, -0.059f);
  const float vr = 0.9277f - 3.6224f / (b - 2.f);
  const float lia = logf(1.1239f + 1.1328f / (b - 3.4f));  // ln(1 / alpha)
  for (uint32_t i = 0; i < 64; ++i) {
    const uint4 w = rng_block(seed, q, d, i, stream);
    const float U = uni53_f32(w.x, w.y) - 0.5f, V = uni53_f32(w.z, w.w);
    const float us = 0.5f - fabsf(U);
    const float T = 2.f * a / us + b;
    const float y = T * U;
    const float yerr = fabsf(T) * fmaf(fabsf(U), fmaf(3e-7f, 1.f / us, 4e-6f), 2e-7f) + 1e-6f;
    const float xr = (y + frac) + 0.43f;
    const float xe = yerr + fmaf(fabsf(xr), 2.5e-7f, 1e-7f) + le;
    const float kr = floorf(xr - xe);
    if (floorf(xr + xe) != kr) return -1;
    const float mu = 3e-7f, mv = 8e-7f;
    const bool c1t = us - 0.07f > mu, c1f = 0.07f - us > mu, c2t = vr - V > mv, c2f = V - vr > mv;
    if (c1t && c2t) return (int)(Lf + kr);
    if (!(c1f || c2f)) return -1;
    if (Lf + kr < 0.f) continue;
    const bool d1t = 0.013f - us > mu, d1f = us - 0.013f > mu, d2t = V - us > mu, d2f = us - V > mu;
    if (d1t && d2t) continue;
    if (!(d1f || d2f)) return -1;
    // slow acceptance: ln V + ln(1/alpha) - ln(a / us^2 + b) <= ln p(k)
    const float lhs = logf(V) + lia - logf(a / (us * us) + b);
    const float elhs = fmaf(1e-6f, fabsf(lhs), 6e-6f) + 3e-7f / us;
    float erhs;
    const float rhs = log_poisson_pmf_f32(kr, Lf, frac, erhs);
    if (lhs + elhs < rhs - erhs) return (int)(Lf + kr);
    if (lhs - elhs > rhs + erhs) continue;
    return -1;
  }
  return -1;
}

// A Poisson count: k when the FP32 draw decided it, else (k < 0) the FP64 value x.
struct Count {
  int k;
  float xf;
  double x;
  __device__ float f32() const { return k >= 0 ? (float)k : xf; }
  __device__ double f64() const { return k >= 0 ? (double)k : x; }
};
__device__ __forceinline__ Count exact_count(double x) { return Count{-1, (float)x, x}; }

// Poisson draw whose mean is known in FP32 (l within le of it), with the exact mean computed
// only when needed (lam_exact(): FP64, the definition's value): dim means never touch FP64.
template <typename LamExact>
static __device__ Count poisson_f32mean(float l, float le, LamExact lam_exact, uint64_t seed, uint32_t q, uint32_t d,
                                        uint32_t stream) {
  if (l + le <= 0.f) return Count{0, 0.f, 0.0};  // the mean is <= 0: no photons
  if (l - le > 0.f && l + le < 10.f) {
    const int k = inversion_f32(l, le / l, seed, q, d, stream);
    if (k >= 0) return Count{k, 0.f, 0.0};
  }
  return exact_count(poisson_filtered(lam_exact(), seed, q, d, stream));
}

}  // namespace e2e
