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
// same integers.  The kernels reach those decisions by filtered evaluation: they first
// compute each decided quantity in FP32 together with a bound on its distance from the FP64
// value; only when the FP32 value lies within that bound of the decision boundary (about one
// draw in 1e4 .. 1e5) is the draw redone in FP64.  Photon noise into FP32 electrons or ADU
// (the common case) runs in two passes: the first issues no FP64 instruction and lists the
// pairs it cannot decide, the second redoes only those pairs in FP64; FP64 electrons and
// expected values (no shot noise) take the one-pass kernel, which redoes draws inline.
#include <cstdint>

#include "e2e_kernels.h"
#include "philox.cuh"

namespace e2e {

struct NoiseArgs {
  uint64_t seed, pattern_seed;
  double dark, prnu, ron, xtalk, gain, bias;
  int saturation, poisson;
  float dark32, inv_gain32, ron32, xtalk32, bias32, sat32;  // FP32 copies for the filtered path
};

// ------------------------------------------------------------------ kernels

// Pixel response R = 1 + prnu z of every pixel (FP64, the fixed pattern; computed once per
// model, pattern seed and prnu and kept by the library).
__global__ void __launch_bounds__(256) k_prnu_map(double* R, float* R32, float* R32lo, int H, int W, int det,
                                                  uint64_t pattern_seed, double prnu) {
  const int half = (W + 1) / 2;
  const int64_t n = (int64_t)H * half;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / half), c = (int)(t - (int64_t)r * half);
    double z0, z1;
    normal_pair(pattern_seed, (uint32_t)t, (uint32_t)det, 0, z0, z1);
    const double r0 = __dadd_rn(1.0, __dmul_rn(prnu, z0)), r1 = __dadd_rn(1.0, __dmul_rn(prnu, z1));
    R[(int64_t)r * W + c] = r0;
    R32[(int64_t)r * W + c] = (float)r0;
    R32lo[(int64_t)r * W + c] = (float)(r0 - (double)(float)r0);  // R as a double-float pair
    if (W - 1 - c != c) {
      R[(int64_t)r * W + (W - 1 - c)] = r1;
      R32[(int64_t)r * W + (W - 1 - c)] = (float)r1;
      R32lo[(int64_t)r * W + (W - 1 - c)] = (float)(r1 - (double)(float)r1);
    }
  }
}

// One thread per mirror pair.  TO = double: electrons in FP64 (exact read-out noise);
// float: electrons rounded to FP32 (FP32 read-out noise, within a few ulp of FP64);
// uint16_t: ADU, exact (filtered, FP64 read-out noise where the rounding is too close).
// Eight CTAs per SM (32 registers, full occupancy): the draws are latency-bound (dependent
// Philox, transcendental and filter chains), and the resident warps outweigh the spills this
// costs.  A 9216^2 frame, minimum CTAs per SM 2 (90 registers) / 3 / 4 / 5 / 6 / 8:
// 2.05 / 1.68 / 1.55 / 1.47 / 1.42 / 1.35 ms, the same ADU bits each time.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256, 8) k_noise(const NoiseArgs a, const TI* __restrict__ src, int64_t src_pitch,
                                               const double* __restrict__ R, const float* __restrict__ R32, TO* dst,
                                               int64_t dst_pitch, int H, int W, int det) {
  const int half = (W + 1) / 2;
  const int n = H * half;  // < 2^31 (the launcher checks)
  const float inv_gain = a.inv_gain32;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int r = t / half, c = t - r * half;
    const uint32_t q = (uint32_t)t;
    const int cm = W - 1 - c;
    const bool two = cm != c;
    const TI* srow = src + (int64_t)r * src_pitch;
    const TI S0 = srow[c], S1 = two ? srow[cm] : (TI)0;
    const int64_t i0 = (int64_t)r * W + c, i1 = (int64_t)r * W + cm;
    // the mean lam = max(R S + dark, 0): exactly (FP64) when a decision needs it, else in FP32
    auto lam_exact0 = [&]() {
      const double l = __dadd_rn(__dmul_rn(R ? R[i0] : 1.0, (double)S0), a.dark);
      return l > 0.0 ? l : 0.0;
    };
    auto lam_exact1 = [&]() {
      const double l = __dadd_rn(__dmul_rn(R ? R[i1] : 1.0, (double)S1), a.dark);
      return l > 0.0 ? l : 0.0;
    };
    Count n0, n1{0, 0.f, 0.0};
    if (a.poisson) {
      const float rs0 = (R32 ? R32[i0] : 1.f) * (float)S0, rs1 = two ? (R32 ? R32[i1] : 1.f) * (float)S1 : 0.f;
      const float l0 = rs0 + a.dark32, l1 = rs1 + a.dark32;
      // |l - lam| <= 2.4e-7 (|R S| + dark): R and S rounded to FP32, one product, one sum (bound 6e-7)
      const float le0 = 6e-7f * (fabsf(rs0) + fabsf(a.dark32)) + 1e-37f;
      const float le1 = 6e-7f * (fabsf(rs1) + fabsf(a.dark32)) + 1e-37f;
      n0 = poisson_f32mean(l0, le0, lam_exact0, a.seed, q, (uint32_t)det, 2);
      if (two) n1 = poisson_f32mean(l1, le1, lam_exact1, a.seed, q, (uint32_t)det, 3);
    } else {
      n0 = exact_count(lam_exact0());
      n1 = exact_count(two ? lam_exact1() : 0.0);
    }
    TO* drow = dst + (int64_t)r * dst_pitch;
    if constexpr (sizeof(TO) == 8) {  // FP64 electrons: exact read-out noise
      double g0, g1;
      normal_pair(a.seed, q, (uint32_t)det, 1, g0, g1);
      const double m0 = two ? __dadd_rn(n0.f64(), __dmul_rn(a.xtalk, n1.f64())) : __dadd_rn(n0.f64(), 0.0);
      drow[c] = (TO)__dadd_rn(m0, __dmul_rn(a.ron, g0));
      if (two) drow[cm] = (TO)__dadd_rn(__dadd_rn(n1.f64(), __dmul_rn(a.xtalk, n0.f64())), __dmul_rn(a.ron, g1));
    } else {
      float g0, g1, eg;
      normal_pair_f32(a.seed, q, (uint32_t)det, 1, g0, g1, eg);
      const float ron = a.ron32, xt = a.xtalk32, nf0 = n0.f32(), nf1 = n1.f32();
      const float e0 = fmaf(ron, g0, fmaf(xt, two ? nf1 : 0.f, nf0));
      const float e1 = fmaf(ron, g1, fmaf(xt, nf0, nf1));
      if constexpr (sizeof(TO) == 4) {
        drow[c] = (TO)e0;
        if (two) drow[cm] = (TO)e1;
      } else {  // ADU = clamp(floor((bias + E / gain) + 1/2)), decided exactly
        const float ig = inv_gain, bias = a.bias32;
        bool exact = false;
        float t[2] = {fmaf(e0, ig, bias) + 0.5f, fmaf(e1, ig, bias) + 0.5f};
        const float ee[2] = {e0, e1};
        float v[2];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const float xn = fabsf(xt) * (s2 ? nf0 : nf1);
          const float mt = fmaf(fmaf(fabsf(ee[s2]), 4e-7f, fmaf(fabsf(ron), eg, xn * 2e-7f)), ig,
                                fmaf(fabsf(t[s2]), 4e-7f, 1e-6f));
          const float lo = floorf(t[s2] - mt);
          exact = exact || (lo != floorf(t[s2] + mt));
          v[s2] = lo;
        }
        if (exact) {  // too close to a rounding boundary: FP64 read-out noise, as the definition
          double g0d, g1d;
          normal_pair(a.seed, q, (uint32_t)det, 1, g0d, g1d);
          const double d0 = n0.f64(), d1 = n1.f64();
          const double m0 = two ? __dadd_rn(d0, __dmul_rn(a.xtalk, d1)) : __dadd_rn(d0, 0.0);
          const double m1 = __dadd_rn(d1, __dmul_rn(a.xtalk, d0));
          // clamped to [-1, 65536] first: integers there are exact in FP32
          const double vd0 = floor(__dadd_rn(__dadd_rn(a.bias, __ddiv_rn(__dadd_rn(m0, __dmul_rn(a.ron, g0d)), a.gain)), 0.5));
          const double vd1 = floor(__dadd_rn(__dadd_rn(a.bias, __ddiv_rn(__dadd_rn(m1, __dmul_rn(a.ron, g1d)), a.gain)), 0.5));
          v[0] = (float)fmin(fmax(vd0, -1.0), 65536.0);
          v[1] = (float)fmin(fmax(vd1, -1.0), 65536.0);
        }
        const float sat = a.sat32;
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) v[s2] = fminf(fmaxf(v[s2], 0.f), sat);
        drow[c] = (TO)v[0];
        if (two) drow[cm] = (TO)v[1];
      }
    }
  }
}

// ------------------------------------------------------------------ two-pass form
//
// Photon noise into FP32 electrons or ADU (the common case): a first pass decides every pair
// in FP32 and double-float arithmetic alone -- the mean lam = R S + dark as a double-float from
// the response map's (hi, lo) words, inversion below 10, PTRS from 10 up with its slow
// acceptance test bounded too, the ADU rounding -- and appends the pairs where some comparison
// is too close to call to a list, writing nothing for them.  A second pass redoes the listed
// pairs entirely in FP64 (the definition).  So the first pass issues no FP64 instruction (FP32
// sources; an FP64 source is split into a double-float), and the FP64 work runs densely, one
// listed pair per thread.

// lam = max(R S + dark, 0) as a double-float (lh, ll) and a bound le on its distance from the
// FP64 definition's value (both within ~2^-44 of the exact product and sum).
__device__ __forceinline__ void mean_df(float rh, float rl, float sh, float sl, float dh, float dl, float& lh,
                                        float& ll, float& le) {
  const float ph = rh * sh;
  const float pe = fmaf(rh, sl, fmaf(rl, sh, fmaf(rh, sh, -ph)));
  const float t = ph + dh;
  const float bb = t - ph;
  const float e = ((ph - (t - bb)) + (dh - bb)) + (pe + dl);
  lh = t + e;
  ll = e - (lh - t);
  le = fmaf(1e-13f, fabsf(ph) + fabsf(dh), 1e-37f);
}

template <typename TI>
__device__ __forceinline__ void split_src(TI v, float& h, float& l) {
  if constexpr (sizeof(TI) == 4) {
    h = v;
    l = 0.f;
  } else {
    h = (float)v;
    l = (float)(v - (double)h);
  }
}

// Poisson count of mean (lh, ll) +- le decided in FP32, or -1.
__device__ __forceinline__ int count_f32(float lh, float ll, float le, uint64_t seed, uint32_t q, uint32_t d,
                                         uint32_t stream) {
  if (lh + le <= 0.f) return 0;  // the mean is <= 0: no photons
  if (lh - le <= 0.f) return -1;
  if (lh + le < 10.f) return inversion_f32(lh, 6e-8f + le / lh, seed, q, d, stream);
  if (lh - le < 10.f) return -1;  // which sampler applies is too close to call
  float Lf = floorf(lh), frac = (lh - Lf) + ll;
  if (frac < 0.f) {
    Lf -= 1.f;
    frac += 1.f;
  } else if (frac >= 1.f) {
    Lf += 1.f;
    frac -= 1.f;
  }
  return ptrs_f32(Lf, frac, le, seed, q, d, stream);
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(256, 8) k_noise_first(const NoiseArgs a, const TI* __restrict__ src,
                                                     int64_t src_pitch, const float* __restrict__ R32,
                                                     const float* __restrict__ R32lo, TO* dst, int64_t dst_pitch,
                                                     int H, int W, int det, unsigned* __restrict__ list,
                                                     unsigned* __restrict__ n_list, float dark_lo) {
  const int half = (W + 1) / 2;
  const int n = H * half;  // < 2^31 (the launcher checks)
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int r = t / half, c = t - r * half;
    const uint32_t q = (uint32_t)t;
    const int cm = W - 1 - c;
    const bool two = cm != c;
    const TI* srow = src + (int64_t)r * src_pitch;
    const int64_t i0 = (int64_t)r * W + c, i1 = (int64_t)r * W + cm;
    float sh0, sl0, sh1 = 0.f, sl1 = 0.f;
    split_src(srow[c], sh0, sl0);
    if (two) split_src(srow[cm], sh1, sl1);
    float lh, ll, le;
    mean_df(R32 ? R32[i0] : 1.f, R32 ? R32lo[i0] : 0.f, sh0, sl0, a.dark32, dark_lo, lh, ll, le);
    const int k0 = count_f32(lh, ll, le, a.seed, q, (uint32_t)det, 2);
    int k1 = 0;
    if (two) {
      mean_df(R32 ? R32[i1] : 1.f, R32 ? R32lo[i1] : 0.f, sh1, sl1, a.dark32, dark_lo, lh, ll, le);
      k1 = count_f32(lh, ll, le, a.seed, q, (uint32_t)det, 3);
    }
    bool defer = k0 < 0 || k1 < 0;
    float v[2] = {0.f, 0.f};
    if (!defer) {
      float g0, g1, eg;
      normal_pair_f32(a.seed, q, (uint32_t)det, 1, g0, g1, eg);
      const float ron = a.ron32, xt = a.xtalk32, nf0 = (float)k0, nf1 = (float)k1;
      const float e0 = fmaf(ron, g0, fmaf(xt, two ? nf1 : 0.f, nf0));
      const float e1 = fmaf(ron, g1, fmaf(xt, nf0, nf1));
      if constexpr (sizeof(TO) == 4) {
        v[0] = e0;
        v[1] = e1;
      } else {  // ADU = clamp(floor((bias + E / gain) + 1/2)), decided exactly or deferred
        const float ig = a.inv_gain32, bias = a.bias32;
        const float tt[2] = {fmaf(e0, ig, bias) + 0.5f, fmaf(e1, ig, bias) + 0.5f};
        const float ee[2] = {e0, e1};
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const float xn = fabsf(xt) * (s2 ? nf0 : nf1);
          const float mt = fmaf(fmaf(fabsf(ee[s2]), 4e-7f, fmaf(fabsf(ron), eg, xn * 2e-7f)), ig,
                                fmaf(fabsf(tt[s2]), 4e-7f, 1e-6f));
          const float lo = floorf(tt[s2] - mt);
          defer = defer || (lo != floorf(tt[s2] + mt));
          v[s2] = fminf(fmaxf(lo, 0.f), a.sat32);
        }
      }
    }
    if (defer) {
      list[atomicAdd(n_list, 1u)] = q;
      continue;
    }
    TO* drow = dst + (int64_t)r * dst_pitch;
    drow[c] = (TO)v[0];
    if (two) drow[cm] = (TO)v[1];
  }
}

// The listed pairs, entirely in FP64: the definition (exact counts, FP64 normals, exact ADU).
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_noise_redo(const NoiseArgs a, const TI* __restrict__ src, int64_t src_pitch,
                                                  const double* __restrict__ R, TO* dst, int64_t dst_pitch, int H,
                                                  int W, int det, const unsigned* __restrict__ list,
                                                  const unsigned* __restrict__ n_list) {
  const int half = (W + 1) / 2;
  const unsigned nl = *n_list;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < nl; e += gridDim.x * blockDim.x) {
    const int t = (int)list[e];
    const int r = t / half, c = t - r * half;
    const uint32_t q = (uint32_t)t;
    const int cm = W - 1 - c;
    const bool two = cm != c;
    const TI* srow = src + (int64_t)r * src_pitch;
    const int64_t i0 = (int64_t)r * W + c, i1 = (int64_t)r * W + cm;
    const double l0 = __dadd_rn(__dmul_rn(R ? R[i0] : 1.0, (double)srow[c]), a.dark);
    const double d0 = poisson_draw(l0 > 0.0 ? l0 : 0.0, a.seed, q, (uint32_t)det, 2);
    double d1 = 0.0;
    if (two) {
      const double l1 = __dadd_rn(__dmul_rn(R ? R[i1] : 1.0, (double)srow[cm]), a.dark);
      d1 = poisson_draw(l1 > 0.0 ? l1 : 0.0, a.seed, q, (uint32_t)det, 3);
    }
    double g0, g1;
    normal_pair(a.seed, q, (uint32_t)det, 1, g0, g1);
    const double m0 = two ? __dadd_rn(d0, __dmul_rn(a.xtalk, d1)) : __dadd_rn(d0, 0.0);
    const double m1 = __dadd_rn(d1, __dmul_rn(a.xtalk, d0));
    const double E0 = __dadd_rn(m0, __dmul_rn(a.ron, g0)), E1 = __dadd_rn(m1, __dmul_rn(a.ron, g1));
    TO* drow = dst + (int64_t)r * dst_pitch;
    if constexpr (sizeof(TO) == 4) {
      drow[c] = (TO)E0;
      if (two) drow[cm] = (TO)E1;
    } else {
      const double vd0 = floor(__dadd_rn(__dadd_rn(a.bias, __ddiv_rn(E0, a.gain)), 0.5));
      const double vd1 = floor(__dadd_rn(__dadd_rn(a.bias, __ddiv_rn(E1, a.gain)), 0.5));
      drow[c] = (TO)fmin(fmax(vd0, 0.0), (double)a.saturation);
      if (two) drow[cm] = (TO)fmin(fmax(vd1, 0.0), (double)a.saturation);
    }
  }
}

static int64_t grid_blocks(int64_t n) {
  int64_t blocks = (n + 255) / 256;
  return blocks > 152 * 16 ? 152 * 16 : blocks;
}

template <typename TI, typename TO>
static cudaError_t launch_noise_t(const NoiseArgs& a, const void* src, int64_t sp, const double* R, const float* R32,
                                  void* dst, int64_t dp, int H, int W, int det, cudaStream_t st) {
  const int64_t n = (int64_t)H * ((W + 1) / 2);
  if (n == 0) return cudaSuccess;
  if (n > INT32_MAX - 256 * grid_blocks(n)) return cudaErrorInvalidValue;  // the kernel indexes in 32 bits
  k_noise<TI, TO><<<(unsigned)grid_blocks(n), 256, 0, st>>>(a, (const TI*)src, sp, R, R32, (TO*)dst, dp, H, W, det);
  return cudaGetLastError();
}

cudaError_t launch_prnu_map(double* R, float* R32, float* R32lo, int H, int W, int det, uint64_t pattern_seed,
                            double prnu, cudaStream_t st) {
  const int64_t n = (int64_t)H * ((W + 1) / 2);
  if (n == 0) return cudaSuccess;
  k_prnu_map<<<(unsigned)grid_blocks(n), 256, 0, st>>>(R, R32, R32lo, H, W, det, pattern_seed, prnu);
  return cudaGetLastError();
}

template <typename TI, typename TO>
static cudaError_t launch_two_pass_t(const NoiseArgs& a, float dark_lo, const void* src, int64_t sp, const double* R,
                                     const float* R32, const float* R32lo, void* dst, int64_t dp, int H, int W,
                                     int det, unsigned* list, unsigned* n_list, cudaStream_t st) {
  const int64_t n = (int64_t)H * ((W + 1) / 2);
  if (n == 0) return cudaSuccess;
  if (n > INT32_MAX - 256 * grid_blocks(n)) return cudaErrorInvalidValue;  // the kernel indexes in 32 bits
  cudaError_t e = cudaMemsetAsync(n_list, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_noise_first<TI, TO><<<(unsigned)grid_blocks(n), 256, 0, st>>>(a, (const TI*)src, sp, R32, R32lo, (TO*)dst, dp, H,
                                                                   W, det, list, n_list, dark_lo);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_noise_redo<TI, TO><<<152 * 4, 256, 0, st>>>(a, (const TI*)src, sp, R, (TO*)dst, dp, H, W, det, list, n_list);
  return cudaGetLastError();
}

cudaError_t launch_noise_two_pass(uint64_t seed, uint64_t pattern_seed, double dark, double prnu, double ron,
                                  double xtalk, double gain, double bias, int saturation, int src_dtype,
                                  const void* src, int64_t src_pitch, const double* R, const float* R32,
                                  const float* R32lo, int dst_dtype, void* dst, int64_t dst_pitch, int H, int W,
                                  int det, unsigned* list, unsigned* n_list, cudaStream_t st) {
  const NoiseArgs a{seed,        pattern_seed, dark,        prnu,        ron,         xtalk,
                    gain,        bias,         saturation,  1,           (float)dark, (float)(1.0 / gain),
                    (float)ron,  (float)xtalk, (float)bias, (float)saturation};
  const float dark_lo = (float)(dark - (double)(float)dark);
#define E2E_N(SI, TI, DI, TO) \
  if (src_dtype == SI && dst_dtype == DI)  \
    return launch_two_pass_t<TI, TO>(a, dark_lo, src, src_pitch, R, R32, R32lo, dst, dst_pitch, H, W, det, list, n_list, st);
  E2E_N(0, float, 0, float) E2E_N(0, float, 2, uint16_t) E2E_N(1, double, 0, float) E2E_N(1, double, 2, uint16_t)
#undef E2E_N
  return cudaErrorInvalidValue;
}

cudaError_t launch_noise(uint64_t seed, uint64_t pattern_seed, double dark, double prnu, double ron, double xtalk,
                         double gain, double bias, int saturation, int poisson, int src_dtype, const void* src,
                         int64_t src_pitch, const double* R, const float* R32, int dst_dtype, void* dst,
                         int64_t dst_pitch, int H, int W, int det, cudaStream_t st) {
  const NoiseArgs a{seed,        pattern_seed, dark,        prnu,        ron,         xtalk,
                    gain,        bias,         saturation,  poisson,     (float)dark, (float)(1.0 / gain),
                    (float)ron,  (float)xtalk, (float)bias, (float)saturation};
#define E2E_N(SI, TI, DI, TO) \
  if (src_dtype == SI && dst_dtype == DI)  \
    return launch_noise_t<TI, TO>(a, src, src_pitch, R, R32, dst, dst_pitch, H, W, det, st);
  E2E_N(0, float, 0, float) E2E_N(0, float, 1, double) E2E_N(0, float, 2, uint16_t)
  E2E_N(1, double, 0, float) E2E_N(1, double, 1, double) E2E_N(1, double, 2, uint16_t)
#undef E2E_N
  return cudaErrorInvalidValue;
}

}  // namespace e2e
