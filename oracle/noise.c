/*
 * Detector noise stage of the synthetic echellogram -- TEST INFRASTRUCTURE ONLY (oracle).
 *
 * Sec. 2.2 ends the simulation by adding photon noise and the detector's own noises --
 * dark current, read-out noise, non-uniform pixel response and cross-talk -- to the final
 * synthetic frame.  The paper gives no formulas.  The reading written out here (and,
 * independently, by the GPU kernel) is, for detector d of width W and pixel (r, c):
 *
 *   R      = 1 + prnu * z                    pixel response (fixed pattern, pattern seed)
 *   lam    = max(R * S + dark, 0)            expected electrons, S = the rendered frame
 *   N      ~ Poisson(lam)                    photon and dark shot noise (or N = lam)
 *   M      = N + xtalk * N'                  N' = the mirror pixel (r, W-1-c), read by the
 *                                            other amplifier of a two-output detector; the
 *                                            middle column of an odd width has no mirror
 *   E      = M + ron * g                     electrons after read-out
 *   ADU    = clamp(floor(bias + E / gain + 1/2), 0, saturation)
 *
 * Random numbers are counter based (Philox4x32-10, Salmon, Moraes, Dror and Shaw, SC'11),
 * so every draw is a pure function of (key, counter) and the GPU can draw any pixel in any
 * order.  Pixels are visited in mirror pairs q = r * ceil(W/2) + c, c < ceil(W/2):
 *
 *   z (left, right) = Box-Muller of block (key = pattern seed, counter = (q, d, 0, 0))
 *   g (left, right) = Box-Muller of block (key = seed,         counter = (q, d, 0, 1))
 *   N of side s     : blocks (key = seed, counter = (q, d, i, 2 + s)), i = 0, 1, ...
 *
 * A block is four 32-bit words w0..w3; u(a, b) = ((a >> 5) 2^26 + (b >> 6) + 1/2) 2^-53 is
 * a uniform on (0, 1).  Box-Muller: rho = sqrt(-2 ln u(w0, w1)), phase = 2 pi u(w2, w3),
 * left = rho cos(phase), right = rho sin(phase).  Poisson: for lam < 10, inversion by
 * sequential search with u(w0, w1) of block 0; for lam >= 10, Hormann's transformed
 * rejection with squeeze (PTRS, Insurance Math. Econom. 12 (1993) 39-45), one block per
 * trial (U = u(w0, w1) - 1/2, V = u(w2, w3)), at most 64 trials (then round(lam)).
 * Every decision is taken in FP64.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>

#define NOISE_PI 3.14159265358979323846

/* Philox4x32-10: ten rounds of the bijection, the key bumped by the Weyl constants between
 * rounds (SC'11, Sec. 3.2). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

double oracle_uniform53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) / 9007199254740992.0;
}
#define uni oracle_uniform53

void oracle_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t w[4]) {
  const uint32_t ctr[4] = {c0, c1, c2, c3};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, w);
}
#define block oracle_block

void oracle_normal_pair_ctr(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double* left,
                            double* right) {
  uint32_t w[4];
  block(seed, c0, c1, c2, c3, w);
  const double rho = sqrt(-2.0 * log(uni(w[0], w[1])));
  const double ph = 2.0 * NOISE_PI * uni(w[2], w[3]);
  *left = rho * cos(ph);
  *right = rho * sin(ph);
}

void oracle_normal_pair(uint64_t seed, uint32_t q, uint32_t d, uint32_t stream, double* left, double* right) {
  uint32_t w[4];
  block(seed, q, d, 0, stream, w);
  const double rho = sqrt(-2.0 * log(uni(w[0], w[1])));
  const double ph = 2.0 * NOISE_PI * uni(w[2], w[3]);
  *left = rho * cos(ph);
  *right = rho * sin(ph);
}

long oracle_poisson(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t side) {
  return oracle_poisson_stream(lam, seed, q, d, 2 + side);
}

long oracle_poisson_stream(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t stream) {
  if (!(lam > 0.0)) return 0;
  uint32_t w[4];
  if (lam < 10.0) {
    block(seed, q, d, 0, stream, w);
    const double u = uni(w[0], w[1]);
    long k = 0;
    double p = exp(-lam), F = p;
    while (u > F && k < 200) {
      ++k;
      p *= lam / (double)k;
      F += p;
    }
    return k;
  }
  const double slam = sqrt(lam), loglam = log(lam);
  const double b = 0.931 + 2.53 * slam;
  const double a = -0.059 + 0.02483 * b;
  const double invalpha = 1.1239 + 1.1328 / (b - 3.4);
  const double vr = 0.9277 - 3.6224 / (b - 2.0);
  for (uint32_t i = 0; i < 64; ++i) {
    block(seed, q, d, i, stream, w);
    const double U = uni(w[0], w[1]) - 0.5, V = uni(w[2], w[3]);
    const double us = 0.5 - fabs(U);
    const double k = floor((2.0 * a / us + b) * U + lam + 0.43);
    if (us >= 0.07 && V <= vr) return (long)k;
    if (k < 0.0 || (us < 0.013 && V > us)) continue;
    if (log(V) + log(invalpha) - log(a / (us * us) + b) <= -lam + k * loglam - lgamma(k + 1.0)) return (long)k;
  }
  return (long)floor(lam + 0.5);
}

int oracle_add_noise(int H, int W, int row0, int det, const double* S, const oracle_noise* p, double* E,
                     int32_t* adu, double* counts) {
  if (H < 0 || W < 0 || row0 < 0 || !p || (!E && !adu)) return -1;
  const int half = (W + 1) / 2;
  for (int r = 0; r < H; ++r)
    for (int c = 0; c < half; ++c) {
      const uint32_t q = (uint32_t)((int64_t)(row0 + r) * half + c);
      const int cm = W - 1 - c;
      const int two = cm != c;  /* the pair has a right pixel */
      double z[2], g[2], n[2];
      oracle_normal_pair(p->pattern_seed, q, (uint32_t)det, 0, &z[0], &z[1]);
      oracle_normal_pair(p->seed, q, (uint32_t)det, 1, &g[0], &g[1]);
      for (int s = 0; s < 1 + two; ++s) {
        const int col = s ? cm : c;
        double lam = (1.0 + p->prnu * z[s]) * S[(int64_t)r * W + col] + p->dark;
        if (!(lam > 0.0)) lam = 0.0;
        n[s] = p->poisson ? (double)oracle_poisson(lam, p->seed, q, (uint32_t)det, (uint32_t)s) : lam;
        if (counts) counts[(int64_t)r * W + col] = n[s];
      }
      for (int s = 0; s < 1 + two; ++s) {
        const int col = s ? cm : c;
        const double m = n[s] + (two ? p->xtalk * n[1 - s] : 0.0);
        const double e = m + p->ron * g[s];
        if (E) E[(int64_t)r * W + col] = e;
        if (adu) {
          double v = floor(p->bias + e / p->gain + 0.5);
          if (v < 0.0) v = 0.0;
          if (v > (double)p->saturation) v = (double)p->saturation;
          adu[(int64_t)r * W + col] = (int32_t)v;
        }
      }
    }
  return 0;
}
