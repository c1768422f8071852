/*
 * Photon Monte-Carlo rendering -- TEST INFRASTRUCTURE ONLY (oracle).
 *
 * Sec. 2.2 contrasts the stamp method with the direct tracing of individual photons drawn
 * from the input spectrum, with an assumed illumination of the entrance fiber and an
 * analytic PSF, to non-integer detector positions binned into pixels.  The reading written
 * out here (and, independently, by the GPU kernel), for order-slice i (its position in the
 * model) and wavelength bin j of n bins:
 *
 *   N_ij ~ Poisson(flux[j] * dlam * U),  U = sum_k u_k     counter (j, i, trial, 4)
 *   photon p = 0 .. N_ij - 1:
 *     block (j, i, p, 5): v = u(w0, w1), t = u(w2, w3)
 *     block (j, i, p, 6): c = u(w0, w1)
 *     k  = the first slit point with c U <= u_0 + .. + u_k (sequential, FP64)
 *     lt = (2 (j + v) - n) / n,   s = (2 (k + t) - n_s) / n_s
 *     (x_c, y_c) = the spectral-format polynomials at (lt, s)
 *     block (j, i, p, 7): Box-Muller pair (z1, z2)
 *     separable PSF: x = x_c + sigma_x(lt) z1,  y = y_c + sigma_y(lt) z2
 *     rotated PSF:   x = x_c + g_x z1,  y = y_c + beta g_x z1 + s_c z2  (the covariance of the
 *                    axes sigma_a, sigma_b rotated by theta, as x-marginal and y | x)
 *     counted in pixel (floor(x + 1/2), floor(y + 1/2)) when that lies on the detector.
 *
 * Every random number is keyed by the seed and indexed by (bin, slice, photon, stream), so
 * the frame does not depend on the order of evaluation.  Unlike the stamps, the PSF here is
 * not truncated to a window.
 *
 * A two-dimensional fiber (n_aper > 1) counts as n_aper order-slices, one per aperture row l,
 * numbered in model order (slice i's rows follow the rows of the slices before it): row l has
 * the slit weights u[l n_slit + k] and every one of its photons sits at t_l = -1 + (2l + 1) /
 * n_aper, its image moved by t_l (ax(lt), ay(lt)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

static int n_coeffs(int d) { return (d + 1) * (d + 2) / 2; }

static int cidx(int a, int b) {
  int t = a + b;
  return t * (t + 1) / 2 + b;
}

static double poly(const double* c, int degree, double lt, double s) {
  double sum = 0.0;
  for (int a = 0; a <= degree; ++a)
    for (int b = 0; a + b <= degree; ++b) sum += c[cidx(a, b)] * pow(lt, a) * pow(s, b);
  return sum;
}

int oracle_render_photons(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s, int psf,
                          uint64_t seed, uint32_t* const* counts, uint64_t* total) {
  if (n_det <= 0 || n_slices < 0 || !counts) return -1;
  for (int d = 0; d < n_det; ++d) memset(counts[d], 0, sizeof(uint32_t) * (size_t)H[d] * W[d]);
  for (int i = 0; i < n_slices; ++i)
    if (s[i].detector < 0 || s[i].detector >= n_det || s[i].n_lambda < 1 || s[i].n_slit < 1) return -1;
  (void)n_coeffs;
  uint64_t tot = 0;
  int n_rows = 0;  /* (slice, aperture row) pairs: the photon streams' slice index */
  for (int i = 0; i < n_slices; ++i) n_rows += s[i].n_aper > 1 ? s[i].n_aper : 1;
  int* row_slice = (int*)malloc(sizeof(int) * (n_rows > 0 ? n_rows : 1));
  int* row_l = (int*)malloc(sizeof(int) * (n_rows > 0 ? n_rows : 1));
  for (int i = 0, r = 0; i < n_slices; ++i)
    for (int l = 0; l < (s[i].n_aper > 1 ? s[i].n_aper : 1); ++l, ++r) {
      row_slice[r] = i;
      row_l[r] = l;
    }
  /* rows in parallel; integer counts, so the result does not depend on the threads */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : tot)
#endif
  for (int i = 0; i < n_rows; ++i) {
    const oracle_slice* S = &s[row_slice[i]];
    const int l = row_l[i];
    const double* u = S->u + (size_t)l * S->n_slit;
    const double tl = S->n_aper > 1 ? -1.0 + (2.0 * l + 1.0) / S->n_aper : 0.0;
    const int h = H[S->detector], w = W[S->detector];
    uint32_t* frame = counts[S->detector];
    const double dl = (S->lambda_hi - S->lambda_lo) / S->n_lambda;
    double U = 0.0;
    for (int k = 0; k < S->n_slit; ++k) U += u[k];
    const double c = cos(S->theta), sn = sin(S->theta);
    for (int j = 0; j < S->n_lambda; ++j) {
      const double lam_j = S->lambda_lo + (j + 0.5) * dl;  /* bin centre: the blaze weight */
      const long N = oracle_poisson_stream(S->flux[j] * oracle_blaze(S, lam_j) * dl * U, seed, (uint32_t)j,
                                           (uint32_t)i, 4);
      tot += (uint64_t)N;
      for (long p = 0; p < N; ++p) {
        uint32_t wa[4], wb[4];
        oracle_block(seed, (uint32_t)j, (uint32_t)i, (uint32_t)p, 5, wa);
        oracle_block(seed, (uint32_t)j, (uint32_t)i, (uint32_t)p, 6, wb);
        const double v = oracle_uniform53(wa[0], wa[1]), t = oracle_uniform53(wa[2], wa[3]);
        const double cu = oracle_uniform53(wb[0], wb[1]) * U;
        int k = 0;
        double acc = u[0];
        while (cu > acc && k < S->n_slit - 1) {
          ++k;
          acc += u[k];
        }
        const double lt = (2.0 * ((double)j + v) - S->n_lambda) / S->n_lambda;
        const double sk = (2.0 * ((double)k + t) - S->n_slit) / S->n_slit;
        const double xc = poly(S->cx, S->degree, lt, sk) + tl * (S->ax[0] + S->ax[1] * lt + S->ax[2] * lt * lt);
        const double yc = poly(S->cy, S->degree, lt, sk) + tl * (S->ay[0] + S->ay[1] * lt + S->ay[2] * lt * lt);
        const double sa = S->sx[0] + S->sx[1] * lt + S->sx[2] * lt * lt;
        const double sb = S->sy[0] + S->sy[1] * lt + S->sy[2] * lt * lt;
        double z1, z2;
        oracle_normal_pair_ctr(seed, (uint32_t)j, (uint32_t)i, (uint32_t)p, 7, &z1, &z2);
        double x, y;
        if (psf == ORACLE_PSF_SEPARABLE) {
          x = xc + sa * z1;
          y = yc + sb * z2;
        } else {
          const double vx = sa * sa * c * c + sb * sb * sn * sn, vy = sa * sa * sn * sn + sb * sb * c * c;
          const double cxy = (sa * sa - sb * sb) * sn * c;
          const double gx = sqrt(vx), beta = cxy / vx, sc = sqrt(vy - beta * cxy);
          const double dx = gx * z1;
          x = xc + dx;
          y = yc + beta * dx + sc * z2;
        }
        const double fx = floor(x + 0.5), fy = floor(y + 0.5);
        if (fx >= 0.0 && fx < (double)w && fy >= 0.0 && fy < (double)h) {
#ifdef _OPENMP
#pragma omp atomic
#endif
          frame[(int64_t)fy * w + (int64_t)fx] += 1u;
        }
      }
    }
  }
  free(row_slice);
  free(row_l);
  if (total) *total = tot;
  return 0;
}
