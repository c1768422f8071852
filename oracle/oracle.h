/*
 * FP64 CPU oracle for the echelle frame renderer -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The product renderer never calls it and shares no code,
 * header, table or constant with it.
 *
 * What it computes (paper Sec. 2, Sec. 2.2): the synthetic echellogram is the
 * superposition, over a wavelength grid, of the images of the fiber (a normalised
 * illumination profile scaled by the photons of the sample), each image being the
 * PSF integrated over the detector pixels.  Written out for one order-slice o:
 *
 *   I[r][i] += sum_j sum_k  w_ojk * integral over pixel (i, r) of PSF_ojk(x - x_c, y - y_c)
 *
 * restricted to the K x K pixel window centred on the pixel that contains the
 * mapped position (x_c, y_c), in FP64 with libm erfc.
 */
#ifndef E2E_ORACLE_H
#define E2E_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_PSF_SEPARABLE = 0, ORACLE_PSF_ELLIPTICAL = 1, ORACLE_PSF_TABLE = 2 };

typedef struct {
  int detector;
  int degree;       /* total degree of the (lt, s) -> (x, y) polynomials */
  int K;            /* odd window size in pixels */
  int n_lambda;     /* wavelength samples of the order */
  int n_slit;       /* slit points */
  double lambda_lo, lambda_hi;
  const double* cx; /* (degree+1)(degree+2)/2 coefficients, ordered by total degree, then a descending */
  const double* cy;
  double sx[3];     /* PSF width polynomial (quadratic in lt), pixels */
  double sy[3];
  double theta;     /* rotation of the elliptical PSF axes, radians */
  const double* u;  /* slit weights: n_slit of them, or n_slit per aperture row (row-major) */
  const double* flux; /* n_lambda flux samples (photons / Angstrom) at the bin centres */
  double blaze_order;  /* blaze B(lambda) = sinc^2(m (1 - lambda_b / lambda)) weights every
                          sample (0 = none); lambda_b = blaze_lambda */
  double blaze_lambda;
  /* Two-dimensional fiber sub-aperture (Sec. 2.2: each image is the fiber's spatial profile
   * convolved with the PSF; n_aper <= 1: a one-dimensional pseudo-slit in s).  With n_aper > 1
   * the sub-aperture points are (s_k, t_l), t_l = -1 + (2l + 1)/n_aper at the row centres, with
   * weights u[l n_slit + k], and the point's image moves by t_l (ax(lt), ay(lt)) px, ax and ay
   * quadratics in lt (the fiber image's half-extent along its second axis). */
  int n_aper;
  double ax[3], ay[3];
  /* ORACLE_PSF_TABLE: tabulated PSF maps at n_field wavelengths field_lt[f] (increasing, in
   * [-1, 1]); map f is map_size^2 samples maps[f][v][u] of the PSF density at offsets
   * ((u - c)/q, (v - c)/q) px from the PSF centre, c = (map_size - 1)/2, q = map_oversample;
   * the density between samples is their bilinear interpolant (zero beyond the grid), and
   * between field nodes the PSF is the linear blend in lt of the two unit-mass maps around
   * it.  A stamp's pixel values are that density's integrals over the pixels for the PSF
   * centred at the stamp's exact mapped position. */
  int n_field;
  const double* field_lt;
  int map_size;
  double map_oversample;
  const double* maps;
} oracle_slice;

/* Render every order-slice into its detector frame.  frames[d] points to H[d]*W[d]
 * doubles (row-major, row = y); they are overwritten.  n_threads <= 0 uses all cores.
 * Returns 0, or -1 on an invalid argument. */
int oracle_render(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s,
                  int psf, double** frames, int n_threads);

/* Effective-PSF value (the pixel integral of map f's bilinear density, normalised to unit
 * integral) of window pixel (m, n), relative to the window's centre pixel, for a PSF centred
 * at sub-pixel offset (phx, phy) from that pixel's centre. */
double oracle_epsf_pixel(const oracle_slice* s, int f, double phx, double phy, int m, int n);

/* The same for all K x K window pixels at once (out[n*K + m]). */
void oracle_epsf_window(const oracle_slice* s, int f, double phx, double phy, double* out);

/* Blaze weight of the slice at wavelength lam (1 when it has none). */
double oracle_blaze(const oracle_slice* s, double lam);

/* Sub-aperture points of an order-slice: n_slit, or n_slit x n_aper for a 2-D fiber; a
 * point index kk stands for slit point kk % n_slit of aperture row kk / n_slit. */
int oracle_points(const oracle_slice* s);

/* Mapped position and PSF widths of stamp (j, kk) of one order-slice (kk a point index). */
void oracle_map(const oracle_slice* s, int j, int k, double* x_c, double* y_c, double* sig_x,
                double* sig_y, double* weight);

/* The K*K pixel values of one stamp (row-major n*K+m, pixel (i0+m, r0+n)), and its window origin. */
void oracle_stamp(const oracle_slice* s, int psf, int j, int k, double* out, int* i0, int* r0);

/* Stamps whose mapped centre lies within `margin` px of a half-integer in x or y (window-rule
 * ties): up to max_out (j, k, axis) triples in out; returns the count. */
int oracle_window_ties(const oracle_slice* s, double margin, int max_out, int* out);

/* P(a < Z < b) for a standard normal Z, a <= b. */
double oracle_normal_interval(double a, double b);

/* Bivariate standard normal CDF P(X < h, Y < k) with correlation rho (|rho| <= 0.95). */
double oracle_bvn_cdf(double h, double k, double rho);

/* P(h0 < X < h1, k0 < Y < k1) for the standard bivariate normal with correlation rho. */
double oracle_bvn_rect(double h0, double h1, double k0, double k1, double rho);

/* n-point Gauss-Legendre nodes and weights on [-1, 1]. */
void oracle_gauss_legendre(int n, double* x, double* w);

/* Pixel integral of a separable Gaussian by the paper's sub-pixel sampling (Sec. 2.2):
 * density evaluated at the centres of an nsub x nsub grid of sub-pixels, times the
 * sub-pixel area.  Pixel (i, r) relative to a centre at (xc, yc). */
double oracle_subpixel_sample(double xc, double yc, double sigx, double sigy, int i, int r, int nsub);

/* Gradient of L = sum over pixels of (I - T)^2 with respect to every order-slice's
 * cx, cy (n_c each), sx, sy (3 each), holding each stamp's window origin fixed at
 * the one the forward render picks.  T has the frames' layout.  Outputs are
 * concatenated per order-slice in the order they are given.  Returns L. */
double oracle_loss_grad(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s,
                        const double* const* target, double* g_cx, double* g_cy, double* g_sx,
                        double* g_sy, int n_threads);

/* Vector-Jacobian product of the render: given dL/dI per detector (frames' layout), the
 * gradient sum over pixels of dL/dI * dI/dtheta for every order-slice's cx, cy, sx, sy, with
 * window origins held at the forward render's.  Returns 0, or -1 on an invalid argument. */
int oracle_vjp(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s,
               const double* const* dLdI, double* g_cx, double* g_cy, double* g_sx, double* g_sy, int n_threads);

/* ---------------------------------------------------------------- detector noise (noise.c) */

#include <stdint.h>

typedef struct {
  uint64_t seed;          /* frame seed: photon / dark shot noise and read-out noise */
  uint64_t pattern_seed;  /* fixed-pattern seed: pixel response non-uniformity */
  double dark;            /* mean dark electrons per pixel over the exposure */
  double prnu;            /* relative rms of the pixel response */
  double ron;             /* read-out noise rms, electrons */
  double xtalk;           /* fraction of the mirror pixel's electrons added */
  double gain;            /* electrons per ADU */
  double bias;            /* ADU offset */
  int32_t saturation;     /* ADU ceiling */
  int32_t poisson;        /* 1 = Poisson draws, 0 = expected values */
} oracle_noise;

/* Philox4x32-10 block for counter ctr and key; the block of counter (c0, c1, c2, c3) under
 * the key of a 64-bit seed; the 53-bit uniform on (0, 1) made from two of its words. */
void oracle_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t w[4]);
double oracle_uniform53(uint32_t a, uint32_t b);
/* Box-Muller pair from the block of counter (c0, c1, c2, c3). */
void oracle_normal_pair_ctr(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double* left,
                            double* right);
/* Poisson(lam) from blocks (q, d, trial, stream), trial = 0, 1, ... */
long oracle_poisson_stream(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t stream);
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Box-Muller pair of standard normals from block (seed, (q, d, 0, stream)). */
void oracle_normal_pair(uint64_t seed, uint32_t q, uint32_t d, uint32_t stream, double* left, double* right);
/* Poisson(lam) draw of side `side` of pair q on detector d. */
long oracle_poisson(double lam, uint64_t seed, uint32_t q, uint32_t d, uint32_t side);
/* Noise stage of rows row0 .. row0+H-1 of one detector frame of width W (S: H x W expected
 * electrons, row-major): electrons E and/or ADU (either may be NULL), and optionally the
 * Poisson counts.  Returns 0 or -1. */
int oracle_add_noise(int H, int W, int row0, int det, const double* S, const oracle_noise* p, double* E,
                     int32_t* adu, double* counts);

/* ---------------------------------------------------------------- photon Monte-Carlo (photons.c) */

/* Photon-by-photon rendering of every order-slice (the alternative of Sec. 2.2): per slice
 * index i and wavelength bin j, N ~ Poisson(flux[j] dlam sum_k u_k) photons; photon p takes
 * a wavelength uniform in its bin, a slit point k with probability u_k / sum u and a position
 * uniform in that point's bin, the PSF offset of a bivariate normal, and is counted in the
 * pixel containing it.  counts[d] (H x W, row-major) are overwritten; *total = photons drawn.
 * Returns 0, or -1 on an invalid argument. */
int oracle_render_photons(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s, int psf,
                          uint64_t seed, uint32_t* const* counts, uint64_t* total);

#ifdef __cplusplus
}
#endif
#endif
