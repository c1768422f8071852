/*
 * FP64 CPU oracle for the echelle frame renderer -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the product path never does.  It is deliberately plain: direct monomial sums, libm
 * erfc, one stamp at a time, loops in the order the definition is written.
 *
 * Method (paper Sec. 2 and Sec. 2.2): the frame is the sum, over the wavelength grid
 * of every order and fiber, of the fiber image projected on the detector; each fiber
 * image is the pixel-integrated convolution of the fiber profile with the PSF.  The
 * fiber profile is a set of slit points s_k with normalised weights u_k (Sec. 2.1:
 * a normalised illumination profile multiplied at the end by the photons of the
 * sample).  Readings where the paper is silent (polynomial spectral format, sample
 * placement, window rule, truncation without renormalisation) are the ones listed in
 * the design notes and repeated at each function below.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* Index of monomial lt^a s^b: ordered by total degree t = a+b, then a descending. */
static int coeff_index(int a, int b) {
  int t = a + b;
  return t * (t + 1) / 2 + b;
}

/* Plain definition of the spectral-format polynomial: sum over a+b <= d of c_ab lt^a s^b. */
static double poly2(const double* c, int degree, double lt, double s) {
  double sum = 0.0;
  for (int a = 0; a <= degree; ++a)
    for (int b = 0; a + b <= degree; ++b) sum += c[coeff_index(a, b)] * pow(lt, a) * pow(s, b);
  return sum;
}

static double quad(const double* c, double lt) { return c[0] + c[1] * lt + c[2] * lt * lt; }

/* Standard normal CDF written with erfc so that the lower tail keeps relative precision. */
static double Phi(double t) { return 0.5 * erfc(-t / sqrt(2.0)); }

double oracle_normal_interval(double a, double b) {
  /* P(a < Z < b).  When both ends are on the same side of the mean, take the
   * difference of the two (small) tail probabilities on that side. */
  if (a >= 0.0) return Phi(-a) - Phi(-b);
  if (b <= 0.0) return Phi(b) - Phi(a);
  return 1.0 - Phi(a) - Phi(-b);
}

static double phi(double t) { return exp(-0.5 * t * t) / sqrt(2.0 * ORACLE_PI); }

/* ---------------------------------------------------------------- Gauss-Legendre */

void oracle_gauss_legendre(int n, double* x, double* w) {
  /* Roots of the Legendre polynomial P_n by Newton's method from the usual cosine
   * guesses; P_n and P_{n-1} from the three-term recurrence
   * k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}, and P_n' = n (z P_n - P_{n-1}) / (z^2 - 1). */
  for (int i = 0; i < n; ++i) {
    double z = cos(ORACLE_PI * (i + 0.75) / (n + 0.5));
    double pn = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      pn = p1;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-15) {
        /* one more evaluation at the converged root for the weight */
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ---------------------------------------------------------------- bivariate normal */

/* P(X < h, Y < k) for unit-variance (X, Y) with correlation rho, by Plackett's identity
 * dF/drho = bivariate density, integrated from rho = 0 with the substitution
 * rho = sin(t) (the form Drezner & Wesolowsky and Genz use):
 *   F = Phi(h) Phi(k) + 1/(2 pi) * int_0^{asin rho} exp(-(h^2 + k^2 - 2 h k sin t) / (2 cos^2 t)) dt
 * The integral is taken with 20-point Gauss-Legendre quadrature. */
double oracle_bvn_cdf(double h, double k, double rho) {
  static double gx[20], gw[20];
  static int init = 0;
  if (!init) {
#ifdef _OPENMP
#pragma omp critical(oracle_gl_init)
#endif
    {
      if (!init) {
        oracle_gauss_legendre(20, gx, gw);
        init = 1;
      }
    }
  }
  double base = Phi(h) * Phi(k);
  if (rho == 0.0) return base;
  double top = asin(rho);
  double half = 0.5 * top, sum = 0.0;
  for (int i = 0; i < 20; ++i) {
    double t = half * (gx[i] + 1.0);
    double st = sin(t), ct = cos(t);
    sum += gw[i] * exp(-(h * h + k * k - 2.0 * h * k * st) / (2.0 * ct * ct));
  }
  return base + sum * half / (2.0 * ORACLE_PI);
}

double oracle_bvn_rect(double h0, double h1, double k0, double k1, double rho) {
  /* Reflect an interval that lies wholly above the mean (X -> -X flips the sign of rho),
   * so that the four corner probabilities are small tail values and the
   * inclusion-exclusion keeps relative precision. */
  if (h0 >= 0.0) {
    double t = -h1;
    h1 = -h0;
    h0 = t;
    rho = -rho;
  }
  if (k0 >= 0.0) {
    double t = -k1;
    k1 = -k0;
    k0 = t;
    rho = -rho;
  }
  return oracle_bvn_cdf(h1, k1, rho) - oracle_bvn_cdf(h0, k1, rho) - oracle_bvn_cdf(h1, k0, rho) +
         oracle_bvn_cdf(h0, k0, rho);
}

/* ---------------------------------------------------------------- mapping */

/* Blaze of the order at wavelength lam: the grating's single-groove diffraction envelope in the
 * order's phase variable nu = m (1 - lambda_b / lam), sinc^2(nu) with sinc(x) = sin(pi x)/(pi x)
 * (the paper weights each order by its blaze profile, computed analytically, Sec. 4.2). */
double oracle_blaze(const oracle_slice* s, double lam) {
  if (s->blaze_order == 0.0) return 1.0;
  const double nu = s->blaze_order * (1.0 - s->blaze_lambda / lam);
  if (nu == 0.0) return 1.0;
  const double sc = sin(ORACLE_PI * nu) / (ORACLE_PI * nu);
  return sc * sc;
}

int oracle_points(const oracle_slice* s) { return s->n_slit * (s->n_aper > 1 ? s->n_aper : 1); }

/* Sample j of n_lambda sits at the centre of the j-th equal bin of [lambda_lo, lambda_hi]
 * (the wavelength grid of Sec. 2); the polynomial variable is that wavelength normalised
 * to [-1, 1].  Slit point k of n_slit sits at the centre of the k-th equal bin of [-1, 1].
 * The weight is flux density x bin width x slit weight (Sec. 2.1: normalised profile times
 * the photons in the sample's wavelength range).  For a 2-D fiber, point kk is slit point
 * k = kk % n_slit of aperture row l = kk / n_slit, at t_l = -1 + (2l + 1)/n_aper, and its
 * image moves by t_l (ax(lt), ay(lt)). */
void oracle_map(const oracle_slice* s, int j, int kk, double* x_c, double* y_c, double* sig_x,
                double* sig_y, double* weight) {
  const int k = kk % s->n_slit, l = kk / s->n_slit;
  double dl = (s->lambda_hi - s->lambda_lo) / s->n_lambda;
  double lam = s->lambda_lo + (j + 0.5) * dl;
  double lt = 2.0 * (lam - s->lambda_lo) / (s->lambda_hi - s->lambda_lo) - 1.0;
  double sk = -1.0 + (2.0 * k + 1.0) / s->n_slit;
  double tl = s->n_aper > 1 ? -1.0 + (2.0 * l + 1.0) / s->n_aper : 0.0;
  *x_c = poly2(s->cx, s->degree, lt, sk) + tl * quad(s->ax, lt);
  *y_c = poly2(s->cy, s->degree, lt, sk) + tl * quad(s->ay, lt);
  *sig_x = quad(s->sx, lt);
  *sig_y = quad(s->sy, lt);
  *weight = s->flux[j] * dl * s->u[kk] * oracle_blaze(s, lam);
}

/* Window rule: the K x K window is centred on the pixel containing the mapped point;
 * pixel i spans [i - 1/2, i + 1/2), so that pixel is floor(x_c + 1/2). */
static int window_origin(double c, int K) { return (int)floor(c + 0.5) - K / 2; }

/* Covariance of the elliptical PSF: widths sa, sb along axes rotated by theta. */
static void ellipse_cov(double sa, double sb, double theta, double* vx, double* vy, double* cxy) {
  double c = cos(theta), s = sin(theta);
  *vx = sa * sa * c * c + sb * sb * s * s;
  *vy = sa * sa * s * s + sb * sb * c * c;
  *cxy = (sa * sa - sb * sb) * s * c;
}

/* ---------------------------------------------------------------- tabulated PSF */

/* Integral of the unit tent max(0, 1 - |t|) from -inf to t. */
static double tent_cdf(double t) {
  if (t <= -1.0) return 0.0;
  if (t <= 0.0) return 0.5 * (1.0 + t) * (1.0 + t);
  if (t <= 1.0) return 1.0 - 0.5 * (1.0 - t) * (1.0 - t);
  return 1.0;
}

/* Integral over [a, b) (px, PSF-relative) of the tent of map sample u: the bilinear density is
 * sum_uv S_uv tent(q x - (u - c)) tent(q y - (v - c)), so a pixel integral factorises into
 * x-weights of the columns times y-weights of the rows. */
static double tent_weight(double a, double b, int u, double c, double q) {
  const double xu = (u - c) / q;
  return (tent_cdf(q * (b - xu)) - tent_cdf(q * (a - xu))) / q;
}

double oracle_epsf_pixel(const oracle_slice* s, int f, double phx, double phy, int m, int n) {
  const int M = s->map_size, H = s->K / 2;
  const double q = s->map_oversample, c = 0.5 * (M - 1);
  const double* S = s->maps + (size_t)f * M * M;
  double norm = 0.0;
  for (int i = 0; i < M * M; ++i) norm += S[i];
  norm /= q * q;  /* integral of the bilinear density */
  const double ax = m - H - 0.5 - phx, bx = ax + 1.0, ay = n - H - 0.5 - phy, by = ay + 1.0;
  double sum = 0.0;
  for (int v = 0; v < M; ++v) {
    const double wy = tent_weight(ay, by, v, c, q);
    if (wy == 0.0) continue;
    for (int u = 0; u < M; ++u) sum += S[(size_t)v * M + u] * tent_weight(ax, bx, u, c, q) * wy;
  }
  return sum / norm;
}

/* All K x K pixel integrals of map f's normalised bilinear density for the PSF centred at
 * sub-pixel offset (phx, phy) from the window's centre pixel: the same sum as
 * oracle_epsf_pixel, with the column weights of every window column and the row weights of
 * every window row formed once, and the loops kept to the samples whose tents meet the pixel
 * (every other term is exactly zero). */
void oracle_epsf_window(const oracle_slice* s, int f, double phx, double phy, double* out) {
  const int M = s->map_size, K = s->K, H = K / 2;
  const double q = s->map_oversample, c = 0.5 * (M - 1);
  const double* S = s->maps + (size_t)f * M * M;
  double norm = 0.0;
  for (int i = 0; i < M * M; ++i) norm += S[i];
  norm /= q * q;
  double* X = (double*)malloc(sizeof(double) * (size_t)K * M);
  double* Y = (double*)malloc(sizeof(double) * (size_t)K * M);
  int* span = (int*)malloc(sizeof(int) * 4 * (size_t)K);
  for (int m = 0; m < K; ++m) {
    const double ax = m - H - 0.5 - phx, ay = m - H - 0.5 - phy;
    int xl = M, xh = -1, yl = M, yh = -1;
    for (int u = 0; u < M; ++u) {
      X[(size_t)m * M + u] = tent_weight(ax, ax + 1.0, u, c, q);
      Y[(size_t)m * M + u] = tent_weight(ay, ay + 1.0, u, c, q);
      if (X[(size_t)m * M + u] != 0.0) {
        if (u < xl) xl = u;
        xh = u;
      }
      if (Y[(size_t)m * M + u] != 0.0) {
        if (u < yl) yl = u;
        yh = u;
      }
    }
    span[4 * m] = xl;
    span[4 * m + 1] = xh;
    span[4 * m + 2] = yl;
    span[4 * m + 3] = yh;
  }
  for (int n = 0; n < K; ++n)
    for (int m = 0; m < K; ++m) {
      double sum = 0.0;
      for (int v = span[4 * n + 2]; v <= span[4 * n + 3]; ++v) {
        const double wy = Y[(size_t)n * M + v];
        for (int u = span[4 * m]; u <= span[4 * m + 1]; ++u)
          sum += S[(size_t)v * M + u] * X[(size_t)m * M + u] * wy;
      }
      out[n * K + m] = sum / norm;
    }
  free(X);
  free(Y);
  free(span);
}

/* Stamp of a tabulated PSF (Sec. 2.1: PSF maps given per field point; Sec. 2.2: each image is
 * the PSF integrated over the pixels): the pixel integrals of the normalised maps at the two
 * field nodes around the sample's lt (the end node beyond the ends), each at the stamp's exact
 * sub-pixel centre (fx, fy), blended linearly in lt, times the weight. */
static void table_stamp(const oracle_slice* s, double lt, double fx, double fy, double w, double* out) {
  const int K = s->K, F = s->n_field;
  int f0 = 0, f1 = 0;
  double wf = 0.0;
  if (lt <= s->field_lt[0]) {
    f0 = f1 = 0;
  } else if (lt >= s->field_lt[F - 1]) {
    f0 = f1 = F - 1;
  } else {
    while (f0 + 1 < F && s->field_lt[f0 + 1] <= lt) ++f0;
    f1 = f0 + 1 < F ? f0 + 1 : f0;
    if (f1 != f0) wf = (lt - s->field_lt[f0]) / (s->field_lt[f1] - s->field_lt[f0]);
  }
  double* e0 = (double*)malloc(sizeof(double) * 2 * (size_t)K * K);
  double* e1 = e0 + (size_t)K * K;
  oracle_epsf_window(s, f0, fx, fy, e0);
  if (wf != 0.0) oracle_epsf_window(s, f1, fx, fy, e1);
  for (int i = 0; i < K * K; ++i) out[i] = w * ((1.0 - wf) * e0[i] + (wf != 0.0 ? wf * e1[i] : 0.0));
  free(e0);
}

void oracle_stamp(const oracle_slice* s, int psf, int j, int k, double* out, int* i0p, int* r0p) {
  double xc, yc, sx, sy, w;
  oracle_map(s, j, k, &xc, &yc, &sx, &sy, &w);
  int K = s->K;
  int i0 = window_origin(xc, K), r0 = window_origin(yc, K);
  *i0p = i0;
  *r0p = r0;
  if (psf == ORACLE_PSF_TABLE) {
    const double dl = (s->lambda_hi - s->lambda_lo) / s->n_lambda;
    const double lam = s->lambda_lo + (j + 0.5) * dl;
    const double lt = 2.0 * (lam - s->lambda_lo) / (s->lambda_hi - s->lambda_lo) - 1.0;
    table_stamp(s, lt, xc - (i0 + K / 2), yc - (r0 + K / 2), w, out);
  } else if (psf == ORACLE_PSF_SEPARABLE) {
    for (int n = 0; n < K; ++n) {
      double ay = oracle_normal_interval((r0 + n - 0.5 - yc) / sy, (r0 + n + 0.5 - yc) / sy);
      for (int m = 0; m < K; ++m) {
        double ax = oracle_normal_interval((i0 + m - 0.5 - xc) / sx, (i0 + m + 0.5 - xc) / sx);
        out[n * K + m] = w * ax * ay;
      }
    }
  } else {
    double vx, vy, cxy;
    ellipse_cov(sx, sy, s->theta, &vx, &vy, &cxy);
    double gx = sqrt(vx), gy = sqrt(vy), rho = cxy / (gx * gy);
    for (int n = 0; n < K; ++n)
      for (int m = 0; m < K; ++m) {
        double h0 = (i0 + m - 0.5 - xc) / gx, h1 = (i0 + m + 0.5 - xc) / gx;
        double k0 = (r0 + n - 0.5 - yc) / gy, k1 = (r0 + n + 0.5 - yc) / gy;
        out[n * K + m] = w * oracle_bvn_rect(h0, h1, k0, k1, rho);
      }
  }
}

/* Stamps of one order-slice whose mapped centre lies within `margin` px of a pixel edge
 * (a half-integer) in x or y: there the window rule floor(c + 1/2) can round either way between
 * two evaluations of c that differ by rounding, so two correct renderers may place the window
 * one pixel apart (a flip).  Writes up to max_out (j, k, axis) triples to out (axis 0 = x,
 * 1 = y) and returns the number of such (stamp, axis) pairs. */
int oracle_window_ties(const oracle_slice* s, double margin, int max_out, int* out) {
  int n = 0;
  for (int j = 0; j < s->n_lambda; ++j)
    for (int k = 0; k < oracle_points(s); ++k) {
      double c[2], sx, sy, w;
      oracle_map(s, j, k, &c[0], &c[1], &sx, &sy, &w);
      for (int a = 0; a < 2; ++a) {
        const double d = (c[a] + 0.5) - floor(c[a] + 0.5);
        if (d < margin || 1.0 - d < margin) {
          if (n < max_out) {
            out[3 * n] = j;
            out[3 * n + 1] = k;
            out[3 * n + 2] = a;
          }
          ++n;
        }
      }
    }
  return n;
}

double oracle_subpixel_sample(double xc, double yc, double sigx, double sigy, int i, int r, int nsub) {
  double h = 1.0 / nsub, sum = 0.0;
  for (int q = 0; q < nsub; ++q)
    for (int p = 0; p < nsub; ++p) {
      double x = i - 0.5 + (p + 0.5) * h, y = r - 0.5 + (q + 0.5) * h;
      sum += phi((x - xc) / sigx) / sigx * phi((y - yc) / sigy) / sigy;
    }
  return sum * h * h;
}

/* ---------------------------------------------------------------- render */

typedef struct {
  int x0, y0, w, h; /* clipped band of the detector touched by the slice */
  double* buf;
} band_t;

static int n_coeffs(int d) { return (d + 1) * (d + 2) / 2; }

static int valid_slice(const oracle_slice* s, int n_det) {
  if (s->detector < 0 || s->detector >= n_det) return 0;
  if (s->K < 1 || s->K % 2 == 0 || s->n_lambda < 0 || s->n_slit < 0 || s->degree < 0 || s->n_aper < 0) return 0;
  if (!(s->lambda_hi > s->lambda_lo)) return 0;
  return 1;
}

/* Render one slice into a private band of its detector (rows/cols it can touch). */
static void render_slice(const oracle_slice* s, int psf, int H, int W, band_t* band) {
  int K = s->K;
  int xmin = W, xmax = -1, ymin = H, ymax = -1;
  for (int j = 0; j < s->n_lambda; ++j)
    for (int k = 0; k < oracle_points(s); ++k) {
      double xc, yc, sx, sy, w;
      oracle_map(s, j, k, &xc, &yc, &sx, &sy, &w);
      int i0 = window_origin(xc, K), r0 = window_origin(yc, K);
      if (i0 < xmin) xmin = i0;
      if (i0 + K - 1 > xmax) xmax = i0 + K - 1;
      if (r0 < ymin) ymin = r0;
      if (r0 + K - 1 > ymax) ymax = r0 + K - 1;
    }
  if (xmin < 0) xmin = 0;
  if (ymin < 0) ymin = 0;
  if (xmax > W - 1) xmax = W - 1;
  if (ymax > H - 1) ymax = H - 1;
  band->buf = NULL;
  band->w = band->h = 0;
  if (xmax < xmin || ymax < ymin) return;
  band->x0 = xmin;
  band->y0 = ymin;
  band->w = xmax - xmin + 1;
  band->h = ymax - ymin + 1;
  band->buf = (double*)calloc((size_t)band->w * band->h, sizeof(double));
  double* st = (double*)malloc(sizeof(double) * K * K);
  const double dl = (s->lambda_hi - s->lambda_lo) / s->n_lambda;
  for (int j = 0; j < s->n_lambda; ++j)
    for (int k = 0; k < oracle_points(s); ++k) {
      int i0, r0;
      if (psf == ORACLE_PSF_TABLE) {
        double xc, yc, sx, sy, w;
        oracle_map(s, j, k, &xc, &yc, &sx, &sy, &w);
        i0 = window_origin(xc, K);
        r0 = window_origin(yc, K);
        const double lam = s->lambda_lo + (j + 0.5) * dl;
        const double lt = 2.0 * (lam - s->lambda_lo) / (s->lambda_hi - s->lambda_lo) - 1.0;
        table_stamp(s, lt, xc - (i0 + K / 2), yc - (r0 + K / 2), w, st);
      } else {
        oracle_stamp(s, psf, j, k, st, &i0, &r0);
      }
      for (int n = 0; n < K; ++n) {
        int r = r0 + n;
        if (r < band->y0 || r >= band->y0 + band->h) continue; /* outside the frame: dropped */
        for (int m = 0; m < K; ++m) {
          int i = i0 + m;
          if (i < band->x0 || i >= band->x0 + band->w) continue;
          band->buf[(size_t)(r - band->y0) * band->w + (i - band->x0)] += st[n * K + m];
        }
      }
    }
  free(st);
}

int oracle_render(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s, int psf,
                  double** frames, int n_threads) {
  if (n_det <= 0 || n_slices < 0) return -1;
  for (int i = 0; i < n_slices; ++i)
    if (!valid_slice(&s[i], n_det)) return -1;
  for (int d = 0; d < n_det; ++d) memset(frames[d], 0, sizeof(double) * (size_t)H[d] * W[d]);
  band_t* bands = (band_t*)calloc(n_slices > 0 ? n_slices : 1, sizeof(band_t));
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#else
  (void)n_threads;
#endif
  for (int i = 0; i < n_slices; ++i) render_slice(&s[i], psf, H[s[i].detector], W[s[i].detector], &bands[i]);
  /* merge the private bands in slice order so the result does not depend on threads */
  for (int i = 0; i < n_slices; ++i) {
    band_t* b = &bands[i];
    if (!b->buf) continue;
    double* f = frames[s[i].detector];
    int w = W[s[i].detector];
    for (int r = 0; r < b->h; ++r)
      for (int c = 0; c < b->w; ++c) f[(size_t)(b->y0 + r) * w + b->x0 + c] += b->buf[(size_t)r * b->w + c];
    free(b->buf);
  }
  free(bands);
  return 0;
}

/* ---------------------------------------------------------------- gradient */

/* d/dx_c of P(e0 < X < e1), X ~ N(x_c, sig^2): -(phi(u1) - phi(u0)) / sig, u = (e - x_c)/sig.
 * d/dsig of the same:                         -(u1 phi(u1) - u0 phi(u0)) / sig. */
static void slice_grad(const oracle_slice* s, int H, int W, const double* R, double* gcx, double* gcy,
                       double* gsx, double* gsy) {
  int K = s->K, nc = n_coeffs(s->degree);
  double* ax = (double*)malloc(sizeof(double) * K);
  double* ay = (double*)malloc(sizeof(double) * K);
  double* dax = (double*)malloc(sizeof(double) * K);
  double* day = (double*)malloc(sizeof(double) * K);
  double* sax = (double*)malloc(sizeof(double) * K);
  double* say = (double*)malloc(sizeof(double) * K);
  for (int c = 0; c < nc; ++c) gcx[c] = gcy[c] = 0.0;
  for (int p = 0; p < 3; ++p) gsx[p] = gsy[p] = 0.0;
  for (int j = 0; j < s->n_lambda; ++j)
    for (int k = 0; k < oracle_points(s); ++k) {
      double xc, yc, sx, sy, w;
      oracle_map(s, j, k, &xc, &yc, &sx, &sy, &w);
      int i0 = window_origin(xc, K), r0 = window_origin(yc, K);
      for (int m = 0; m < K; ++m) {
        double u0 = (i0 + m - 0.5 - xc) / sx, u1 = (i0 + m + 0.5 - xc) / sx;
        ax[m] = oracle_normal_interval(u0, u1);
        dax[m] = -(phi(u1) - phi(u0)) / sx;
        sax[m] = -(u1 * phi(u1) - u0 * phi(u0)) / sx;
        double v0 = (r0 + m - 0.5 - yc) / sy, v1 = (r0 + m + 0.5 - yc) / sy;
        ay[m] = oracle_normal_interval(v0, v1);
        day[m] = -(phi(v1) - phi(v0)) / sy;
        say[m] = -(v1 * phi(v1) - v0 * phi(v0)) / sy;
      }
      double gx = 0, gy = 0, gsig_x = 0, gsig_y = 0;
      for (int n = 0; n < K; ++n) {
        int r = r0 + n;
        if (r < 0 || r >= H) continue;
        for (int m = 0; m < K; ++m) {
          int i = i0 + m;
          if (i < 0 || i >= W) continue;
          double res = R[(size_t)r * W + i];
          gx += res * w * dax[m] * ay[n];
          gy += res * w * ax[m] * day[n];
          gsig_x += res * w * sax[m] * ay[n];
          gsig_y += res * w * ax[m] * say[n];
        }
      }
      double dl = (s->lambda_hi - s->lambda_lo) / s->n_lambda;
      double lam = s->lambda_lo + (j + 0.5) * dl;
      double lt = 2.0 * (lam - s->lambda_lo) / (s->lambda_hi - s->lambda_lo) - 1.0;
      double sk = -1.0 + (2.0 * (k % s->n_slit) + 1.0) / s->n_slit;  /* the point's slit coordinate */
      for (int a = 0; a <= s->degree; ++a)
        for (int b = 0; a + b <= s->degree; ++b) {
          double mono = pow(lt, a) * pow(sk, b);
          gcx[coeff_index(a, b)] += gx * mono;
          gcy[coeff_index(a, b)] += gy * mono;
        }
      for (int p = 0; p < 3; ++p) {
        gsx[p] += gsig_x * pow(lt, p);
        gsy[p] += gsig_y * pow(lt, p);
      }
    }
  free(ax); free(ay); free(dax); free(day); free(sax); free(say);
}

int oracle_vjp(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s,
               const double* const* dLdI, double* g_cx, double* g_cy, double* g_sx, double* g_sy, int n_threads) {
  if (n_det <= 0 || n_slices < 0) return -1;
  for (int i = 0; i < n_slices; ++i)
    if (!valid_slice(&s[i], n_det)) return -1;
  int* off = (int*)malloc(sizeof(int) * (n_slices + 1));
  off[0] = 0;
  for (int i = 0; i < n_slices; ++i) off[i + 1] = off[i] + n_coeffs(s[i].degree);
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#else
  (void)n_threads;
#endif
  for (int i = 0; i < n_slices; ++i)
    slice_grad(&s[i], H[s[i].detector], W[s[i].detector], dLdI[s[i].detector], g_cx + off[i], g_cy + off[i],
               g_sx + 3 * i, g_sy + 3 * i);
  free(off);
  return 0;
}

double oracle_loss_grad(int n_det, const int* H, const int* W, int n_slices, const oracle_slice* s,
                        const double* const* target, double* g_cx, double* g_cy, double* g_sx, double* g_sy,
                        int n_threads) {
  double** frames = (double**)malloc(sizeof(double*) * n_det);
  for (int d = 0; d < n_det; ++d) frames[d] = (double*)malloc(sizeof(double) * (size_t)H[d] * W[d]);
  if (oracle_render(n_det, H, W, n_slices, s, ORACLE_PSF_SEPARABLE, frames, n_threads) != 0) {
    for (int d = 0; d < n_det; ++d) free(frames[d]);
    free(frames);
    return NAN;
  }
  double loss = 0.0;
  for (int d = 0; d < n_det; ++d)
    for (size_t p = 0; p < (size_t)H[d] * W[d]; ++p) {
      double r = frames[d][p] - target[d][p];
      loss += r * r;
      frames[d][p] = 2.0 * r; /* dL/dI */
    }
  int* off = (int*)malloc(sizeof(int) * (n_slices + 1));
  off[0] = 0;
  for (int i = 0; i < n_slices; ++i) off[i + 1] = off[i] + n_coeffs(s[i].degree);
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#else
  (void)n_threads;
#endif
  for (int i = 0; i < n_slices; ++i)
    slice_grad(&s[i], H[s[i].detector], W[s[i].detector], frames[s[i].detector], g_cx + off[i], g_cy + off[i],
               g_sx + 3 * i, g_sy + 3 * i);
  free(off);
  for (int d = 0; d < n_det; ++d) free(frames[d]);
  free(frames);
  return loss;
}
