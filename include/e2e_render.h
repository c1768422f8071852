/*
 * e2e_render.h -- C ABI of the GB300 echelle frame renderer.
 *
 * The library renders the raw detector frame of a fiber-fed echelle spectrograph
 * from a source spectrum, as the image simulator of arXiv:2008.05858 does (Sec. 2.2):
 * the frame is the superposition, over a wavelength grid, of the images of the fiber
 * projected on the detector, each image being the PSF integrated over the pixels.
 *
 * Model of one order-slice o (one trace: detector, diffraction order, fiber, slice):
 *   - wavelength samples j = 0..n_lambda-1 at the centres of n_lambda equal bins of
 *     [lambda_lo, lambda_hi]; lt_j = that wavelength normalised to [-1, 1];
 *   - slit points k = 0..n_slit-1 at the centres of n_slit equal bins of s in [-1, 1];
 *   - a stamp (o, j, k) has weight  w = flux_o[j] * (lambda_hi - lambda_lo)/n_lambda * u_k
 *     (Sec. 2.1: normalised illumination profile u times the photons of the sample);
 *   - its centre is (x_c, y_c) = (P_x(lt_j, s_k), P_y(lt_j, s_k)), with P the total-degree
 *     polynomials given by cx/cy (the spectral format of Sec. 2.1, here in polynomial form);
 *   - its PSF is a Gaussian with widths sigma_x(lt), sigma_y(lt) (quadratics in lt; Sec. 2.1
 *     models the PSF analytically as an asymmetric Gaussian), axis-aligned
 *     (E2E_PSF_SEPARABLE) or with axes rotated by theta (E2E_PSF_ELLIPTICAL);
 *   - it deposits into the K x K pixel window centred on pixel (floor(x_c+1/2),
 *     floor(y_c+1/2)) the exact integral of the PSF over each pixel (pixel i spans
 *     [i-1/2, i+1/2)); flux outside the window is not deposited (no renormalisation),
 *     pixels outside the detector are dropped.
 *
 * Conventions: every function returns 0 (E2E_OK) or a negative E2E_E* code; the text of
 * the last error of the calling thread is in e2e_last_error().  No C++ exception crosses
 * the ABI.  Ids are opaque 64-bit handles.  The caller keeps ownership of every array it
 * passes; the library copies what it keeps.  All work is asynchronous on the CUDA stream
 * given (a cudaStream_t; NULL = legacy default stream) unless stated otherwise.
 */
#ifndef E2E_RENDER_H
#define E2E_RENDER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ error codes */
#define E2E_OK 0
#define E2E_EINVAL -1    /* invalid argument or model */
#define E2E_ENOMEM -2    /* device memory exhausted */
#define E2E_ECUDA -3     /* a CUDA call failed; see e2e_last_error() */
#define E2E_ENOTFOUND -4 /* unknown id */
#define E2E_EBUSY -5     /* reserved (queued jobs report E2E_JOB_QUEUED in e2e_job_info) */
#define E2E_ETOOBIG -6   /* serving: job can never fit the memory pool */
#define E2E_ETIMEOUT -7  /* serving: wait timed out */
#define E2E_ECANCELLED -8
#define E2E_EDEVICE -9   /* debug checks: a kernel found a deposit its plan did not foresee */

/* ------------------------------------------------------------------ enums */
enum { E2E_PSF_SEPARABLE = 0, E2E_PSF_ELLIPTICAL = 1, E2E_PSF_TABLE = 2 };
/* E2E_PREC_MIXED: the mapping's per-sample coefficients in FP64, its polynomial in the slit
 *                 coordinate in double-float FP32 (within ~1e-10 px of FP64); FP32 PSF stamps
 *                 from double-float edge arguments; FP32 sums
 *                 over runs of <= 16 stamps in registers; each item's box summed exactly in
 *                 52-bit fixed point (shared-memory integer atomics) and stored as an FP32
 *                 (hi, lo) pair; boxes merged into the frame with TwoSum compensation (the
 *                 fast path: per-pixel error <= 1e-6 relative against the FP64 definition).
 * E2E_PREC_FP64:  everything in FP64, one thread per stamp, FP64 global atomics (baseline). */
enum { E2E_PREC_MIXED = 0, E2E_PREC_FP64 = 1 };
enum { E2E_F32 = 0, E2E_F64 = 1, E2E_U16 = 2 /* detector ADU, e2e_add_noise output only */ };

/* ------------------------------------------------------------------ limits */
#define E2E_MAX_DEGREE 8  /* polynomial total degree */
#define E2E_MAX_K 15      /* window size (odd) */

typedef struct e2e_ctx e2e_ctx;

typedef struct {
  size_t pool_bytes; /* cap on the device scratch the context may hold (0 = no cap) */
  int32_t max_inflight; /* serving: jobs on the device at once (0 = default 4) */
  int32_t debug_checks; /* 1 = the mixed-precision kernels count every deposit that falls
                           outside its work item's planned box (or a run that outgrows its
                           planned tile) while on the detector; such deposits are dropped,
                           never written out of bounds.  The render then synchronises its
                           stream and returns E2E_EDEVICE if any were found. */
  int32_t kernel_timing; /* 1 = record CUDA events around each kernel of a render (see e2e_kernel_times) */
} e2e_opts;

/* One order-slice (trace).  Arrays are read during e2e_load_model only. */
typedef struct {
  int32_t detector;    /* index into the model's detectors */
  int32_t order;       /* diffraction order number (matches spectra) */
  int32_t fiber;       /* fiber id (matches spectra) */
  int32_t slice;       /* pupil slice id (informational) */
  int32_t degree;      /* total degree d of the (lt, s) polynomials, 0..E2E_MAX_DEGREE */
  int32_t K;           /* window size, odd, 1..E2E_MAX_K */
  int32_t n_lambda;    /* wavelength samples, >= 1 */
  int32_t n_slit;      /* slit points, >= 1 */
  double lambda_lo, lambda_hi; /* wavelength range (lambda_hi > lambda_lo) */
  const double* cx;    /* (d+1)(d+2)/2 coefficients of x, index(a,b) = t(t+1)/2 + b, t = a+b,
                          multiplying lt^a s^b (ordered by total degree, then a descending) */
  const double* cy;    /* same for y */
  double sigma_x[3];   /* PSF width (px) = c0 + c1 lt + c2 lt^2; must stay > 0 on [-1, 1] */
  double sigma_y[3];
  double theta;        /* E2E_PSF_ELLIPTICAL: rotation of the PSF axes (radians); with
                          vx, vy, cxy the rotated covariance at a sample, the shear
                          eps = cxy / sqrt(vx (vx vy - cxy^2)) must satisfy |eps| <= 0.2 at
                          every wavelength sample (about |theta| <= 20 deg for widths in
                          [1.2, 2.0] px): the renderers expand the conditional profile of
                          y given x in eps * tau over one pixel column */
  const double* slit_weights; /* n_slit weights u_k (finite), per aperture row with n_aper > 1 */
  double blaze_order;  /* echelle blaze of the order (the paper computes each order's blaze
                          profile analytically, Sec. 4.2): every sample's weight is multiplied by
                          B(lambda) = sinc^2(nu), nu = blaze_order * (1 - blaze_lambda / lambda),
                          sinc(x) = sin(pi x) / (pi x), at the sample's wavelength; 0 = no blaze */
  double blaze_lambda; /* blaze wavelength of the order (> 0 when blaze_order != 0) */
  /* E2E_PSF_TABLE: the PSF as tabulated maps (Sec. 2.1: the spectrograph unit delivers PSF
   * maps per projected fiber image; here sampled densities at field points along the order).
   * Map f samples the PSF density at offsets ((u - c)/q, (v - c)/q) px from the PSF centre,
   * c = (map_size - 1)/2, q = map_oversample; between samples the density is their bilinear
   * interpolant (zero beyond the grid); between field nodes the PSF is the linear blend in lt
   * of the two nodes' unit-mass maps (the end node beyond the ends).  A stamp's pixel values
   * are that density's integrals over the pixels for the PSF centred at the stamp's exact
   * position (Sec. 2.2).  For an integer q each pixel integral is a biquadratic in the
   * sub-pixel phase within cells of 1/q px; the library tabulates the biquadratics' exact
   * coefficients at load time (n_field x (q + 1)^2 x 9 x K^2 values in FP64 and FP32), so no
   * phase interpolation error enters. */
  int32_t n_field;          /* field nodes (>= 1) */
  const double* field_lt;   /* their normalised wavelengths, strictly increasing, in [-1, 1] */
  int32_t map_size;         /* M >= 2: each map is M x M samples, row v, column u */
  double map_oversample;    /* q: samples per pixel, an integer 1..32;
                               n_field x (q + 1)^2 must stay <= 65535 */
  const double* maps;       /* n_field * M * M densities, finite, >= 0, each map's sum > 0 */
  /* Two-dimensional fiber sub-aperture (Sec. 2.2: each fiber image is the fiber's spatial
   * profile convolved with the PSF).  n_aper <= 1: a one-dimensional pseudo-slit in s, and
   * slit_weights holds n_slit values.  n_aper > 1: aperture rows t_l = -1 + (2l + 1)/n_aper;
   * slit_weights holds n_slit values per row, row-major (u[l n_slit + k]), and the image of
   * point (s_k, t_l) is the pseudo-slit's at s_k moved by t_l (aper_x(lt), aper_y(lt)) px,
   * aper_x and aper_y quadratics c0 + c1 lt + c2 lt^2.  The library renders such a slice as
   * n_aper one-dimensional slices, one per row, whose lt^q s^0 coefficients are moved by
   * t_l aper_q (their degree raised to 2 where aper has a quadratic term): the stamp numbering
   * of e2e_window_origins and the photon renderer's streams count those rows as slices, in
   * model order.  The aperture itself (aper_x, aper_y) is not differentiated by the adjoint. */
  int32_t n_aper;           /* 0..64 */
  double aper_x[3];
  double aper_y[3];
} e2e_order_slice;

typedef struct {
  int32_t n_detectors;
  const int32_t* height; /* rows per detector (y) */
  const int32_t* width;  /* columns per detector (x) */
  int32_t n_slices;
  const e2e_order_slice* slices;
  int32_t psf;           /* E2E_PSF_SEPARABLE, E2E_PSF_ELLIPTICAL or E2E_PSF_TABLE */
} e2e_model_desc;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  opts may be NULL (defaults).
 * Errors: E2E_EINVAL (bad device), E2E_ECUDA. */
int e2e_create(e2e_ctx** out, int32_t device, const e2e_opts* opts);

/* Destroy a context and free everything it owns (models, spectra, frames, scratch).
 * Synchronises the device first.  NULL is a no-op. */
void e2e_destroy(e2e_ctx* ctx);

/* Text of the last error reported to the calling thread ("" if none).  Valid until the
 * thread's next failing call. */
const char* e2e_last_error(void);

/* ------------------------------------------------------------------ resident data */

/* Load an optical model (the spectral-format database of Sec. 2.1, which the paper
 * computes once and reuses across simulations): validates it (degree, K odd, widths > 0 on
 * [-1, 1], finite coefficients, |eps| <= 0.2 for the elliptical PSF), copies it to the
 * device and plans the tiled render (synchronous; uses the context's device).  Resident per
 * model: the slices, the plan (items, merge tiles and their lists), and per wavelength sample
 * of every slice (degree + 3) x 16 bytes of precomputed mapping coefficients and PSF constants
 * (261 MB for a 9216^2 frame of 340 slices x 6000 samples at degree 5); the tabulated PSF adds
 * its coefficient tables.
 * Errors: E2E_EINVAL, E2E_ENOMEM, E2E_ECUDA. */
int e2e_load_model(e2e_ctx* ctx, const e2e_model_desc* desc, uint64_t* model_id);
int e2e_unload_model(e2e_ctx* ctx, uint64_t model_id);

/* Load the spectrum of one fiber: n_orders orders (order_ids), order i holding n_lambda[i]
 * flux samples (photons per Angstrom at the bin centres of that order's order-slices),
 * packed consecutively in `flux`.  Copied to the device (synchronous).
 * Errors: E2E_EINVAL (non-finite flux, duplicate order), E2E_ENOMEM, E2E_ECUDA. */
int e2e_load_spectrum(e2e_ctx* ctx, int32_t fiber, int32_t n_orders, const int32_t* order_ids,
                      const int32_t* n_lambda, const double* flux, uint64_t* spec_id);
int e2e_unload_spectrum(e2e_ctx* ctx, uint64_t spec_id);

/* ------------------------------------------------------------------ render */

/* Render every detector of `model` lit by the spectra `spec_ids` (one per fiber used by
 * the model; each order-slice takes the row of its fiber's spectrum for its order, whose
 * length must equal its n_lambda).  The frame is the image model of Sec. 2.2: for every
 * order-slice, wavelength sample and slit (sub-aperture) point, the PSF integrated over each
 * pixel of the K x K window around the point's mapped position (spectral format of Sec.
 * 2.1), weighted by the sampled flux times the bin width times the point's weight, summed.
 *   dst[d]: device pointer to detector d's frame, row-major, dtype E2E_F32 or E2E_F64,
 *           pitch_elems[d] elements between rows (pitch_elems may be NULL = width).
 *           Every pixel of the frame is written.
 *   precision: E2E_PREC_MIXED or E2E_PREC_FP64.
 * Asynchronous on `stream`; scratch comes from the context and is released in stream
 * order.  Errors: E2E_EINVAL, E2E_ENOTFOUND, E2E_ENOMEM, E2E_ECUDA. */
int e2e_render(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t precision,
               int32_t dtype, void* const* dst, const int64_t* pitch_elems, void* stream);

/* As e2e_render (the Sec. 2.2 frame), into frames the library allocates (stream-ordered, from the device's
 * memory pool, on `stream`) and owns until e2e_release_frame. */
int e2e_render_alloc(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids,
                     int32_t precision, int32_t dtype, void* stream, uint64_t* frame_id);

/* Copy detector `detector` of a library-owned frame (the Sec. 2.2 frame of e2e_render_alloc;
 * height*width elements of its dtype,
 * row-major) to dst (device or host memory, `bytes` must equal the frame's size).
 * Stream-ordered on `stream`, after the frame's render wherever that was enqueued; a host
 * destination is complete when the stream is.
 * e2e_release_frame returns the buffers to the pool after every enqueued use of the frame
 * (its render and fetches) has completed; it does not block the caller. */
int e2e_fetch_frame(e2e_ctx* ctx, uint64_t frame_id, int32_t detector, void* dst, int32_t dst_is_device,
                    size_t bytes, void* stream);
int e2e_release_frame(e2e_ctx* ctx, uint64_t frame_id);

/* Render every detector of `model` (the Sec. 2.2 frame, as e2e_render) into HOST memory, overlapping the
 * device-to-host copy with the render: the mixed-precision frame is rendered in up to 16
 * bands of rows (whole merge tiles, the same fraction of every detector), and each band is
 * copied to host_dst[d] as soon as its pixels are final, while later bands still render.
 * The pixels equal those e2e_render writes for the same model and spectra.  E2E_PREC_FP64
 * renders the whole frame first and then copies it.
 *   host_dst[d]: host pointer to detector d's frame, row-major, dtype E2E_F32 or E2E_F64,
 *                pitch_elems[d] elements between rows (pitch_elems may be NULL = width).
 *                Page-locked memory (cudaHostAlloc / cudaHostRegister) lets the copies run
 *                asynchronously; pageable memory is accepted, but then each band's copy
 *                blocks the calling thread until that band is done.  Device memory is
 *                rejected (E2E_EINVAL).
 * The frame is complete when `stream` is.  Scratch (the device frame, box store) comes from
 * the context, in stream order on `stream`; the library's own side streams wait for work
 * enqueued on `stream` before the call and `stream` waits for them.
 * Errors: E2E_EINVAL, E2E_ENOTFOUND, E2E_ENOMEM, E2E_ECUDA, E2E_EDEVICE (debug checks). */
int e2e_render_host(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t precision,
                    int32_t dtype, void* const* host_dst, const int64_t* pitch_elems, void* stream);

/* ------------------------------------------------------------------ differentiation */

/* Gradient of a frame loss L with respect to the optical model, for calibration fitting:
 * the vector-Jacobian product  g = sum over pixels of dL/dI * dI/dtheta  of the render of a
 * separable-PSF model lit by spec_ids, for theta = every order-slice's mapping coefficients
 * (cx, cy) and PSF-width coefficients (sigma_x, sigma_y).  Each stamp's window is held at the
 * origin the forward render picks (the frame is piecewise smooth in the coefficients; its
 * jumps where a centre crosses a pixel edge are excluded).  The pixel-integral derivatives
 * follow from the PSF model of Sec. 2.1/2.2: dA/dx_c = -(phi(u1) - phi(u0))/sigma and
 * dA/dsigma = -(u1 phi(u1) - u0 phi(u0))/sigma for a pixel between edges u0 < u1.
 *   dldi[d]: device pointer to detector d's dL/dI (dtype E2E_F32 / E2E_F64, pitch_elems[d]
 *            elements per row; pitch_elems may be NULL = width).
 *   g_cx, g_cy: device FP64 arrays of sum over slices of (d+1)(d+2)/2 entries, the slices'
 *            coefficient vectors concatenated in model order; g_sx, g_sy: 3 per slice.  They
 *            are overwritten.
 *   frozen_windows: NULL, or a device array of 2 int32 per stamp, (i0, r0) in the stamp order
 *            of e2e_window_origins, 8-byte aligned: the windows are then held at these
 *            origins instead of those the mapping picks (the gradient of the frame that
 *            e2e_render_frozen renders with them).  Origins are expected within a pixel or so
 *            of the mapping's own (for instance those of the unperturbed model in a central-
 *            difference check, or of an earlier fitting iteration); stamps whose own window
 *            lies wholly off the detector are skipped.
 * Asynchronous on `stream`.  Errors: E2E_EINVAL (elliptical PSF, bad arguments),
 * E2E_ENOTFOUND, E2E_ENOMEM, E2E_ECUDA. */
int e2e_render_adjoint(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t dtype,
                       const void* const* dldi, const int64_t* pitch_elems, double* g_cx, double* g_cy,
                       double* g_sx, double* g_sy, const int32_t* frozen_windows, void* stream);

/* Window origins of every stamp of a resident model: origins[2 s] = i0 and origins[2 s + 1] = r0,
 * the lower-left pixel of stamp s's K x K window, floor(x_c + 1/2) - K/2 (likewise in y), with
 * x_c mapped in FP64.  Stamps are numbered slice by slice in model order, then by wavelength
 * sample j, then by slit point k: s = sum of earlier slices' n_lambda n_slit + j n_slit + k.
 * The truncated frame jumps where a centre crosses a pixel edge; holding the windows at these
 * origins (e2e_render_frozen, e2e_render_adjoint) gives the smooth frame whose derivative the
 * adjoint computes (window re-centring is excluded from the gradient).
 *   origins: device array of 2 x (number of stamps) int32, 8-byte aligned.
 * Asynchronous on `stream`.  Errors: E2E_EINVAL, E2E_ENOTFOUND, E2E_ECUDA. */
int e2e_window_origins(e2e_ctx* ctx, uint64_t model_id, int32_t* origins, void* stream);

/* Render (FP64, separable PSF) with every stamp's window held at the given origins instead of
 * the one its mapped centre picks: the forward companion of the adjoint's frozen windows, for
 * central-difference checks and fitting with fixed windows.  Pixel integrals are exact for
 * any origin (the stamp's centre need not lie in the window's centre pixel).
 *   frozen_windows: device array in the layout of e2e_window_origins (8-byte aligned).
 * Other arguments as for e2e_render with precision E2E_PREC_FP64.
 * Errors: E2E_EINVAL (not a separable-PSF model, bad arguments), E2E_ENOTFOUND, E2E_ENOMEM,
 * E2E_ECUDA. */
int e2e_render_frozen(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids,
                      const int32_t* frozen_windows, int32_t dtype, void* const* dst, const int64_t* pitch_elems,
                      void* stream);

/* Replace the mapping and PSF-width coefficients of a resident model (host arrays laid out
 * as the gradients of e2e_render_adjoint), validate them as e2e_load_model does, and re-plan.
 * Synchronous: waits for the device before replacing what in-flight work may read.
 * Errors: E2E_EINVAL (the model keeps its old coefficients), E2E_ENOTFOUND, E2E_ECUDA. */
int e2e_update_model(e2e_ctx* ctx, uint64_t model_id, const double* cx, const double* cy, const double* sx,
                     const double* sy);

/* ------------------------------------------------------------------ photon Monte-Carlo */

/* Render by tracing individual photons (the alternative to the stamp method that Sec. 2.2
 * describes: photons drawn from the spectrum with an assumed fiber illumination and an
 * analytic PSF, binned into pixels).  For order-slice i and wavelength bin j:
 *   N_ij ~ Poisson(flux[j] * dlam * sum_k u_k) photons; photon p gets a wavelength uniform in
 *   its bin, a slit point k with probability u_k / sum u and a position uniform in that
 *   point's bin, the spectral-format mapping, a PSF offset (the model's separable or rotated
 *   Gaussian, not truncated), and is counted in the pixel containing it if on the detector.
 * Draws come from Philox4x32-10 keyed by `seed`, indexed by (bin, slice, photon, stream): the
 * frame is a pure function of (model, spectra, seed).
 *   dst[d]: device uint32 frames (overwritten), pitch_elems as for e2e_render;
 *   total_photons: host pointer or NULL; when given, the call waits for the stream and
 *                  stores the number of photons drawn (on and off the detectors).
 * Slit weights must be >= 0.  Errors: E2E_EINVAL, E2E_ENOTFOUND, E2E_ENOMEM, E2E_ECUDA. */
int e2e_render_photons(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, uint64_t seed,
                       uint32_t* const* dst, const int64_t* pitch_elems, uint64_t* total_photons, void* stream);

/* ------------------------------------------------------------------ detector noise */

/* Noise stage applied to rendered frames (Sec. 2.2 ends the simulation by adding photon
 * noise, dark current, read-out noise, pixel response non-uniformity and cross-talk to the
 * synthetic frame; it gives no formulas, this is the model used).  For detector d of width W,
 * pixel (r, c), rendered value S (expected electrons):
 *   lam = max((1 + prnu z) S + dark_e, 0);  N ~ Poisson(lam) (N = lam when poisson = 0);
 *   M = N + xtalk N(r, W-1-c)  (the mirror pixel, read by the other amplifier of a two-output
 *       detector; the middle column of an odd width has none);
 *   E = M + ron_e g;  ADU = clamp(floor(bias + E / gain + 1/2), 0, saturation);
 * z (fixed pattern, from pattern_seed) and g (from seed) are standard normals.  Draws come
 * from Philox4x32-10 keyed by the seeds with counter (pair, detector, trial, stream), so a
 * frame is a pure function of (S, parameters, seeds): the same on every launch shape. */
typedef struct {
  uint64_t seed;          /* frame seed: shot noise and read-out noise */
  uint64_t pattern_seed;  /* fixed-pattern seed: pixel response */
  double dark_e;          /* mean dark electrons per pixel over the exposure, >= 0 */
  double prnu;            /* relative rms of the pixel response, >= 0 */
  double ron_e;           /* read-out noise rms (electrons), >= 0 */
  double xtalk;           /* cross-talk fraction, |xtalk| < 1 */
  double gain;            /* electrons per ADU, > 0 (E2E_U16 output) */
  double bias;            /* ADU offset (E2E_U16 output) */
  int32_t saturation;     /* ADU ceiling, 0..65535 (E2E_U16 output) */
  int32_t poisson;        /* 1 = Poisson shot noise, 0 = expected values */
} e2e_noise_params;

/* Apply the noise stage to every detector frame of `model` (sizes from the model).
 *   src[d]: device frame of expected electrons, src_dtype E2E_F32 or E2E_F64, src_pitch[d]
 *           elements between rows (NULL = width);
 *   dst[d]: device output, dst_dtype E2E_F32 / E2E_F64 (electrons) or E2E_U16 (ADU),
 *           dst_pitch as src; dst may be src (same dtype and pitch) for in-place noise.
 * Asynchronous on `stream`.  Errors: E2E_EINVAL, E2E_ENOTFOUND, E2E_ECUDA. */
int e2e_add_noise(e2e_ctx* ctx, uint64_t model_id, const e2e_noise_params* params, int32_t src_dtype,
                  const void* const* src, const int64_t* src_pitch, int32_t dst_dtype, void* const* dst,
                  const int64_t* dst_pitch, void* stream);

/* ------------------------------------------------------------------ serving */

/* The paper spreads many simulation jobs over cloud workers (Sec. 3); here one GPU serves a
 * stream of render jobs of uneven size.
 * A persistent request loop (a host thread per context) renders jobs with continuous
 * batching: a job that arrives while others run is admitted as soon as a slot (a CUDA stream)
 * and enough of the memory budget are free, and its kernels then run on the device
 * concurrently with the jobs already in flight.  Models and spectra stay resident.  A job's
 * frame is bitwise the same whether it ran alone or in the mix (the renderer is
 * deterministic). */
typedef struct {
  int32_t max_inflight; /* slots (streams); 0 = the context's max_inflight */
  size_t budget_bytes;  /* device memory the in-flight jobs may hold (scratch + library frames);
                           0 = the context's pool_bytes, or else 90% of the free HBM at start */
  int64_t express_stamps; /* jobs of at most this many stamps are "express": admitted before
                             any queued regular job and run on high-priority streams, so
                             small jobs do not wait behind full frames (0 = one FIFO class) */
  int32_t express_slots;  /* with express jobs: slots regular jobs leave free for them
                             (0 = max_inflight / 4, at least 1; at most max_inflight - 1) */
} e2e_server_cfg;

typedef struct {
  uint64_t model_id;
  int32_t n_spec;
  const uint64_t* spec_ids;  /* copied at submit */
  int32_t precision;         /* E2E_PREC_MIXED or E2E_PREC_FP64 */
  int32_t dtype;             /* E2E_F32 or E2E_F64 */
  void* const* dst;          /* per-detector device frames (copied at submit), or NULL: the library
                                allocates the job's frames (e2e_job_info.frame_id; fetch with
                                e2e_fetch_frame, free with e2e_release_frame) */
  const int64_t* pitch_elems;  /* as for e2e_render; may be NULL */
} e2e_job;

enum { E2E_JOB_DONE = 0, E2E_JOB_RUNNING = 1, E2E_JOB_QUEUED = 2 };

typedef struct {
  int32_t status;        /* E2E_JOB_DONE / RUNNING / QUEUED, or a negative error code */
  double submit_ms;      /* host times, ms since the server started */
  double admit_ms;
  double done_ms;
  double device_ms;      /* CUDA-event time from the job's first kernel to its last */
  int64_t budget_bytes;  /* memory the job held while in flight */
  uint64_t frame_id;     /* library-owned frames, else 0 */
  int64_t stamps;
} e2e_job_info;

/* Start the loop.  Errors: E2E_EINVAL (already running), E2E_ECUDA, E2E_ENOMEM. */
int e2e_server_start(e2e_ctx* ctx, const e2e_server_cfg* cfg);
/* Queue a job.  Validates it (model, spectra, dtype); a job whose memory can never fit the
 * budget is refused with E2E_ETOOBIG.  Thread-safe. */
int e2e_submit(e2e_ctx* ctx, const e2e_job* job, uint64_t* request_id);
/* Non-blocking status (info may be NULL).  Returns E2E_OK, or E2E_ENOTFOUND. */
int e2e_poll(e2e_ctx* ctx, uint64_t request_id, e2e_job_info* info);
/* Wait up to timeout_ms (< 0: forever) for a job to finish: E2E_OK when done (info filled),
 * E2E_ETIMEOUT if it has not finished in time, or the job's error. */
int e2e_wait(e2e_ctx* ctx, uint64_t request_id, int32_t timeout_ms, e2e_job_info* info);
/* Cancel a job that is still queued (E2E_ECANCELLED afterwards); running jobs finish. */
int e2e_cancel(e2e_ctx* ctx, uint64_t request_id);
/* Forget a finished job's record (its library frames stay until e2e_release_frame). */
int e2e_forget(e2e_ctx* ctx, uint64_t request_id);
/* Stop admitting, wait for every admitted job, stop the loop.  Queued jobs are cancelled. */
int e2e_server_stop(e2e_ctx* ctx);

/* Shape of the mixed-precision plan chosen for a model (for reports/tests): chunk of
 * wavelength samples per work item, slit points per register run, tile slack, number of
 * work items, tile size of the merge, and bytes of scratch one render needs. */
typedef struct {
  int32_t chunk_lambda, run_slit, slack_x, slack_y;
  int64_t n_items, n_tiles, scratch_bytes;
  int32_t tile_w, tile_h, boxes_per_cta, max_box_area;
} e2e_plan_info;
int e2e_model_plan(e2e_ctx* ctx, uint64_t model_id, e2e_plan_info* info);

/* Kernel timing (contexts created with kernel_timing = 1): durations in milliseconds of the
 * kernels of the context's most recent render, measured with CUDA events recorded on the
 * render's stream around each launch.  Blocks until those events complete.  Writes up to
 * `cap` entries: names[i] points to a static string naming the kernel; *n receives the
 * number of kernels.  Errors: E2E_EINVAL (timing not enabled), E2E_ECUDA. */
int e2e_kernel_times(e2e_ctx* ctx, const char** names, float* ms, int32_t cap, int32_t* n);

/* Render without allocating (no counterpart in the paper: a deployment convenience).
 * Some callers cannot allocate device memory while they run: a process whose device memory
 * is already reserved by another runtime (for instance a deep-learning framework's caching
 * allocator holding most of the GPU), or a real-time pipeline that must not allocate after
 * start-up because an allocation can block the stream or fail mid-observation.  This entry
 * point renders like e2e_render with precision E2E_PREC_MIXED, but takes its scratch (the
 * per-item box store and the small launch tables) from a fixed buffer of
 * E2E_STATIC_SCRATCH_BYTES that the library holds in device memory on every GPU it is loaded
 * on, until the process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - A model whose scratch (e2e_plan_info.scratch_bytes plus a few KB of tables) exceeds the
 *     buffer is rejected with E2E_ETOOBIG and a message giving both sizes.
 *   - The first call on a device looks up the buffer's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.
 *   - All calls share the one buffer and it keeps the previous call's contents; nothing in
 *     it needs to start at zero (every call rewrites all it reads).  Calls whose work
 *     overlaps on the GPU (different streams, or another thread) race on the buffer: order
 *     them on one stream or synchronise between them.
 *   - The frames are bitwise those of e2e_render with E2E_PREC_MIXED (same kernels, same
 *     exact box sums, same merge order).  Kernel timing and debug checks work as there: the
 *     timing events come from the context's pool and the check counter was allocated with
 *     the context.
 * Arguments as for e2e_render (dst/pitch per detector, dtype E2E_F32 or E2E_F64).
 * Errors: E2E_EINVAL, E2E_ENOTFOUND, E2E_ETOOBIG, E2E_ECUDA, E2E_EDEVICE (debug checks). */
#define E2E_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
int e2e_render_static(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t dtype,
                      void* const* dst, const int64_t* pitch_elems, void* stream);

/* Diagnostic: out[i] = the FP32 Gaussian tail erfc(|u[i]|) the renderer's mixed-precision
 * kernels use (the pixel integral of Sec. 2.2 is a difference of two such tails), with u[i]
 * taken as a double-float (hi = (float)u, lo = (float)(u - hi)).  u_dev (n doubles) and
 * out_dev (n floats) are device pointers; asynchronous on `stream`.  Errors: E2E_EINVAL,
 * E2E_ECUDA. */
int e2e_eval_tail(const double* u_dev, int64_t n, float* out_dev, void* stream);

/* Diagnostic: as e2e_eval_tail, with the cheaper rational the separable kernel uses on the
 * edges one or more pixels from a stamp's centre when the model's widest PSF (at most ~2.12 px)
 * keeps those edges' arguments at or above 0.4 in log2 units (|u| >= 0.4 / sqrt(log2 e) ~=
 * 0.333, the range the rational is fitted on; outside it the result is unspecified).  Same
 * arguments, layout and errors as e2e_eval_tail. */
int e2e_eval_tail_far(const double* u_dev, int64_t n, float* out_dev, void* stream);

/* Diagnostic (no counterpart in the paper): the fused multiply-add probe behind the roofline
 * of the ALU-bound renderers.  Launches `blocks` CTAs of 256 threads, each thread running 8
 * independent FMA chains of `iters` steps in FP64 (fp64 != 0) or FP32, and writes one value
 * per thread to sink_dev (blocks * 256 elements of that type, device memory).  *fmas receives
 * the number of FMAs the launch performs; the caller times it (CUDA events on `stream`) to get
 * the pipe's FMA rate.  Errors: E2E_EINVAL, E2E_ECUDA. */
int e2e_fma_probe(int32_t fp64, int32_t blocks, int32_t iters, void* sink_dev, int64_t* fmas, void* stream);

#ifdef __cplusplus
}
#endif
#endif
