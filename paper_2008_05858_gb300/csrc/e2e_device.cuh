// Device-side data layout and inline math shared by the renderer's kernels.
//
// The model of the paper's image simulator (Sec. 2.2): the frame is the superposition,
// over a wavelength grid, of pixel-integrated fiber images; the fiber image of one
// wavelength sample is a set of slit points, each a PSF "stamp" centred where the
// spectral-format polynomial maps (lambda, s), weighted by flux x bin width x the
// normalised slit illumination (Sec. 2.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define E2E_MAXC 45  // (8+1)(8+2)/2 coefficients for total degree 8

namespace e2e {

// One order-slice as the kernels read it (copied once per model; __ldg'd).
struct DevSlice {
  double cx[E2E_MAXC];  // x(lt, s) coefficients, index(a,b) = t(t+1)/2 + b
  double cy[E2E_MAXC];
  double sx[3], sy[3];  // PSF width quadratics in lt (px)
  double dlam;          // wavelength bin width (lambda_hi - lambda_lo) / n_lambda
  double cos_t, sin_t;  // elliptical PSF axis rotation
  double blaze_m, blaze_lc;  // blaze function: order (0 = none) and blaze wavelength
  double lambda_lo;          // start of the wavelength range
  int32_t degree, K, n_lambda, n_slit;
  int32_t det, H, W, flux_slot;  // detector, its size, index into the per-render flux table
  int64_t u_off;                 // offset of this slice's slit weights in the model's weight array
  int64_t stamp_off;             // first global stamp index of this slice (FP64 path)
  int32_t coef_off;              // offset of this slice's cx / cy in the concatenated gradients
  int32_t index;                 // position of the slice in the model
  // per-sample table, built once per model (k_sample_tables): for wavelength sample j, the
  // degree + 3 float4 at samples + j (degree + 3): the s-polynomial's coefficients P_b(lt_j)
  // as split_xy pairs (b = 0..degree), then two float4 of PSF constants (see sample_tables.cu)
  const float4* samples;
};

// A mixed-path work item: a block of wavelength samples x a block of slit points of one
// slice; its stamps' windows, clipped to the detector, lie in box (bx0, by0, bw, bh).
struct Item {
  int32_t slice, j0, nj, k0, nk;  // wavelength samples [j0, j0+nj), slit points [k0, k0+nk)
  int32_t bx0, by0, bw, bh;
  int32_t pad;
  int64_t store_off;  // offset (elements) of this item's box in the render's box store
};

// Tabulated-PSF slice: its maps, field nodes and per-cell phase polynomials in the model's
// arrays.  The sub-pixel phase range [-1/2, 1/2] of each axis is cut into n_cell cells of
// width 1/q (q + 1 cells, the end ones half as wide, when map_size is even); per field node,
// cell (cy, cx) and window pixel the table holds the 9 coefficients of the pixel integral's
// biquadratic in the cell.
struct TableSlice {
  int64_t tab_off;    // first FP64 entry (n_field x n_cell^2 x 9 rows of K^2)
  int64_t tab_off32;  // first FP32 entry (n_field x n_cell^2 x 9 rows of table_row32(K) floats)
  int64_t map_off;    // first map sample (n_field x M^2)
  int32_t field_off;  // first field node
  int32_t n_field, map_size, K;
  int32_t q;          // map samples per pixel (an integer)
  int32_t n_cell;     // phase cells per axis
  int32_t half;       // 1 when map_size is even (cells start half a cell into the phase range)
  int32_t pad;
};

// Floats per FP32 table row: the K^2 window pixels padded to a multiple of 32, so that every
// row starts on a 128-byte line and a warp's 32 consecutive reads touch 4 sectors, not 5.
__host__ __device__ constexpr int table_row32(int K) { return (K * K + 31) / 32 * 32; }

// Output tile of the merge: tile (tx, ty) of detector det lists items[list_off .. list_off+n).
struct Tile {
  int32_t det, x0, y0, n;
  int64_t list_off;
};

__host__ __device__ inline int coeff_index(int a, int b) {
  int t = a + b;
  return t * (t + 1) / 2 + b;
}

// Normalised wavelength of bin-centred sample j of n: lt = (2j + 1 - n) / n in [-1, 1].
// Numerator and denominator are exact in FP64, so this is correctly rounded.
__device__ __forceinline__ double norm_sample(int j, int n) { return (double)(2 * j + 1 - n) / (double)n; }

// Per-wavelength-sample coefficients of the polynomial in s: P_b(lt) = sum_a c_ab lt^a
// (Horner in lt), b = 0..d.  x(lt, s) is then sum_b P_b s^b.
__device__ __forceinline__ double poly_lt_for_b(const double* c, int degree, int b, double lt) {
  double p = 0.0;
  for (int a = degree - b; a >= 0; --a) p = fma(p, lt, c[coeff_index(a, b)]);
  return p;
}

// Window-centre marker for a mapped coordinate outside |v| < 2^15 px (or not finite): the
// stamp lies off every detector and deposits nothing.
constexpr int kOffFrame = -(1 << 28);

// Split an FP64 pixel coordinate into the window-centre pixel floor(v + 1/2) and the
// offset v - that pixel in [-1/2, 1/2] as FP32, using integer operations on the bits of
// v + 1.5*2^16 (one FP64 add): for |v| < 2^15 the sum has the fixed exponent 16, so its low
// 52 mantissa bits are (v + 2^15) in fixed point with 36 fractional bits.  Anything else
// (including NaN) returns kOffFrame.  The offset keeps 32 fractional bits before rounding
// to FP32.
__device__ __forceinline__ void split_coord(double v, int& c, float& f) {
  const double magic = 98304.0;  // 1.5 * 2^16
  const double t = v + magic;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(t);
  if ((bits >> 52) != 1039ull) {  // sign 0, biased exponent 1023 + 16
    c = kOffFrame;
    f = 0.f;
    return;
  }
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;  // (v + 2^15) * 2^36
  m += (1ull << 35);                                   // + 1/2 pixel
  c = (int)(m >> 36) - 32768;
  const long long frac = (long long)(m & 0xFFFFFFFFFull) - (1ll << 35);  // in [-2^35, 2^35)
  f = (float)(int)(frac >> 4) * 2.3283064365386963e-10f;                 // * 2^-32
}

// Clamp a mapped coordinate for the plain FP64 renderer (far off-frame stamps are dropped).
__device__ __forceinline__ double clamp_coord(double v) {
  return fmin(fmax(v, -16000.0), 16000.0);
}

// x(s) = sum_b P_b s^b by Horner in s, for the (uniform) degree d: straight-line FMAs.
__device__ __forceinline__ double horner_s(const double* P, int d, double s) {
  switch (d) {
    case 0: return P[0];
    case 1: return fma(P[1], s, P[0]);
    case 2: return fma(fma(P[2], s, P[1]), s, P[0]);
    case 3: return fma(fma(fma(P[3], s, P[2]), s, P[1]), s, P[0]);
    case 4: return fma(fma(fma(fma(P[4], s, P[3]), s, P[2]), s, P[1]), s, P[0]);
    case 5: return fma(fma(fma(fma(fma(P[5], s, P[4]), s, P[3]), s, P[2]), s, P[1]), s, P[0]);
    case 6: return fma(fma(fma(fma(fma(fma(P[6], s, P[5]), s, P[4]), s, P[3]), s, P[2]), s, P[1]), s, P[0]);
    case 7:
      return fma(fma(fma(fma(fma(fma(fma(P[7], s, P[6]), s, P[5]), s, P[4]), s, P[3]), s, P[2]), s, P[1]), s, P[0]);
    default:
      return fma(fma(fma(fma(fma(fma(fma(fma(P[8], s, P[7]), s, P[6]), s, P[5]), s, P[4]), s, P[3]), s, P[2]), s,
                     P[1]),
                 s, P[0]);
  }
}

}  // namespace e2e
