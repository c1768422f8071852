// Per-sample tables of a resident model, built once per model (at load and after an update).
//
// Every mixed-precision kernel and the planner need, per wavelength sample lt_j of an
// order-slice, the coefficients P_b(lt_j) of the mapping's polynomial in s (Horner in lt of
// the spectral format, Sec. 2.1) and a few PSF constants.  Computed in FP64 in each CTA's
// prologue they ran on 32 of the CTA's threads while the rest waited, on a pipe with 1/64 of
// the FP32 rate; here one thread per (slice, sample) computes them once per model.  Row j of
// a slice (DevSlice::samples + j (degree + 3)):
//
//   [0, degree]   split_xy(P_b of x, P_b of y), b = 0..degree (double-float pairs)
//   [degree + 1]  separable PSF: 1/(sqrt2 sigma) sqrt(log2 e) of x and y as (hi, lo) pairs;
//                 elliptical: the same for the x-marginal and the conditional width s_c;
//                 tabulated: the field nodes f0, f1 around lt (as int bits) and the weight of f1
//   [degree + 2]  elliptical: beta as (hi, lo), eps, -log2(e) / vx; else zero
#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "mixed_common.cuh"
#include "tail_coeffs.h"

namespace e2e {

__global__ void __launch_bounds__(256) k_sample_tables(const DevSlice* __restrict__ slices, int psf,
                                                       const TableSlice* __restrict__ ts,
                                                       const double* __restrict__ field_lt) {
  const DevSlice& S = slices[blockIdx.y];
  const int d = S.degree, w = d + 3;
  float4* rows = const_cast<float4*>(S.samples);
  const double inv_nl = 1.0 / (double)S.n_lambda;
  const double kq = kSqrtLog2eD * 0.70710678118654752440;  // edge arguments in log2 units
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n_lambda; j += gridDim.x * blockDim.x) {
    const double lt = norm_sample_r(j, S.n_lambda, inv_nl);
    float4* row = rows + (int64_t)j * w;
    for (int b = 0; b <= d; ++b) row[b] = split_xy(poly_lt_for_b(S.cx, d, b, lt), poly_lt_for_b(S.cy, d, b, lt));
    float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0;
    if (psf == 1) {  // elliptical
      const EllipParams p = ellip_params(S, lt);
      const float2 gx = split_df(kq / p.gx), gc = split_df(kq / p.sc), be = split_df(p.beta);
      e0 = make_float4(gx.x, gx.y, gc.x, gc.y);
      e1 = make_float4(be.x, be.y, (float)p.eps, (float)(-1.44269504088896340736 / p.vx));
    } else if (psf == 2) {  // tabulated: field nodes and weight
      const TableSlice& T = ts[blockIdx.y];
      int f0, f1;
      double wf;
      field_weight(field_lt + T.field_off, T.n_field, lt, f0, f1, wf);
      e0 = make_float4(__int_as_float(f0), __int_as_float(f1), (float)wf, 0.f);  // read back as int4
    } else {
      const double sgx = fma(fma(S.sx[2], lt, S.sx[1]), lt, S.sx[0]);
      const double sgy = fma(fma(S.sy[2], lt, S.sy[1]), lt, S.sy[0]);
      const float2 gx = split_df(kq / sgx), gy = split_df(kq / sgy);
      e0 = make_float4(gx.x, gx.y, gy.x, gy.y);
    }
    row[d + 1] = e0;
    row[d + 2] = e1;
  }
}

cudaError_t launch_sample_tables(const DevSlice* slices, int n_slices, int max_lambda, int psf, const TableSlice* ts,
                                 const double* field_lt, cudaStream_t st) {
  if (n_slices == 0 || max_lambda == 0) return cudaSuccess;
  const int bx = (max_lambda + 255) / 256 < 64 ? (max_lambda + 255) / 256 : 64;
  k_sample_tables<<<dim3(bx, n_slices), 256, 0, st>>>(slices, psf, ts, field_lt);
  return cudaGetLastError();
}

}  // namespace e2e
