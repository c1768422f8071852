// Plain FP64 renderer: one thread per stamp, FP64 mapping and erfc, FP64 atomic deposits.
//
// It is the straightforward GPU form of the image model (Sec. 2.2: the frame is the sum
// over wavelength samples and slit points of pixel-integrated PSF stamps) and the
// baseline the mixed-precision tiled renderer is measured against.
#include "e2e_device.cuh"
#include "e2e_kernels.h"

namespace e2e {

// P(a < Z < b) for a standard normal Z from the two edge values E = erfc(|t|/sqrt2):
// on one side of the mean the two tail probabilities are subtracted (no cancellation
// against 1), across the mean 1 minus both tails.
__device__ __forceinline__ double interval_from_erfc(double ta, double tb, double ea, double eb) {
  if (ta >= 0.0) return 0.5 * (ea - eb);
  if (tb <= 0.0) return 0.5 * (eb - ea);
  return 1.0 - 0.5 * (ea + eb);
}

// frozen (nullable): window origins (i0, r0) per stamp of the model, in stamp order (slice, then
// wavelength sample, then slit point), used instead of the windows the mapping picks.
template <int K>
__global__ void __launch_bounds__(256) k_render_fp64(const DevSlice* __restrict__ slices,
                                                     const double* const* __restrict__ flux_tab,
                                                     const double* __restrict__ u_all, double* const* acc,
                                                     const int64_t* __restrict__ pitch,
                                                     const int2* __restrict__ frozen) {
  const DevSlice& S = slices[blockIdx.y];
  if (S.K != K) return;  // launched once per window size over all slices
  const double* flux = flux_tab[S.flux_slot];
  const double* u = u_all + S.u_off;
  const int64_t n = (int64_t)S.n_lambda * S.n_slit;
  double* frame = acc[S.det];
  const int64_t P = pitch[S.det];
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / S.n_slit);
    const int k = (int)(idx - (int64_t)j * S.n_slit);
    const double lt = norm_sample(j, S.n_lambda);
    const double s = norm_sample(k, S.n_slit);
    // x = sum_b P_b(lt) s^b, Horner in s over Horner-in-lt coefficients
    double x = 0.0, y = 0.0;
    for (int b = S.degree; b >= 0; --b) {
      x = fma(x, s, poly_lt_for_b(S.cx, S.degree, b, lt));
      y = fma(y, s, poly_lt_for_b(S.cy, S.degree, b, lt));
    }
    const double sgx = fma(fma(S.sx[2], lt, S.sx[1]), lt, S.sx[0]);
    const double sgy = fma(fma(S.sy[2], lt, S.sy[1]), lt, S.sy[0]);
    const double w = flux[j] * S.dlam * u[k];
    x = clamp_coord(x);
    y = clamp_coord(y);
    int i0 = (int)floor(x + 0.5) - K / 2;
    int r0 = (int)floor(y + 0.5) - K / 2;
    if (frozen) {
      const int2 o = frozen[S.stamp_off + idx];
      i0 = o.x;
      r0 = o.y;
    }
    if (i0 + K <= 0 || i0 >= S.W || r0 + K <= 0 || r0 >= S.H) continue;
    const double ix = 1.0 / sgx, iy = 1.0 / sgy;
    double ax[K], ay[K];
    {
      double tp = ((double)i0 - 0.5 - x) * ix;
      double ep = erfc(fabs(tp) * 0.70710678118654752440);
#pragma unroll
      for (int m = 0; m < K; ++m) {
        double tn = ((double)(i0 + m) + 0.5 - x) * ix;
        double en = erfc(fabs(tn) * 0.70710678118654752440);
        ax[m] = w * interval_from_erfc(tp, tn, ep, en);
        tp = tn;
        ep = en;
      }
    }
    {
      double tp = ((double)r0 - 0.5 - y) * iy;
      double ep = erfc(fabs(tp) * 0.70710678118654752440);
#pragma unroll
      for (int m = 0; m < K; ++m) {
        double tn = ((double)(r0 + m) + 0.5 - y) * iy;
        double en = erfc(fabs(tn) * 0.70710678118654752440);
        ay[m] = interval_from_erfc(tp, tn, ep, en);
        tp = tn;
        ep = en;
      }
    }
#pragma unroll
    for (int nn = 0; nn < K; ++nn) {
      const int r = r0 + nn;
      if (r < 0 || r >= S.H) continue;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const int i = i0 + m;
        if (i < 0 || i >= S.W) continue;
        atomicAdd(frame + (int64_t)r * P + i, ax[m] * ay[nn]);
      }
    }
  }
}

// Window origins (i0, r0) of every stamp of the model as the FP64 renderer picks them.
__global__ void __launch_bounds__(256) k_window_origins(const DevSlice* __restrict__ slices, int2* __restrict__ out) {
  const DevSlice& S = slices[blockIdx.y];
  const int64_t n = (int64_t)S.n_lambda * S.n_slit;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / S.n_slit);
    const int k = (int)(idx - (int64_t)j * S.n_slit);
    const double lt = norm_sample(j, S.n_lambda);
    const double s = norm_sample(k, S.n_slit);
    double x = 0.0, y = 0.0;
    for (int b = S.degree; b >= 0; --b) {
      x = fma(x, s, poly_lt_for_b(S.cx, S.degree, b, lt));
      y = fma(y, s, poly_lt_for_b(S.cy, S.degree, b, lt));
    }
    x = clamp_coord(x);
    y = clamp_coord(y);
    out[S.stamp_off + idx] = make_int2((int)floor(x + 0.5) - S.K / 2, (int)floor(y + 0.5) - S.K / 2);
  }
}

cudaError_t launch_window_origins(int n_slices, int64_t max_stamps, const DevSlice* slices, int2* out,
                                  cudaStream_t st) {
  if (n_slices == 0 || max_stamps == 0) return cudaSuccess;
  int64_t bx = (max_stamps + 255) / 256;
  if (bx > 4096) bx = 4096;
  k_window_origins<<<dim3((unsigned)bx, (unsigned)n_slices), 256, 0, st>>>(slices, out);
  return cudaGetLastError();
}

// FP64 accumulation frame -> output frame of the requested dtype and pitch.
template <typename T>
__global__ void k_convert(const double* __restrict__ src, int64_t src_pitch, T* __restrict__ dst, int64_t dst_pitch,
                          int H, int W) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)H * W;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / W), c = (int)(idx - (int64_t)r * W);
    dst[(int64_t)r * dst_pitch + c] = (T)src[(int64_t)r * src_pitch + c];
  }
}

cudaError_t launch_render_fp64(int K, int n_slices, int64_t max_stamps, const DevSlice* slices,
                               const double* const* flux_tab, const double* u_all, double* const* acc,
                               const int64_t* pitch, cudaStream_t st, const int2* frozen) {
  if (n_slices == 0 || max_stamps == 0) return cudaSuccess;
  int64_t bx = (max_stamps + 255) / 256;
  if (bx > 4096) bx = 4096;
  dim3 grid((unsigned)bx, (unsigned)n_slices);
  switch (K) {
#define E2E_CASE(KK) \
  case KK: k_render_fp64<KK><<<grid, 256, 0, st>>>(slices, flux_tab, u_all, acc, pitch, frozen); break;
    E2E_CASE(1) E2E_CASE(3) E2E_CASE(5) E2E_CASE(7) E2E_CASE(9) E2E_CASE(11) E2E_CASE(13) E2E_CASE(15)
#undef E2E_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_convert(const double* src, int64_t src_pitch, void* dst, int dtype, int64_t dst_pitch, int H,
                           int W, cudaStream_t st) {
  int64_t n = (int64_t)H * W;
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (dtype == 0)
    k_convert<float><<<(unsigned)blocks, 256, 0, st>>>(src, src_pitch, (float*)dst, dst_pitch, H, W);
  else
    k_convert<double><<<(unsigned)blocks, 256, 0, st>>>(src, src_pitch, (double*)dst, dst_pitch, H, W);
  return cudaGetLastError();
}

}  // namespace e2e
