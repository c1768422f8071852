// Blaze weighting of the spectra.  The paper weights each order by the blaze profile of the
// echelle grating, computed analytically (Sec. 4.2); here an order-slice may carry a blaze
// function B(lambda) = sinc^2(nu), nu = m (1 - lambda_b / lambda), sinc(x) = sin(pi x) / (pi x)
// (m the order, lambda_b its blaze wavelength), which multiplies the weight of every sample
// at the sample's wavelength.  The renderers read spectra through a per-slice table of flux
// pointers; for a blazed model that table is redirected to B(lambda_j) * flux[j], made here
// once per render, so every renderer (stamps, FP64, adjoint, photons) sees the same weights.
#include "e2e_device.cuh"
#include "e2e_kernels.h"

namespace e2e {

__global__ void __launch_bounds__(256) k_blaze(const DevSlice* __restrict__ slices, int n_slices,
                                               const double* const* __restrict__ flux_in,
                                               const int64_t* __restrict__ bin_off, double* __restrict__ out) {
  const int64_t nb = bin_off[n_slices];
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_slices - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bin_off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const DevSlice& S = slices[lo];
    const int j = (int)(b - bin_off[lo]);
    double B = 1.0;
    if (S.blaze_m != 0.0) {
      const double lam = __dadd_rn(S.lambda_lo, __dmul_rn((double)j + 0.5, S.dlam));  // bin centre
      const double nu = __dmul_rn(S.blaze_m, __dadd_rn(1.0, -__ddiv_rn(S.blaze_lc, lam)));
      const double sc = nu == 0.0 ? 1.0 : __ddiv_rn(sinpi(nu), __dmul_rn(3.14159265358979323846, nu));
      B = __dmul_rn(sc, sc);
    }
    out[b] = __dmul_rn(flux_in[lo][j], B);
  }
}

cudaError_t launch_blaze(const DevSlice* slices, int n_slices, const double* const* flux_in, const int64_t* bin_off,
                         int64_t n_bins, double* out, cudaStream_t st) {
  if (n_bins == 0) return cudaSuccess;
  int64_t blocks = (n_bins + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_blaze<<<(unsigned)blocks, 256, 0, st>>>(slices, n_slices, flux_in, bin_off, out);
  return cudaGetLastError();
}

// Flag (flag = 1) if any of the n values is not finite: the check e2e_load_spectrum makes of
// an uploaded spectrum, on the device instead of a host pass over the host copy.
__global__ void __launch_bounds__(256) k_flag_nonfinite(const double* __restrict__ p, int64_t n, int* flag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

cudaError_t launch_flag_nonfinite(const double* p, int64_t n, int* flag, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_flag_nonfinite<<<(unsigned)blocks, 256, 0, st>>>(p, n, flag);
  return cudaGetLastError();
}

}  // namespace e2e
