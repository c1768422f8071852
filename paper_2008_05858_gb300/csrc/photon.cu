// Photon Monte-Carlo renderer: the alternative to the stamp method that Sec. 2.2 describes
// (photons drawn from the input spectrum, traced with an assumed fiber illumination and an
// analytic PSF to non-integer detector positions, and binned into pixels).
//
// For order-slice i and wavelength bin j (n bins, width dlam):
//   N_ij ~ Poisson(flux[j] dlam U),  U = sum_k u_k            blocks (j, i, trial, 4)
//   photon p < N_ij:  v, t from block (j, i, p, 5);  c from block (j, i, p, 6)
//     slit point k = the first with c U <= u_0 + .. + u_k;  lt = (2 (j + v) - n) / n,
//     s = (2 (k + t) - n_s) / n_s;  (x_c, y_c) = the spectral-format polynomials at (lt, s);
//     (z1, z2) = Box-Muller of block (j, i, p, 7);
//     separable PSF: (x, y) = (x_c + sigma_x z1, y_c + sigma_y z2); rotated PSF: the
//     x-marginal and y | x of the rotated covariance, x = x_c + g_x z1,
//     y = y_c + beta g_x z1 + s_c z2;
//     counted in pixel (floor(x + 1/2), floor(y + 1/2)) if that is on the detector.
//
// Four kernels: the photon count of every bin (one thread per bin, the Poisson sampler of
// philox.cuh), an exclusive scan of the counts, a guide table from evenly spaced photon numbers
// to their bins, and one thread per photon, which finds its bin by binary search in the scan
// between two guide entries, so that every photon is a pure function of
// (seed, bin, slice, index) whatever the launch shape.  The pixel decisions are taken in FP64;
// counts are added with 32-bit integer atomics (exact, order-independent).
#include <climits>
#include <cstdint>

#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "philox.cuh"

namespace e2e {

// FP32 copy of a slice's mapping coefficients and the bounds its fast path uses: per
// coordinate 45 coefficients, then sum_a a |c_a0| (bounds the divided difference of the b = 0
// polynomial) and sum_{b >= 1} |c_ab| (bounds the slit terms); then the PSF-width
// coefficients sigma_x[0..2], sigma_y[0..2], the slit-weight total and one pad, all rounded
// to FP32 once on the host.
constexpr int kCfExtra = 2 * (E2E_MAXC + 2);
constexpr int kCf = kCfExtra + 8;

// Per bin: the photon count, and the bin centre's position at s = 0 in FP64, split into the
// nearest integer and an FP32 remainder (the anchor the FP32 fast path adds small terms to).
__global__ void __launch_bounds__(256) k_photon_bins(const DevSlice* __restrict__ slices, int n_slices,
                                                     const double* const* __restrict__ flux_tab,
                                                     const double* __restrict__ usum, const int64_t* __restrict__ bin_off,
                                                     uint64_t seed, uint64_t* __restrict__ counts,
                                                     int4* __restrict__ anchors, int* __restrict__ bin_slice) {
  const int64_t nb = bin_off[n_slices];
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_slices - 1;
    while (lo < hi) {  // slice owning bin b
      const int mid = (lo + hi + 1) >> 1;
      if (bin_off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const DevSlice& S = slices[lo];
    bin_slice[b] = lo;
    const int j = (int)(b - bin_off[lo]);
    const double lam = __dmul_rn(__dmul_rn(flux_tab[S.flux_slot][j], S.dlam), usum[lo]);
    counts[b] = (uint64_t)poisson_filtered(lam, seed, (uint32_t)j, (uint32_t)S.index, 4);
    const double ltj = norm_sample(j, S.n_lambda);
    const double X0 = poly_lt_for_b(S.cx, S.degree, 0, ltj), Y0 = poly_lt_for_b(S.cy, S.degree, 0, ltj);
    const bool ok = fabs(X0) < 1e9 && fabs(Y0) < 1e9;
    const double Xi = ok ? rint(X0) : 0.0, Yi = ok ? rint(Y0) : 0.0;
    anchors[b] = make_int4(ok ? (int)Xi : INT_MIN, __float_as_int((float)(X0 - Xi)), (int)Yi,
                           __float_as_int((float)(Y0 - Yi)));
  }
}

// ---------------------------------------------------------------- exclusive scan (uint64)

constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t v, uint64_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) s_warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  return v + (warp > 0 ? s_warp[warp - 1] : 0);
}

// Per-block exclusive scan of in[] into out[], block totals into sums[].
__global__ void __launch_bounds__(kScanThreads) k_scan_local(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                             int64_t n, uint64_t* __restrict__ sums) {
  __shared__ uint64_t s_warp[32];
  const int64_t i = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;
  const uint64_t v = i < n ? in[i] : 0;
  const uint64_t inc = block_inclusive_scan(v, s_warp);
  if (i < n) out[i] = inc - v;
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = inc;
}

// One block: exclusive scan of the block totals in place; total into *total.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint64_t* __restrict__ sums, int64_t nblocks,
                                                            uint64_t* __restrict__ total) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nblocks; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const uint64_t v = i < nblocks ? sums[i] : 0;
    const uint64_t inc = block_inclusive_scan(v, s_warp);
    const uint64_t carry = s_carry;
    if (i < nblocks) sums[i] = carry + inc - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) s_carry = carry + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(uint64_t* __restrict__ out, int64_t n,
                                                           const uint64_t* __restrict__ sums,
                                                           const uint64_t* __restrict__ total) {
  const int64_t i = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
  if (i == n) out[n] = *total;
}

// ---------------------------------------------------------------- photons

// Bin holding photon p: the last b in [lo, hi] with offsets[b] <= p.
__device__ __forceinline__ int64_t photon_bin(const uint64_t* __restrict__ offsets, uint64_t p, int64_t lo, int64_t hi) {
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// guide[g] = the bin of photon floor(g total / G), g = 0 .. G (G = kPhotonGuide): photon p
// lies in a bin between guide[g] and guide[g + 1] for g = floor(p G / total), so its search
// covers the few bins of one guide step instead of all of them.  Products g total and p G stay
// below 2^64 for totals below kGuidedPhotons; beyond, photons search all bins.
constexpr uint64_t kGuidedPhotons = 1ull << 44;
__global__ void __launch_bounds__(256) k_photon_guide(const uint64_t* __restrict__ offsets, int64_t nb,
                                                      int64_t* __restrict__ guide) {
  const uint64_t total = offsets[nb];
  if (total >= kGuidedPhotons) return;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= kPhotonGuide; g += gridDim.x * blockDim.x)
    guide[g] = photon_bin(offsets, (uint64_t)g * total / kPhotonGuide, 0, nb - 1);
}

// The photon's pixel by the definition, in FP64 (fx, fy: the pixel's column and row).
__device__ void photon_exact(const DevSlice& S, const double* __restrict__ C, double U, int psf, uint64_t seed,
                             uint32_t j, uint32_t si, uint32_t pp, const uint4& wa, const uint4& wb, double& fxo,
                             double& fyo) {
  const double v = uni53(wa.x, wa.y), t = uni53(wa.z, wa.w);
  const double cu = __dmul_rn(uni53(wb.x, wb.y), U);
  int k0 = 0, k1 = S.n_slit - 1;  // slit point: the first k with cu <= C_k, else the last
  while (k0 < k1) {
    const int mid = (k0 + k1) >> 1;
    if (cu <= C[mid]) k1 = mid; else k0 = mid + 1;
  }
  const double n = (double)S.n_lambda, ns = (double)S.n_slit;
  const double lt = __ddiv_rn(__dadd_rn(__dmul_rn(2.0, __dadd_rn((double)j, v)), -n), n);
  const double s = __ddiv_rn(__dadd_rn(__dmul_rn(2.0, __dadd_rn((double)k0, t)), -ns), ns);
  double px[9], py[9];
#pragma unroll
  for (int bb = 0; bb <= 8; ++bb) {
    px[bb] = bb <= S.degree ? poly_lt_for_b(S.cx, S.degree, bb, lt) : 0.0;
    py[bb] = bb <= S.degree ? poly_lt_for_b(S.cy, S.degree, bb, lt) : 0.0;
  }
  const double xc = horner_s(px, S.degree, s), yc = horner_s(py, S.degree, s);
  const double sa = fma(fma(S.sx[2], lt, S.sx[1]), lt, S.sx[0]);
  const double sb = fma(fma(S.sy[2], lt, S.sy[1]), lt, S.sy[0]);
  double z1, z2;
  normal_pair_ctr(seed, j, si, pp, 7, z1, z2);
  double x, y;
  if (psf == 0) {
    x = __dadd_rn(xc, __dmul_rn(sa, z1));
    y = __dadd_rn(yc, __dmul_rn(sb, z2));
  } else {
    const double a2 = sa * sa, b2 = sb * sb, c = S.cos_t, sn = S.sin_t;
    const double vx = a2 * c * c + b2 * sn * sn, vy = a2 * sn * sn + b2 * c * c, cxy = (a2 - b2) * sn * c;
    const double gx = sqrt(vx), beta = cxy / vx, sc = sqrt(vy - beta * cxy);
    const double dx = __dmul_rn(gx, z1);
    x = __dadd_rn(xc, dx);
    y = __dadd_rn(__dadd_rn(yc, __dmul_rn(beta, dx)), __dmul_rn(sc, z2));
  }
  fxo = floor(__dadd_rn(x, 0.5));
  fyo = floor(__dadd_rn(y, 0.5));
}

// Offset of the photon from the bin's anchor along one coordinate, in FP32, and a bound on its
// distance from the exact value: delta * Q(lt, lt_j) for the b = 0 polynomial (its divided
// difference, so no large terms cancel) plus the slit terms sum_{b>=1} P_b(lt) s^b.  D is the
// slice's degree, a template parameter so that only its terms are evaluated.
template <int D>
__device__ __forceinline__ float photon_offset(const float* cf, float lt, float ltj, float delta, float s,
                                               float& mag) {
  float q[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) q[a] = 0.f;
  // q_a = c_a0 + ltj q_{a+1} (a = D .. 1), Q = sum_a q_a lt^(a-1)
  float acc = 0.f;
#pragma unroll
  for (int a = D; a >= 1; --a) {
    acc = fmaf(ltj, acc, cf[a * (a + 1) / 2]);  // index(a, 0) = a(a+1)/2
    q[a - 1] = acc;
  }
  float Q = 0.f;
#pragma unroll
  for (int a = D; a >= 1; --a) Q = fmaf(Q, lt, q[a - 1]);
  // slit terms: Horner in s over P_b(lt), b = D .. 1
  float sb = 0.f;
#pragma unroll
  for (int b = D; b >= 1; --b) {
    float pb = 0.f;
#pragma unroll
    for (int a = D - b; a >= 0; --a) pb = fmaf(pb, lt, cf[(a + b) * (a + b + 1) / 2 + b]);
    sb = fmaf(sb, s, pb);
  }
  sb *= s;
  mag = fabsf(delta) * cf[E2E_MAXC] + cf[E2E_MAXC + 1];
  return fmaf(delta, Q, sb);
}

// Both coordinates' offsets for a slice of degree d (0 .. E2E_MAX_DEGREE).
__device__ __forceinline__ void photon_offsets(int d, const float* cf, float lt, float ltj, float delta, float s,
                                               float& ox, float& oy, float& mx, float& my) {
  switch (d) {
#define E2E_PO(D)                                                                   \
  case D:                                                                           \
    ox = photon_offset<D>(cf, lt, ltj, delta, s, mx);                               \
    oy = photon_offset<D>(cf + E2E_MAXC + 2, lt, ltj, delta, s, my);                \
    return;
    E2E_PO(0) E2E_PO(1) E2E_PO(2) E2E_PO(3) E2E_PO(4) E2E_PO(5) E2E_PO(6) E2E_PO(7)
#undef E2E_PO
    default:
      ox = photon_offset<8>(cf, lt, ltj, delta, s, mx);
      oy = photon_offset<8>(cf + E2E_MAXC + 2, lt, ltj, delta, s, my);
  }
}

// Four CTAs of 256 per SM (64 registers): the photons are latency-bound on their dependent
// Philox, search and coefficient loads; at the 80 registers the compiler picks unbounded, three
// CTAs fit and 1e9 photons took 75 ms against 32 ms.
#ifndef E2E_PHOTON_MIN_BLOCKS
#define E2E_PHOTON_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(256, E2E_PHOTON_MIN_BLOCKS) k_photons(const DevSlice* __restrict__ slices, int n_slices,
                                                 const double* __restrict__ ucum, const double* __restrict__ usum,
                                                 const int64_t* __restrict__ bin_off,
                                                 const uint64_t* __restrict__ offsets, int psf, uint64_t seed,
                                                 uint32_t* const* __restrict__ dst, const int64_t* __restrict__ pitch,
                                                 const float* __restrict__ ucum32, const float* __restrict__ cf32,
                                                 const int4* __restrict__ anchors, const int* __restrict__ bin_slice,
                                                 const int64_t* __restrict__ guide) {
  const int64_t nb = bin_off[n_slices];
  const uint64_t total = offsets[nb];
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (uint64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nb - 1;
    if (total < kGuidedPhotons) {
      const uint64_t g = p * kPhotonGuide / total;  // g < G since p < total
      lo = guide[g];
      hi = guide[g + 1];
    }
    const int64_t b = photon_bin(offsets, p, lo, hi);
    const int sl = bin_slice[b];
    const DevSlice& S = slices[sl];
    const uint32_t j = (uint32_t)(b - bin_off[sl]);
    const uint32_t pp = (uint32_t)(p - offsets[b]);
    const uint32_t si = (uint32_t)S.index;
    const uint4 wa = rng_block(seed, j, si, pp, 5), wb = rng_block(seed, j, si, pp, 6);
    const int4 an = anchors[b];
    double fx = 0.0, fy = 0.0;
    int ix = -1, iy = -1;
    bool exact = psf != 0 || an.x == INT_MIN;
    if (!exact) {
      // FP32 fast path: every decision is checked against its error bound; a photon too close
      // to a slit-point boundary or a pixel edge is redone in FP64 below
      const float* C32 = ucum32 + S.u_off;
      const float* cf = cf32 + (int64_t)sl * kCf;
      const float* ce = cf + kCfExtra;
      const float cu = uni53_f32(wb.x, wb.y) * ce[6];
      int k0 = 0, k1 = S.n_slit - 1;
      while (k0 < k1) {
        const int mid = (k0 + k1) >> 1;
        if (cu <= C32[mid]) k1 = mid; else k0 = mid + 1;
      }
      const float tol = 5e-7f * fabsf(cu) + 1e-30f;
      if (k0 < S.n_slit - 1 && !(C32[k0] - cu > tol)) exact = true;
      if (k0 > 0 && !(cu - C32[k0 - 1] > tol)) exact = true;
      const float n = (float)S.n_lambda, ns = (float)S.n_slit;
      const float delta = (2.f * uni53_f32(wa.x, wa.y) - 1.f) / n;
      const float ltj = (float)(2 * (int)j + 1 - S.n_lambda) / n;
      const float lt = ltj + delta;
      const float s = (2.f * ((float)k0 + uni53_f32(wa.z, wa.w)) - ns) / ns;
      float z1, z2, eg;
      normal_pair_f32_ctr(seed, j, si, pp, 7, z1, z2, eg);
      const float sx = fmaf(fmaf(ce[2], lt, ce[1]), lt, ce[0]);
      const float sy = fmaf(fmaf(ce[5], lt, ce[4]), lt, ce[3]);
      float mx, my, ox, oy;
      photon_offsets(S.degree, cf, lt, ltj, delta, s, ox, oy, mx, my);
      ox += sx * z1;
      oy += sy * z2;
      const float rx = __int_as_float(an.y) + ox + 0.5f, ry = __int_as_float(an.w) + oy + 0.5f;
      const float ein = 4e-7f * ((cf[E2E_MAXC] / n) + (float)S.degree * cf[E2E_MAXC + 1] / ns);
      const float einy = 4e-7f * ((cf[2 * E2E_MAXC + 2] / n) + (float)S.degree * cf[2 * E2E_MAXC + 3] / ns);
      const float ex = 1e-5f * (mx + fabsf(sx * z1) + 1.f) + ein + 1.5f * sx * eg;
      const float ey = 1e-5f * (my + fabsf(sy * z2) + 1.f) + einy + 1.5f * sy * eg;
      const float kx = floorf(rx - ex), ky = floorf(ry - ey);
      if (kx != floorf(rx + ex) || ky != floorf(ry + ey)) exact = true;
      if (!(fabsf(kx) < 0x1p30f && fabsf(ky) < 0x1p30f)) exact = true;  // also NaN
      ix = exact ? -1 : an.x + (int)kx;  // integers below 2^30: exact conversions, no overflow
      iy = exact ? -1 : an.z + (int)ky;
    }
    if (exact) {
      photon_exact(S, ucum + S.u_off, usum[sl], psf, seed, j, si, pp, wa, wb, fx, fy);
      const bool in = fx >= 0.0 && fx < (double)S.W && fy >= 0.0 && fy < (double)S.H;
      ix = in ? (int)fx : -1;
      iy = in ? (int)fy : -1;
    }
    if (ix >= 0 && ix < S.W && iy >= 0 && iy < S.H) atomicAdd(dst[S.det] + (int64_t)iy * pitch[S.det] + ix, 1u);
  }
}

static unsigned grid_for(uint64_t n, int threads, uint64_t cap) {
  const uint64_t b = n / threads + (n % threads ? 1 : 0);  // no overflow for any n
  return (unsigned)(b == 0 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_photon_bins(const DevSlice* slices, int n_slices, const double* const* flux_tab, const double* usum,
                               const int64_t* bin_off, int64_t n_bins, uint64_t seed, uint64_t* counts,
                               int4* anchors, int* bin_slice, cudaStream_t st) {
  if (n_bins == 0) return cudaSuccess;
  k_photon_bins<<<grid_for((uint64_t)n_bins, 256, 152 * 64), 256, 0, st>>>(slices, n_slices, flux_tab, usum, bin_off,
                                                                         seed, counts, anchors, bin_slice);
  return cudaGetLastError();
}

cudaError_t launch_photon_guide(const uint64_t* offsets, int64_t n_bins, int64_t* guide, cudaStream_t st) {
  if (n_bins == 0) return cudaSuccess;
  k_photon_guide<<<(kPhotonGuide + 1 + 255) / 256, 256, 0, st>>>(offsets, n_bins, guide);
  return cudaGetLastError();
}

size_t scan_scratch_elems(int64_t n) { return (size_t)((n + kScanThreads - 1) / kScanThreads) + 1; }

cudaError_t launch_scan_exclusive(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* scratch, cudaStream_t st) {
  const int64_t nblocks = (n + kScanThreads - 1) / kScanThreads;
  uint64_t* total = scratch + nblocks;
  if (nblocks > 0) k_scan_local<<<(unsigned)nblocks, kScanThreads, 0, st>>>(in, out, n, scratch);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(scratch, nblocks, total);
  k_scan_add<<<(unsigned)(n / kScanThreads + 1), kScanThreads, 0, st>>>(out, n, scratch, total);
  return cudaGetLastError();
}

size_t photon_coef_floats() { return (size_t)kCf; }

cudaError_t launch_photons(const DevSlice* slices, int n_slices, const double* ucum, const double* usum,
                           const int64_t* bin_off, const uint64_t* offsets, int psf, uint64_t seed,
                           uint32_t* const* dst, const int64_t* pitch, uint64_t max_photons, const float* ucum32,
                           const float* cf32, const int4* anchors, const int* bin_slice, const int64_t* guide,
                           cudaStream_t st) {
  if (max_photons == 0) return cudaSuccess;
  k_photons<<<grid_for(max_photons, 256, 152 * 32), 256, 0, st>>>(slices, n_slices, ucum, usum, bin_off, offsets, psf,
                                                                   seed, dst, pitch, ucum32, cf32, anchors, bin_slice,
                                                                   guide);
  return cudaGetLastError();
}

}  // namespace e2e
