// Adjoint of the separable render: the vector-Jacobian product of the frame with respect to
// the spectral-format polynomial coefficients and the PSF-width coefficients.
//
// For calibration fitting (matching rendered frames to observed ones) the gradient of a
// frame loss L with respect to the optical model is needed.  With dL/dI given per pixel and
// each stamp's window held at the origin the forward render chose, a stamp (w, A_x, A_y)
// contributes
//   dL/dx_c = w sum_m dA_x[m]/dx_c S_x[m],  S_x[m] = sum_n dL/dI[r0+n][i0+m] A_y[n]
//   dL/dsx  = w sum_m dA_x[m]/dsx  S_x[m]   (and likewise in y with S_y[n] = sum_m dL/dI A_x[m])
// where, for a pixel between edges e0 < e1 and u = (e - x_c)/sigma,
//   dA/dx_c = -(phi(u1) - phi(u0)) / sigma,   dA/dsigma = -(u1 phi(u1) - u0 phi(u0)) / sigma,
// and the chain rule through x_c = sum c_ab lt^a s^b and sigma = sum p_q lt^q gives the
// coefficient gradients.  With frozen windows (origins given per stamp, e.g. those of an
// earlier render) a stamp's centre may lie beyond its window's centre pixel, so the profile
// picks each pixel's formula by the signs of its edges, and window pixels outside the item's
// box are read from the frame.  The work decomposition is the forward's (items, boxes): dL/dI over
// the item's box is staged in shared memory, each lane takes a run of slit points of one
// wavelength sample, gathers its stamps' windows, and the per-run sums are reduced over the
// warp in FP32 and over the warp's tasks and the CTA in FP64 before one global FP64 add per
// coefficient per CTA.  An item's warp
// tasks are spread over gridDim.y CTAs (each stages the item's dL/dI), so that small grids
// still fill the GPU.
#include <algorithm>

#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "mixed_common.cuh"
#include "phi32.cuh"

namespace e2e {

constexpr int kAdjThreads = 128;
constexpr int kAdjWarps = kAdjThreads / 32;

struct AdjArgs {
  const DevSlice* slices;
  const double* const* flux_tab;
  const double* u_all;
  const Item* items;
  const void* const* dldi;  // per detector
  const int64_t* pitch;
  int dtype;                // 0 f32, 1 f64
  int B;
  int nk_max;               // largest number of slit points in an item
  double* g_cx;
  double* g_cy;
  double* g_sx;
  double* g_sy;
  const int2* frozen;       // nullable: window origins (i0, r0) per stamp of the model
};

__device__ __forceinline__ float2 split_pair(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// Profile of one axis of a stamp's K-pixel window: A[m] (pixel integrals), and the pixel
// integrals' derivatives with respect to the centre (dA) and the width (sA).
template <int K>
__device__ __forceinline__ void axis_profile(float f, float gh, float gl, float inv_sigma, float* A, float* dA,
                                             float* sA) {
  constexpr int H = K / 2;
  float E[K + 1], Fv[K + 1], ph[K + 1], u[K + 1];
  const float inv_sqrt2pi = 0.398942280401432678f;
#pragma unroll
  for (int m = 0; m <= K; ++m) {
    float wh, wl, dens;
    const float e = (float)(m - H) - 0.5f;
    edge_arg(e, f, gh, gl, wh, wl);
    E[m] = tail2_dens(wh, wl, dens);
    ph[m] = dens * inv_sqrt2pi;
    u[m] = (e - f) * inv_sigma;
    if (m >= H - 1 && m <= H + 2) Fv[m] = fabsf(wh) < kErfMaxArg ? erf_small(wh) : 1.f - E[m];
  }
#pragma unroll
  for (int m = 0; m < K; ++m) {
    float v;
    if (m < H - 1) v = E[m + 1] - E[m];
    else if (m == H - 1) v = Fv[m] - Fv[m + 1];
    else if (m == H) v = Fv[m] + Fv[m + 1];
    else if (m == H + 1) v = Fv[m + 1] - Fv[m];
    else v = E[m] - E[m + 1];
    A[m] = 0.5f * v;
    dA[m] = -(ph[m + 1] - ph[m]) * inv_sigma;
    sA[m] = -(u[m + 1] * ph[m + 1] - u[m] * ph[m]) * inv_sigma;
  }
}

// The same for a window whose centre pixel need not contain the stamp's centre (frozen
// windows; |f| < K/2 + 1/2): pixels on one side of the centre take differences of tails, the
// pixel across it a sum of erf, and a pixel whose inner edge lies within kErfMaxArg of the
// centre a difference of erf.
template <int K>
__device__ __forceinline__ void axis_profile_any(float f, float gh, float gl, float inv_sigma, float* A, float* dA,
                                                 float* sA) {
  constexpr int H = K / 2;
  float E[K + 1], Fv[K + 1], ph[K + 1], u[K + 1], W[K + 1];
  const float inv_sqrt2pi = 0.398942280401432678f;
#pragma unroll
  for (int m = 0; m <= K; ++m) {
    const float e = (float)(m - H) - 0.5f;
    // e - f exactly as a pair (TwoSum: |f| may exceed |e|), times g = gh + gl
    const float dh = e - f;
    const float bb = dh - e;
    const float dl = (e - (dh - bb)) + (-f - bb);
    const float wh = dh * gh;
    const float wl = fmaf(dh, gh, -wh) + fmaf(dh, gl, dl * gh);
    float dens;
    E[m] = tail2_dens(wh, wl, dens);
    ph[m] = dens * inv_sqrt2pi;
    u[m] = dh * inv_sigma;
    W[m] = wh;
    Fv[m] = fabsf(wh) < kErfMaxArg ? erf_small(wh) : 1.f - E[m];
  }
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const float a0 = W[m], a1 = W[m + 1];
    float v;
    if (a0 >= 0.f) v = a0 < kErfMaxArg ? Fv[m + 1] - Fv[m] : E[m] - E[m + 1];          // right of the centre
    else if (a1 <= 0.f) v = -a1 < kErfMaxArg ? Fv[m] - Fv[m + 1] : E[m + 1] - E[m];    // left of it
    else v = Fv[m] + Fv[m + 1];                                                        // across it
    A[m] = 0.5f * v;
    dA[m] = -(ph[m + 1] - ph[m]) * inv_sigma;
    sA[m] = -(u[m + 1] * ph[m + 1] - u[m] * ph[m]) * inv_sigma;
  }
}

template <int K, bool FROZEN>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint(const AdjArgs a) {
  constexpr int H = K / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const Item it = a.items[blockIdx.x];
  const DevSlice& S = a.slices[it.slice];
  const int area = it.bw * it.bh;
  const int d = S.degree, nc = (d + 1) * (d + 2) / 2;
  const int ncoef = 2 * nc + 6;
  const int nrc = (it.nk + a.B - 1) / a.B;
  const int njb = (it.nj + 31) / 32;
  const int ntask = njb * nrc;
  if ((int)blockIdx.y * kAdjWarps >= ntask) return;  // no task of this item for this CTA
  float* R = reinterpret_cast<float*>(smem);                            // dL/dI over the box
  const size_t o_red = ((size_t)area * 4 + 15) & ~(size_t)15;
  double* red = reinterpret_cast<double*>(smem + o_red);                // [warps][ncoef]
  double* tabS = red + kAdjWarps * ncoef;                               // s of the item's slit points
  float2* tabU = reinterpret_cast<float2*>(tabS + a.nk_max);           // their weights, (hi, lo)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    const int64_t P = a.pitch[S.det];
    for (int p = tid; p < area; p += kAdjThreads) {
      const int gy = p / it.bw, gx = p - gy * it.bw;
      const int64_t off = (int64_t)(it.by0 + gy) * P + (it.bx0 + gx);
      R[p] = a.dtype == 0 ? static_cast<const float*>(a.dldi[S.det])[off]
                          : (float)static_cast<const double*>(a.dldi[S.det])[off];
    }
    for (int q = tid; q < kAdjWarps * ncoef; q += kAdjThreads) red[q] = 0.0;
    const double* u = a.u_all + S.u_off;
    const double inv_ns = 1.0 / (double)S.n_slit;
    for (int kk = tid; kk < it.nk; kk += kAdjThreads) {
      tabS[kk] = (double)(2 * (it.k0 + kk) + 1 - S.n_slit) * inv_ns;
      tabU[kk] = split_pair(u[it.k0 + kk]);
    }
  }
  __syncthreads();
  const double* flux = a.flux_tab[S.flux_slot];
  const double inv_nl = 1.0 / (double)S.n_lambda;
  for (int task = blockIdx.y * kAdjWarps + warp; task < ntask; task += gridDim.y * kAdjWarps) {
    const int jj = (task % njb) * 32 + lane;
    const bool jvalid = jj < it.nj;
    const int j = it.j0 + jj;
    const int k0 = it.k0 + (task / njb) * a.B;
    const int nb = min(a.B, it.k0 + it.nk - k0);
    float Hx[9], Hy[9], Gsx = 0.f, Gsy = 0.f;
#pragma unroll
    for (int b = 0; b < 9; ++b) Hx[b] = Hy[b] = 0.f;
    double lt = 0.0;
    if (jvalid) {
      lt = (double)(2 * j + 1 - S.n_lambda) * inv_nl;
      // P_b(lt) of x and y as split_xy pairs (the planner's mapping), degree <= 8, and the
      // edge-argument scales, from the per-model sample tables
      const float4* row = S.samples + (int64_t)j * (d + 3);
      float4 P[9];
#pragma unroll
      for (int b = 0; b <= 8; ++b) P[b] = b <= d ? row[b] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 g = row[d + 1];
      const float2 gx = make_float2(g.x, g.y), gy = make_float2(g.z, g.w);
      const double sgx = fma(fma(S.sx[2], lt, S.sx[1]), lt, S.sx[0]);
      const double sgy = fma(fma(S.sy[2], lt, S.sy[1]), lt, S.sy[0]);
      const float isx = (float)(1.0 / sgx), isy = (float)(1.0 / sgy);
      const float2 wj = split_pair(flux[j] * S.dlam);
      for (int b = 0; b < nb; ++b) {
        const int k = k0 + b;
        const double sd = tabS[k - it.k0];
        int ci, ri;
        float fx, fy;
        float2 mh, ml;
        map_xy_df_regs(P, d, split_df(sd), mh, ml);
        split_coord_df(mh.x, ml.x, ci, fx);
        split_coord_df(mh.y, ml.y, ri, fy);
        if (ci == kOffFrame || ri == kOffFrame) continue;
        const float2 uk = tabU[k - it.k0];
        const float w = fmaf(wj.x, uk.x, fmaf(wj.x, uk.y, wj.y * uk.x));
        float Ax[K], dAx[K], sAx[K], Ay[K], dAy[K], sAy[K];
        if constexpr (FROZEN) {
          const int2 o = a.frozen[S.stamp_off + (int64_t)j * S.n_slit + k];
          ci = o.x + H;
          ri = o.y + H;
          fx = (mh.x - (float)ci) + ml.x;  // h - c exact (|h - c| small against h), one rounding
          fy = (mh.y - (float)ri) + ml.y;
          axis_profile_any<K>(fx, gx.x, gx.y, isx, Ax, dAx, sAx);
          axis_profile_any<K>(fy, gy.x, gy.y, isy, Ay, dAy, sAy);
        } else {
          axis_profile<K>(fx, gx.x, gx.y, isx, Ax, dAx, sAx);
          axis_profile<K>(fy, gy.x, gy.y, isy, Ay, dAy, sAy);
        }
        // gather dL/dI over the window (with the forward's windows, pixels outside the box lie
        // outside the detector; frozen windows may reach detector pixels beyond the box, which
        // are read from the frame)
        float Sx[K], Sy[K];
#pragma unroll
        for (int m = 0; m < K; ++m) Sx[m] = 0.f;
        const int bx = ci - H - it.bx0, by = ri - H - it.by0;
#pragma unroll
        for (int n = 0; n < K; ++n) {
          float sy = 0.f;
          const int gy = by + n;
          if (FROZEN || (gy >= 0 && gy < it.bh)) {
#pragma unroll
            for (int m = 0; m < K; ++m) {
              const int gx2 = bx + m;
              float r = 0.f;
              if (gy >= 0 && gy < it.bh && gx2 >= 0 && gx2 < it.bw) {
                r = R[gy * it.bw + gx2];
              } else if (FROZEN) {
                const int X = it.bx0 + gx2, Y = it.by0 + gy;
                if (X >= 0 && X < S.W && Y >= 0 && Y < S.H) {
                  const int64_t off = (int64_t)Y * a.pitch[S.det] + X;
                  r = a.dtype == 0 ? static_cast<const float*>(a.dldi[S.det])[off]
                                   : (float)static_cast<const double*>(a.dldi[S.det])[off];
                }
              }
              sy = fmaf(r, Ax[m], sy);
              Sx[m] = fmaf(r, Ay[n], Sx[m]);
            }
          }
          Sy[n] = sy;
        }
        float gxc = 0.f, gsx = 0.f, gyc = 0.f, gsy = 0.f;
#pragma unroll
        for (int m = 0; m < K; ++m) {
          gxc = fmaf(dAx[m], Sx[m], gxc);
          gsx = fmaf(sAx[m], Sx[m], gsx);
          gyc = fmaf(dAy[m], Sy[m], gyc);
          gsy = fmaf(sAy[m], Sy[m], gsy);
        }
        gxc *= w;
        gyc *= w;
        Gsx = fmaf(w, gsx, Gsx);
        Gsy = fmaf(w, gsy, Gsy);
        // powers of s for the chain rule through x_c = sum_b P_b(lt) s^b
        const float s = (float)sd;
        float sp = 1.f;
#pragma unroll
        for (int bb = 0; bb < 9; ++bb) {
          if (bb <= d) {
            Hx[bb] = fmaf(gxc, sp, Hx[bb]);
            Hy[bb] = fmaf(gyc, sp, Hy[bb]);
          }
          sp *= s;
        }
      }
    }
    // coefficient gradients of this run: dL/dc_ab = lt^a H_b, dL/ds_q = lt^q G_s.  The warp's
    // 32 samples are summed in FP32 (|lt| <= 1; the run sums are FP32 already), the partials
    // of the warp's tasks in FP64
    const float ltf = (float)lt;
    for (int t = 0; t <= d; ++t)
      for (int bb = 0; bb <= t; ++bb) {
        const int aa = t - bb;
        float lp = 1.f;
        for (int q = 0; q < aa; ++q) lp *= ltf;
        float hx = 0.f, hy = 0.f;
#pragma unroll
        for (int q = 0; q < 9; ++q)
          if (q == bb) {
            hx = Hx[q];
            hy = Hy[q];
          }
        float vx = lp * hx, vy = lp * hy;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          vx += __shfl_xor_sync(0xffffffffu, vx, o);
          vy += __shfl_xor_sync(0xffffffffu, vy, o);
        }
        if (lane == 0) {
          const int idx = t * (t + 1) / 2 + bb;
          red[warp * ncoef + idx] += (double)vx;
          red[warp * ncoef + nc + idx] += (double)vy;
        }
      }
    {
      float lp = 1.f;
      for (int q = 0; q < 3; ++q) {
        float vx = lp * Gsx, vy = lp * Gsy;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          vx += __shfl_xor_sync(0xffffffffu, vx, o);
          vy += __shfl_xor_sync(0xffffffffu, vy, o);
        }
        if (lane == 0) {
          red[warp * ncoef + 2 * nc + q] += (double)vx;
          red[warp * ncoef + 2 * nc + 3 + q] += (double)vy;
        }
        lp *= ltf;
      }
    }
  }
  __syncthreads();
  for (int q = tid; q < ncoef; q += kAdjThreads) {
    double v = 0.0;
    for (int w2 = 0; w2 < kAdjWarps; ++w2) v += red[w2 * ncoef + q];
    if (v == 0.0) continue;
    if (q < nc) atomicAdd(a.g_cx + S.coef_off + q, v);
    else if (q < 2 * nc) atomicAdd(a.g_cy + S.coef_off + q - nc, v);
    else if (q < 2 * nc + 3) atomicAdd(a.g_sx + 3 * S.index + (q - 2 * nc), v);
    else atomicAdd(a.g_sy + 3 * S.index + (q - 2 * nc - 3), v);
  }
}

// 2-D fibers: the gradients of a parent slice are the sums over its aperture rows' slices
// (each row's mapping is the parent's plus a displacement independent of the coefficients);
// one CTA per parent, rows summed in order.  fold = first_sub[n_parent + 1] | sub coef_off[n_sub] |
// parent coef_off[n_parent] | parent n_coef[n_parent].
__global__ void k_fold_gradients(int n_parent, int n_sub, const int* __restrict__ fold,
                                 const double* __restrict__ gcx_e, const double* __restrict__ gcy_e,
                                 const double* __restrict__ gsx_e, const double* __restrict__ gsy_e, double* gcx,
                                 double* gcy, double* gsx, double* gsy) {
  const int p = blockIdx.x;
  if (p >= n_parent) return;
  const int* first = fold;
  const int* sub_off = fold + n_parent + 1;
  const int* par_off = sub_off + n_sub;
  const int* par_nc = par_off + n_parent;
  const int q0 = first[p], q1 = first[p + 1], nc = par_nc[p];
  for (int e = threadIdx.x; e < 2 * nc + 6; e += blockDim.x) {
    double v = 0.0;
    if (e < 2 * nc) {
      const double* g = e < nc ? gcx_e : gcy_e;
      const int c = e < nc ? e : e - nc;
      for (int q = q0; q < q1; ++q) v += g[sub_off[q] + c];
      (e < nc ? gcx : gcy)[par_off[p] + c] = v;
    } else {
      const int k = e - 2 * nc;
      const double* g = k < 3 ? gsx_e : gsy_e;
      for (int q = q0; q < q1; ++q) v += g[3 * q + k % 3];
      (k < 3 ? gsx : gsy)[3 * p + k % 3] = v;
    }
  }
}

cudaError_t launch_fold_gradients(int n_parent, int n_sub, const int* fold, const double* gcx_e, const double* gcy_e,
                                  const double* gsx_e, const double* gsy_e, double* gcx, double* gcy, double* gsx,
                                  double* gsy, cudaStream_t st) {
  if (n_parent == 0) return cudaSuccess;
  k_fold_gradients<<<n_parent, 64, 0, st>>>(n_parent, n_sub, fold, gcx_e, gcy_e, gsx_e, gsy_e, gcx, gcy, gsx, gsy);
  return cudaGetLastError();
}

size_t adjoint_smem_bytes(int max_area, int max_deg, int nk_max, int nj_max) {
  (void)nj_max;
  const int nc = (max_deg + 1) * (max_deg + 2) / 2;
  return (((size_t)max_area * 4 + 15) & ~(size_t)15) + (size_t)kAdjWarps * (2 * nc + 6) * 8 + (size_t)nk_max * 16;
}

int adjoint_parts(int max_tasks) { return std::max(1, std::min(4, (max_tasks + kAdjWarps - 1) / kAdjWarps)); }

template <int K>
static cudaError_t launch_adj(const AdjArgs& a, int n_items, int parts, size_t smem, cudaStream_t st) {
  auto kern = a.frozen ? k_adjoint<K, true> : k_adjoint<K, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(n_items, parts), kAdjThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(int K, const DevSlice* slices, const double* const* flux_tab, const double* u_all,
                           const Item* items, int n_items, const void* const* dldi, const int64_t* pitch, int dtype,
                           int B, int nk_max, int parts, double* g_cx, double* g_cy, double* g_sx, double* g_sy,
                           size_t smem, cudaStream_t st, const int2* frozen) {
  if (n_items == 0) return cudaSuccess;
  AdjArgs a{slices, flux_tab, u_all, items, dldi, pitch, dtype, B, nk_max, g_cx, g_cy, g_sx, g_sy, frozen};
  switch (K) {
    case 1: return launch_adj<1>(a, n_items, parts, smem, st);
    case 3: return launch_adj<3>(a, n_items, parts, smem, st);
    case 5: return launch_adj<5>(a, n_items, parts, smem, st);
    case 7: return launch_adj<7>(a, n_items, parts, smem, st);
    case 9: return launch_adj<9>(a, n_items, parts, smem, st);
    case 11: return launch_adj<11>(a, n_items, parts, smem, st);
    case 13: return launch_adj<13>(a, n_items, parts, smem, st);
    case 15: return launch_adj<15>(a, n_items, parts, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace e2e
