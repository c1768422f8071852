// Mixed-precision tiled renderer (separable Gaussian PSF) and the halo merge.
//
// Work item = one order-slice x a block of wavelength samples x a block of slit points.
// Inside the item, each lane owns a *run* of B consecutive slit points of one wavelength
// sample: the run's stamps land within a (K+DX) x (K+DY) pixel tile (the plan checks this for
// every run of the model), so the lane accumulates their outer products w * A_x (x) A_y in
// FP32 registers and flushes the tile once per run into the item's box in shared memory.
// The box holds 52-bit fixed-point sums (two 32-bit words per pixel, scaled by a power of
// two above the item's total flux) updated with integer atomics: the accumulation is exact
// and independent of the order of the flushes.  At the end the box is written, in FP64, to a
// scratch "box store".  The merge kernel then owns every output pixel: it adds, with
// compensated summation, the boxes of all items overlapping its tile, in item order, and
// writes the frame once.  No global atomics; the frame does not depend on scheduling.
//
// Precision (the paper's fidelity target, Sec. 2.2, is a photocenter shift below ~1e-5 px):
// mapping in FP64, the centre split exactly into an integer pixel and an FP32 offset, PSF
// pixel integrals in FP32 with double-float edge arguments (phi32.cuh), FP32 sums over one
// run (<= B stamps) in registers, exact fixed-point sums per item, FP64 across items.
#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "phi32.cuh"

namespace e2e {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Horner in s over the per-sample coefficients P_b(lt), b = 0..d (same sequence of FMAs
// in the plan and the render, so both see identical window origins).
__device__ __forceinline__ double horner_s(const double* P, int d, double s) {
  double x = 0.0;
#pragma unroll
  for (int b = 8; b >= 0; --b)
    if (b <= d) x = fma(x, s, P[b]);
  return x;
}

// ------------------------------------------------------------------------------ plan

// One thread per (slice, wavelength sample j, block of 16 slit points): map the stamps
// exactly as the render will, and record (a) per (32-sample block, 16-point block) of each
// slice the bounding box of the stamps' windows, (b) per slice the largest spread of window
// origins over any aligned run of B = 1, 2, 4, 8, 16 consecutive slit points.
__global__ void k_plan(const DevSlice* __restrict__ slices, int n_slices, const int64_t* __restrict__ task_off,
                       int4* __restrict__ bbox, const int64_t* __restrict__ bbox_off,
                       int* __restrict__ spans /* [n_slices][5][2] */) {
  const int64_t n_tasks = task_off[n_slices];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tasks; t += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_slices - 1;
    while (lo < hi) {  // slice owning task t
      int mid = (lo + hi + 1) >> 1;
      if (task_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const DevSlice& S = slices[lo];
    const int nkb = (S.n_slit + 15) / 16;
    const int64_t local = t - task_off[lo];
    const int j = (int)(local / nkb), kb = (int)(local - (int64_t)j * nkb);
    const double lt = norm_sample(j, S.n_lambda);
    double px[9], py[9];
#pragma unroll
    for (int b = 0; b <= 8; ++b) {
      px[b] = b <= S.degree ? poly_lt_for_b(S.cx, S.degree, b, lt) : 0.0;
      py[b] = b <= S.degree ? poly_lt_for_b(S.cy, S.degree, b, lt) : 0.0;
    }
    int xmn = 1 << 30, xmx = -(1 << 30), ymn = 1 << 30, ymx = -(1 << 30);
    int rxmn[5], rxmx[5], rymn[5], rymx[5], spx[5], spy[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) { rxmn[q] = rymn[q] = 1 << 30; rxmx[q] = rymx[q] = -(1 << 30); spx[q] = spy[q] = 0; }
    const int k0 = kb * 16, k1 = min(k0 + 16, S.n_slit);
    for (int k = k0; k < k1; ++k) {
      const double s = norm_sample(k, S.n_slit);
      int ci, ri;
      float fx, fy;
      split_coord(clamp_coord(horner_s(px, S.degree, s)), ci, fx);
      split_coord(clamp_coord(horner_s(py, S.degree, s)), ri, fy);
      xmn = min(xmn, ci); xmx = max(xmx, ci); ymn = min(ymn, ri); ymx = max(ymx, ri);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int B = 1 << q;
        rxmn[q] = min(rxmn[q], ci); rxmx[q] = max(rxmx[q], ci);
        rymn[q] = min(rymn[q], ri); rymx[q] = max(rymx[q], ri);
        if (((k + 1) % B) == 0 || k + 1 == k1) {  // end of an aligned run
          spx[q] = max(spx[q], rxmx[q] - rxmn[q]);
          spy[q] = max(spy[q], rymx[q] - rymn[q]);
          rxmn[q] = rymn[q] = 1 << 30; rxmx[q] = rymx[q] = -(1 << 30);
        }
      }
    }
    const int h = S.K / 2;
    int4* bb = bbox + bbox_off[lo] + (int64_t)(j / 32) * nkb + kb;
    atomicMin(&bb->x, xmn - h);
    atomicMax(&bb->y, xmx + h);
    atomicMin(&bb->z, ymn - h);
    atomicMax(&bb->w, ymx + h);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      atomicMax(&spans[(lo * 5 + q) * 2 + 0], spx[q]);
      atomicMax(&spans[(lo * 5 + q) * 2 + 1], spy[q]);
    }
  }
}

// ------------------------------------------------------------------------------ render

struct MixedArgs {
  const DevSlice* slices;
  const double* const* flux_tab;
  const double* u_all;
  const Item* items;
  double* store;
  int B;        // slit points per run
  int JB;       // 32-sample blocks per item
  int max_deg;  // largest degree among the launched slices
};

constexpr int kSplit = 22;  // fixed point: value * 2^P = hi * 2^22 + lo, lo in [0, 2^22)

template <int K, int DX, int DY>
__global__ void __launch_bounds__(kThreads) k_render_mixed(const MixedArgs a) {
  constexpr int RX = K + DX, RY = K + DY, H = K / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const Item it = a.items[blockIdx.x];
  const DevSlice& S = a.slices[it.slice];
  const int area = it.bw * it.bh;
  const int J = 32 * a.JB;
  const int nd = S.degree + 1;
  // shared layout: per-sample tables | run staging | box hi words | box lo words
  double* tabP = reinterpret_cast<double*>(smem);  // [J][2][nd]
  double* tabW = tabP + (size_t)J * 2 * nd;         // [J] flux x bin width / 4
  float4* tabG = reinterpret_cast<float4*>(tabW + J);  // [J] (gx hi, gx lo, gy hi, gy lo), g = 1/(sqrt2 sigma)
  int4* stage = reinterpret_cast<int4*>(tabG + J);  // [B][kThreads]
  int* boxh = reinterpret_cast<int*>(stage + (size_t)a.B * kThreads);
  unsigned* boxl = reinterpret_cast<unsigned*>(boxh + area);
  __shared__ double s_red[kWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int p = tid; p < area; p += kThreads) {
    boxh[p] = 0;
    boxl[p] = 0u;
  }
  const double* flux = a.flux_tab[S.flux_slot];
  const double* u = a.u_all + S.u_off;
  for (int q = tid; q < it.nj * 2 * nd; q += kThreads) {
    const int jj = q / (2 * nd), r = q - jj * 2 * nd, axis = r / nd, b = r - axis * nd;
    const double lt = norm_sample(it.j0 + jj, S.n_lambda);
    tabP[q] = poly_lt_for_b(axis ? S.cy : S.cx, S.degree, b, lt);
  }
  // flux bound of the item: sum over its stamps of |w| (bounds every pixel of its box)
  double usum = 0.0;
  for (int k = lane; k < it.nk; k += 32) usum += fabs(u[it.k0 + k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) usum += __shfl_xor_sync(0xffffffffu, usum, o);
  double wsum = 0.0;
  for (int jj = tid; jj < it.nj; jj += kThreads) {
    const double lt = norm_sample(it.j0 + jj, S.n_lambda);
    const double sgx = fma(fma(S.sx[2], lt, S.sx[1]), lt, S.sx[0]);
    const double sgy = fma(fma(S.sy[2], lt, S.sy[1]), lt, S.sy[0]);
    const double gx = 0.70710678118654752440 / sgx, gy = 0.70710678118654752440 / sgy;
    const float gxh = (float)gx, gyh = (float)gy;
    tabG[jj] = make_float4(gxh, (float)(gx - (double)gxh), gyh, (float)(gy - (double)gyh));
    const double wj = flux[it.j0 + jj] * S.dlam;
    tabW[jj] = wj * 0.25;  // 0.25: the profiles below are 2x the pixel integrals
    wsum += fabs(wj);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  if (lane == 0) s_red[warp] = wsum;
  __syncthreads();
  double total = 0.0;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) total += s_red[q];
  total *= usum;
  // scale 2^P with |box sums| <= total < 2^(52-P); clamp so 2^P stays a normal FP32
  int ex = 0;
  frexp(total, &ex);
  const int P = total > 0.0 ? max(-100, min(100, 52 - ex)) : 0;
  const float sc = ldexpf(1.f, P), sc_hi = ldexpf(1.f, P - kSplit);

  const int nrc = (it.nk + a.B - 1) / a.B;
  const int jbs = (it.nj + 31) / 32;  // 32-sample blocks of this item (<= a.JB)
  const int ntask = jbs * nrc;
  for (int task = warp; task < ntask && total > 0.0; task += kWarps) {
    const int jj = (task % jbs) * 32 + lane;
    if (jj >= it.nj) continue;
    const int k0 = it.k0 + (task / jbs) * a.B;
    const int nb = min(a.B, it.k0 + it.nk - k0);
    double px[9], py[9];
#pragma unroll
    for (int b = 0; b <= 8; ++b) {
      px[b] = b < nd ? tabP[(jj * 2 + 0) * nd + b] : 0.0;
      py[b] = b < nd ? tabP[(jj * 2 + 1) * nd + b] : 0.0;
    }
    int xmn = 1 << 30, ymn = 1 << 30;
    for (int b = 0; b < nb; ++b) {
      const double s = norm_sample(k0 + b, S.n_slit);
      int ci, ri;
      float fx, fy;
      split_coord(clamp_coord(horner_s(px, S.degree, s)), ci, fx);
      split_coord(clamp_coord(horner_s(py, S.degree, s)), ri, fy);
      xmn = min(xmn, ci);
      ymn = min(ymn, ri);
      stage[b * kThreads + tid] = make_int4(ci, ri, __float_as_int(fx), __float_as_int(fy));
    }
    const float4 g = tabG[jj];
    const double wj = tabW[jj];
    float acc[RY][RX];
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
      for (int c = 0; c < RX; ++c) acc[r][c] = 0.f;
    for (int b = 0; b < nb; ++b) {
      const int4 st = stage[b * kThreads + tid];
      const int ox = st.x - xmn, oy = st.y - ymn;  // 0..DX, 0..DY
      const float fx = __int_as_float(st.z), fy = __int_as_float(st.w);
      const float w = (float)(wj * u[k0 + b]);
      float wax[RX], ay[RY];
      {
        float th, tl;
        edge_arg((float)(-ox - H) - 0.5f, fx, g.x, g.y, th, tl);
        float ep = erfc_df(th, tl), tp = th;
#pragma unroll
        for (int c = 0; c < RX; ++c) {
          edge_arg((float)(c + 1 - ox - H) - 0.5f, fx, g.x, g.y, th, tl);
          const float en = erfc_df(th, tl);
          const float v = twice_interval(tp, th, ep, en);
          wax[c] = (c >= ox && c < ox + K) ? w * v : 0.f;
          tp = th;
          ep = en;
        }
      }
      {
        float th, tl;
        edge_arg((float)(-oy - H) - 0.5f, fy, g.z, g.w, th, tl);
        float ep = erfc_df(th, tl), tp = th;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          edge_arg((float)(r + 1 - oy - H) - 0.5f, fy, g.z, g.w, th, tl);
          const float en = erfc_df(th, tl);
          const float v = twice_interval(tp, th, ep, en);
          ay[r] = (r >= oy && r < oy + K) ? v : 0.f;
          tp = th;
          ep = en;
        }
      }
#pragma unroll
      for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int c = 0; c < RX; ++c) acc[r][c] = fmaf(ay[r], wax[c], acc[r][c]);
    }
    // flush the run tile into the box as exact fixed-point increments
    const int gx0 = xmn - H - it.bx0, gy0 = ymn - H - it.by0;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int gy = gy0 + r;
      if (gy < 0 || gy >= it.bh) continue;
#pragma unroll
      for (int c = 0; c < RX; ++c) {
        const int gxp = gx0 + c;
        const float v = acc[r][c];
        if (gxp >= 0 && gxp < it.bw && v != 0.f) {
          const float hf = floorf(v * sc_hi);
          const float lf = fmaf(-hf, 4194304.f, v * sc);
          atomicAdd(boxh + gy * it.bw + gxp, __float2int_rz(hf));
          atomicAdd(boxl + gy * it.bw + gxp, __float2uint_rn(lf));
        }
      }
    }
  }
  __syncthreads();
  double* out = a.store + it.store_off;
  const double inv = ldexp(1.0, -P);
  for (int p = tid; p < area; p += kThreads)
    out[p] = fma((double)boxh[p], 4194304.0, (double)boxl[p]) * inv;
}

size_t mixed_smem_bytes(int area, int JB, int B, int nd) {
  const int J = 32 * JB;
  size_t bytes = (size_t)J * 2 * nd * 8 + (size_t)J * 8 + (size_t)J * 16;
  bytes = (bytes + 15) & ~(size_t)15;
  bytes += (size_t)B * kThreads * 16;
  bytes += (size_t)area * 8;
  return bytes;
}

// ------------------------------------------------------------------------------ merge

// One CTA per output tile: sum, in item order and with Neumaier compensation, the FP64
// boxes of the items overlapping the tile, convert and write every pixel once.
template <typename T>
__global__ void __launch_bounds__(256) k_merge(const Tile* __restrict__ tiles, const int32_t* __restrict__ lists,
                                               const Item* __restrict__ items, const double* __restrict__ store,
                                               T* const* dst, const int64_t* __restrict__ pitch, const int* __restrict__ dims) {
  const Tile t = tiles[blockIdx.x];
  const int H = dims[2 * t.det], W = dims[2 * t.det + 1];
  const int tx = threadIdx.x & (kTileW - 1), ty0 = threadIdx.x / kTileW;
  constexpr int kRows = kTileW * kTileH / 256;  // pixels per thread
  double sum[kRows], comp[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) sum[q] = comp[q] = 0.0;
  const int x = t.x0 + tx;
  for (int n = 0; n < t.n; ++n) {
    const Item it = items[lists[t.list_off + n]];
    const int gx = x - it.bx0;
    if (gx < 0 || gx >= it.bw) continue;
    const double* box = store + it.store_off;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const int gy = t.y0 + ty0 + q * (256 / kTileW) - it.by0;
      if (gy >= 0 && gy < it.bh) {
        const double v = box[(int64_t)gy * it.bw + gx];
        const double s = sum[q] + v;
        comp[q] += fabs(sum[q]) >= fabs(v) ? (sum[q] - s) + v : (v - s) + sum[q];
        sum[q] = s;
      }
    }
  }
  if (x >= W) return;
  T* frame = dst[t.det];
  const int64_t P = pitch[t.det];
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int y = t.y0 + ty0 + q * (256 / kTileW);
    if (y < H) frame[(int64_t)y * P + x] = (T)(sum[q] + comp[q]);
  }
}

// ------------------------------------------------------------------------------ launchers

cudaError_t launch_plan(const DevSlice* slices, int n_slices, const int64_t* task_off, int64_t n_tasks,
                        int4* bbox, const int64_t* bbox_off, int* spans, cudaStream_t st) {
  if (n_tasks == 0) return cudaSuccess;
  int64_t blocks = (n_tasks + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_plan<<<(unsigned)blocks, 256, 0, st>>>(slices, n_slices, task_off, bbox, bbox_off, spans);
  return cudaGetLastError();
}

template <int K, int DX, int DY>
static cudaError_t launch_one(const MixedArgs& a, int n_items, size_t smem, cudaStream_t st) {
  auto kern = k_render_mixed<K, DX, DY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_items, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

bool mixed_variant_supported(int K, int DX, int DY) {
  if (K < 1 || K > 15 || (K % 2) == 0) return false;
  if (DX == 0 && DY == 0) return true;
  if (DX == 1 && DY == 1) return K <= 13;
  if (DX == 2 && DY == 2) return K <= 11;
  return false;
}

cudaError_t launch_render_mixed(int K, int DX, int DY, const DevSlice* slices, const double* const* flux_tab,
                                const double* u_all, const Item* items, int n_items, double* store, int B, int JB,
                                int max_deg, size_t smem, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  MixedArgs a{slices, flux_tab, u_all, items, store, B, JB, max_deg};
#define E2E_V(KK, X, Y) \
  if (K == KK && DX == X && DY == Y) return launch_one<KK, X, Y>(a, n_items, smem, st);
  E2E_V(1, 0, 0) E2E_V(3, 0, 0) E2E_V(5, 0, 0) E2E_V(7, 0, 0) E2E_V(9, 0, 0) E2E_V(11, 0, 0) E2E_V(13, 0, 0)
  E2E_V(15, 0, 0)
  E2E_V(1, 1, 1) E2E_V(3, 1, 1) E2E_V(5, 1, 1) E2E_V(7, 1, 1) E2E_V(9, 1, 1) E2E_V(11, 1, 1) E2E_V(13, 1, 1)
  E2E_V(1, 2, 2) E2E_V(3, 2, 2) E2E_V(5, 2, 2) E2E_V(7, 2, 2) E2E_V(9, 2, 2) E2E_V(11, 2, 2)
#undef E2E_V
  return cudaErrorInvalidValue;
}

cudaError_t launch_merge(const Tile* tiles, int n_tiles, const int32_t* lists, const Item* items, const double* store,
                         void* const* dst, int dtype, const int64_t* pitch, const int* dims, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  if (dtype == 0)
    k_merge<float><<<n_tiles, 256, 0, st>>>(tiles, lists, items, store, (float* const*)dst, pitch, dims);
  else
    k_merge<double><<<n_tiles, 256, 0, st>>>(tiles, lists, items, store, (double* const*)dst, pitch, dims);
  return cudaGetLastError();
}

}  // namespace e2e
