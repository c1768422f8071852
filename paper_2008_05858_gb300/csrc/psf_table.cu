// Tabulated PSF: per-cell phase polynomials of the exact pixel integrals, and the stamp
// renderers that read them.
//
// A slice's PSF is given as maps (Sec. 2.1: the spectrograph unit delivers PSF maps per
// projected fiber image) at field nodes lt_f along the order: map f samples the density at
// offsets ((u - c)/q, (v - c)/q) px from the PSF centre, c = (M - 1)/2, and the density
// between samples is the bilinear interpolant, sum_uv S_uv T(q x - (u - c)) T(q y - (v - c))
// with T the unit tent.  A stamp's pixel value is that density's integral over the pixel for
// the PSF centred at the stamp's position (Sec. 2.2), which factorises:
//
//   I = sum_v sum_u S_uv X_u Y_v / norm,  X_u = (G(q (b - x_u)) - G(q (a - x_u))) / q,
//   G(t) = integral of the tent up to t (0, (1+t)^2/2, 1 - (1-t)^2/2, 1),  norm = sum S / q^2.
//
// As a function of the centre's sub-pixel phase ph (pixel edges at half-integers minus ph),
// X_u is piecewise quadratic, with knots where an edge crosses a knot of a tent: at
// ph = 1/2 - (k + c)/q.  For an integer q these knots are the same for every pixel of the
// window: cells of width 1/q, starting at ph = -1/2 for odd M, half a cell later for even M
// (then the first and last cells are half cells).  Within a cell pair (x, y) the pixel
// integral is therefore exactly a biquadratic in the phase.  At load time k_epsf_build
// evaluates it at the 3 x 3 nodes of every cell (its ends and midpoint per axis) in FP64 and
// stores the biquadratic's coefficients in the centred variable tau in [-1/2, 1/2]:
//
//   f(tau) = T1 + tau (T2 - T0) + tau^2 2 (T0 - 2 T1 + T2)   (per axis; tensor product in 2-D),
//
// in FP64 and FP32.  A stamp evaluates it by Horner in tau_x, tau_y (the terms after the first
// are small, so FP32 keeps a few-ulp error), for the two field nodes around its wavelength (the
// end node beyond the ends), blended linearly in lt: 18 table reads per pixel, and no
// interpolation error in the phase.
#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "mixed_common.cuh"

namespace e2e {

__device__ __forceinline__ double tent_cdf(double t) {
  if (t <= -1.0) return 0.0;
  if (t <= 0.0) return 0.5 * (1.0 + t) * (1.0 + t);
  if (t <= 1.0) return 1.0 - 0.5 * (1.0 - t) * (1.0 - t);
  return 1.0;
}

// One block per (slice, node): the map's norm, sum S / q^2.
__global__ void __launch_bounds__(256) k_map_norm(const TableSlice* __restrict__ ts, const double* __restrict__ maps,
                                                  double* __restrict__ norms) {
  const TableSlice& t = ts[blockIdx.x];
  const int f = blockIdx.y;
  if (f >= t.n_field) return;
  const int M = t.map_size;
  const double* S = maps + t.map_off + (int64_t)f * M * M;
  double sum = 0.0;
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) sum += S[i];
  __shared__ double red[256];
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) norms[t.field_off + f] = red[0] / ((double)t.q * t.q);
}

// Phase of node a (0, 1, 2: start, midpoint, end) of cell i on one axis: in units of 1/q from
// the cell grid's origin, cell i spans [max(i, h), min(i + 1, q + h)] with h = 1/2 for even
// maps (half cells at both ends), and ph = r / q - 1/2 - h / q.
__device__ __forceinline__ double cell_node_phase(const TableSlice& t, int i, int a) {
  const double h = t.half ? 0.5 : 0.0;
  const double lo = fmax((double)i, h), hi = fmin((double)(i + 1), (double)t.q + h);
  const double r = a == 0 ? lo : (a == 1 ? 0.5 * (lo + hi) : hi);
  return (r - h) / t.q - 0.5;
}

// Pixel integral of map f's normalised density over window pixel (m, n) for the PSF centred
// at phase (phx, phy) from the centre pixel's centre.
__device__ double epsf_pixel(const TableSlice& t, const double* S, double norm, int m, int n, double phx,
                             double phy) {
  const int H = t.K / 2, M = t.map_size;
  const double q = (double)t.q, c = 0.5 * (M - 1);
  const double ax = m - H - 0.5 - phx, bx = ax + 1.0, ay = n - H - 0.5 - phy, by = ay + 1.0;
  // samples whose tents meet [a, b): c + q a - 1 < u < c + q b + 1
  const int u0 = max(0, (int)floor(c + q * ax - 1.0)), u1 = min(M - 1, (int)ceil(c + q * bx + 1.0));
  const int v0 = max(0, (int)floor(c + q * ay - 1.0)), v1 = min(M - 1, (int)ceil(c + q * by + 1.0));
  double sum = 0.0;
  for (int v = v0; v <= v1; ++v) {
    const double yv = (v - c) / q;
    const double wy = (tent_cdf(q * (by - yv)) - tent_cdf(q * (ay - yv))) / q;
    if (wy == 0.0) continue;
    double row = 0.0;
    for (int u = u0; u <= u1; ++u) {
      const double xu = (u - c) / q;
      row += S[(int64_t)v * M + u] * ((tent_cdf(q * (bx - xu)) - tent_cdf(q * (ax - xu))) / q);
    }
    sum += row * wy;
  }
  return sum / norm;
}

// One block per (slice, node, phase cell (cy, cx)): thread (n, m) integrates the map over
// window pixel (m, n) at the cell's 3 x 3 phase nodes and stores the biquadratic's 9
// coefficients C[p][r] (power p of tau_y, r of tau_x) as rows p * 3 + r.
__global__ void __launch_bounds__(128) k_epsf_build(const TableSlice* __restrict__ ts, const double* __restrict__ maps,
                                                    const double* __restrict__ norms, int max_cells,
                                                    double* __restrict__ T64, float* __restrict__ T32) {
  const TableSlice& t = ts[blockIdx.x];
  const int f = blockIdx.y / (max_cells * max_cells);
  const int cell = blockIdx.y - f * max_cells * max_cells;
  const int cyi = cell / max_cells, cxi = cell - cyi * max_cells;
  if (f >= t.n_field || cyi >= t.n_cell || cxi >= t.n_cell) return;
  const int K = t.K, KK = K * K, M = t.map_size;
  const double* S = maps + t.map_off + (int64_t)f * M * M;
  const double norm = norms[t.field_off + f];
  double phx[3], phy[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    phx[a] = cell_node_phase(t, cxi, a);
    phy[a] = cell_node_phase(t, cyi, a);
  }
  const int64_t row0 = (((int64_t)f * t.n_cell + cyi) * t.n_cell + cxi) * 9;
  const int KR = table_row32(K);
  for (int e = threadIdx.x; e < KK; e += blockDim.x) {
    const int n = e / K, m = e - n * K;
    double T[3][3];  // T[y node][x node]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) T[a][b] = epsf_pixel(t, S, norm, m, n, phx[b], phy[a]);
    // per axis: coefficients of 1, tau, tau^2 from the nodes at tau = -1/2, 0, 1/2
    double R[3][3];  // R[y node][x power]
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R[a][0] = T[a][1];
      R[a][1] = T[a][2] - T[a][0];
      R[a][2] = 2.0 * (T[a][0] - 2.0 * T[a][1] + T[a][2]);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double c0 = R[1][r], c1 = R[2][r] - R[0][r], c2 = 2.0 * (R[0][r] - 2.0 * R[1][r] + R[2][r]);
      const double cp[3] = {c0, c1, c2};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int64_t row = row0 + p * 3 + r;
        T64[t.tab_off + row * KK + e] = cp[p];
        T32[t.tab_off32 + row * KR + e] = (float)cp[p];
      }
    }
  }
}

cudaError_t launch_epsf_build(const TableSlice* ts, int n_slices, int max_field, int max_cells, const double* maps,
                              double* norms, double* T64, float* T32, cudaStream_t st) {
  if (n_slices == 0) return cudaSuccess;
  k_map_norm<<<dim3(n_slices, max_field), 256, 0, st>>>(ts, maps, norms);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_epsf_build<<<dim3(n_slices, max_field * max_cells * max_cells), 128, 0, st>>>(ts, maps, norms, max_cells, T64,
                                                                                    T32);
  return cudaGetLastError();
}

// Cell and centred coordinate tau in [-1/2, 1/2] of sub-pixel phase ph on one axis (FP64: the
// phase is the FP64 mapped coordinate minus its window-centre pixel).
__device__ __forceinline__ void phase_cell(const TableSlice& t, double ph, int& cell, double& tau) {
  const double h = t.half ? 0.5 : 0.0;
  const double r = (ph + 0.5) * t.q + h;
  int i = (int)floor(r);
  i = min(t.n_cell - 1, max(0, i));
  const double lo = fmax((double)i, h), hi = fmin((double)(i + 1), (double)t.q + h);
  cell = i;
  tau = (r - lo) * (hi - lo < 1.0 ? 2.0 : 1.0) - 0.5;  // cells are 1 or 1/2 wide
}

// ------------------------------------------------------------------ mixed precision

// The biquadratic C[p][r] tau_y^p tau_x^r (rows p * 3 + r) by Horner in tau_x, then tau_y.
__device__ __forceinline__ float biquad(const float* c, float tx, float ty) {
  const float r0 = fmaf(tx, fmaf(tx, c[2], c[1]), c[0]);
  const float r1 = fmaf(tx, fmaf(tx, c[5], c[4]), c[3]);
  const float r2 = fmaf(tx, fmaf(tx, c[8], c[7]), c[6]);
  return fmaf(ty, fmaf(ty, r2, r1), r0);
}

constexpr int kTThreads = 128;
constexpr int kTWarps = kTThreads / 32;

struct TableLayout {
  size_t tabP, tabS, tabW, tabU, tabF, stage, stagew, boxh, boxl, total;
  __host__ __device__ TableLayout(int J, int NK, int nd, int area) {
    size_t o = 0;
    tabP = o; o += (size_t)J * nd * 16;        // P_b(lt) of x and y, split_xy pairs
    tabS = o; o += (size_t)NK * 8;              // s, (hi, lo) floats
    tabW = o; o += (size_t)J * 8;
    tabU = o; o += (size_t)NK * 8;
    o = (o + 15) & ~(size_t)15;
    tabF = o; o += (size_t)J * 16;              // (f0, f1, weight of f1, -) per sample
    stage = o; o += (size_t)kTWarps * 32 * 16;   // per staged stamp: origin, table row offsets
    stagew = o; o += (size_t)kTWarps * 32 * 16;  // tau_x, tau_y and the two nodes' weights
    boxh = o; o += (size_t)area * 4;
    boxl = o; o += (size_t)area * 4;
    total = o;
  }
};

struct TableArgs {
  MixedArgs m;
  const TableSlice* ts;
  const float* T32;
  const double* field_lt;
};

// One CTA per work item (<= 32 samples x <= 16 slit points); the warp's 32 stamps are mapped
// into staging, then taken one after the other by the whole warp: each lane evaluates its
// pixels' biquadratics in the stamp's phase cell at the two field nodes around its
// wavelength, blends them, sums them over stamps with the same window origin, and deposits
// the sums into the item's box as exact fixed point.
template <int K>
__global__ void __launch_bounds__(kTThreads) k_render_table(const TableArgs ta) {
  const MixedArgs& a = ta.m;
  constexpr int KK = K * K;
  extern __shared__ __align__(16) unsigned char smem[];
  const Item it = a.items[blockIdx.x];
  const DevSlice& S = a.slices[it.slice];
  const TableSlice& TS = ta.ts[it.slice];
  const int area = it.bw * it.bh;
  const int nd = S.degree + 1;
  const TableLayout L(32, a.nk_max, a.max_deg + 1, area);
  float4* tabP = reinterpret_cast<float4*>(smem + L.tabP);
  float2* tabS = reinterpret_cast<float2*>(smem + L.tabS);
  float2* tabW = reinterpret_cast<float2*>(smem + L.tabW);
  float2* tabU = reinterpret_cast<float2*>(smem + L.tabU);
  int4* tabF = reinterpret_cast<int4*>(smem + L.tabF);
  int4* stage = reinterpret_cast<int4*>(smem + L.stage);
  float4* stagew = reinterpret_cast<float4*>(smem + L.stagew);
  int* boxh = reinterpret_cast<int*>(smem + L.boxh);
  unsigned* boxl = reinterpret_cast<unsigned*>(smem + L.boxl);
  __shared__ double s_w[kTWarps], s_u[kTWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int p = tid; p < area; p += kTThreads) {
    boxh[p] = 0;
    boxl[p] = 0u;
  }
  const double* flux = a.flux_tab[S.flux_slot];
  const double* u = a.u_all + S.u_off;
  const double inv_ns = 1.0 / (double)S.n_slit;
  double usum = 0.0;
  for (int kk = tid; kk < it.nk; kk += kTThreads) {
    const double uk = u[it.k0 + kk];
    tabS[kk] = split_df(norm_sample_r(it.k0 + kk, S.n_slit, inv_ns));
    tabU[kk] = split_df(uk);
    usum += fabs(uk);
  }
  {  // mapping coefficients and field nodes of the item's samples (per-model tables)
    const int w = nd + 2;
    const float4* rows = S.samples + (int64_t)it.j0 * w;
    for (int e = tid; e < it.nj * w; e += kTThreads) {
      const int jj = e / w, b = e - jj * w;
      if (b < nd) tabP[jj * nd + b] = rows[e];
      else if (b == nd) tabF[jj] = reinterpret_cast<const int4*>(rows)[e];
    }
  }
  double wsum = 0.0;
  for (int jj = tid; jj < it.nj; jj += kTThreads) {
    const double wj = flux[it.j0 + jj] * S.dlam;
    tabW[jj] = split_df(wj);
    wsum += fabs(wj);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    usum += __shfl_xor_sync(0xffffffffu, usum, o);
  }
  if (lane == 0) {
    s_w[warp] = wsum;
    s_u[warp] = usum;
  }
  __syncthreads();
  double wtot = 0.0, utot = 0.0;
#pragma unroll
  for (int q = 0; q < kTWarps; ++q) {
    wtot += s_w[q];
    utot += s_u[q];
  }
  const double total = wtot * utot;
  int ex = 0;
  frexp(total, &ex);
  const int Psh = total > 0.0 ? max(-100, min(100, 52 - ex)) : 0;
  const float sc = ldexpf(1.f, Psh), sc_hi = ldexpf(1.f, Psh - 22);
  constexpr int KR = table_row32(K);  // floats per table row
  const float* T = ta.T32 + TS.tab_off32;
  // a cell's 9 coefficient rows are consecutive; n_field n_cell^2 <= 65535, so offsets fit 32 bits
  const int cell_stride = 9 * KR;
  const int node_stride = TS.n_cell * TS.n_cell * cell_stride;

  const int nst = it.nj * it.nk;
  int4* wst = stage + warp * 32;
  float4* wsw = stagew + warp * 32;
  // Each lane owns the pixels e = lane, lane + 32, ... of the window.  Consecutive stamps of a
  // warp are consecutive slit points of one sample, whose windows often share their origin:
  // a lane adds its pixels' values in FP32 registers while the origin stays the same (at most
  // kTRun stamps) and deposits them into the box when it moves.
  constexpr int NI = (KK + 31) / 32;
  constexpr int kTRun = 16;
  float acc[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) acc[i] = 0.f;
  int cx = kOffFrame, cy = kOffFrame, n_acc = 0;  // warp-uniform: origin and stamps held
  auto flush = [&]() {
    const int bxs = cx - K / 2 - it.bx0, bys = cy - K / 2 - it.by0;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int e = lane + 32 * i;
      if (e >= KK) break;
      const int n = e / K, m = e - n * K;
      const int bx = bxs + m, by = bys + n;
      const float v = acc[i];
      acc[i] = 0.f;
      if (bx < 0 || bx >= it.bw || by < 0 || by >= it.bh) {
        if (a.err) {
          const int X = it.bx0 + bx, Y = it.by0 + by;
          if (X >= 0 && X < S.W && Y >= 0 && Y < S.H) atomicAdd(a.err, 1);
        }
        continue;
      }
      box_deposit(boxh + by * it.bw + bx, boxl + by * it.bw + bx, v, sc, sc_hi);
    }
  };
  for (int base = warp * 32; base < nst && total > 0.0; base += kTWarps * 32) {
    {
      // lane i maps stamp base + i and prepares what the whole warp needs of it: the window
      // origin, the offsets of its phase cell's coefficient rows at its two field nodes, the
      // cell coordinates tau_x, tau_y and the nodes' weights (linear in wavelength, times the
      // stamp weight)
      const int idx = base + lane;
      int ci = kOffFrame, ri = kOffFrame, aoff = 0, boff = 0;
      float4 cw = make_float4(0.f, 0.f, 0.f, 0.f);
      if (idx < nst) {
        const int jj = idx / it.nk;
        const int kk = idx - jj * it.nk;
        float2 mh, ml;  // the centre as double-floats, as the planner maps it
        map_xy_df(tabP + jj * nd, S.degree, tabS[kk], mh, ml);
        float fx, fy;
        split_coord_df(mh.x, ml.x, ci, fx);
        split_coord_df(mh.y, ml.y, ri, fy);
        const float2 wj = tabW[jj], uk = tabU[kk];
        const float w = fmaf(wj.x, uk.x, fmaf(wj.x, uk.y, wj.y * uk.x));
        const int4 fw = tabF[jj];
        int cxi = 0, cyi = 0;
        double tx = 0.0, ty = 0.0;
        if (ci != kOffFrame && ri != kOffFrame) {
          // the phase v - c exactly in FP64 (h - c is exact in FP32, the low word adds exactly)
          phase_cell(TS, (double)(mh.x - (float)ci) + (double)ml.x, cxi, tx);
          phase_cell(TS, (double)(mh.y - (float)ri) + (double)ml.y, cyi, ty);
        }
        const float wf1 = __int_as_float(fw.z);
        cw = make_float4((float)tx, (float)ty, (1.f - wf1) * w, wf1 * w);
        const int row = (cyi * TS.n_cell + cxi) * cell_stride;
        aoff = fw.x * node_stride + row;
        boff = fw.y * node_stride + row;
      }
      wst[lane] = make_int4(ci, ri, aoff, boff);
      wsw[lane] = cw;
    }
    __syncwarp();
    const int nb = min(32, nst - base);
    // stamp by stamp (warp-uniform): a pixel costs 18 coalesced table reads (9 coefficients at
    // each of two field nodes) and 18 FMAs
    for (int b = 0; b < nb; ++b) {
      const int4 st = wst[b];
      if (st.x == kOffFrame || st.y == kOffFrame) continue;
      if (st.x != cx || st.y != cy || n_acc == kTRun) {
        if (n_acc) flush();
        cx = st.x;
        cy = st.y;
        n_acc = 0;
      }
      ++n_acc;
      const float4 cw = wsw[b];
      const float* A = T + st.z;   // node f0
      const float* Bn = T + st.w;  // node f1
      // two pixel groups at a time: their 36 reads first, then the evaluations
#pragma unroll
      for (int i0 = 0; i0 < NI; i0 += 2) {
        float ca[2][9], cb[2][9];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = lane + 32 * (i0 + h);
          if (i0 + h < NI && e < KK) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              ca[h][k] = __ldg(A + e + k * KR);
              cb[h][k] = __ldg(Bn + e + k * KR);
            }
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = lane + 32 * (i0 + h);
          if (i0 + h >= NI || e >= KK) break;
          const float va = biquad(ca[h], cw.x, cw.y), vb = biquad(cb[h], cw.x, cw.y);
          acc[i0 + h] += fmaf(cw.w, vb, cw.z * va);  // the stamp's value first, then one rounding
        }
      }
    }
    __syncwarp();
  }
  if (n_acc) flush();
  __syncthreads();
  float2* out = a.store + it.store_off;
  const float inv = ldexpf(1.f, -Psh);
  for (int p = tid; p < area; p += kTThreads) out[p] = fixed_to_pair(boxh[p], boxl[p], inv);
}

size_t table_smem_bytes(int area, int nk_max, int nd) { return TableLayout(32, nk_max, nd, area).total; }

template <int K>
static cudaError_t launch_table_one(const TableArgs& a, int n_items, size_t smem, cudaStream_t st) {
  auto kern = k_render_table<K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_items, kTThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_render_table(int K, const DevSlice* slices, const TableSlice* ts, const float* T32,
                                const double* field_lt, const double* const* flux_tab, const double* u_all,
                                const Item* items, int n_items, float2* store, int nk_max, int max_deg, size_t smem,
                                cudaStream_t st, int* err) {
  if (n_items == 0) return cudaSuccess;
  TableArgs a{MixedArgs{slices, flux_tab, u_all, items, store, 0, 1, nk_max, max_deg, err}, ts,
              T32, field_lt};
  switch (K) {
#define E2E_CASE(KK) \
  case KK: return launch_table_one<KK>(a, n_items, smem, st);
    E2E_CASE(1) E2E_CASE(3) E2E_CASE(5) E2E_CASE(7) E2E_CASE(9) E2E_CASE(11) E2E_CASE(13) E2E_CASE(15)
#undef E2E_CASE
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------ FP64

// One thread per stamp: FP64 mapping, FP64 coefficient tables and evaluation, FP64 atomics.
template <int K>
__global__ void __launch_bounds__(256) k_render_fp64_table(const DevSlice* __restrict__ slices,
                                                           const TableSlice* __restrict__ ts,
                                                           const double* __restrict__ T64,
                                                           const double* __restrict__ field_lt,
                                                           const double* const* __restrict__ flux_tab,
                                                           const double* __restrict__ u_all, double* const* acc,
                                                           const int64_t* __restrict__ pitch) {
  const DevSlice& S = slices[blockIdx.y];
  if (S.K != K) return;
  const TableSlice& TS = ts[blockIdx.y];
  const double* flux = flux_tab[S.flux_slot];
  const double* u = u_all + S.u_off;
  const int64_t n = (int64_t)S.n_lambda * S.n_slit;
  double* frame = acc[S.det];
  const int64_t Pf = pitch[S.det];
  constexpr int KK = K * K, H = K / 2;
  const int64_t node_stride = (int64_t)TS.n_cell * TS.n_cell * 9 * KK;
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
    const double ci = floor(x + 0.5), ri = floor(y + 0.5);
    const int i0 = (int)ci - H, r0 = (int)ri - H;
    if (i0 + K <= 0 || i0 >= S.W || r0 + K <= 0 || r0 >= S.H) continue;
    const double w = flux[j] * S.dlam * u[k];
    int f0, f1;
    double wf;
    field_weight(field_lt + TS.field_off, TS.n_field, lt, f0, f1, wf);
    int cxi, cyi;
    double tx, ty;
    phase_cell(TS, x - ci, cxi, tx);
    phase_cell(TS, y - ri, cyi, ty);
    const int64_t row = (int64_t)(cyi * TS.n_cell + cxi) * 9 * KK;
    const double* T0 = T64 + TS.tab_off + (int64_t)f0 * node_stride + row;
    const double* T1 = T64 + TS.tab_off + (int64_t)f1 * node_stride + row;
    for (int nn = 0; nn < K; ++nn) {
      const int r = r0 + nn;
      if (r < 0 || r >= S.H) continue;
      for (int m = 0; m < K; ++m) {
        const int i = i0 + m;
        if (i < 0 || i >= S.W) continue;
        const int e = nn * K + m;
        double v = 0.0;
        for (int side = 0; side < 2; ++side) {
          const double we = side ? wf : 1.0 - wf;
          if (we == 0.0) continue;
          const double* C = (side ? T1 : T0) + e;
          double rp[3];
          for (int p = 0; p < 3; ++p)
            rp[p] = fma(tx, fma(tx, C[(p * 3 + 2) * KK], C[(p * 3 + 1) * KK]), C[(p * 3) * KK]);
          v += we * fma(ty, fma(ty, rp[2], rp[1]), rp[0]);
        }
        atomicAdd(frame + (int64_t)r * Pf + i, w * v);
      }
    }
  }
}

cudaError_t launch_render_fp64_table(int K, int n_slices, int64_t max_stamps, const DevSlice* slices,
                                     const TableSlice* ts, const double* T64, const double* field_lt,
                                     const double* const* flux_tab, const double* u_all, double* const* acc,
                                     const int64_t* pitch, cudaStream_t st) {
  if (n_slices == 0 || max_stamps == 0) return cudaSuccess;
  int64_t bx = (max_stamps + 255) / 256;
  if (bx > 4096) bx = 4096;
  dim3 grid((unsigned)bx, (unsigned)n_slices);
  switch (K) {
#define E2E_CASE(KK) \
  case KK: k_render_fp64_table<KK><<<grid, 256, 0, st>>>(slices, ts, T64, field_lt, flux_tab, u_all, acc, pitch); break;
    E2E_CASE(1) E2E_CASE(3) E2E_CASE(5) E2E_CASE(7) E2E_CASE(9) E2E_CASE(11) E2E_CASE(13) E2E_CASE(15)
#undef E2E_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace e2e
