// Mixed-precision tiled renderer (separable Gaussian PSF), its planner and the tile merge kernel.
//
// Work item = one order-slice x a block of wavelength samples x a block of slit points.
// Inside the item, a quad of lanes owns a *run* of B consecutive slit points of one wavelength
// sample: the run's stamps land within a (K+DX) x (K+DY) pixel tile (the plan checks this for
// every run of the model), so the quad accumulates their outer products w * A_x (x) A_y in
// FP32 registers (a quarter of the tile's rows per lane) and flushes the tile once per run
// into the item's box in shared memory.
// The box holds 52-bit fixed-point sums (two 32-bit words per pixel, scaled by a power of
// two above the item's total flux) updated with integer atomics: the accumulation is exact
// and independent of the order of the flushes.  At the end the box is written to a scratch
// "box store" as unevaluated FP32 pairs (hi + lo, ~48 bits).  Each output tile is then merged
// once (merge_tile.cuh): the boxes of all items overlapping it are added in item order with
// compensated summation and the frame is written once, either by the render CTA that finishes
// the tile's last item (fused) or by the merge kernel below.  No global atomics on the frame;
// the frame does not depend on scheduling.
//
// Precision (the paper's fidelity target, Sec. 2.2, is a photocenter shift below ~1e-5 px):
// per-sample mapping coefficients in FP64 (per-model tables), the polynomial in s in
// double-float FP32, the centre split exactly into an integer pixel and an FP32 offset, PSF
// pixel integrals in FP32 with double-float edge arguments (phi32.cuh), FP32 sums over one
// run (<= B stamps) in registers, exact fixed-point sums per item, compensated (TwoSum) sums
// of FP32 pairs across items.
#include "render_mixed.cuh"

namespace e2e {

// ------------------------------------------------------------------------------ plan

// One thread per (slice, wavelength sample j, block of 16 slit points): map the stamps
// exactly as the render will (map_stamp_df), and record (a) per (32-sample block, 16-point block) of each
// slice the bounding box of the stamps' windows, (b) per slice the largest spread of window
// origins over any aligned run of B = 1, 2, 4, 8, 16 consecutive slit points.  Stamps that
// map off every detector (kOffFrame) are ignored.
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
    const double inv_ns = 1.0 / (double)S.n_slit;
    const float4* row = S.samples + (int64_t)j * (S.degree + 3);  // per-model sample tables
    float4 P[9];  // degree <= 8
#pragma unroll
    for (int b = 0; b <= 8; ++b) P[b] = b <= S.degree ? row[b] : make_float4(0.f, 0.f, 0.f, 0.f);
    int xmn = 1 << 30, xmx = -(1 << 30), ymn = 1 << 30, ymx = -(1 << 30);
    int rxmn[5], rxmx[5], rymn[5], rymx[5], spx[5], spy[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) { rxmn[q] = rymn[q] = 1 << 30; rxmx[q] = rymx[q] = -(1 << 30); spx[q] = spy[q] = 0; }
    const int k0 = kb * 16, k1 = min(k0 + 16, S.n_slit);
    for (int k = k0; k < k1; ++k) {
      int ci, ri;
      float fx, fy;
      float2 mh, ml;
      map_xy_df_regs(P, S.degree, split_df(norm_sample_r(k, S.n_slit, inv_ns)), mh, ml);
      split_coord_df(mh.x, ml.x, ci, fx);
      split_coord_df(mh.y, ml.y, ri, fy);
      const bool on = ci != kOffFrame && ri != kOffFrame;
      if (on) {
        xmn = min(xmn, ci); xmx = max(xmx, ci); ymn = min(ymn, ri); ymx = max(ymx, ri);
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int B = 1 << q;
        if (on) {
          rxmn[q] = min(rxmn[q], ci); rxmx[q] = max(rxmx[q], ci);
          rymn[q] = min(rymn[q], ri); rymx[q] = max(rymx[q], ri);
        }
        if (((k + 1) % B) == 0 || k + 1 == k1) {  // end of an aligned run
          if (rxmx[q] >= rxmn[q]) {
            spx[q] = max(spx[q], rxmx[q] - rxmn[q]);
            spy[q] = max(spy[q], rymx[q] - rymn[q]);
          }
          rxmn[q] = rymn[q] = 1 << 30; rxmx[q] = rymx[q] = -(1 << 30);
        }
      }
    }
    if (xmx >= xmn) {
      const int h = S.K / 2;
      int4* bb = bbox + bbox_off[lo] + (int64_t)(j / 32) * nkb + kb;
      atomicMin(&bb->x, xmn - h);
      atomicMax(&bb->y, xmx + h);
      atomicMin(&bb->z, ymn - h);
      atomicMax(&bb->w, ymx + h);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      atomicMax(&spans[(lo * 5 + q) * 2 + 0], spx[q]);
      atomicMax(&spans[(lo * 5 + q) * 2 + 1], spy[q]);
    }
  }
}

size_t mixed_smem_bytes(int area, int JB, int nk_max, int B, int nd) {
  return MixedLayout(32 * JB, nk_max, nd, B, area).total;
}


// ------------------------------------------------------------------------------ merge

// One CTA of 256 threads per output tile (merge_tile.cuh).  Tiles that no item touches are zeros.
template <typename T>
__global__ void __launch_bounds__(256) k_merge(const Tile* __restrict__ tiles, const int32_t* __restrict__ lists,
                                               const Item* __restrict__ items, const float2* __restrict__ store,
                                               T* const* dst, const int64_t* __restrict__ pitch, const int* __restrict__ dims) {
  const Tile t = tiles[blockIdx.x];
  merge_tile<256, false, T>(t, lists, items, store, dst[t.det], pitch[t.det], dims[2 * t.det], dims[2 * t.det + 1],
                            threadIdx.x);
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


bool mixed_variant_supported(int K, int DX, int DY) {
  if (K < 1 || K > 15 || (K % 2) == 0) return false;
  if (DX == 0 && DY == 0) return true;
  if (DX == 1 && DY == 1) return K <= 13;
  if (DX == 1 && DY == 2) return K <= 13;
  if (DX == 1 && DY == 3) return K <= 11;
  if (DX == 2 && DY == 2) return K <= 9;
  return false;
}

cudaError_t launch_render_mixed(int K, int DX, int DY, const DevSlice* slices, const double* const* flux_tab,
                                const double* u_all, const Item* items, int n_items, float2* store, int B, int JB,
                                int nk_max, int max_deg, int far_tails, size_t smem, cudaStream_t st, int* err,
                                const MergeArgs* mg) {
  if (n_items == 0) return cudaSuccess;
  MixedArgs a{slices, flux_tab, u_all, items, store, B, JB, nk_max, max_deg, err, far_tails};
  const MergeArgs g = mg ? *mg : MergeArgs{};
  if (far_tails && K >= 3) return launch_render_mixed_far(K, DX, DY, err != nullptr, a, g, n_items, smem, st);
  if (err) return launch_render_mixed_checked(K, DX, DY, a, g, n_items, smem, st);
#define E2E_V(KK, X, Y) \
  if (K == KK && DX == X && DY == Y) return launch_one<KK, X, Y, false, false>(a, g, n_items, smem, st);
  E2E_MIXED_VARIANTS(E2E_V)
#undef E2E_V
  return cudaErrorInvalidValue;
}

cudaError_t launch_merge(const Tile* tiles, int n_tiles, const int32_t* lists, const Item* items, const float2* store,
                         void* const* dst, int dtype, const int64_t* pitch, const int* dims, cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  if (dtype == 0)
    k_merge<float><<<n_tiles, 256, 0, st>>>(tiles, lists, items, store, (float* const*)dst, pitch, dims);
  else
    k_merge<double><<<n_tiles, 256, 0, st>>>(tiles, lists, items, store, (double* const*)dst, pitch, dims);
  return cudaGetLastError();
}

}  // namespace e2e
