// The tile merge of the tiled renderers: the boxes of the items overlapping one 64x32 output
// tile are added per pixel in item order with compensated summation (TwoSum on the FP32
// pairs, Neumaier's correction carried in a second word), converted and written once.  One
// device function serves the standalone merge kernel (256 threads per tile) and the fused
// merge at the end of the separable render kernel (128 threads), so both give the same bits.
//
// Fused merge: every tile counts its finished items.  A render CTA, after writing its box,
// fences, adds one to the count of each tile the box overlaps, and the CTA that brings a
// tile's count to the tile's number of items merges that tile.  Nothing waits: the last
// arrival does the work, and the counts are zeroed before each render.  Tiles that no item
// overlaps are written as zeros by the standalone kernel over the plan's zero-tile list.
#pragma once
#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "mixed_common.cuh"

namespace e2e {

// Merge tile t with NT threads (thread index tid); box reads bypass L1 when CG (the boxes were
// written by other CTAs during this launch).
template <int NT, bool CG, typename T>
__device__ __forceinline__ void merge_tile(const Tile& t, const int32_t* __restrict__ lists,
                                           const Item* __restrict__ items, const float2* store, T* frame, int64_t P,
                                           int H, int W, int tid) {
  constexpr int kRows = kTileW * kTileH / NT;  // pixels per thread
  constexpr int kStep = NT / kTileW;
  const int tx = tid & (kTileW - 1), ty0 = tid / kTileW;
  const int x = t.x0 + tx;
  if (t.n == 0) {
    if (x < W) {
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        const int y = t.y0 + ty0 + q * kStep;
        if (y < H) frame[(int64_t)y * P + x] = (T)0;
      }
    }
    return;
  }
  float sum[kRows], comp[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) sum[q] = comp[q] = 0.f;
  for (int n = 0; n < t.n; ++n) {
    const Item it = items[lists[t.list_off + n]];
    const int gx = x - it.bx0;
    if (gx < 0 || gx >= it.bw) continue;
    const float2* box = store + it.store_off;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const int gy = t.y0 + ty0 + q * kStep - it.by0;
      if (gy >= 0 && gy < it.bh) {
        const float2 v = CG ? __ldcg(box + (int64_t)gy * it.bw + gx) : box[(int64_t)gy * it.bw + gx];
        float s, e;
        two_sum(sum[q], v.x, s, e);
        sum[q] = s;
        comp[q] += e + v.y;
      }
    }
  }
  if (x >= W) return;
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int y = t.y0 + ty0 + q * kStep;
    if (y < H) frame[(int64_t)y * P + x] = sizeof(T) == 8 ? (T)((double)sum[q] + (double)comp[q]) : (T)(sum[q] + comp[q]);
  }
}

// End of a render CTA of NT threads that has written item `it`'s box (every thread's stores
// issued): count the item into its tiles and merge the tiles it completes.
template <int NT>
__device__ void fused_merge_epilogue(const MergeArgs& g, const float2* store, const Item& it, int det) {
  __shared__ int s_tiles[NT];
  __shared__ int s_n;
  const Item* __restrict__ items = g.items;
  __threadfence();  // this thread's box stores are visible device-wide
  __syncthreads();  // ... and every thread's, before any count of this CTA
  const int W = g.dims[2 * det + 1], H = g.dims[2 * det];
  const int ntx_det = (W + kTileW - 1) / kTileW;
  const int tx0 = it.bx0 / kTileW, tx1 = (it.bx0 + it.bw - 1) / kTileW;
  const int ty0 = it.by0 / kTileH, ty1 = (it.by0 + it.bh - 1) / kTileH;
  const int ntx = tx1 - tx0 + 1, n = ntx * (ty1 - ty0 + 1);
  for (int base = 0; base < n; base += NT) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int i = base + (int)threadIdx.x;
    if (i < n) {
      const int ty = ty0 + i / ntx, tx = tx0 + i % ntx;
      const int tile = g.tile_of[g.grid_off[det] + ty * ntx_det + tx];
      __threadfence();  // release: the CTA's box (ordered before this thread by the barrier)
      if (atomicAdd(&g.count[tile], 1) + 1 == g.tiles[tile].n) {
        __threadfence();  // acquire: the other items' boxes, released before their counts
        s_tiles[atomicAdd(&s_n, 1)] = tile;
      }
    }
    __syncthreads();
    const int m = s_n;
    if (m > 0) {
      __threadfence();  // the other items' boxes, counted before ours, are visible to this CTA
      for (int k = 0; k < m; ++k) {
        const Tile t = g.tiles[s_tiles[k]];
        if (g.dtype == 0)
          merge_tile<NT, true, float>(t, g.lists, items, store, static_cast<float*>(g.dst[t.det]), g.pitch[t.det], H, W,
                                      threadIdx.x);
        else
          merge_tile<NT, true, double>(t, g.lists, items, store, static_cast<double*>(g.dst[t.det]), g.pitch[t.det], H,
                                       W, threadIdx.x);
      }
    }
    __syncthreads();  // s_tiles and s_n are reused by the next chunk
  }
}

}  // namespace e2e
