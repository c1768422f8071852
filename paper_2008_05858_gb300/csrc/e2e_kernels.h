// Host-callable launchers of the renderer's kernels (internal to the library).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "e2e_device.cuh"

namespace e2e {

constexpr int kTileW = 64;  // merge tile (pixels); 256 threads x 8 pixels
constexpr int kTileH = 32;
constexpr int kStaticSmemReserve = 1024;  // static shared memory of the render kernels (bytes, upper bound)

// The fused tile merge of the separable render kernel (merge_tile.cuh): per-tile item counts,
// the plan's tiles and lists, and the frames.  count == nullptr: no fused merge.
struct MergeArgs {
  const Item* items;        // the plan's items (the tile lists hold indices into this array)
  const Tile* tiles;
  const int32_t* lists;     // CSR item lists of the tiles (item order)
  const int32_t* tile_of;   // tile index of (detector, tile row, tile column)
  const int32_t* grid_off;  // per detector: its first entry in tile_of
  const int* dims;          // per detector: (H, W)
  int* count;               // per tile: items finished, zero before the render
  void* const* dst;         // frames
  const int64_t* pitch;     // their pitches (elements)
  int dtype;                // 0 = FP32 frame, 1 = FP64 frame
  const Tile* zero_tiles;   // tiles no item overlaps: written as zeros by the launch's last
  int n_zero;               // n_zero CTAs (0 = none in this launch)
};

cudaError_t launch_render_fp64(int K, int n_slices, int64_t max_stamps, const DevSlice* slices,
                               const double* const* flux_tab, const double* u_all, double* const* acc,
                               const int64_t* pitch, cudaStream_t st, const int2* frozen = nullptr);
cudaError_t launch_window_origins(int n_slices, int64_t max_stamps, const DevSlice* slices, int2* out,
                                  cudaStream_t st);
cudaError_t launch_convert(const double* src, int64_t src_pitch, void* dst, int dtype, int64_t dst_pitch, int H,
                           int W, cudaStream_t st);

cudaError_t launch_plan(const DevSlice* slices, int n_slices, const int64_t* task_off, int64_t n_tasks,
                        int4* bbox, const int64_t* bbox_off, int* spans, cudaStream_t st);
bool mixed_variant_supported(int K, int DX, int DY);
size_t mixed_smem_bytes(int area, int JB, int nk_max, int B, int nd);
cudaError_t launch_render_mixed(int K, int DX, int DY, const DevSlice* slices, const double* const* flux_tab,
                                const double* u_all, const Item* items, int n_items, float2* store, int B, int JB,
                                int nk_max, int max_deg, int far_tails, size_t smem, cudaStream_t st,
                                int* err = nullptr, const MergeArgs* mg = nullptr);
cudaError_t launch_merge(const Tile* tiles, int n_tiles, const int32_t* lists, const Item* items, const float2* store,
                         void* const* dst, int dtype, const int64_t* pitch, const int* dims, cudaStream_t st);

size_t ellip_smem_bytes(int area, int nk_max, int nd, int k_min);
cudaError_t launch_render_ellip(int K, const DevSlice* slices, const double* const* flux_tab, const double* u_all,
                                const Item* items, int n_items, float2* store, int nk_max, int max_deg, size_t smem,
                                cudaStream_t st, int* err = nullptr);
cudaError_t launch_render_fp64_ellip(int K, int n_slices, int64_t max_stamps, const DevSlice* slices,
                                     const double* const* flux_tab, const double* u_all, double* const* acc,
                                     const int64_t* pitch, cudaStream_t st);

cudaError_t launch_prnu_map(double* R, float* R32, float* R32lo, int H, int W, int det, uint64_t pattern_seed,
                            double prnu, cudaStream_t st);
cudaError_t launch_noise_two_pass(uint64_t seed, uint64_t pattern_seed, double dark, double prnu, double ron,
                                  double xtalk, double gain, double bias, int saturation, int src_dtype,
                                  const void* src, int64_t src_pitch, const double* R, const float* R32,
                                  const float* R32lo, int dst_dtype, void* dst, int64_t dst_pitch, int H, int W,
                                  int det, unsigned* list, unsigned* n_list, cudaStream_t st);
cudaError_t launch_noise(uint64_t seed, uint64_t pattern_seed, double dark, double prnu, double ron, double xtalk,
                         double gain, double bias, int saturation, int poisson, int src_dtype, const void* src,
                         int64_t src_pitch, const double* R, const float* R32, int dst_dtype, void* dst,
                         int64_t dst_pitch, int H, int W, int det, cudaStream_t st);

cudaError_t launch_epsf_build(const TableSlice* ts, int n_slices, int max_field, int max_cells, const double* maps,
                              double* norms, double* T64, float* T32, cudaStream_t st);
size_t table_smem_bytes(int area, int nk_max, int nd);
cudaError_t launch_render_table(int K, const DevSlice* slices, const TableSlice* ts, const float* T32,
                                const double* field_lt, const double* const* flux_tab, const double* u_all,
                                const Item* items, int n_items, float2* store, int nk_max, int max_deg, size_t smem,
                                cudaStream_t st, int* err = nullptr);
cudaError_t launch_render_fp64_table(int K, int n_slices, int64_t max_stamps, const DevSlice* slices,
                                     const TableSlice* ts, const double* T64, const double* field_lt,
                                     const double* const* flux_tab, const double* u_all, double* const* acc,
                                     const int64_t* pitch, cudaStream_t st);
// per-sample mapping coefficients and PSF constants of every slice (DevSlice::samples);
// psf 0 separable, 1 elliptical, 2 tabulated (ts and field_lt used only then)
cudaError_t launch_sample_tables(const DevSlice* slices, int n_slices, int max_lambda, int psf, const TableSlice* ts,
                                 const double* field_lt, cudaStream_t st);
cudaError_t launch_flag_nonfinite(const double* p, int64_t n, int* flag, cudaStream_t st);
cudaError_t launch_blaze(const DevSlice* slices, int n_slices, const double* const* flux_in, const int64_t* bin_off,
                         int64_t n_bins, double* out, cudaStream_t st);
cudaError_t launch_photon_bins(const DevSlice* slices, int n_slices, const double* const* flux_tab, const double* usum,
                               const int64_t* bin_off, int64_t n_bins, uint64_t seed, uint64_t* counts,
                               int4* anchors, int* bin_slice, cudaStream_t st);
constexpr int kPhotonGuide = 1 << 20;  // entries of the photon -> bin guide table (+1)
cudaError_t launch_photon_guide(const uint64_t* offsets, int64_t n_bins, int64_t* guide, cudaStream_t st);
size_t photon_coef_floats();
size_t scan_scratch_elems(int64_t n);
cudaError_t launch_scan_exclusive(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* scratch, cudaStream_t st);
cudaError_t launch_photons(const DevSlice* slices, int n_slices, const double* ucum, const double* usum,
                           const int64_t* bin_off, const uint64_t* offsets, int psf, uint64_t seed,
                           uint32_t* const* dst, const int64_t* pitch, uint64_t max_photons, const float* ucum32,
                           const float* cf32, const int4* anchors, const int* bin_slice, const int64_t* guide,
                           cudaStream_t st);

size_t adjoint_smem_bytes(int max_area, int max_deg, int nk_max, int nj_max);
cudaError_t launch_fold_gradients(int n_parent, int n_sub, const int* fold, const double* gcx_e, const double* gcy_e,
                                  const double* gsx_e, const double* gsy_e, double* gcx, double* gcy, double* gsx,
                                  double* gsy, cudaStream_t st);
int adjoint_parts(int max_tasks);  // CTAs per item sharing its warp tasks
cudaError_t launch_adjoint(int K, const DevSlice* slices, const double* const* flux_tab, const double* u_all,
                           const Item* items, int n_items, const void* const* dldi, const int64_t* pitch, int dtype,
                           int B, int nk_max, int parts, double* g_cx, double* g_cy, double* g_sx, double* g_sy,
                           size_t smem, cudaStream_t st, const int2* frozen = nullptr);

}  // namespace e2e
