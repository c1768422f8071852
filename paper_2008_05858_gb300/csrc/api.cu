// C ABI and host runtime of the echelle frame renderer: contexts, resident optical models
// (with their tiled-render plan) and spectra, render jobs, library-owned frames.
//
// The spectral-format "database" of the paper (Sec. 2.1) is computed once and reused across
// simulations; here an optical model is validated, copied to the device and planned once
// (e2e_load_model), spectra are resident too, and a render only launches kernels.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/e2e_render.h"
#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "tail_coeffs.h"

using namespace e2e;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? E2E_ENOMEM : E2E_ECUDA;
}

// An NVTX range around one stage of the runtime (visible to profilers that record NVTX; a
// pointer check otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define E2E_CK(call)                                       \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

struct SliceHost {
  e2e_order_slice d;
  std::vector<double> cx, cy, u, field_lt, maps;
};

struct Plan {
  bool ok = false;
  int B = 1, DX = 0, DY = 0, JB = 1, NB = 8, max_area = 0, max_deg = 0, nk_max = 1;
  int far_tails = 0;  // separable kernel: every tail edge's argument within the cheaper rational's fit
  std::vector<Item> items;  // host copy
  int64_t store_elems = 0;
  size_t smem = 0;
  // device
  Item* d_items = nullptr;
  Tile* d_tiles = nullptr;
  int32_t* d_lists = nullptr;
  int n_tiles = 0;
  // items grouped by K (one kernel launch per group)
  struct Group {
    int K, first, count;
  };
  std::vector<Group> groups;
  // y-bands: within each K group the items are ordered by the band of their box's first row,
  // and the merge tiles by band, so band b of every detector is final once the items of bands
  // <= b are rendered (no item reaches above its box)
  int n_bands = 1;
  std::vector<int> band_tile_rows;  // per detector: tile rows per band
  std::vector<int> seg_first;       // [group * n_bands + band]: first item of the segment
  std::vector<int> seg_count;
  std::vector<int> tile_first;      // [n_bands + 1]: merge tiles of each band
  // fused merge: tile index of each (detector, tile row, tile column), and the tiles that no
  // item overlaps (written as zeros by the merge kernel)
  int32_t* d_tile_of = nullptr;
  int32_t* d_grid_off = nullptr;
  Tile* d_zero_tiles = nullptr;
  int n_zero_tiles = 0;
};

constexpr int kBands = 16;  // y-bands of a frame rendered into host memory

struct Model {
  int n_det = 0, psf = 0;
  std::vector<int> H, W;
  std::vector<SliceHost> slices;
  std::vector<DevSlice> dev;  // host copy of d_slices
  int coef_total = 0;
  DevSlice* d_slices = nullptr;
  double* d_u = nullptr;
  double* d_ucum = nullptr;     // running sums of the slit weights (photon renderer)
  double* d_usum = nullptr;     // their totals, per slice
  float* d_ucum32 = nullptr;    // FP32 copies for the photon fast path
  float* d_cf32 = nullptr;      // FP32 mapping coefficients and bounds per slice (photon fast path)
  int64_t* d_bin_off = nullptr; // first wavelength bin of each slice (photon renderer, blaze)
  std::vector<int64_t> bin_off;
  int64_t n_bins = 0;
  bool u_nonneg = true;
  bool has_blaze = false;  // some slice weights its samples by a blaze function
  // tabulated PSF: per-slice layout, field nodes, effective-PSF tables (FP64 and FP32)
  TableSlice* d_ts = nullptr;
  double* d_field = nullptr;
  double* d_T64 = nullptr;
  float* d_T32 = nullptr;
  int* d_dims = nullptr;  // [det][2] = (H, W)
  int64_t max_stamps = 0;
  int64_t n_stamps = 0;  // stamps of all slices (the length of a window-origin list)
  std::vector<int> Ks;    // distinct K values
  Plan plan;
  // 2-D fiber sub-apertures: the caller's ("parent") slices and the one-dimensional slices,
  // one per aperture row, the library renders in their place (sub-slice q of parent
  // parent_of[q], row t_of[q]); identity when no slice has n_aper > 1
  bool expanded = false;
  std::vector<int> parent_of, first_sub, parent_nc, parent_coef_off;
  std::vector<double> t_of, apx, apy;  // apx/apy: 3 per parent
  int parent_coef_total = 0;
  int* d_fold = nullptr;  // first_sub | sub coef_off | parent coef_off | parent nc (adjoint folding)
  float4* d_stab = nullptr;  // per-sample tables of every slice (DevSlice::samples)
};

struct Spectrum {
  int fiber = 0;
  std::map<int, std::pair<int64_t, int>> rows;  // order -> (offset, n_lambda)
  double* d_flux = nullptr;
};

// A library-owned frame.  Its buffers come from the stream-ordered pool; `ready` marks the
// last use enqueued on any stream (the render, then each fetch), so a fetch on another stream
// and the release both wait for it without synchronising the device.
struct Frame {
  int dtype = 0;
  std::vector<int> H, W;
  std::vector<void*> ptrs;
  cudaEvent_t ready = nullptr;
};

}  // namespace

namespace {
struct Server;
}

struct e2e_ctx {
  int device = 0;
  std::unique_ptr<Server> server;
  e2e_opts opts{};
  std::mutex mu;
  uint64_t next_id = 1;
  std::map<uint64_t, std::unique_ptr<Model>> models;
  std::map<uint64_t, std::unique_ptr<Spectrum>> spectra;
  std::map<uint64_t, std::unique_ptr<Frame>> frames;
  cudaMemPool_t pool = nullptr;
  cudaStream_t free_stream = nullptr;  // where library frames are returned to the pool
  // spectrum uploads: pool allocation, copy and finiteness check on their own stream
  std::mutex load_mu;
  cudaStream_t load_stream = nullptr;
  int* d_flag = nullptr;
  int* h_flag = nullptr;  // page-locked
  int* d_err = nullptr;                // debug checks: deposits outside the planned boxes
  struct NoisePattern {                // pixel response map of a model's detectors (FP64)
    uint64_t pattern_seed = 0;
    double prnu = 0.0;
    std::vector<double*> R;
    std::vector<float*> R32;
  };
  std::map<uint64_t, NoisePattern> patterns;  // by model id
  // kernel timing of the most recent render (opts.kernel_timing)
  struct Timed {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> event_pool;
  // banded render into host memory (e2e_render_host): two render streams, a high-priority
  // merge stream, a copy stream and per-band events, created on first use
  cudaStream_t band_st[2] = {nullptr, nullptr};
  cudaStream_t merge_st = nullptr, copy_st = nullptr;
  std::vector<cudaEvent_t> band_ev;
};

namespace {

// ---------------------------------------------------------------- serving state
struct Job {
  uint64_t id = 0;
  uint64_t model = 0;
  std::vector<uint64_t> spec;
  std::vector<void*> dst;  // empty: library-owned frames
  std::vector<int64_t> pitch;
  int precision = 0, dtype = 0;
  int status = E2E_JOB_QUEUED;
  int err = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  float device_ms = 0.f;
  int64_t budget = 0, stamps = 0;
  uint64_t frame_id = 0;
  int slot = -1;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool finished_on_device = false;
  bool express = false;  // small job: admitted before regular ones, high-priority stream
};

struct Server {
  e2e_ctx* ctx = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;       // wakes the loop
  std::condition_variable cv_done;  // wakes waiters
  bool stopping = false;
  std::deque<uint64_t> queue;     // regular jobs, FIFO
  std::deque<uint64_t> express;   // jobs of <= express_stamps stamps, FIFO, admitted first
  int64_t express_stamps = 0;
  int express_slots = 0;  // slots regular jobs may not take
  std::map<uint64_t, Job> jobs;
  std::vector<cudaStream_t> slots;     // lowest stream priority
  std::vector<cudaStream_t> slots_hi;  // highest stream priority (express jobs)
  std::vector<uint64_t> slot_job;  // 0 = free
  size_t budget = 0, in_use = 0;
  uint64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int n_coeffs(int d) { return (d + 1) * (d + 2) / 2; }

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Minimum of c0 + c1 t + c2 t^2 over t in [-1, 1].
double quad_min(const double* c) {
  double m = std::min(c[0] - c[1] + c[2], c[0] + c[1] + c[2]);
  if (c[2] > 0) {
    double t = -c[1] / (2 * c[2]);
    if (t > -1 && t < 1) m = std::min(m, c[0] + c[1] * t + c[2] * t * t);
  }
  return m;
}

// Maximum of c0 + c1 t + c2 t^2 over t in [-1, 1].
double quad_max(const double* c) {
  const double n[3] = {-c[0], -c[1], -c[2]};
  return -quad_min(n);
}

constexpr double kMaxEllipEps = 0.2;

int validate_slice(const e2e_order_slice& s, int n_det, int psf, int idx) {
  char buf[256];
  auto bad = [&](const char* why) {
    snprintf(buf, sizeof buf, "order-slice %d: %s", idx, why);
    return fail(E2E_EINVAL, buf);
  };
  if (s.detector < 0 || s.detector >= n_det) return bad("detector index out of range");
  if (s.degree < 0 || s.degree > E2E_MAX_DEGREE) return bad("degree out of range 0..8");
  if (s.K < 1 || s.K > E2E_MAX_K || s.K % 2 == 0) return bad("K must be odd and in 1..15");
  if (s.n_lambda < 1 || s.n_slit < 1) return bad("n_lambda and n_slit must be >= 1");
  if (s.n_slit > 65536 || s.n_lambda > (1 << 28)) return bad("n_lambda or n_slit too large");
  if (!std::isfinite(s.lambda_lo) || !std::isfinite(s.lambda_hi) || !(s.lambda_hi > s.lambda_lo))
    return bad("lambda range must be finite with lambda_hi > lambda_lo");
  if (!s.cx || !s.cy || !s.slit_weights) return bad("null coefficient or weight array");
  const int nc = n_coeffs(s.degree);
  if (!finite_all(s.cx, nc) || !finite_all(s.cy, nc)) return bad("non-finite mapping coefficient");
  if (!finite_all(s.sigma_x, 3) || !finite_all(s.sigma_y, 3)) return bad("non-finite PSF width coefficient");
  if (quad_min(s.sigma_x) <= 0 || quad_min(s.sigma_y) <= 0) return bad("PSF width must stay > 0 on [-1, 1]");
  if (s.n_aper < 0 || s.n_aper > 64) return bad("n_aper must be 0..64");
  if (!finite_all(s.aper_x, 3) || !finite_all(s.aper_y, 3)) return bad("non-finite aperture displacement");
  if (!finite_all(s.slit_weights, (int64_t)s.n_slit * (s.n_aper > 1 ? s.n_aper : 1)))
    return bad("non-finite slit weight");
  if (!std::isfinite(s.blaze_order) || (s.blaze_order != 0.0 && !(s.blaze_lambda > 0.0 && std::isfinite(s.blaze_lambda))))
    return bad("blaze: finite order and a positive, finite blaze wavelength required");
  if (psf == E2E_PSF_TABLE) {
    if (s.n_field < 1 || !s.field_lt || !s.maps) return bad("tabulated PSF needs n_field >= 1 and maps");
    if (s.map_size < 2 || s.map_size > 4096) return bad("map_size must be 2..4096");
    if (!(s.map_oversample >= 1.0 && s.map_oversample <= 32.0) || s.map_oversample != std::floor(s.map_oversample))
      return bad("map_oversample must be an integer 1..32 (samples per pixel)");
    for (int f = 0; f < s.n_field; ++f) {
      if (!std::isfinite(s.field_lt[f]) || s.field_lt[f] < -1.0 || s.field_lt[f] > 1.0 ||
          (f > 0 && !(s.field_lt[f] > s.field_lt[f - 1])))
        return bad("field_lt must be strictly increasing in [-1, 1]");
      double sum = 0.0;
      const double* mp = s.maps + (size_t)f * s.map_size * s.map_size;
      for (int i = 0; i < s.map_size * s.map_size; ++i) {
        if (!std::isfinite(mp[i]) || mp[i] < 0.0) return bad("PSF map samples must be finite and >= 0");
        sum += mp[i];
      }
      if (!(sum > 0.0)) return bad("every PSF map needs a positive sum");
    }
  }
  if (psf == E2E_PSF_ELLIPTICAL) {
    if (!std::isfinite(s.theta)) return bad("non-finite theta");
    // The elliptical renderers expand the conditional profile of y given x in eps * tau,
    // |tau| <= 1/2 within a pixel column; eps = beta / s_c must stay within the range where
    // the truncated series is exact to FP32 (checked at every wavelength sample).
    const double c = std::cos(s.theta), sn = std::sin(s.theta);
    for (int j = 0; j < s.n_lambda; ++j) {
      const double lt = (double)(2 * j + 1 - s.n_lambda) / (double)s.n_lambda;
      const double sa = (s.sigma_x[2] * lt + s.sigma_x[1]) * lt + s.sigma_x[0];
      const double sb = (s.sigma_y[2] * lt + s.sigma_y[1]) * lt + s.sigma_y[0];
      const double vx = sa * sa * c * c + sb * sb * sn * sn, vy = sa * sa * sn * sn + sb * sb * c * c;
      const double cxy = (sa * sa - sb * sb) * sn * c;
      const double eps = cxy / vx / std::sqrt(vy - cxy * cxy / vx);
      if (!(std::fabs(eps) <= kMaxEllipEps)) return bad("elliptical PSF too strongly sheared: |cxy / sqrt(vx (vx vy - cxy^2))| must stay <= 0.2");
    }
  }
  return E2E_OK;
}

Model* find_model(e2e_ctx* ctx, uint64_t id) {
  auto it = ctx->models.find(id);
  return it == ctx->models.end() ? nullptr : it->second.get();
}

void free_plan(Plan& p) {
  cudaFree(p.d_items);
  cudaFree(p.d_tiles);
  cudaFree(p.d_lists);
  cudaFree(p.d_tile_of);
  cudaFree(p.d_grid_off);
  cudaFree(p.d_zero_tiles);
  p = Plan{};
}

void free_model(Model* m) {
  cudaFree(m->d_slices);
  cudaFree(m->d_u);
  cudaFree(m->d_ucum);
  cudaFree(m->d_usum);
  cudaFree(m->d_ucum32);
  cudaFree(m->d_cf32);
  cudaFree(m->d_bin_off);
  cudaFree(m->d_ts);
  cudaFree(m->d_field);
  cudaFree(m->d_T64);
  cudaFree(m->d_T32);
  cudaFree(m->d_dims);
  cudaFree(m->d_fold);
  cudaFree(m->d_stab);
  free_plan(m->plan);
}

template <typename T>
int upload(T** dptr, const T* src, size_t n) {
  *dptr = nullptr;
  if (n == 0) return E2E_OK;
  E2E_CK(cudaMalloc((void**)dptr, n * sizeof(T)));
  E2E_CK(cudaMemcpy(*dptr, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return E2E_OK;
}

// ------------------------------------------------------------------ planning

// Relative cost per stamp of a tile variant of the separable kernel: a lane evaluates the
// K+1 edges of one axis of a stamp's window (~30 FP32 operations and 2 SFU operations per
// edge) and shifts it into the tile (two selects per pixel); the quad of lanes that owns the
// run accumulates the (K+DX) x (K+DY) tile, a quarter of its rows per lane, and once per run
// of B stamps maps the run, clears and flushes the tile (~30 operations per tile pixel:
// calibrated on the full-detector frame, K = 11, where runs of 16 / 8 / 4 stamps took 7.41 /
// 9.30 / 10.18 ms); tiles above 84 accumulators per lane halve the occupancy.
double variant_cost(int K, int DX, int DY, int B) {
  const int D = std::max(DX, DY);
  const double edges = 2.0 * (K + 1);
  const double tile = (double)(K + DX) * (K + DY);
  double c = edges * 30.0 + 2.0 * (K + D) + tile + tile * 30.0 / B;
  if ((K + DX) * ((K + DY + 3) / 4) > 84) c *= 1.6;
  return c;
}

// Phase-cell tables of a tabulated-PSF model, built on the device at load time.
int build_psf_tables(Model* m) {
  NvtxRange nvtx_("e2e psf tables");
  const int ns = (int)m->slices.size();
  std::vector<TableSlice> ts(ns);
  std::vector<double> field, maps;
  int64_t tab = 0, tab32 = 0;
  int max_field = 1, max_cells = 1;
  for (int i = 0; i < ns; ++i) {
    const e2e_order_slice& s = m->slices[i].d;
    TableSlice& t = ts[i];
    t.tab_off = tab;
    t.tab_off32 = tab32;
    t.map_off = (int64_t)maps.size();
    t.field_off = (int32_t)field.size();
    t.n_field = s.n_field;
    t.map_size = s.map_size;
    t.K = s.K;
    t.q = (int32_t)s.map_oversample;  // validated to be an integer in 1..32
    t.half = s.map_size % 2 == 0 ? 1 : 0;
    t.n_cell = t.q + t.half;
    t.pad = 0;
    field.insert(field.end(), s.field_lt, s.field_lt + s.n_field);
    maps.insert(maps.end(), s.maps, s.maps + (size_t)s.n_field * s.map_size * s.map_size);
    const int64_t rows = (int64_t)s.n_field * t.n_cell * t.n_cell * 9;
    tab += rows * s.K * s.K;
    tab32 += rows * table_row32(s.K);
    max_field = std::max(max_field, s.n_field);
    max_cells = std::max(max_cells, t.n_cell);
  }
  if ((int64_t)max_field * max_cells * max_cells > 65535)
    return fail(E2E_EINVAL, "too many field nodes x phase cells (n_field x (q + 1)^2 must stay <= 65535)");
  double* d_maps = nullptr;
  double* d_norms = nullptr;
  int rc = upload(&m->d_ts, ts.data(), ts.size());
  if (rc == E2E_OK) rc = upload(&m->d_field, field.data(), field.size());
  if (rc == E2E_OK) rc = upload(&d_maps, maps.data(), maps.size());
  if (rc == E2E_OK && cudaMalloc((void**)&d_norms, std::max<size_t>(1, field.size()) * sizeof(double)) != cudaSuccess)
    rc = fail(E2E_ENOMEM, "map norms");
  if (rc == E2E_OK && (cudaMalloc((void**)&m->d_T64, std::max<int64_t>(1, tab) * sizeof(double)) != cudaSuccess ||
                       cudaMalloc((void**)&m->d_T32, std::max<int64_t>(1, tab32) * sizeof(float)) != cudaSuccess))
    rc = fail(E2E_ENOMEM, "PSF tables");
  if (rc == E2E_OK) {  // the FP32 rows' padding is never read; zero it all the same
    const cudaError_t e = cudaMemset(m->d_T32, 0, std::max<int64_t>(1, tab32) * sizeof(float));
    if (e != cudaSuccess) rc = cuda_fail(e, "PSF tables");
  }
  if (rc == E2E_OK) {
    cudaError_t e = launch_epsf_build(m->d_ts, ns, max_field, max_cells, d_maps, d_norms, m->d_T64, m->d_T32, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "PSF table build");
  }
  cudaFree(d_maps);
  cudaFree(d_norms);
  return rc;
}

// Bands and merge tiles of a planned model (every model, including one without slices, whose
// tiles are all empty and merge to zeros).
int plan_bands_and_tiles(Model* m) {
  Plan& P = m->plan;
  std::vector<int> tile_base(m->n_det + 1, 0);
  std::vector<int> ntx(m->n_det), nty(m->n_det);
  int max_ty = 1;
  for (int d = 0; d < m->n_det; ++d) {
    ntx[d] = (m->W[d] + kTileW - 1) / kTileW;
    nty[d] = (m->H[d] + kTileH - 1) / kTileH;
    tile_base[d + 1] = tile_base[d] + ntx[d] * nty[d];
    max_ty = std::max(max_ty, nty[d]);
  }

  // ---- y-bands: order each K group's items by the band of their first row (stable, so the
  // items of one band keep the slice-major order) and lay out their boxes in that order
  P.n_bands = std::min(kBands, max_ty);
  P.band_tile_rows.assign(m->n_det, 1);
  for (int d = 0; d < m->n_det; ++d) P.band_tile_rows[d] = (nty[d] + P.n_bands - 1) / P.n_bands;
  auto band_of = [&](const Item& it) {
    const int d = m->slices[it.slice].d.detector;
    return (it.by0 / kTileH) / P.band_tile_rows[d];
  };
  P.seg_first.assign(P.groups.size() * P.n_bands, 0);
  P.seg_count.assign(P.groups.size() * P.n_bands, 0);
  for (size_t g = 0; g < P.groups.size(); ++g) {
    auto first = P.items.begin() + P.groups[g].first;
    std::stable_sort(first, first + P.groups[g].count,
                     [&](const Item& a, const Item& b) { return band_of(a) < band_of(b); });
    for (int n = P.groups[g].first; n < P.groups[g].first + P.groups[g].count; ++n) {
      const int b = band_of(P.items[n]);
      if (P.seg_count[g * P.n_bands + b]++ == 0) P.seg_first[g * P.n_bands + b] = n;
    }
  }
  {
    int64_t off = 0;
    for (auto& it : P.items) {
      it.store_off = off;
      off += (int64_t)it.bw * it.bh;
    }
  }

  // ---- merge tiles: every tile of every detector, with the items overlapping it, in band order
  std::vector<Tile> tiles;
  std::vector<std::vector<int32_t>> lists;
  lists.resize(tile_base[m->n_det]);
  for (size_t n = 0; n < P.items.size(); ++n) {
    const Item& it = P.items[n];
    const int d = m->slices[it.slice].d.detector;
    for (int ty = it.by0 / kTileH; ty <= (it.by0 + it.bh - 1) / kTileH; ++ty)
      for (int tx = it.bx0 / kTileW; tx <= (it.bx0 + it.bw - 1) / kTileW; ++tx)
        lists[tile_base[d] + ty * ntx[d] + tx].push_back((int32_t)n);
  }
  std::vector<int32_t> flat;
  P.tile_first.clear();
  for (int b = 0; b < P.n_bands; ++b) {
    P.tile_first.push_back((int)tiles.size());
    for (int d = 0; d < m->n_det; ++d)
      for (int ty = b * P.band_tile_rows[d]; ty < std::min(nty[d], (b + 1) * P.band_tile_rows[d]); ++ty)
        for (int tx = 0; tx < ntx[d]; ++tx) {
          const auto& l = lists[tile_base[d] + ty * ntx[d] + tx];
          Tile t{d, tx * kTileW, ty * kTileH, (int)l.size(), (int64_t)flat.size()};
          flat.insert(flat.end(), l.begin(), l.end());
          tiles.push_back(t);
        }
  }
  P.tile_first.push_back((int)tiles.size());
  P.n_tiles = (int)tiles.size();
  std::vector<int32_t> tile_of(tile_base[m->n_det]), grid_off(tile_base.begin(), tile_base.end() - 1);
  std::vector<Tile> zero_tiles;
  for (size_t i = 0; i < tiles.size(); ++i) {
    const Tile& t = tiles[i];
    tile_of[tile_base[t.det] + (t.y0 / kTileH) * ntx[t.det] + t.x0 / kTileW] = (int32_t)i;
    if (t.n == 0) zero_tiles.push_back(t);
  }
  P.n_zero_tiles = (int)zero_tiles.size();
  int rc = upload(&P.d_items, P.items.data(), P.items.size());
  if (rc == E2E_OK) rc = upload(&P.d_tiles, tiles.data(), tiles.size());
  if (rc == E2E_OK) rc = upload(&P.d_lists, flat.data(), flat.size());
  if (rc == E2E_OK) rc = upload(&P.d_tile_of, tile_of.data(), tile_of.size());
  if (rc == E2E_OK) rc = upload(&P.d_grid_off, grid_off.data(), grid_off.size());
  if (rc == E2E_OK) rc = upload(&P.d_zero_tiles, zero_tiles.data(), zero_tiles.size());
  if (rc != E2E_OK) return rc;
  P.ok = true;
  return E2E_OK;
}

// Per-sample tables (mapping coefficients in s and PSF constants at each wavelength sample)
// of every slice, rebuilt on the device whenever the model's coefficients change.
int build_sample_tables(Model* m) {
  const int ns = (int)m->slices.size();
  int64_t total = 0;
  int max_lambda = 0;
  std::vector<int64_t> off(ns);
  for (int i = 0; i < ns; ++i) {
    off[i] = total;
    total += (int64_t)m->dev[i].n_lambda * (m->dev[i].degree + 3);
    max_lambda = std::max(max_lambda, m->dev[i].n_lambda);
  }
  if (!m->d_stab) E2E_CK(cudaMalloc((void**)&m->d_stab, (size_t)total * sizeof(float4)));
  for (int i = 0; i < ns; ++i) m->dev[i].samples = m->d_stab + off[i];
  E2E_CK(cudaMemcpy(m->d_slices, m->dev.data(), ns * sizeof(DevSlice), cudaMemcpyHostToDevice));
  const int psf = m->psf == E2E_PSF_ELLIPTICAL ? 1 : m->psf == E2E_PSF_TABLE ? 2 : 0;
  E2E_CK(launch_sample_tables(m->d_slices, ns, max_lambda, psf, m->d_ts, m->d_field, 0));
  E2E_CK(cudaDeviceSynchronize());
  return E2E_OK;
}

int plan_model(Model* m) {
  NvtxRange nvtx_("e2e plan");
  Plan& P = m->plan;
  const int ns = (int)m->slices.size();
  const bool ellip = m->psf != E2E_PSF_SEPARABLE;  // item shape of the non-separable kernels
  if (ns == 0) return plan_bands_and_tiles(m);
  if (int rc0 = build_sample_tables(m); rc0 != E2E_OK) return rc0;
  // ---- device pass: exact window origins of every stamp
  std::vector<int64_t> task_off(ns + 1, 0), bb_off(ns + 1, 0);
  std::vector<int> n_jb(ns), n_k16(ns);
  for (int i = 0; i < ns; ++i) {
    const auto& s = m->slices[i].d;
    n_jb[i] = (s.n_lambda + 31) / 32;
    n_k16[i] = (s.n_slit + 15) / 16;
    task_off[i + 1] = task_off[i] + (int64_t)s.n_lambda * n_k16[i];
    bb_off[i + 1] = bb_off[i] + (int64_t)n_jb[i] * n_k16[i];
  }
  int64_t *d_task_off = nullptr, *d_bb_off = nullptr;
  int4* d_bbox = nullptr;
  int* d_spans = nullptr;
  std::vector<int4> bbox(bb_off[ns], make_int4(1 << 30, -(1 << 30), 1 << 30, -(1 << 30)));
  std::vector<int> spans(ns * 10, 0);
  int rc = upload(&d_task_off, task_off.data(), task_off.size());
  if (rc == E2E_OK) rc = upload(&d_bb_off, bb_off.data(), bb_off.size());
  if (rc == E2E_OK) rc = upload(&d_bbox, bbox.data(), bbox.size());
  if (rc == E2E_OK) rc = upload(&d_spans, spans.data(), spans.size());
  if (rc == E2E_OK) {
    cudaError_t e = launch_plan(m->d_slices, ns, d_task_off, task_off[ns], d_bbox, d_bb_off, d_spans, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(bbox.data(), d_bbox, bbox.size() * sizeof(int4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(spans.data(), d_spans, spans.size() * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "plan kernel");
  }
  cudaFree(d_task_off);
  cudaFree(d_bb_off);
  cudaFree(d_bbox);
  cudaFree(d_spans);
  if (rc != E2E_OK) return rc;

  // ---- tile variant and run length (one for the whole model; per-K kernels).  The
  // elliptical kernel has no run tiles: one item per (32-sample, 16-point) block.
  int K = 0;
  for (auto& s : m->slices) K = std::max(K, s.d.K);
  double best = 1e300;
  int bB = 1, bDX = 0, bDY = 0;
  const int variants[5][2] = {{0, 0}, {1, 1}, {1, 2}, {1, 3}, {2, 2}};
  for (int q = 0; q <= 4 && !ellip; ++q) {  // B = 1..16
    const int B = 1 << q;
    int sx = 0, sy = 0;
    for (int i = 0; i < ns; ++i) {
      sx = std::max(sx, spans[(i * 5 + q) * 2 + 0]);
      sy = std::max(sy, spans[(i * 5 + q) * 2 + 1]);
    }
    for (auto& v : variants) {
      bool ok = true;
      for (int k : m->Ks) ok = ok && mixed_variant_supported(k, v[0], v[1]);
      if (!ok || sx > v[0] || sy > v[1]) continue;
      const double c = variant_cost(K, v[0], v[1], B);
      if (c < best) {
        best = c;
        bB = B;
        bDX = v[0];
        bDY = v[1];
      }
    }
  }
  P.B = bB;
  // The tail edges (off the centre pixel) sit at |e - f| >= 1 px from a stamp's centre, i.e. at
  // arguments w >= sqrt(log2 e) / (sqrt 2 sigma) in log2 units: when the model's widest PSF
  // keeps that at or above the cheaper rational's lower end (sigma <= 2.12 px), the separable
  // kernel takes that rational on them (a margin of 1e-3 on the width covers the FP32 rounding
  // of the per-sample constants).
  {
    double smax = 0.0;
    for (auto& s : m->slices) smax = std::max(smax, std::max(quad_max(s.d.sigma_x), quad_max(s.d.sigma_y)));
    const double limit = kSqrtLog2eD / (std::sqrt(2.0) * (double)kTailFarMinArg);
    P.far_tails = !ellip && smax <= limit * (1.0 - 1e-3) ? 1 : 0;
  }
  P.DX = bDX;
  P.DY = bDY;
  P.max_deg = 0;
  for (auto& s : m->slices) P.max_deg = std::max(P.max_deg, s.d.degree);

  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

  // ---- items: (32-sample blocks) x (16-point blocks); at most 16 warp tasks (<= 512 runs,
  // which keeps the fixed-point low words of a box below 2^31) and a box that fits on chip
  for (int jb_cap = 8; jb_cap >= 1; jb_cap /= 2) {
    int64_t store = 0;
    P.items.clear();
    P.groups.clear();
    P.JB = 1;
    for (int Kg : m->Ks) {
      Plan::Group g{Kg, (int)P.items.size(), 0};
      for (int i = 0; i < ns; ++i) {
        const auto& s = m->slices[i].d;
        if (s.K != Kg) continue;
        const int nrc_full = (s.n_slit + P.B - 1) / P.B;
        int KC = nrc_full <= 16 ? n_k16[i] : P.B;  // 16-point blocks per item
        const int nrc = std::min(nrc_full, (KC * 16 + P.B - 1) / P.B);
        int JB = std::max(1, std::min(jb_cap, std::min((8 + nrc - 1) / nrc, 16 / nrc)));
        if (ellip) KC = JB = 1;  // <= 512 stamps: <= 512 deposits per box pixel
        P.JB = std::max(P.JB, JB);
        for (int b0 = 0; b0 < n_jb[i]; b0 += JB)
          for (int c0 = 0; c0 < n_k16[i]; c0 += KC) {
            int4 u = make_int4(1 << 30, -(1 << 30), 1 << 30, -(1 << 30));
            for (int b = b0; b < std::min(n_jb[i], b0 + JB); ++b)
              for (int c = c0; c < std::min(n_k16[i], c0 + KC); ++c) {
                const int4 v = bbox[bb_off[i] + (int64_t)b * n_k16[i] + c];
                u.x = std::min(u.x, v.x);
                u.y = std::max(u.y, v.y);
                u.z = std::min(u.z, v.z);
                u.w = std::max(u.w, v.w);
              }
            const int Wd = m->W[s.detector], Hd = m->H[s.detector];
            const int x0 = std::max(u.x, 0), x1 = std::min(u.y, Wd - 1);
            const int y0 = std::max(u.z, 0), y1 = std::min(u.w, Hd - 1);
            if (x1 < x0 || y1 < y0) continue;  // every window of the item is off the detector
            Item it{};
            it.slice = i;
            it.j0 = b0 * 32;
            it.nj = std::min(s.n_lambda, (b0 + JB) * 32) - it.j0;
            it.k0 = c0 * 16;
            it.nk = std::min(s.n_slit, (c0 + KC) * 16) - it.k0;
            it.bx0 = x0;
            it.by0 = y0;
            it.bw = x1 - x0 + 1;
            it.bh = y1 - y0 + 1;
            it.store_off = store;
            store += (int64_t)it.bw * it.bh;
            P.items.push_back(it);
            g.count++;
          }
      }
      P.groups.push_back(g);
    }
    P.store_elems = store;
    P.max_area = 0;
    P.nk_max = 1;
    for (auto& it : P.items) {
      P.max_area = std::max(P.max_area, it.bw * it.bh);
      P.nk_max = std::max(P.nk_max, it.nk);
    }
    P.smem = m->psf == E2E_PSF_TABLE ? table_smem_bytes(P.max_area, P.nk_max, P.max_deg + 1)
             : ellip ? ellip_smem_bytes(P.max_area, P.nk_max, P.max_deg + 1, m->Ks.empty() ? 15 : m->Ks.front())
                     : mixed_smem_bytes(P.max_area, P.JB, P.nk_max, P.B, P.max_deg + 1);
    if ((int)P.smem + kStaticSmemReserve <= optin) break;
    if (jb_cap == 1)
      return fail(E2E_EINVAL, "trace footprint of a work item exceeds on-chip memory (area " +
                                  std::to_string(P.max_area) + " px)");
  }
  P.NB = 1;
  return plan_bands_and_tiles(m);
}

// ------------------------------------------------------------------ render

// Bracket one kernel launch with events when the context records kernel timings.
struct KernelTimer {
  e2e_ctx* ctx;
  cudaStream_t st;
  size_t idx = (size_t)-1;
  KernelTimer(e2e_ctx* c, cudaStream_t s, const char* name) : ctx(c), st(s) {
    if (!ctx->opts.kernel_timing) return;
    e2e_ctx::Timed t{name, nullptr, nullptr};
    for (cudaEvent_t* e : {&t.a, &t.b}) {
      if (!ctx->event_pool.empty()) {
        *e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
      } else if (cudaEventCreate(e) != cudaSuccess) {
        return;
      }
    }
    cudaEventRecord(t.a, st);
    idx = ctx->timed.size();
    ctx->timed.push_back(t);
  }
  ~KernelTimer() {
    if (idx != (size_t)-1) cudaEventRecord(ctx->timed[idx].b, st);
  }
};

void reset_timing(e2e_ctx* ctx) {
  for (auto& t : ctx->timed) {
    ctx->event_pool.push_back(t.a);
    ctx->event_pool.push_back(t.b);
  }
  ctx->timed.clear();
}

struct Scratch {
  std::vector<void*> blocks;
  cudaStream_t st;
  ~Scratch() {
    for (void* p : blocks) cudaFreeAsync(p, st);
  }
  cudaError_t get(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) blocks.push_back(*p);
    return e;
  }
};

int resolve_flux(e2e_ctx* ctx, Model* m, int n_spec, const uint64_t* spec_ids, std::vector<const double*>& table) {
  std::map<int, Spectrum*> byfiber;
  if (n_spec < 0 || (n_spec > 0 && !spec_ids)) return fail(E2E_EINVAL, "bad spectrum list");
  for (int i = 0; i < n_spec; ++i) {
    auto it = ctx->spectra.find(spec_ids[i]);
    if (it == ctx->spectra.end()) return fail(E2E_ENOTFOUND, "unknown spectrum id");
    if (byfiber.count(it->second->fiber)) return fail(E2E_EINVAL, "two spectra for one fiber");
    byfiber[it->second->fiber] = it->second.get();
  }
  table.resize(m->slices.size());
  for (size_t i = 0; i < m->slices.size(); ++i) {
    const auto& s = m->slices[i].d;
    auto f = byfiber.find(s.fiber);
    if (f == byfiber.end()) return fail(E2E_EINVAL, "no spectrum for fiber " + std::to_string(s.fiber));
    auto r = f->second->rows.find(s.order);
    if (r == f->second->rows.end())
      return fail(E2E_EINVAL, "spectrum of fiber " + std::to_string(s.fiber) + " lacks order " + std::to_string(s.order));
    if (r->second.second != s.n_lambda)
      return fail(E2E_EINVAL, "spectrum length differs from n_lambda for order " + std::to_string(s.order));
    table[i] = f->second->d_flux + r->second.first;
  }
  return E2E_OK;
}

// Blazed model: redirect the flux table to B(lambda_j) * flux[j], computed into `out`
// (n_bins doubles) with `d_in` (n_slices pointers) as the upload of the original table.
int blaze_into(Model* m, std::vector<const double*>& table, double* out, const double** d_in, cudaStream_t st) {
  E2E_CK(cudaMemcpyAsync(d_in, table.data(), table.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  E2E_CK(launch_blaze(m->d_slices, (int)m->slices.size(), d_in, m->d_bin_off, m->n_bins, out, st));
  for (size_t i = 0; i < table.size(); ++i) table[i] = out + m->bin_off[i];
  return E2E_OK;
}

int blaze_scratch(Model* m, std::vector<const double*>& table, Scratch& sc, cudaStream_t st) {
  if (!m->has_blaze || table.empty()) return E2E_OK;
  double* out = nullptr;
  const double** d_in = nullptr;
  E2E_CK(sc.get((void**)&out, (size_t)m->n_bins * sizeof(double)));
  E2E_CK(sc.get((void**)&d_in, table.size() * sizeof(double*)));
  return blaze_into(m, table, out, d_in, st);
}

// Render items [first, first + count) of the model's plan (all of PSF width K) into the box
// store, on `st`; with mg (separable PSF only), each CTA also merges the tiles its item
// completes.
cudaError_t launch_items(e2e_ctx* ctx, Model* m, int K, int first, int count, const double** d_table, float2* store,
                         cudaStream_t st, const MergeArgs* mg = nullptr) {
  const Plan& P = m->plan;
  if (m->psf == E2E_PSF_TABLE)
    return launch_render_table(K, m->d_slices, m->d_ts, m->d_T32, m->d_field, d_table, m->d_u,
                               P.d_items + first, count, store, P.nk_max, P.max_deg, P.smem, st, ctx->d_err);
  if (m->psf == E2E_PSF_ELLIPTICAL)
    return launch_render_ellip(K, m->d_slices, d_table, m->d_u, P.d_items + first, count, store, P.nk_max,
                               P.max_deg, P.smem, st, ctx->d_err);
  return launch_render_mixed(K, P.DX, P.DY, m->d_slices, d_table, m->d_u, P.d_items + first, count, store, P.B,
                             P.JB, P.nk_max, P.max_deg, P.far_tails, P.smem, st, ctx->d_err, mg);
}

int render_impl(e2e_ctx* ctx, Model* m, int n_spec, const uint64_t* spec_ids, int precision, int dtype,
                void* const* dst, const int64_t* pitch_in, cudaStream_t st, const int2* frozen = nullptr) {
  NvtxRange nvtx_("e2e render");
  if (dtype != E2E_F32 && dtype != E2E_F64) return fail(E2E_EINVAL, "dtype must be E2E_F32 or E2E_F64");
  if (precision != E2E_PREC_MIXED && precision != E2E_PREC_FP64) return fail(E2E_EINVAL, "bad precision");
  if (!dst) return fail(E2E_EINVAL, "null destination list");
  std::vector<int64_t> pitch(m->n_det);
  for (int d = 0; d < m->n_det; ++d) {
    if (!dst[d]) return fail(E2E_EINVAL, "null destination frame");
    pitch[d] = pitch_in ? pitch_in[d] : m->W[d];
    if (pitch[d] < m->W[d]) return fail(E2E_EINVAL, "pitch smaller than width");
  }
  std::vector<const double*> table;
  int rc = resolve_flux(ctx, m, n_spec, spec_ids, table);
  if (rc != E2E_OK) return rc;
  const bool ellip = m->psf == E2E_PSF_ELLIPTICAL;
  const bool tab = m->psf == E2E_PSF_TABLE;

  if (ctx->opts.kernel_timing) reset_timing(ctx);
  Scratch sc{{}, st};
  rc = blaze_scratch(m, table, sc, st);
  if (rc != E2E_OK) return rc;
  const double** d_table = nullptr;
  int64_t* d_pitch = nullptr;
  void** d_dst = nullptr;
  E2E_CK(sc.get((void**)&d_table, table.size() * sizeof(double*)));
  E2E_CK(sc.get((void**)&d_pitch, pitch.size() * sizeof(int64_t)));
  E2E_CK(sc.get((void**)&d_dst, m->n_det * sizeof(void*)));
  E2E_CK(cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_pitch, pitch.data(), pitch.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_dst, dst, m->n_det * sizeof(void*), cudaMemcpyHostToDevice, st));

  if (precision == E2E_PREC_FP64) {
    // accumulate in FP64: straight into an FP64 destination, else into scratch + convert
    std::vector<double*> acc(m->n_det);
    std::vector<int64_t> apitch(m->n_det);
    for (int d = 0; d < m->n_det; ++d) {
      if (dtype == E2E_F64) {
        acc[d] = (double*)dst[d];
        apitch[d] = pitch[d];
        E2E_CK(cudaMemset2DAsync(acc[d], pitch[d] * 8, 0, (size_t)m->W[d] * 8, m->H[d], st));
      } else {
        E2E_CK(sc.get((void**)&acc[d], (size_t)m->H[d] * m->W[d] * 8));
        apitch[d] = m->W[d];
        E2E_CK(cudaMemsetAsync(acc[d], 0, (size_t)m->H[d] * m->W[d] * 8, st));
      }
    }
    double** d_acc = nullptr;
    int64_t* d_apitch = nullptr;
    E2E_CK(sc.get((void**)&d_acc, acc.size() * sizeof(double*)));
    E2E_CK(sc.get((void**)&d_apitch, apitch.size() * sizeof(int64_t)));
    E2E_CK(cudaMemcpyAsync(d_acc, acc.data(), acc.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
    E2E_CK(cudaMemcpyAsync(d_apitch, apitch.data(), apitch.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    for (int K : m->Ks) {
      // one launch per K over all slices; slices of another K exit at once
      KernelTimer kt(ctx, st, tab ? "render_fp64_table" : ellip ? "render_fp64_ellip" : "render_fp64");
      if (tab)
        E2E_CK(launch_render_fp64_table(K, (int)m->slices.size(), m->max_stamps, m->d_slices, m->d_ts, m->d_T64,
                                        m->d_field, d_table, m->d_u, d_acc, d_apitch, st));
      else if (ellip)
        E2E_CK(launch_render_fp64_ellip(K, (int)m->slices.size(), m->max_stamps, m->d_slices, d_table, m->d_u,
                                        d_acc, d_apitch, st));
      else
        E2E_CK(launch_render_fp64(K, (int)m->slices.size(), m->max_stamps, m->d_slices, d_table, m->d_u, d_acc,
                                  d_apitch, st, frozen));
    }
    if (dtype == E2E_F32)
      for (int d = 0; d < m->n_det; ++d) {
        KernelTimer kt(ctx, st, "convert");
        E2E_CK(launch_convert(acc[d], apitch[d], dst[d], dtype, pitch[d], m->H[d], m->W[d], st));
      }
    return E2E_OK;
  }

  // mixed precision
  Plan& P = m->plan;
  if (!P.ok) return fail(E2E_EINVAL, "model has no mixed-precision plan");
  float2* store = nullptr;
  E2E_CK(sc.get((void**)&store, (size_t)P.store_elems * sizeof(float2)));
  if (ctx->d_err) E2E_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  if (!tab && !ellip) {
    // separable PSF: the render CTA that finishes a tile's last item merges the tile; the
    // tiles no item overlaps are written as zeros first
    int* count = nullptr;
    E2E_CK(sc.get((void**)&count, (size_t)P.n_tiles * sizeof(int)));
    if (count) E2E_CK(cudaMemsetAsync(count, 0, (size_t)P.n_tiles * sizeof(int), st));
    const MergeArgs mg{P.d_items, P.d_tiles, P.d_lists, P.d_tile_of, P.d_grid_off, m->d_dims, count, d_dst, d_pitch,
                       dtype == E2E_F32 ? 0 : 1, nullptr, 0};
    bool zeros = false;  // the zero tiles ride as extra CTAs at the end of the first non-empty launch
    for (auto& g : P.groups) {
      MergeArgs mgg = mg;
      if (!zeros && g.count > 0) {
        mgg.zero_tiles = P.d_zero_tiles;
        mgg.n_zero = P.n_zero_tiles;
        zeros = true;
      }
      KernelTimer kt(ctx, st, "render_mixed");
      E2E_CK(launch_items(ctx, m, g.K, g.first, g.count, d_table, store, st, &mgg));
    }
    if (!zeros) {  // no item at all: every tile is a zero tile
      KernelTimer kt(ctx, st, "merge_zero");
      E2E_CK(launch_merge(P.d_zero_tiles, P.n_zero_tiles, P.d_lists, P.d_items, store, d_dst, dtype, d_pitch,
                          m->d_dims, st));
    }
  } else {
    for (auto& g : P.groups) {
      KernelTimer kt(ctx, st, tab ? "render_table" : "render_ellip");
      E2E_CK(launch_items(ctx, m, g.K, g.first, g.count, d_table, store, st));
    }
    KernelTimer kt(ctx, st, "merge");
    E2E_CK(launch_merge(P.d_tiles, P.n_tiles, P.d_lists, P.d_items, store, d_dst, dtype, d_pitch, m->d_dims, st));
  }
  if (ctx->d_err) {  // debug checks: wait for the render and report unplanned deposits
    int n_bad = 0;
    E2E_CK(cudaMemcpyAsync(&n_bad, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    E2E_CK(cudaStreamSynchronize(st));
    if (n_bad) return fail(E2E_EDEVICE, std::to_string(n_bad) + " deposits fell outside the planned boxes");
  }
  return E2E_OK;
}

// Streams and events of the banded host render, created once per context.
int ensure_band_streams(e2e_ctx* ctx) {
  if (ctx->copy_st) return E2E_OK;
  int lo = 0, hi = 0;
  E2E_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  for (cudaStream_t& s : ctx->band_st) E2E_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  E2E_CK(cudaStreamCreateWithPriority(&ctx->merge_st, cudaStreamNonBlocking, hi));
  E2E_CK(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking));
  ctx->band_ev.assign(1 + 2 * kBands + 4, nullptr);  // fork, per band rendered / merged, 4 stream ends
  for (cudaEvent_t& e : ctx->band_ev) E2E_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return E2E_OK;
}

// Rows [r0, r1) of detector d that belong to band b of the plan.
void band_rows(const Model* m, int d, int b, int& r0, int& r1) {
  const int rows = m->plan.band_tile_rows[d] * kTileH;
  r0 = std::min(m->H[d], b * rows);
  r1 = std::min(m->H[d], (b + 1) * rows);
}

// Mixed-precision render into host memory, band by band: the items of band b render on one of
// two streams (consecutive bands alternate, so one band's last CTAs overlap the next band's
// first), the merge of band b's tiles follows on a high-priority stream once the bands <= b
// are rendered, and the copy of band b's rows to the host follows on a copy stream, while
// later bands still render.  (Fusing the merge into the band renders, as e2e_render does,
// made the whole step slower here: each band's launch then ends only after its merges.)
// The frame is the one e2e_render writes: same items, same order, same merge.
int render_host_banded(e2e_ctx* ctx, Model* m, int n_spec, const uint64_t* spec_ids, int dtype, void* const* host,
                       const std::vector<int64_t>& pitch, cudaStream_t st) {
  NvtxRange nvtx_("e2e render host");
  Plan& P = m->plan;
  if (!P.ok) return fail(E2E_EINVAL, "model has no mixed-precision plan");
  std::vector<const double*> table;
  int rc = resolve_flux(ctx, m, n_spec, spec_ids, table);
  if (rc != E2E_OK) return rc;
  rc = ensure_band_streams(ctx);
  if (rc != E2E_OK) return rc;
  const size_t es = dtype == E2E_F32 ? 4 : 8;
  Scratch sc{{}, st};
  rc = blaze_scratch(m, table, sc, st);
  if (rc != E2E_OK) return rc;
  std::vector<void*> frame(m->n_det);
  std::vector<int64_t> fpitch(m->W.begin(), m->W.end());
  for (int d = 0; d < m->n_det; ++d) E2E_CK(sc.get(&frame[d], (size_t)m->H[d] * m->W[d] * es));
  const double** d_table = nullptr;
  int64_t* d_pitch = nullptr;
  void** d_dst = nullptr;
  float2* store = nullptr;
  E2E_CK(sc.get((void**)&d_table, table.size() * sizeof(double*)));
  E2E_CK(sc.get((void**)&d_pitch, fpitch.size() * sizeof(int64_t)));
  E2E_CK(sc.get((void**)&d_dst, m->n_det * sizeof(void*)));
  E2E_CK(sc.get((void**)&store, (size_t)P.store_elems * sizeof(float2)));
  E2E_CK(cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_pitch, fpitch.data(), fpitch.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_dst, frame.data(), m->n_det * sizeof(void*), cudaMemcpyHostToDevice, st));
  if (ctx->d_err) E2E_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  // events: [0] fork, [1 + b] band b rendered, [1 + kBands + b] band b merged, then the
  // ends of the two render streams, the merge stream and the copy stream
  cudaEvent_t* ev = ctx->band_ev.data();
  cudaStream_t R[2] = {ctx->band_st[0], ctx->band_st[1]}, M = ctx->merge_st, C = ctx->copy_st;
  E2E_CK(cudaEventRecord(ev[0], st));
  for (cudaStream_t s : {R[0], R[1], M, C}) E2E_CK(cudaStreamWaitEvent(s, ev[0], 0));
  // From here on `st` must wait for the side streams before the scratch is released, on
  // every return path (an error path joins in the destructor, its own errors then moot).
  struct Join {
    cudaStream_t st, side[4];
    cudaEvent_t* end;
    bool done = false;
    cudaError_t run() {
      done = true;
      for (int i = 0; i < 4; ++i) {
        cudaError_t e = cudaEventRecord(end[i], side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, end[i], 0);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    ~Join() {
      if (!done) run();
    }
  } join{st, {R[0], R[1], M, C}, ev + 1 + 2 * kBands};
  const int nb = P.n_bands;
  for (int b = 0; b < nb; ++b) {
    cudaStream_t r = R[b & 1];
    for (size_t g = 0; g < P.groups.size(); ++g) {
      const int cnt = P.seg_count[g * nb + b];
      if (cnt) E2E_CK(launch_items(ctx, m, P.groups[g].K, P.seg_first[g * nb + b], cnt, d_table, store, r));
    }
    E2E_CK(cudaEventRecord(ev[1 + b], r));
    E2E_CK(cudaStreamWaitEvent(M, ev[1 + b], 0));  // bands < b: waited for by earlier merges
    E2E_CK(launch_merge(P.d_tiles + P.tile_first[b], P.tile_first[b + 1] - P.tile_first[b], P.d_lists, P.d_items,
                        store, d_dst, dtype, d_pitch, m->d_dims, M));
    E2E_CK(cudaEventRecord(ev[1 + kBands + b], M));
    E2E_CK(cudaStreamWaitEvent(C, ev[1 + kBands + b], 0));
    for (int d = 0; d < m->n_det; ++d) {
      int r0, r1;
      band_rows(m, d, b, r0, r1);
      if (r1 > r0)
        E2E_CK(cudaMemcpy2DAsync(static_cast<char*>(host[d]) + (size_t)r0 * pitch[d] * es, (size_t)pitch[d] * es,
                                 static_cast<const char*>(frame[d]) + (size_t)r0 * m->W[d] * es, (size_t)m->W[d] * es,
                                 (size_t)m->W[d] * es, (size_t)(r1 - r0), cudaMemcpyDeviceToHost, C));
    }
  }
  E2E_CK(join.run());
  return E2E_OK;
}

}  // namespace

// ====================================================================== C ABI

namespace {
// Library-owned frames for model m, allocated in stream order on st.
int alloc_frame(const Model* m, int dtype, cudaStream_t st, std::unique_ptr<Frame>& out) {
  auto f = std::make_unique<Frame>();
  f->dtype = dtype;
  f->H = m->H;
  f->W = m->W;
  const size_t es = dtype == E2E_F32 ? 4 : 8;
  cudaError_t e = cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming);
  for (int d = 0; d < m->n_det && e == cudaSuccess; ++d) {
    void* p = nullptr;
    e = cudaMallocAsync(&p, (size_t)m->H[d] * m->W[d] * es, st);
    if (e == cudaSuccess) f->ptrs.push_back(p);
  }
  if (e != cudaSuccess) {
    for (void* q : f->ptrs) cudaFreeAsync(q, st);
    if (f->ready) cudaEventDestroy(f->ready);
    return cuda_fail(e, "frame allocation");
  }
  out = std::move(f);
  return E2E_OK;
}

// Return a frame's buffers to the pool once its last recorded use has completed.
void free_frame(e2e_ctx* ctx, Frame* f) {
  if (f->ready) cudaStreamWaitEvent(ctx->free_stream, f->ready, 0);
  for (void* p : f->ptrs) cudaFreeAsync(p, ctx->free_stream);
  f->ptrs.clear();
  if (f->ready) cudaEventDestroy(f->ready);
  f->ready = nullptr;
}

}  // namespace

extern "C" {

const char* e2e_last_error(void) { return g_err.c_str(); }

int e2e_create(e2e_ctx** out, int32_t device, const e2e_opts* opts) {
  if (!out) return fail(E2E_EINVAL, "null output pointer");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(E2E_EINVAL, "no such CUDA device");
  DeviceGuard g(device);
  auto* c = new (std::nothrow) e2e_ctx;
  if (!c) return fail(E2E_ENOMEM, "host allocation failed");
  c->device = device;
  if (opts) c->opts = *opts;
  if (c->opts.max_inflight <= 0) c->opts.max_inflight = 4;
  // keep freed scratch in the stream-ordered pool instead of returning it to the driver
  if (cudaDeviceGetDefaultMemPool(&c->pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  e = cudaStreamCreateWithFlags(&c->free_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->load_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_flag, sizeof(int));
  if (e == cudaSuccess && c->opts.debug_checks) e = cudaMalloc((void**)&c->d_err, sizeof(int));
  if (e == cudaSuccess && c->d_err) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    if (c->free_stream) cudaStreamDestroy(c->free_stream);
    if (c->load_stream) cudaStreamDestroy(c->load_stream);
    cudaFree(c->d_flag);
    cudaFreeHost(c->h_flag);
    cudaFree(c->d_err);
    delete c;
    return cuda_fail(e, "context setup");
  }
  *out = c;
  return E2E_OK;
}

void e2e_destroy(e2e_ctx* ctx) {
  if (!ctx) return;
  if (ctx->server) e2e_server_stop(ctx);
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto& kv : ctx->models) free_model(kv.second.get());
    for (auto& kv : ctx->spectra) cudaFreeAsync(kv.second->d_flux, ctx->load_stream);
    cudaStreamSynchronize(ctx->load_stream);
    cudaStreamDestroy(ctx->load_stream);
    cudaFree(ctx->d_flag);
    cudaFreeHost(ctx->h_flag);
    for (auto& kv : ctx->frames) free_frame(ctx, kv.second.get());
    for (auto& kv : ctx->patterns) {
      for (double* p : kv.second.R) cudaFree(p);
      for (float* p : kv.second.R32) cudaFree(p);
    }
    cudaStreamSynchronize(ctx->free_stream);
    cudaStreamDestroy(ctx->free_stream);
    cudaFree(ctx->d_err);
    reset_timing(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->band_ev) cudaEventDestroy(e);
    for (cudaStream_t s : {ctx->band_st[0], ctx->band_st[1], ctx->merge_st, ctx->copy_st})
      if (s) cudaStreamDestroy(s);
  }
  delete ctx;
}

// The one-dimensional slices that render a model's 2-D fibers: parent slice p with n_aper > 1
// becomes one slice per aperture row l, its coefficients of lt^q s^0 moved by t_l aper_q
// (degree raised to 2 where the aperture has a quadratic term, to 1 for a linear one) and its
// slit weights the row's.  cx, cy: parent coefficient arrays (caller layout) or nullptr for
// the descriptors' own.  Descriptors point into `store`.
void expand_fibers(const e2e_model_desc* desc, const double* cx_in, const double* cy_in,
                   std::vector<e2e_order_slice>& out, std::vector<std::vector<double>>& store, Model* m) {
  out.clear();
  store.clear();
  m->parent_of.clear();
  m->first_sub.assign(1, 0);
  m->parent_nc.clear();
  m->parent_coef_off.clear();
  m->t_of.clear();
  m->apx.clear();
  m->apy.clear();
  m->expanded = false;
  int off = 0;
  for (int i = 0; i < desc->n_slices; ++i) {
    const e2e_order_slice& s = desc->slices[i];
    const int nc = n_coeffs(s.degree);
    m->parent_nc.push_back(nc);
    m->parent_coef_off.push_back(off);
    const double* pcx = cx_in ? cx_in + off : s.cx;
    const double* pcy = cy_in ? cy_in + off : s.cy;
    off += nc;
    for (int q = 0; q < 3; ++q) {
      m->apx.push_back(s.aper_x[q]);
      m->apy.push_back(s.aper_y[q]);
    }
    const int rows = s.n_aper > 1 ? s.n_aper : 1;
    if (rows > 1) m->expanded = true;
    int deg = s.degree;
    if (rows > 1) {
      if (s.aper_x[2] != 0.0 || s.aper_y[2] != 0.0) deg = std::max(deg, 2);
      else if (s.aper_x[1] != 0.0 || s.aper_y[1] != 0.0) deg = std::max(deg, 1);
    }
    for (int l = 0; l < rows; ++l) {
      const double t = rows > 1 ? -1.0 + (2.0 * l + 1.0) / rows : 0.0;
      const int ncs = n_coeffs(deg);
      std::vector<double> ccx(ncs, 0.0), ccy(ncs, 0.0), uu(s.slit_weights + (size_t)l * s.n_slit,
                                                        s.slit_weights + (size_t)(l + 1) * s.n_slit);
      for (int c = 0; c < nc; ++c) {  // a coefficient's index depends on its (a, b) only
        ccx[c] = pcx[c];
        ccy[c] = pcy[c];
      }
      if (rows > 1)
        for (int q = 0; q <= std::min(deg, 2); ++q) {
          ccx[coeff_index(q, 0)] += t * s.aper_x[q];
          ccy[coeff_index(q, 0)] += t * s.aper_y[q];
        }
      e2e_order_slice e = s;
      e.degree = deg;
      e.n_aper = 0;
      store.push_back(std::move(ccx));
      e.cx = store.back().data();
      store.push_back(std::move(ccy));
      e.cy = store.back().data();
      store.push_back(std::move(uu));
      e.slit_weights = store.back().data();
      out.push_back(e);
      m->parent_of.push_back(i);
      m->t_of.push_back(t);
    }
    m->first_sub.push_back((int)out.size());
  }
  m->parent_coef_total = off;
  // store's vectors were moved in before their data() was taken, and a later push_back moves
  // the vector objects but not their heap buffers: the pointers stay valid
}

int e2e_load_model(e2e_ctx* ctx, const e2e_model_desc* desc_in, uint64_t* model_id) {
  NvtxRange nvtx_("e2e load model");
  if (!ctx || !desc_in || !model_id) return fail(E2E_EINVAL, "null argument");
  if (desc_in->n_detectors < 1 || !desc_in->height || !desc_in->width) return fail(E2E_EINVAL, "need >= 1 detector");
  if (desc_in->n_slices < 0 || (desc_in->n_slices > 0 && !desc_in->slices)) return fail(E2E_EINVAL, "bad slice list");
  if (desc_in->psf != E2E_PSF_SEPARABLE && desc_in->psf != E2E_PSF_ELLIPTICAL && desc_in->psf != E2E_PSF_TABLE)
    return fail(E2E_EINVAL, "bad psf kind");
  for (int d = 0; d < desc_in->n_detectors; ++d)
    if (desc_in->height[d] < 1 || desc_in->width[d] < 1 || desc_in->height[d] > 16000 || desc_in->width[d] > 16000)
      return fail(E2E_EINVAL, "detector size must be 1..16000 px");
  for (int i = 0; i < desc_in->n_slices; ++i) {
    int rc = validate_slice(desc_in->slices[i], desc_in->n_detectors, desc_in->psf, i);
    if (rc != E2E_OK) return rc;
  }
  DeviceGuard g(ctx->device);
  auto m = std::make_unique<Model>();
  // 2-D fibers: render the one-dimensional slice of each aperture row
  std::vector<e2e_order_slice> ex;
  std::vector<std::vector<double>> ex_store;
  expand_fibers(desc_in, nullptr, nullptr, ex, ex_store, m.get());
  e2e_model_desc dexp = *desc_in;
  dexp.n_slices = (int32_t)ex.size();
  dexp.slices = ex.data();
  const e2e_model_desc* desc = &dexp;
  m->n_det = desc->n_detectors;
  m->psf = desc->psf;
  m->H.assign(desc->height, desc->height + m->n_det);
  m->W.assign(desc->width, desc->width + m->n_det);
  std::vector<DevSlice> ds(desc->n_slices);
  std::vector<double> u_all;
  int32_t coef_total = 0;
  for (int i = 0; i < desc->n_slices; ++i) {
    const auto& s = desc->slices[i];
    SliceHost h;
    h.d = s;
    const int nc = n_coeffs(s.degree);
    h.cx.assign(s.cx, s.cx + nc);
    h.cy.assign(s.cy, s.cy + nc);
    h.u.assign(s.slit_weights, s.slit_weights + s.n_slit);
    h.d.cx = h.cx.data();
    h.d.cy = h.cy.data();
    h.d.slit_weights = h.u.data();
    if (desc->psf == E2E_PSF_TABLE) {
      h.field_lt.assign(s.field_lt, s.field_lt + s.n_field);
      h.maps.assign(s.maps, s.maps + (size_t)s.n_field * s.map_size * s.map_size);
      h.d.field_lt = h.field_lt.data();
      h.d.maps = h.maps.data();
    } else {
      h.d.field_lt = nullptr;
      h.d.maps = nullptr;
      h.d.n_field = 0;
    }
    DevSlice& v = ds[i];
    memset(&v, 0, sizeof v);
    for (int c = 0; c < nc; ++c) {
      v.cx[c] = s.cx[c];
      v.cy[c] = s.cy[c];
    }
    for (int c = 0; c < 3; ++c) {
      v.sx[c] = s.sigma_x[c];
      v.sy[c] = s.sigma_y[c];
    }
    v.dlam = (s.lambda_hi - s.lambda_lo) / s.n_lambda;
    v.cos_t = std::cos(s.theta);
    v.sin_t = std::sin(s.theta);
    v.blaze_m = s.blaze_order;
    v.blaze_lc = s.blaze_lambda;
    v.lambda_lo = s.lambda_lo;
    m->has_blaze = m->has_blaze || s.blaze_order != 0.0;
    v.degree = s.degree;
    v.K = s.K;
    v.n_lambda = s.n_lambda;
    v.n_slit = s.n_slit;
    v.det = s.detector;
    v.H = m->H[s.detector];
    v.W = m->W[s.detector];
    v.flux_slot = i;
    v.u_off = (int64_t)u_all.size();
    v.coef_off = coef_total;
    v.index = i;
    v.stamp_off = m->n_stamps;
    m->n_stamps += (int64_t)s.n_lambda * s.n_slit;
    coef_total += nc;
    u_all.insert(u_all.end(), s.slit_weights, s.slit_weights + s.n_slit);
    m->max_stamps = std::max(m->max_stamps, (int64_t)s.n_lambda * s.n_slit);
    if (std::find(m->Ks.begin(), m->Ks.end(), s.K) == m->Ks.end()) m->Ks.push_back(s.K);
    m->slices.push_back(std::move(h));
  }
  std::sort(m->Ks.begin(), m->Ks.end());
  std::vector<int> dims(2 * m->n_det);
  for (int d = 0; d < m->n_det; ++d) {
    dims[2 * d] = m->H[d];
    dims[2 * d + 1] = m->W[d];
  }
  m->dev = ds;
  m->coef_total = coef_total;
  // running sums of the slit weights, each slice summed in order (the photon renderer's slit
  // choice), and the wavelength-bin offsets of the slices
  std::vector<double> ucum(u_all.size()), usum(m->slices.size());
  std::vector<int64_t> bin_off(m->slices.size() + 1, 0);
  for (size_t i = 0; i < m->slices.size(); ++i) {
    const DevSlice& v = ds[i];
    double acc = 0.0;
    for (int k = 0; k < v.n_slit; ++k) {
      const double uk = u_all[v.u_off + k];
      m->u_nonneg = m->u_nonneg && uk >= 0.0;
      acc = k == 0 ? uk : acc + uk;
      ucum[v.u_off + k] = acc;
    }
    usum[i] = acc;
    bin_off[i + 1] = bin_off[i] + v.n_lambda;
  }
  m->n_bins = bin_off.back();
  m->bin_off = bin_off;
  int rc = upload(&m->d_slices, ds.data(), ds.size());
  if (rc == E2E_OK && m->expanded) {  // the adjoint's gradient folding: sub-slices -> parents
    std::vector<int> fold(m->first_sub);
    for (const DevSlice& v : ds) fold.push_back(v.coef_off);
    fold.insert(fold.end(), m->parent_coef_off.begin(), m->parent_coef_off.end());
    fold.insert(fold.end(), m->parent_nc.begin(), m->parent_nc.end());
    rc = upload(&m->d_fold, fold.data(), fold.size());
  }
  if (rc == E2E_OK) rc = upload(&m->d_u, u_all.data(), u_all.size());
  if (rc == E2E_OK) rc = upload(&m->d_ucum, ucum.data(), ucum.size());
  if (rc == E2E_OK) rc = upload(&m->d_usum, usum.data(), usum.size());
  {
    std::vector<float> ucum32(ucum.begin(), ucum.end());
    const size_t nf = photon_coef_floats();
    std::vector<float> cf(nf * m->slices.size(), 0.f);
    for (size_t i = 0; i < m->slices.size(); ++i) {
      const DevSlice& v = ds[i];
      for (int c = 0; c < 2; ++c) {
        const double* co = c ? v.cy : v.cx;
        float* o = cf.data() + i * nf + c * (E2E_MAXC + 2);
        double qb = 0.0, sb = 0.0;
        for (int a = 0; a <= v.degree; ++a)
          for (int b = 0; a + b <= v.degree; ++b) {
            const int t = a + b, idx = t * (t + 1) / 2 + b;
            o[idx] = (float)co[idx];
            if (b == 0) qb += a * std::fabs(co[idx]);
            else sb += std::fabs(co[idx]);
          }
        o[E2E_MAXC] = (float)qb;
        o[E2E_MAXC + 1] = (float)sb;
      }
      float* e = cf.data() + i * nf + 2 * (E2E_MAXC + 2);  // sigma_x, sigma_y, slit-weight total
      for (int k = 0; k < 3; ++k) {
        e[k] = (float)v.sx[k];
        e[3 + k] = (float)v.sy[k];
      }
      e[6] = (float)usum[i];
    }
    if (rc == E2E_OK) rc = upload(&m->d_ucum32, ucum32.data(), ucum32.size());
    if (rc == E2E_OK) rc = upload(&m->d_cf32, cf.data(), cf.size());
  }
  if (rc == E2E_OK) rc = upload(&m->d_bin_off, bin_off.data(), bin_off.size());
  if (rc == E2E_OK && m->psf == E2E_PSF_TABLE) rc = build_psf_tables(m.get());
  if (rc == E2E_OK) rc = upload(&m->d_dims, dims.data(), dims.size());
  if (rc == E2E_OK) rc = plan_model(m.get());
  if (rc != E2E_OK) {
    std::string keep = g_err;
    free_model(m.get());
    g_err = keep;
    return rc;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  *model_id = ctx->next_id++;
  ctx->models[*model_id] = std::move(m);
  return E2E_OK;
}

int e2e_unload_model(e2e_ctx* ctx, uint64_t model_id) {
  if (!ctx) return fail(E2E_EINVAL, "null context");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->models.find(model_id);
  if (it == ctx->models.end()) return fail(E2E_ENOTFOUND, "unknown model id");
  cudaDeviceSynchronize();
  free_model(it->second.get());
  ctx->models.erase(it);
  auto pt = ctx->patterns.find(model_id);
  if (pt != ctx->patterns.end()) {
    for (double* q : pt->second.R) cudaFree(q);
    for (float* q : pt->second.R32) cudaFree(q);
    ctx->patterns.erase(pt);
  }
  return E2E_OK;
}

int e2e_load_spectrum(e2e_ctx* ctx, int32_t fiber, int32_t n_orders, const int32_t* order_ids,
                      const int32_t* n_lambda, const double* flux, uint64_t* spec_id) {
  NvtxRange nvtx_("e2e load spectrum");
  if (!ctx || !spec_id || n_orders < 0 || (n_orders > 0 && (!order_ids || !n_lambda || !flux)))
    return fail(E2E_EINVAL, "null or negative argument");
  auto sp = std::make_unique<Spectrum>();
  sp->fiber = fiber;
  int64_t total = 0;
  for (int i = 0; i < n_orders; ++i) {
    if (n_lambda[i] < 1) return fail(E2E_EINVAL, "n_lambda must be >= 1");
    if (sp->rows.count(order_ids[i])) return fail(E2E_EINVAL, "duplicate order in spectrum");
    sp->rows[order_ids[i]] = {total, n_lambda[i]};
    total += n_lambda[i];
  }
  DeviceGuard g(ctx->device);
  if (total > 0) {
    // from the pool on the load stream; the finiteness check runs on the uploaded copy
    std::lock_guard<std::mutex> lk(ctx->load_mu);
    const size_t bytes = (size_t)total * sizeof(double);
    cudaStream_t ls = ctx->load_stream;
    E2E_CK(ctx->pool ? cudaMallocFromPoolAsync((void**)&sp->d_flux, bytes, ctx->pool, ls)
                     : cudaMallocAsync((void**)&sp->d_flux, bytes, ls));
    cudaError_t e = cudaMemcpyAsync(sp->d_flux, flux, bytes, cudaMemcpyHostToDevice, ls);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ls);
    if (e == cudaSuccess) e = launch_flag_nonfinite(sp->d_flux, total, ctx->d_flag, ls);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ls);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ls);
    if (e != cudaSuccess || *ctx->h_flag) {
      cudaFreeAsync(sp->d_flux, ls);
      cudaStreamSynchronize(ls);
      return e != cudaSuccess ? cuda_fail(e, "spectrum upload") : fail(E2E_EINVAL, "non-finite flux");
    }
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  *spec_id = ctx->next_id++;
  ctx->spectra[*spec_id] = std::move(sp);
  return E2E_OK;
}

int e2e_unload_spectrum(e2e_ctx* ctx, uint64_t spec_id) {
  if (!ctx) return fail(E2E_EINVAL, "null context");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->spectra.find(spec_id);
  if (it == ctx->spectra.end()) return fail(E2E_ENOTFOUND, "unknown spectrum id");
  cudaDeviceSynchronize();  // no render enqueued before this call still reads the spectrum
  cudaFreeAsync(it->second->d_flux, ctx->load_stream);  // back to the pool
  ctx->spectra.erase(it);
  return E2E_OK;
}

int e2e_render(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t precision,
               int32_t dtype, void* const* dst, const int64_t* pitch_elems, void* stream) {
  if (!ctx) return fail(E2E_EINVAL, "null context");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  return render_impl(ctx, m, n_spec, spec_ids, precision, dtype, dst, pitch_elems, (cudaStream_t)stream);
}

int e2e_window_origins(e2e_ctx* ctx, uint64_t model_id, int32_t* origins, void* stream) {
  if (!ctx || !origins) return fail(E2E_EINVAL, "null argument");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  E2E_CK(launch_window_origins((int)m->slices.size(), m->max_stamps, m->d_slices, reinterpret_cast<int2*>(origins),
                               (cudaStream_t)stream));
  return E2E_OK;
}

int e2e_render_frozen(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids,
                      const int32_t* frozen_windows, int32_t dtype, void* const* dst, const int64_t* pitch_elems,
                      void* stream) {
  if (!ctx || !frozen_windows) return fail(E2E_EINVAL, "null argument");
  if (reinterpret_cast<uintptr_t>(frozen_windows) % 8 != 0) return fail(E2E_EINVAL, "frozen_windows must be 8-byte aligned");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  if (m->psf != E2E_PSF_SEPARABLE) return fail(E2E_EINVAL, "frozen windows support the separable PSF");
  return render_impl(ctx, m, n_spec, spec_ids, E2E_PREC_FP64, dtype, dst, pitch_elems, (cudaStream_t)stream,
                     reinterpret_cast<const int2*>(frozen_windows));
}

int e2e_render_alloc(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t precision,
                     int32_t dtype, void* stream, uint64_t* frame_id) {
  if (!ctx || !frame_id) return fail(E2E_EINVAL, "null argument");
  if (dtype != E2E_F32 && dtype != E2E_F64) return fail(E2E_EINVAL, "dtype must be E2E_F32 or E2E_F64");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  std::unique_ptr<Frame> f;
  int rc = alloc_frame(m, dtype, (cudaStream_t)stream, f);
  if (rc != E2E_OK) return rc;
  rc = render_impl(ctx, m, n_spec, spec_ids, precision, dtype, f->ptrs.data(), nullptr, (cudaStream_t)stream);
  cudaEventRecord(f->ready, (cudaStream_t)stream);
  if (rc != E2E_OK) {
    free_frame(ctx, f.get());
    return rc;
  }
  *frame_id = ctx->next_id++;
  ctx->frames[*frame_id] = std::move(f);
  return E2E_OK;
}

int e2e_fetch_frame(e2e_ctx* ctx, uint64_t frame_id, int32_t detector, void* dst, int32_t dst_is_device, size_t bytes,
                    void* stream) {
  if (!ctx || !dst) return fail(E2E_EINVAL, "null argument");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->frames.find(frame_id);
  if (it == ctx->frames.end()) return fail(E2E_ENOTFOUND, "unknown frame id");
  Frame* f = it->second.get();
  if (detector < 0 || detector >= (int)f->ptrs.size()) return fail(E2E_EINVAL, "detector out of range");
  const size_t need = (size_t)f->H[detector] * f->W[detector] * (f->dtype == E2E_F32 ? 4 : 8);
  if (bytes != need) return fail(E2E_EINVAL, "byte count differs from the frame size");
  E2E_CK(cudaStreamWaitEvent((cudaStream_t)stream, f->ready, 0));
  E2E_CK(cudaMemcpyAsync(dst, f->ptrs[detector], bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         (cudaStream_t)stream));
  E2E_CK(cudaEventRecord(f->ready, (cudaStream_t)stream));
  return E2E_OK;
}

int e2e_render_host(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t precision,
                    int32_t dtype, void* const* host_dst, const int64_t* pitch_elems, void* stream) {
  if (!ctx || !host_dst) return fail(E2E_EINVAL, "null argument");
  if (dtype != E2E_F32 && dtype != E2E_F64) return fail(E2E_EINVAL, "dtype must be E2E_F32 or E2E_F64");
  if (precision != E2E_PREC_MIXED && precision != E2E_PREC_FP64) return fail(E2E_EINVAL, "bad precision");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  std::vector<int64_t> pitch(m->n_det);
  for (int d = 0; d < m->n_det; ++d) {
    if (!host_dst[d]) return fail(E2E_EINVAL, "null destination frame");
    pitch[d] = pitch_elems ? pitch_elems[d] : m->W[d];
    if (pitch[d] < m->W[d]) return fail(E2E_EINVAL, "pitch smaller than width");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host_dst[d]) == cudaSuccess) {
      if (at.type == cudaMemoryTypeDevice) return fail(E2E_EINVAL, "destination is device memory (use e2e_render)");
    } else {
      cudaGetLastError();  // an unknown host pointer is host memory
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = dtype == E2E_F32 ? 4 : 8;
  if (precision == E2E_PREC_FP64) {  // render whole, then copy
    Scratch sc{{}, st};
    std::vector<void*> frame(m->n_det);
    for (int d = 0; d < m->n_det; ++d) E2E_CK(sc.get(&frame[d], (size_t)m->H[d] * m->W[d] * es));
    int rc = render_impl(ctx, m, n_spec, spec_ids, precision, dtype, frame.data(), nullptr, st);
    if (rc != E2E_OK) return rc;
    for (int d = 0; d < m->n_det; ++d)
      E2E_CK(cudaMemcpy2DAsync(host_dst[d], (size_t)pitch[d] * es, frame[d], (size_t)m->W[d] * es,
                               (size_t)m->W[d] * es, (size_t)m->H[d], cudaMemcpyDeviceToHost, st));
    return E2E_OK;
  }
  int rc = render_host_banded(ctx, m, n_spec, spec_ids, dtype, host_dst, pitch, st);
  if (rc != E2E_OK) return rc;
  if (ctx->d_err) {  // debug checks: wait for the render and report unplanned deposits
    int n_bad = 0;
    E2E_CK(cudaMemcpyAsync(&n_bad, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    E2E_CK(cudaStreamSynchronize(st));
    if (n_bad) return fail(E2E_EDEVICE, std::to_string(n_bad) + " deposits fell outside the planned boxes");
  }
  return E2E_OK;
}

int e2e_release_frame(e2e_ctx* ctx, uint64_t frame_id) {
  if (!ctx) return fail(E2E_EINVAL, "null context");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->frames.find(frame_id);
  if (it == ctx->frames.end()) return fail(E2E_ENOTFOUND, "unknown frame id");
  free_frame(ctx, it->second.get());
  ctx->frames.erase(it);
  return E2E_OK;
}

int e2e_model_plan(e2e_ctx* ctx, uint64_t model_id, e2e_plan_info* info) {
  if (!ctx || !info) return fail(E2E_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  const Plan& P = m->plan;
  memset(info, 0, sizeof *info);
  info->chunk_lambda = 32 * P.JB;
  info->run_slit = P.B;
  info->slack_x = P.DX;
  info->slack_y = P.DY;
  info->n_items = (int64_t)P.items.size();
  info->n_tiles = P.n_tiles;
  info->scratch_bytes = P.store_elems * 8;
  info->tile_w = kTileW;
  info->tile_h = kTileH;
  info->boxes_per_cta = P.NB;
  info->max_box_area = P.max_area;
  return E2E_OK;
}

// ---------------------------------------------------------------- render without allocating
//
// For callers that cannot allocate device memory mid-run (another runtime owns the GPU's
// memory, or a real-time loop must not block or fail on an allocation), the mixed-precision
// render can take its scratch from this fixed buffer instead of the stream-ordered pool.  It
// lives in device memory on every GPU that loads the library, for the life of the process.
// Host code sees `g_static_scratch` only as a host-side handle: its device address comes
// from cudaGetSymbolAddress, looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_static_scratch[E2E_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
std::map<int, void*> g_static_addr;  // device -> device address of g_static_scratch

int static_scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  auto it = g_static_addr.find(device);
  if (it != g_static_addr.end()) {
    *out = it->second;
    return E2E_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);  // the caller made `device` current
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  g_static_addr[device] = p;
  *out = p;
  return E2E_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }
}  // namespace

int e2e_render_static(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t dtype,
                      void* const* dst, const int64_t* pitch_in, void* stream) {
  if (!ctx) return fail(E2E_EINVAL, "null context");
  if (dtype != E2E_F32 && dtype != E2E_F64) return fail(E2E_EINVAL, "dtype must be E2E_F32 or E2E_F64");
  if (!dst) return fail(E2E_EINVAL, "null destination list");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  if (m->psf != E2E_PSF_SEPARABLE) return fail(E2E_EINVAL, "the fixed-scratch render supports the separable PSF");
  const Plan& P = m->plan;
  if (!P.ok) return fail(E2E_EINVAL, "model has no mixed-precision plan");
  std::vector<int64_t> pitch(m->n_det);
  for (int d = 0; d < m->n_det; ++d) {
    if (!dst[d]) return fail(E2E_EINVAL, "null destination frame");
    pitch[d] = pitch_in ? pitch_in[d] : m->W[d];
    if (pitch[d] < m->W[d]) return fail(E2E_EINVAL, "pitch smaller than width");
  }
  std::vector<const double*> table;
  int rc = resolve_flux(ctx, m, n_spec, spec_ids, table);
  if (rc != E2E_OK) return rc;
  // layout in the fixed buffer: flux table | pitches | destination pointers | box store
  // [| blazed spectra | original flux table]
  const size_t off_table = 0;
  const size_t off_pitch = align256(off_table + table.size() * sizeof(double*));
  const size_t off_dst = align256(off_pitch + pitch.size() * sizeof(int64_t));
  const size_t off_store = align256(off_dst + (size_t)m->n_det * sizeof(void*));
  const size_t off_blaze = align256(off_store + (size_t)P.store_elems * sizeof(float2));
  const size_t off_tin = align256(off_blaze + (m->has_blaze ? (size_t)m->n_bins * sizeof(double) : 0));
  const size_t need = m->has_blaze ? off_tin + table.size() * sizeof(double*) : off_blaze;
  if (need > E2E_STATIC_SCRATCH_BYTES)
    return fail(E2E_ETOOBIG, "model needs " + std::to_string(need) + " bytes of scratch; the fixed buffer holds " +
                                 std::to_string((size_t)E2E_STATIC_SCRATCH_BYTES));
  void* base = nullptr;
  rc = static_scratch_address(ctx->device, &base);
  if (rc != E2E_OK) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  const double** d_table = reinterpret_cast<const double**>(b + off_table);
  int64_t* d_pitch = reinterpret_cast<int64_t*>(b + off_pitch);
  void** d_dst = reinterpret_cast<void**>(b + off_dst);
  float2* store = reinterpret_cast<float2*>(b + off_store);
  cudaStream_t st = (cudaStream_t)stream;
  if (m->has_blaze && !table.empty()) {
    rc = blaze_into(m, table, reinterpret_cast<double*>(b + off_blaze), reinterpret_cast<const double**>(b + off_tin),
                    st);
    if (rc != E2E_OK) return rc;
  }
  if (!table.empty())
    E2E_CK(cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_pitch, pitch.data(), pitch.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_dst, dst, m->n_det * sizeof(void*), cudaMemcpyHostToDevice, st));
  // kernel timings and debug checks as in e2e_render: the timing events come from the
  // context's pool and the error counter was allocated with the context
  if (ctx->opts.kernel_timing) reset_timing(ctx);
  if (ctx->d_err) E2E_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  for (auto& grp : P.groups) {
    KernelTimer kt(ctx, st, "render_mixed");
    E2E_CK(launch_render_mixed(grp.K, P.DX, P.DY, m->d_slices, d_table, m->d_u, P.d_items + grp.first, grp.count,
                               store, P.B, P.JB, P.nk_max, P.max_deg, P.far_tails, P.smem, st, ctx->d_err));
  }
  {
    KernelTimer kt(ctx, st, "merge");
    E2E_CK(launch_merge(P.d_tiles, P.n_tiles, P.d_lists, P.d_items, store, d_dst, dtype, d_pitch, m->d_dims, st));
  }
  if (ctx->d_err) {  // debug checks: wait for the render and report unplanned deposits
    int n_bad = 0;
    E2E_CK(cudaMemcpyAsync(&n_bad, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    E2E_CK(cudaStreamSynchronize(st));
    if (n_bad) return fail(E2E_EDEVICE, std::to_string(n_bad) + " deposits fell outside the planned boxes");
  }
  return E2E_OK;
}

int e2e_render_adjoint(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, int32_t dtype,
                       const void* const* dldi, const int64_t* pitch_in, double* g_cx, double* g_cy, double* g_sx,
                       double* g_sy, const int32_t* frozen_windows, void* stream) {
  NvtxRange nvtx_("e2e adjoint");
  if (!ctx || !dldi || !g_cx || !g_cy || !g_sx || !g_sy) return fail(E2E_EINVAL, "null argument");
  if (dtype != E2E_F32 && dtype != E2E_F64) return fail(E2E_EINVAL, "dtype must be E2E_F32 or E2E_F64");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  if (m->psf != E2E_PSF_SEPARABLE) return fail(E2E_EINVAL, "the adjoint supports the separable PSF");
  if (reinterpret_cast<uintptr_t>(frozen_windows) % 8 != 0) return fail(E2E_EINVAL, "frozen_windows must be 8-byte aligned");
  const Plan& P = m->plan;
  std::vector<int64_t> pitch(m->n_det);
  for (int d = 0; d < m->n_det; ++d) {
    if (!dldi[d]) return fail(E2E_EINVAL, "null dL/dI frame");
    pitch[d] = pitch_in ? pitch_in[d] : m->W[d];
    if (pitch[d] < m->W[d]) return fail(E2E_EINVAL, "pitch smaller than width");
  }
  std::vector<const double*> table;
  int rc = resolve_flux(ctx, m, n_spec, spec_ids, table);
  if (rc != E2E_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ns = m->slices.size();
  Scratch sc{{}, st};
  // 2-D fibers: gradients of the aperture rows' slices in scratch, folded into the caller's
  // (parent) layout at the end
  double *ucx = g_cx, *ucy = g_cy, *usx = g_sx, *usy = g_sy;
  if (m->expanded) {
    const int np = (int)m->parent_nc.size();
    E2E_CK(cudaMemsetAsync(ucx, 0, sizeof(double) * m->parent_coef_total, st));
    E2E_CK(cudaMemsetAsync(ucy, 0, sizeof(double) * m->parent_coef_total, st));
    E2E_CK(cudaMemsetAsync(usx, 0, sizeof(double) * 3 * np, st));
    E2E_CK(cudaMemsetAsync(usy, 0, sizeof(double) * 3 * np, st));
    E2E_CK(sc.get((void**)&g_cx, sizeof(double) * std::max(1, m->coef_total)));
    E2E_CK(sc.get((void**)&g_cy, sizeof(double) * std::max(1, m->coef_total)));
    E2E_CK(sc.get((void**)&g_sx, sizeof(double) * 3 * std::max<size_t>(1, ns)));
    E2E_CK(sc.get((void**)&g_sy, sizeof(double) * 3 * std::max<size_t>(1, ns)));
  }
  E2E_CK(cudaMemsetAsync(g_cx, 0, sizeof(double) * m->coef_total, st));
  E2E_CK(cudaMemsetAsync(g_cy, 0, sizeof(double) * m->coef_total, st));
  E2E_CK(cudaMemsetAsync(g_sx, 0, sizeof(double) * 3 * ns, st));
  E2E_CK(cudaMemsetAsync(g_sy, 0, sizeof(double) * 3 * ns, st));
  if (ns == 0 || P.items.empty()) return E2E_OK;
  rc = blaze_scratch(m, table, sc, st);
  if (rc != E2E_OK) return rc;
  const double** d_table = nullptr;
  int64_t* d_pitch = nullptr;
  const void** d_dldi = nullptr;
  E2E_CK(sc.get((void**)&d_table, table.size() * sizeof(double*)));
  E2E_CK(sc.get((void**)&d_pitch, pitch.size() * sizeof(int64_t)));
  E2E_CK(sc.get((void**)&d_dldi, m->n_det * sizeof(void*)));
  E2E_CK(cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_pitch, pitch.data(), pitch.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_dldi, dldi, m->n_det * sizeof(void*), cudaMemcpyHostToDevice, st));
  int nj_max = 1;
  for (const Item& it : P.items) nj_max = std::max(nj_max, it.nj);
  const size_t smem = adjoint_smem_bytes(P.max_area, P.max_deg, P.nk_max, nj_max);
  int max_tasks = 1;  // warp tasks of the largest item: 32-sample blocks x runs
  for (const Item& it : P.items) max_tasks = std::max(max_tasks, ((it.nj + 31) / 32) * ((it.nk + P.B - 1) / P.B));
  const int parts = adjoint_parts(max_tasks);
  for (auto& grp : P.groups) {
    KernelTimer kt(ctx, st, "adjoint");
    E2E_CK(launch_adjoint(grp.K, m->d_slices, d_table, m->d_u, P.d_items + grp.first, grp.count, d_dldi, d_pitch,
                          dtype == E2E_F32 ? 0 : 1, P.B, P.nk_max, parts, g_cx, g_cy, g_sx, g_sy, smem, st,
                          reinterpret_cast<const int2*>(frozen_windows)));
  }
  if (m->expanded)
    E2E_CK(launch_fold_gradients((int)m->parent_nc.size(), (int)ns, m->d_fold, g_cx, g_cy, g_sx, g_sy, ucx, ucy, usx,
                                 usy, st));
  return E2E_OK;
}

int e2e_update_model(e2e_ctx* ctx, uint64_t model_id, const double* cx_in, const double* cy_in, const double* sx_in,
                     const double* sy_in) {
  if (!ctx || !cx_in || !cy_in || !sx_in || !sy_in) return fail(E2E_EINVAL, "null argument");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  // 2-D fibers: the caller's coefficients are the parents'; each aperture row's slice takes
  // them plus its displacement (as at load), and the parents' widths
  std::vector<double> ecx, ecy, esx, esy;
  const double *cx = cx_in, *cy = cy_in, *sx = sx_in, *sy = sy_in;
  if (m->expanded) {
    ecx.assign(m->coef_total, 0.0);
    ecy.assign(m->coef_total, 0.0);
    esx.assign(3 * m->slices.size(), 0.0);
    esy.assign(3 * m->slices.size(), 0.0);
    for (size_t q = 0; q < m->slices.size(); ++q) {
      const int p = m->parent_of[q], off = m->dev[q].coef_off, po = m->parent_coef_off[p];
      const int ncs = n_coeffs(m->slices[q].d.degree);
      for (int c = 0; c < std::min(ncs, m->parent_nc[p]); ++c) {
        ecx[off + c] = cx_in[po + c];
        ecy[off + c] = cy_in[po + c];
      }
      const double t = m->t_of[q];
      if (t != 0.0)
        for (int a = 0; a <= std::min(m->slices[q].d.degree, 2); ++a) {
          ecx[off + coeff_index(a, 0)] += t * m->apx[3 * p + a];
          ecy[off + coeff_index(a, 0)] += t * m->apy[3 * p + a];
        }
      for (int k = 0; k < 3; ++k) {
        esx[3 * q + k] = sx_in[3 * p + k];
        esy[3 * q + k] = sy_in[3 * p + k];
      }
    }
    cx = ecx.data();
    cy = ecy.data();
    sx = esx.data();
    sy = esy.data();
  }
  // validate on copies first so a rejected update leaves the model untouched
  std::vector<SliceHost> ns = m->slices;
  std::vector<DevSlice> dv = m->dev;
  for (size_t i = 0; i < ns.size(); ++i) {
    SliceHost& h = ns[i];
    const int nc = n_coeffs(h.d.degree);
    const int off = dv[i].coef_off;
    h.cx.assign(cx + off, cx + off + nc);
    h.cy.assign(cy + off, cy + off + nc);
    for (int c = 0; c < 3; ++c) {
      h.d.sigma_x[c] = sx[3 * i + c];
      h.d.sigma_y[c] = sy[3 * i + c];
    }
    h.d.cx = h.cx.data();
    h.d.cy = h.cy.data();
    h.d.slit_weights = h.u.data();
    int rc = validate_slice(h.d, m->n_det, m->psf, (int)i);
    if (rc != E2E_OK) return rc;
    for (int c = 0; c < nc; ++c) {
      dv[i].cx[c] = h.cx[c];
      dv[i].cy[c] = h.cy[c];
    }
    for (int c = 0; c < 3; ++c) {
      dv[i].sx[c] = h.d.sigma_x[c];
      dv[i].sy[c] = h.d.sigma_y[c];
    }
  }
  E2E_CK(cudaDeviceSynchronize());
  if (!dv.empty()) E2E_CK(cudaMemcpy(m->d_slices, dv.data(), dv.size() * sizeof(DevSlice), cudaMemcpyHostToDevice));
  m->slices = std::move(ns);
  for (auto& h : m->slices) {  // re-point the descriptors at the moved vectors
    h.d.cx = h.cx.data();
    h.d.cy = h.cy.data();
    h.d.slit_weights = h.u.data();
  }
  m->dev = dv;
  free_plan(m->plan);
  return plan_model(m);
}

}  // extern "C"

namespace {

struct CallbackPayload {
  Server* srv;
  uint64_t id;
};

void CUDART_CB job_finished(void* p) {
  auto* cp = static_cast<CallbackPayload*>(p);
  {
    std::lock_guard<std::mutex> lk(cp->srv->mu);
    auto it = cp->srv->jobs.find(cp->id);
    if (it != cp->srv->jobs.end()) it->second.finished_on_device = true;
  }
  cp->srv->cv.notify_all();
  delete cp;
}

// Memory a job holds while in flight: its scratch plus library-owned frames.
int64_t job_budget(const Model* m, const Job& j) {
  int64_t b = 64 << 10;  // launch tables
  if (m->has_blaze) b += m->n_bins * 8 + (int64_t)m->slices.size() * 8;  // blazed spectra
  if (j.precision == E2E_PREC_MIXED) b += m->plan.store_elems * 8;
  else if (j.dtype == E2E_F32)
    for (int d = 0; d < m->n_det; ++d) b += (int64_t)m->H[d] * m->W[d] * 8;
  if (j.dst.empty())
    for (int d = 0; d < m->n_det; ++d) b += (int64_t)m->H[d] * m->W[d] * (j.dtype == E2E_F32 ? 4 : 8);
  return b;
}

// Admit queued jobs (FIFO) while a slot and budget are free; launch them on their slots.
void admit_jobs(Server* S, std::unique_lock<std::mutex>& lk) {
  e2e_ctx* ctx = S->ctx;
  while ((!S->queue.empty() || !S->express.empty()) && !S->stopping) {
    std::deque<uint64_t>& q = S->express.empty() ? S->queue : S->express;
    const uint64_t id = q.front();
    Job& j = S->jobs[id];
    if (j.status != E2E_JOB_QUEUED) {  // cancelled
      q.pop_front();
      continue;
    }
    int slot = -1;
    for (size_t q = 0; q < S->slot_job.size(); ++q)
      if (S->slot_job[q] == 0) {
        slot = (int)q;
        break;
      }
    if (slot < 0 || S->in_use + (size_t)j.budget > S->budget) break;
    if (!j.express) {  // keep express_slots free for small jobs
      int regular = 0;
      for (uint64_t sid : S->slot_job) regular += (sid != 0 && !S->jobs[sid].express) ? 1 : 0;
      if (regular >= (int)S->slot_job.size() - S->express_slots) break;
    }
    q.pop_front();
    S->slot_job[slot] = id;
    S->in_use += j.budget;
    j.slot = slot;
    j.status = E2E_JOB_RUNNING;
    j.t_admit = S->now_ms();
    cudaStream_t st = j.express ? S->slots_hi[slot] : S->slots[slot];
    // launch outside the server lock; the context lock guards models and spectra
    lk.unlock();
    int rc = E2E_OK;
    uint64_t frame_id = 0;
    {
      std::lock_guard<std::mutex> clk(ctx->mu);
      Model* m = find_model(ctx, j.model);
      if (!m) rc = fail(E2E_ENOTFOUND, "model unloaded before the job ran");
      std::vector<void*> dst = j.dst;
      std::unique_ptr<Frame> fr;
      if (rc == E2E_OK && dst.empty()) {
        rc = alloc_frame(m, j.dtype, st, fr);
        if (rc == E2E_OK) dst = fr->ptrs;
      }
      if (rc == E2E_OK && cudaEventRecord(j.ev0, st) != cudaSuccess) rc = fail(E2E_ECUDA, "event record");
      if (rc == E2E_OK)
        rc = render_impl(ctx, m, (int)j.spec.size(), j.spec.data(), j.precision, j.dtype, dst.data(),
                         j.pitch.empty() ? nullptr : j.pitch.data(), st);
      if (rc == E2E_OK && cudaEventRecord(j.ev1, st) != cudaSuccess) rc = fail(E2E_ECUDA, "event record");
      if (fr) cudaEventRecord(fr->ready, st);
      if (rc == E2E_OK && fr) {
        frame_id = ctx->next_id++;
        ctx->frames[frame_id] = std::move(fr);
      } else if (fr) {
        free_frame(ctx, fr.get());
      }
    }
    if (rc == E2E_OK) {
      auto* cp = new CallbackPayload{S, id};
      if (cudaLaunchHostFunc(st, job_finished, cp) != cudaSuccess) {
        delete cp;
        rc = fail(E2E_ECUDA, "cudaLaunchHostFunc");
      }
    }
    lk.lock();
    Job& jj = S->jobs[id];
    jj.frame_id = frame_id;
    if (rc != E2E_OK) {  // the job failed to launch: finish it with its error
      cudaStreamSynchronize(st);
      jj.status = rc;
      jj.err = rc;
      jj.t_done = S->now_ms();
      S->slot_job[slot] = 0;
      S->in_use -= jj.budget;
      S->cv_done.notify_all();
    }
  }
}

// Retire jobs whose completion callback ran: times, budget, slot.
void retire_jobs(Server* S) {
  for (size_t q = 0; q < S->slot_job.size(); ++q) {
    const uint64_t id = S->slot_job[q];
    if (!id) continue;
    Job& j = S->jobs[id];
    if (!j.finished_on_device) continue;
    j.t_done = S->now_ms();
    cudaEventElapsedTime(&j.device_ms, j.ev0, j.ev1);
    j.status = E2E_JOB_DONE;
    S->slot_job[q] = 0;
    S->in_use -= j.budget;
    S->cv_done.notify_all();
  }
}

void server_loop(Server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    retire_jobs(S);
    bool busy = false;
    for (uint64_t id : S->slot_job) busy = busy || id != 0;
    if (S->stopping && !busy) break;
    admit_jobs(S, lk);
    S->cv.wait_for(lk, std::chrono::milliseconds(50));
  }
}

}  // namespace

extern "C" {

int e2e_server_start(e2e_ctx* ctx, const e2e_server_cfg* cfg) {
  if (!ctx) return fail(E2E_EINVAL, "null context");
  DeviceGuard g(ctx->device);
  if (ctx->server) return fail(E2E_EINVAL, "server already running");
  auto S = std::make_unique<Server>();
  S->ctx = ctx;
  int slots = (cfg && cfg->max_inflight > 0) ? cfg->max_inflight : ctx->opts.max_inflight;
  if (slots < 1) slots = 1;
  size_t budget = cfg ? cfg->budget_bytes : 0;
  if (!budget) budget = ctx->opts.pool_bytes;
  if (!budget) {
    size_t fr = 0, tot = 0;
    E2E_CK(cudaMemGetInfo(&fr, &tot));
    budget = (size_t)(0.9 * (double)fr);
  }
  S->budget = budget;
  S->express_stamps = cfg ? cfg->express_stamps : 0;
  if (S->express_stamps > 0) {
    const int want = (cfg && cfg->express_slots > 0) ? cfg->express_slots : std::max(1, slots / 4);
    S->express_slots = std::min(want, slots - 1);
  }
  int prio_lo = 0, prio_hi = 0;
  E2E_CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  for (int q = 0; q < slots; ++q) {
    cudaStream_t st, sh;
    E2E_CK(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_lo));
    E2E_CK(cudaStreamCreateWithPriority(&sh, cudaStreamNonBlocking, prio_hi));
    S->slots.push_back(st);
    S->slots_hi.push_back(sh);
    S->slot_job.push_back(0);
  }
  S->t0 = std::chrono::steady_clock::now();
  Server* raw = S.get();
  ctx->server = std::move(S);
  raw->th = std::thread(server_loop, raw);
  return E2E_OK;
}

int e2e_submit(e2e_ctx* ctx, const e2e_job* job, uint64_t* request_id) {
  if (!ctx || !job || !request_id) return fail(E2E_EINVAL, "null argument");
  Server* S = ctx->server.get();
  if (!S) return fail(E2E_EINVAL, "server not running");
  if (job->dtype != E2E_F32 && job->dtype != E2E_F64) return fail(E2E_EINVAL, "bad dtype");
  if (job->precision != E2E_PREC_MIXED && job->precision != E2E_PREC_FP64) return fail(E2E_EINVAL, "bad precision");
  Job j;
  j.model = job->model_id;
  j.precision = job->precision;
  j.dtype = job->dtype;
  if (job->n_spec > 0) j.spec.assign(job->spec_ids, job->spec_ids + job->n_spec);
  {
    std::lock_guard<std::mutex> clk(ctx->mu);
    Model* m = find_model(ctx, job->model_id);
    if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
    std::vector<const double*> table;
    int rc = resolve_flux(ctx, m, (int)j.spec.size(), j.spec.data(), table);
    if (rc != E2E_OK) return rc;
    if (job->dst) {
      j.dst.assign(job->dst, job->dst + m->n_det);
      for (void* p : j.dst)
        if (!p) return fail(E2E_EINVAL, "null destination frame");
      if (job->pitch_elems) j.pitch.assign(job->pitch_elems, job->pitch_elems + m->n_det);
    }
    j.budget = job_budget(m, j);
    for (auto& sl : m->slices) j.stamps += (int64_t)sl.d.n_lambda * sl.d.n_slit;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if ((size_t)j.budget > S->budget)
    return fail(E2E_ETOOBIG, "job needs " + std::to_string(j.budget) + " bytes; the serving budget is " +
                                 std::to_string(S->budget));
  if (S->stopping) return fail(E2E_EINVAL, "server is stopping");
  if (cudaEventCreate(&j.ev0) != cudaSuccess || cudaEventCreate(&j.ev1) != cudaSuccess)
    return fail(E2E_ECUDA, "event creation");
  j.id = S->next_id++;
  j.t_submit = S->now_ms();
  const uint64_t id = j.id;
  S->jobs[id] = std::move(j);
  Job& jq = S->jobs[id];
  jq.express = S->express_stamps > 0 && jq.stamps <= S->express_stamps;
  (jq.express ? S->express : S->queue).push_back(id);
  *request_id = id;
  S->cv.notify_all();
  return E2E_OK;
}

static void fill_info(const Job& j, e2e_job_info* info) {
  if (!info) return;
  info->status = j.status;
  info->submit_ms = j.t_submit;
  info->admit_ms = j.t_admit;
  info->done_ms = j.t_done;
  info->device_ms = j.device_ms;
  info->budget_bytes = j.budget;
  info->frame_id = j.frame_id;
  info->stamps = j.stamps;
}

int e2e_poll(e2e_ctx* ctx, uint64_t request_id, e2e_job_info* info) {
  if (!ctx || !ctx->server) return fail(E2E_EINVAL, "server not running");
  Server* S = ctx->server.get();
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(request_id);
  if (it == S->jobs.end()) return fail(E2E_ENOTFOUND, "unknown request id");
  fill_info(it->second, info);
  return E2E_OK;
}

int e2e_wait(e2e_ctx* ctx, uint64_t request_id, int32_t timeout_ms, e2e_job_info* info) {
  if (!ctx || !ctx->server) return fail(E2E_EINVAL, "server not running");
  Server* S = ctx->server.get();
  std::unique_lock<std::mutex> lk(S->mu);
  auto done = [&] {
    auto it = S->jobs.find(request_id);
    return it == S->jobs.end() || (it->second.status != E2E_JOB_QUEUED && it->second.status != E2E_JOB_RUNNING);
  };
  if (timeout_ms < 0) S->cv_done.wait(lk, done);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    auto it = S->jobs.find(request_id);
    if (it != S->jobs.end()) fill_info(it->second, info);
    return fail(E2E_ETIMEOUT, "job not finished within the timeout");
  }
  auto it = S->jobs.find(request_id);
  if (it == S->jobs.end()) return fail(E2E_ENOTFOUND, "unknown request id");
  fill_info(it->second, info);
  if (it->second.status < 0) return fail(it->second.status, "job failed");
  return E2E_OK;
}

int e2e_cancel(e2e_ctx* ctx, uint64_t request_id) {
  if (!ctx || !ctx->server) return fail(E2E_EINVAL, "server not running");
  Server* S = ctx->server.get();
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(request_id);
  if (it == S->jobs.end()) return fail(E2E_ENOTFOUND, "unknown request id");
  if (it->second.status != E2E_JOB_QUEUED) return fail(E2E_EINVAL, "only queued jobs can be cancelled");
  it->second.status = E2E_ECANCELLED;
  it->second.t_done = S->now_ms();
  S->cv_done.notify_all();
  return E2E_OK;
}

int e2e_forget(e2e_ctx* ctx, uint64_t request_id) {
  if (!ctx || !ctx->server) return fail(E2E_EINVAL, "server not running");
  Server* S = ctx->server.get();
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(request_id);
  if (it == S->jobs.end()) return fail(E2E_ENOTFOUND, "unknown request id");
  if (it->second.status == E2E_JOB_RUNNING || it->second.status == E2E_JOB_QUEUED)
    return fail(E2E_EINVAL, "job still pending");
  cudaEventDestroy(it->second.ev0);
  cudaEventDestroy(it->second.ev1);
  S->jobs.erase(it);
  return E2E_OK;
}

int e2e_server_stop(e2e_ctx* ctx) {
  if (!ctx || !ctx->server) return fail(E2E_EINVAL, "server not running");
  Server* S = ctx->server.get();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    for (auto* qq : {&S->queue, &S->express}) {
      for (uint64_t id : *qq) {
        Job& j = S->jobs[id];
        if (j.status == E2E_JOB_QUEUED) {
          j.status = E2E_ECANCELLED;
          j.t_done = S->now_ms();
        }
      }
      qq->clear();
    }
  }
  S->cv.notify_all();
  S->th.join();
  S->cv_done.notify_all();
  DeviceGuard g(ctx->device);
  for (auto& kv : S->jobs) {
    cudaEventDestroy(kv.second.ev0);
    cudaEventDestroy(kv.second.ev1);
  }
  for (cudaStream_t st : S->slots) cudaStreamDestroy(st);
  for (cudaStream_t st : S->slots_hi) cudaStreamDestroy(st);
  ctx->server.reset();
  return E2E_OK;
}

int e2e_render_photons(e2e_ctx* ctx, uint64_t model_id, int32_t n_spec, const uint64_t* spec_ids, uint64_t seed,
                       uint32_t* const* dst, const int64_t* pitch_elems, uint64_t* total_photons, void* stream) {
  NvtxRange nvtx_("e2e photons");
  if (!ctx || !dst) return fail(E2E_EINVAL, "null argument");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  if (!m->u_nonneg) return fail(E2E_EINVAL, "photon rendering needs slit weights >= 0");
  if (m->psf == E2E_PSF_TABLE) return fail(E2E_EINVAL, "photon rendering supports the analytic PSFs");
  std::vector<int64_t> pitch(m->n_det);
  for (int d = 0; d < m->n_det; ++d) {
    if (!dst[d]) return fail(E2E_EINVAL, "null destination frame");
    pitch[d] = pitch_elems ? pitch_elems[d] : m->W[d];
    if (pitch[d] < m->W[d]) return fail(E2E_EINVAL, "pitch smaller than width");
  }
  std::vector<const double*> table;
  int rc = resolve_flux(ctx, m, n_spec, spec_ids, table);
  if (rc != E2E_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->opts.kernel_timing) reset_timing(ctx);
  for (int d = 0; d < m->n_det; ++d)
    E2E_CK(cudaMemset2DAsync(dst[d], pitch[d] * 4, 0, (size_t)m->W[d] * 4, m->H[d], st));
  if (m->slices.empty()) {
    if (total_photons) *total_photons = 0;
    return E2E_OK;
  }
  Scratch sc{{}, st};
  rc = blaze_scratch(m, table, sc, st);
  if (rc != E2E_OK) return rc;
  const double** d_table = nullptr;
  int64_t* d_pitch = nullptr;
  uint32_t** d_dst = nullptr;
  uint64_t *counts = nullptr, *offsets = nullptr, *scan = nullptr;
  int4* anchors = nullptr;
  int* bin_slice = nullptr;
  int64_t* guide = nullptr;
  E2E_CK(sc.get((void**)&d_table, table.size() * sizeof(double*)));
  E2E_CK(sc.get((void**)&d_pitch, pitch.size() * sizeof(int64_t)));
  E2E_CK(sc.get((void**)&d_dst, m->n_det * sizeof(uint32_t*)));
  E2E_CK(sc.get((void**)&counts, (size_t)m->n_bins * sizeof(uint64_t)));
  E2E_CK(sc.get((void**)&offsets, (size_t)(m->n_bins + 1) * sizeof(uint64_t)));
  E2E_CK(sc.get((void**)&scan, scan_scratch_elems(m->n_bins) * sizeof(uint64_t)));
  E2E_CK(sc.get((void**)&anchors, (size_t)m->n_bins * sizeof(int4)));
  E2E_CK(sc.get((void**)&bin_slice, (size_t)m->n_bins * sizeof(int)));
  E2E_CK(sc.get((void**)&guide, (size_t)(kPhotonGuide + 1) * sizeof(int64_t)));
  E2E_CK(cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_pitch, pitch.data(), pitch.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  E2E_CK(cudaMemcpyAsync(d_dst, dst, m->n_det * sizeof(uint32_t*), cudaMemcpyHostToDevice, st));
  const int ns = (int)m->slices.size();
  {
    KernelTimer kt(ctx, st, "photon_bins");
    E2E_CK(launch_photon_bins(m->d_slices, ns, d_table, m->d_usum, m->d_bin_off, m->n_bins, seed, counts, anchors,
                              bin_slice, st));
  }
  {
    KernelTimer kt(ctx, st, "photon_scan");
    E2E_CK(launch_scan_exclusive(counts, offsets, m->n_bins, scan, st));
    E2E_CK(launch_photon_guide(offsets, m->n_bins, guide, st));
  }
  {
    KernelTimer kt(ctx, st, "photons");
    E2E_CK(launch_photons(m->d_slices, ns, m->d_ucum, m->d_usum, m->d_bin_off, offsets, m->psf, seed, d_dst, d_pitch,
                          UINT64_MAX, m->d_ucum32, m->d_cf32, anchors, bin_slice, guide, st));
  }
  if (total_photons) {
    E2E_CK(cudaMemcpyAsync(total_photons, offsets + m->n_bins, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    E2E_CK(cudaStreamSynchronize(st));
  }
  return E2E_OK;
}

int e2e_add_noise(e2e_ctx* ctx, uint64_t model_id, const e2e_noise_params* p, int32_t src_dtype,
                  const void* const* src, const int64_t* src_pitch, int32_t dst_dtype, void* const* dst,
                  const int64_t* dst_pitch, void* stream) {
  NvtxRange nvtx_("e2e noise");
  if (!ctx || !p || !src || !dst) return fail(E2E_EINVAL, "null argument");
  if (src_dtype != E2E_F32 && src_dtype != E2E_F64) return fail(E2E_EINVAL, "src dtype must be E2E_F32 or E2E_F64");
  if (dst_dtype != E2E_F32 && dst_dtype != E2E_F64 && dst_dtype != E2E_U16) return fail(E2E_EINVAL, "bad dst dtype");
  if (!(p->dark_e >= 0) || !(p->prnu >= 0) || !(p->ron_e >= 0) || !(std::fabs(p->xtalk) < 1) ||
      !std::isfinite(p->bias) || !(p->gain > 0) || !std::isfinite(p->gain) || p->saturation < 0 ||
      p->saturation > 65535 || !std::isfinite(p->dark_e) || !std::isfinite(p->prnu) || !std::isfinite(p->ron_e))
    return fail(E2E_EINVAL, "noise parameters out of range");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  Model* m = find_model(ctx, model_id);
  if (!m) return fail(E2E_ENOTFOUND, "unknown model id");
  for (int d = 0; d < m->n_det; ++d) {
    const int64_t sp = src_pitch ? src_pitch[d] : m->W[d], dp = dst_pitch ? dst_pitch[d] : m->W[d];
    if (!src[d] || !dst[d]) return fail(E2E_EINVAL, "null frame");
    if (sp < m->W[d] || dp < m->W[d]) return fail(E2E_EINVAL, "pitch smaller than width");
    if ((int64_t)m->H[d] * ((m->W[d] + 1) / 2) >= ((int64_t)1 << 32)) return fail(E2E_EINVAL, "frame too large");
    if (src[d] == dst[d] && (src_dtype != dst_dtype || sp != dp))
      return fail(E2E_EINVAL, "in-place noise needs the same dtype and pitch");
  }
  if (ctx->opts.kernel_timing) reset_timing(ctx);
  cudaStream_t st = (cudaStream_t)stream;
  // the pixel response is a fixed pattern: computed once per (model, pattern seed, prnu)
  std::vector<double*> R(m->n_det, nullptr);
  std::vector<float*> R32(m->n_det, nullptr);
  if (p->prnu != 0.0) {
    auto& pat = ctx->patterns[model_id];
    if (pat.R.empty() || pat.pattern_seed != p->pattern_seed || pat.prnu != p->prnu) {
      cudaStreamSynchronize(st);  // a previous pattern may still be read
      for (double* q : pat.R) cudaFree(q);
      for (float* q : pat.R32) cudaFree(q);
      pat.R.assign(m->n_det, nullptr);
      pat.R32.assign(m->n_det, nullptr);
      pat.pattern_seed = p->pattern_seed;
      pat.prnu = p->prnu;
      for (int d = 0; d < m->n_det; ++d) {
        const size_t npx = (size_t)m->H[d] * m->W[d];
        cudaError_t e = cudaMalloc((void**)&pat.R[d], npx * sizeof(double));
        // FP32 words of R: the high words, then the low words (R as double-float pairs)
        if (e == cudaSuccess) e = cudaMalloc((void**)&pat.R32[d], 2 * npx * sizeof(float));
        if (e == cudaSuccess)
          e = launch_prnu_map(pat.R[d], pat.R32[d], pat.R32[d] + npx, m->H[d], m->W[d], d, p->pattern_seed, p->prnu,
                              st);
        if (e != cudaSuccess) {
          for (double* q : pat.R) cudaFree(q);
          for (float* q : pat.R32) cudaFree(q);
          ctx->patterns.erase(model_id);
          return cuda_fail(e, "pixel response map");
        }
      }
    }
    R = pat.R;
    R32 = pat.R32;
  }
  // photon noise into FP32 electrons or ADU: the two-pass form (FP32 first pass, the pairs too
  // close to call redone in FP64 from a compacted list); FP64 electrons and expected values
  // (no shot noise) keep the one-pass kernel, whose FP64 paths are the output's own arithmetic
  const bool two_pass = p->poisson && dst_dtype != E2E_F64;
  Scratch sc{{}, st};
  unsigned* list = nullptr;
  unsigned* n_list = nullptr;
  if (two_pass) {
    int64_t most = 0;
    for (int d = 0; d < m->n_det; ++d) most = std::max(most, (int64_t)m->H[d] * ((m->W[d] + 1) / 2));
    E2E_CK(sc.get((void**)&n_list, sizeof(unsigned)));
    E2E_CK(sc.get((void**)&list, std::max<int64_t>(1, most) * sizeof(unsigned)));
  }
  for (int d = 0; d < m->n_det; ++d) {
    const int64_t sp = src_pitch ? src_pitch[d] : m->W[d], dp = dst_pitch ? dst_pitch[d] : m->W[d];
    KernelTimer kt(ctx, st, "noise");
    if (two_pass) {
      const float* lo = R32[d] ? R32[d] + (size_t)m->H[d] * m->W[d] : nullptr;
      E2E_CK(launch_noise_two_pass(p->seed, p->pattern_seed, p->dark_e, p->prnu, p->ron_e, p->xtalk, p->gain,
                                   p->bias, p->saturation, src_dtype, src[d], sp, R[d], R32[d], lo, dst_dtype, dst[d],
                                   dp, m->H[d], m->W[d], d, list, n_list, st));
    } else {
      E2E_CK(launch_noise(p->seed, p->pattern_seed, p->dark_e, p->prnu, p->ron_e, p->xtalk, p->gain, p->bias,
                          p->saturation, p->poisson, src_dtype, src[d], sp, R[d], R32[d], dst_dtype, dst[d], dp,
                          m->H[d], m->W[d], d, st));
    }
  }
  return E2E_OK;
}

int e2e_kernel_times(e2e_ctx* ctx, const char** names, float* ms, int32_t cap, int32_t* n) {
  if (!ctx || !n) return fail(E2E_EINVAL, "null argument");
  if (!ctx->opts.kernel_timing) return fail(E2E_EINVAL, "context was created without kernel_timing");
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->mu);
  *n = (int32_t)ctx->timed.size();
  for (int32_t i = 0; i < *n && i < cap; ++i) {
    E2E_CK(cudaEventSynchronize(ctx->timed[i].b));
    float t = 0.f;
    E2E_CK(cudaEventElapsedTime(&t, ctx->timed[i].a, ctx->timed[i].b));
    if (names) names[i] = ctx->timed[i].name;
    if (ms) ms[i] = t;
  }
  return E2E_OK;
}

}  // extern "C"
