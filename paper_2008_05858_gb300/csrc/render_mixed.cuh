// The separable-PSF mixed-precision render kernel (see render_mixed.cu), as a template
// instantiated by render_mixed.cu (production) and render_mixed_check.cu (debug checks).
#pragma once
#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "merge_tile.cuh"
#include "mixed_common.cuh"
#include "phi32.cuh"

namespace e2e {

#ifndef E2E_MIXED_THREADS
#define E2E_MIXED_THREADS 128
#endif
constexpr int kThreads = E2E_MIXED_THREADS;  // threads per render CTA
constexpr int kWarps = kThreads / 32;
constexpr int kQuads = kThreads / 4;  // runs in flight per CTA (a quad of lanes per run)
// floats per profile row of the quads' exchange area: 16 used, padded to 80 bytes so that
// the 16-byte chunks written by the lanes of a warp fall in distinct banks
constexpr int kXchStride = 20;

// ------------------------------------------------------------------------------ render


// Shared-memory layout of one CTA (offsets in bytes), identical on host and device.
struct MixedLayout {
  size_t tabP, tabS, tabW, tabU, tabG, stage, xch, boxh, boxl, total;
  __host__ __device__ MixedLayout(int J, int NK, int nd, int B, int area) {
    size_t o = 0;
    tabP = o; o += (size_t)J * nd * 16;      // P_b(lt) of x and y per sample, split_xy pairs
    tabS = o; o += (size_t)NK * 8;            // s of each slit point, (hi, lo) floats
    tabW = o; o += (size_t)J * 8;             // flux x bin width / 4 per sample, (hi, lo) floats
    tabU = o; o += (size_t)NK * 8;            // slit weights, (hi, lo) floats
    o = (o + 15) & ~(size_t)15;
    tabG = o; o += (size_t)J * 16;            // 1/(sqrt2 sigma) of x and y, (hi, lo) each
    stage = o; o += (size_t)B * kQuads * 16;  // mapped stamps of the runs in flight
    xch = o; o += (size_t)kQuads * 4 * kXchStride * 4;  // the quads' profile exchange
    boxh = o; o += (size_t)area * 4;          // fixed-point box, high words
    boxl = o; o += (size_t)area * 4;          // low words
    total = o;
  }
};


#ifndef E2E_MID_TILE_BLOCKS
#define E2E_MID_TILE_BLOCKS 4
#endif
#ifndef E2E_SMALL_TILE_BLOCKS
#define E2E_SMALL_TILE_BLOCKS 4
#endif
// CTAs per SM the register budget is set for (128-thread CTAs): E2E_SMALL_TILE_BLOCKS (4:
// 128 registers) for lane tiles up to 72 accumulators -- every quad tile, at most 16 x 4; five
// CTAs (96 registers) fit without spills but ran slower -- E2E_MID_TILE_BLOCKS up to 84, else 2.
template <int K, int DX, int DY>
constexpr int mixed_min_blocks() {
  return ((K + DX) * ((K + DY + 3) / 4) <= 72 ? E2E_SMALL_TILE_BLOCKS : ((K + DX) * ((K + DY + 3) / 4) <= 84 ? E2E_MID_TILE_BLOCKS : 2)) *
         128 / kThreads;
}

// N consecutive floats from shared memory at p (p 4N-byte aligned when N is 2 or 4).
template <int N>
__device__ __forceinline__ void load_rows(const float* p, float (&v)[N]) {
  if constexpr (N == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (N == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

// The separable kernel's arguments: the render's, then the fused tile merge's.
struct FusedArgs {
  MixedArgs a;
  MergeArgs mg;
};

// CHECK: debug build of the same kernel, counting into a.err every deposit the plan did not
// foresee (the non-checking instantiation carries none of that code).  FAR: the cheaper tail
// rational on every tail edge (the edges one or more pixels from a stamp's centre) when the
// model's widest PSF keeps their arguments within its fit (the plan's far_tails; K = 1 has no
// tail edges and takes FAR = false).
template <int K, int DX, int DY, bool CHECK, bool FAR>
__global__ void __launch_bounds__(kThreads, mixed_min_blocks<K, DX, DY>()) k_render_mixed(const FusedArgs fa) {
  const MixedArgs& a = fa.a;
  const MergeArgs& mg = fa.mg;
  constexpr int RX = K + DX, RY = K + DY, H = K / 2;
  constexpr int D = DX > DY ? DX : DY;  // slack of the profile a lane evaluates
  constexpr int R = K + D;              // pixels of that profile
  constexpr int RY4 = (RY + 3) / 4;     // tile rows accumulated per lane of a quad
  constexpr int RC = (R + 3) / 4;       // 16-byte chunks of a profile in the exchange
  constexpr int RXC = (RX + 3) / 4;     // chunks of an x profile the tile reads
  static_assert(4 * RC <= kXchStride, "profile row exceeds the exchange stride");
  extern __shared__ __align__(16) unsigned char smem[];
  if (mg.n_zero && (int)blockIdx.x >= (int)gridDim.x - mg.n_zero) {  // a tile no item overlaps: zeros
    const Tile t = mg.zero_tiles[blockIdx.x - (gridDim.x - mg.n_zero)];
    const int th = mg.dims[2 * t.det], tw = mg.dims[2 * t.det + 1];
    if (mg.dtype == 0)
      merge_tile<kThreads, false, float>(t, mg.lists, mg.items, a.store, reinterpret_cast<float* const*>(mg.dst)[t.det],
                                         mg.pitch[t.det], th, tw, threadIdx.x);
    else
      merge_tile<kThreads, false, double>(t, mg.lists, mg.items, a.store, reinterpret_cast<double* const*>(mg.dst)[t.det],
                                          mg.pitch[t.det], th, tw, threadIdx.x);
    return;
  }
  const Item it = a.items[blockIdx.x];
  const DevSlice& S = a.slices[it.slice];
  const int area = it.bw * it.bh;
  const int nd = S.degree + 1;
  const MixedLayout L(32 * a.JB, a.nk_max, a.max_deg + 1, a.B, area);
  float4* tabP = reinterpret_cast<float4*>(smem + L.tabP);
  float2* tabS = reinterpret_cast<float2*>(smem + L.tabS);
  float2* tabW = reinterpret_cast<float2*>(smem + L.tabW);
  float2* tabU = reinterpret_cast<float2*>(smem + L.tabU);
  float4* tabG = reinterpret_cast<float4*>(smem + L.tabG);
  int4* stage = reinterpret_cast<int4*>(smem + L.stage);
  float* xch = reinterpret_cast<float*>(smem + L.xch);
  int* boxh = reinterpret_cast<int*>(smem + L.boxh);
  unsigned* boxl = reinterpret_cast<unsigned*>(smem + L.boxl);
  __shared__ double s_w[kWarps], s_u[kWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {  // mapping coefficients and PSF constants of the item's samples (per-model tables), copied
     // to shared memory asynchronously while the box is cleared and the weights are built
    const int w = nd + 2;
    const float4* rows = S.samples + (int64_t)it.j0 * w;
    for (int e = tid; e < it.nj * w; e += kThreads) {
      const int jj = e / w, b = e - jj * w;
      if (b < nd) cp_async16(tabP + jj * nd + b, rows + e);
      else if (b == nd) cp_async16(tabG + jj, rows + e);
    }
  }
  const double* flux = a.flux_tab[S.flux_slot];
  const double* u = a.u_all + S.u_off;
  // this thread's first slit weight and flux, loaded before the box is cleared
  const double u_first = tid < it.nk ? u[it.k0 + tid] : 0.0;
  const double f_first = tid < it.nj ? flux[it.j0 + tid] : 0.0;
  for (int p = tid; p < area; p += kThreads) {
    boxh[p] = 0;
    boxl[p] = 0u;
  }
  const double inv_ns = 1.0 / (double)S.n_slit;
  double usum = 0.0;
  for (int kk = tid; kk < it.nk; kk += kThreads) {
    const double uk = kk == tid ? u_first : u[it.k0 + kk];
    tabS[kk] = split_df(norm_sample_r(it.k0 + kk, S.n_slit, inv_ns));
    tabU[kk] = split_df(uk);
    usum += fabs(uk);
  }
  double wsum = 0.0;
  for (int jj = tid; jj < it.nj; jj += kThreads) {
    const double wj = (jj == tid ? f_first : flux[it.j0 + jj]) * S.dlam;
    tabW[jj] = split_df(wj * 0.25);  // 0.25: the profiles below are 2x the pixel integrals
    wsum += fabs(wj);
  }
  // flux bound of the item: sum over its stamps of |w| (bounds every pixel of its box)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    usum += __shfl_xor_sync(0xffffffffu, usum, o);
  }
  if (lane == 0) {
    s_w[warp] = wsum;
    s_u[warp] = usum;
  }
  cp_async_wait_all();  // this thread's table copies; the barrier then publishes all of them
  __syncthreads();
  double wtot = 0.0, utot = 0.0;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) {
    wtot += s_w[q];
    utot += s_u[q];
  }
  const double total = wtot * utot;
  // scale 2^P with |box sums| <= total < 2^(52-P); clamp so 2^P stays a normal FP32
  int ex = 0;
  frexp(total, &ex);
  const int Psh = total > 0.0 ? max(-100, min(100, 52 - ex)) : 0;
  const float sc = ldexpf(1.f, Psh), sc_hi = ldexpf(1.f, Psh - 22);

  // A quad of lanes owns one run and takes its stamps two at a time: lanes 0 and 1 evaluate
  // the x and y profiles of the even stamp, lanes 2 and 3 those of the odd one (same code,
  // different inputs).  The four profiles go through shared memory, and each lane of the quad
  // accumulates its quarter of the tile's rows from both stamps, in stamp order.
  const int quad = lane >> 2, qi = lane & 3, slot = qi >> 1, axis = qi & 1;
  const int nrc = (it.nk + a.B - 1) / a.B;
  const int njq = (it.nj + 7) / 8;
  const int ntask = njq * nrc;
  int4* mystage = stage + warp * 8 + quad;
  float* qrow = xch + (warp * 8 + quad) * 4 * kXchStride;  // rows: x, y of the even stamp, x, y of the odd
  float* myrow = qrow + (slot * 2 + axis) * kXchStride;
  for (int task = warp; task < ntask && total > 0.0; task += kWarps) {
    const int jj = (task % njq) * 8 + quad;
    const bool jvalid = jj < it.nj;      // uniform over the quad
    const int kk0 = (task / njq) * a.B;  // first slit point of the run, relative to the item
    const int nb = min(a.B, it.nk - kk0);
    // map the run's stamps (double-float), a quarter each, into the staging area; the tile
    // origin is the least window centre of the run's on-frame stamps (reduced over the quad)
    // (a lane's stamps -- at most four: runs hold at most 16 -- mapped together)
    int xmn = 1 << 30, ymn = 1 << 30;
    {
      const float4* Pj = tabP + (jvalid ? jj : 0) * nd;
      float2 sv[4], mh[4], ml[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) sv[u] = tabS[kk0 + min(qi + 4 * u, nb - 1)];
      map_xy_df_n<4>(Pj, S.degree, sv, mh, ml);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = qi + 4 * u;
        if (b < nb) {
          int ci = kOffFrame, ri = kOffFrame;
          float fx = 0.f, fy = 0.f;
          if (jvalid) {
            split_coord_df(mh[u].x, ml[u].x, ci, fx);
            split_coord_df(mh[u].y, ml[u].y, ri, fy);
          }
          mystage[b * kQuads] = make_int4(ci, ri, __float_as_int(fx), __float_as_int(fy));
          if (ci != kOffFrame && ri != kOffFrame) {
            xmn = min(xmn, ci);
            ymn = min(ymn, ri);
          }
        }
      }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      xmn = min(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
      ymn = min(ymn, __shfl_xor_sync(0xffffffffu, ymn, o));
    }
    __syncwarp();
    const float4 g4 = jvalid ? tabG[jj] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float gh = axis ? g4.z : g4.x, gl = axis ? g4.w : g4.y;
    const float2 gl2 = f2(2.f * gl, 2.f * gl);
    const float2 wj = jvalid ? tabW[jj] : make_float2(0.f, 0.f);
    float acc[RY4][RX];
#pragma unroll
    for (int r = 0; r < RY4; ++r)
#pragma unroll
      for (int c = 0; c < RX; ++c) acc[r][c] = 0.f;
    const int nstep = (nb + 1) >> 1;
    for (int step = 0; step < nstep; ++step) {
      const int b = 2 * step + slot;
      const int4 st = b < nb ? mystage[b * kQuads] : make_int4(kOffFrame, kOffFrame, 0, 0);
      const bool on = st.x != kOffFrame && st.y != kOffFrame;
      const int o = on ? (axis ? st.y - ymn : st.x - xmn) : 0;  // window offset in the tile, 0..D
      if constexpr (CHECK) {
        if (o > (axis ? DY : DX)) atomicAdd(a.err, 1);  // the run outgrew the planned tile
      }
      const float f = on ? __int_as_float(axis ? st.w : st.z) : 0.f;
      const float2 uk = tabU[kk0 + min(b, nb - 1)];
      const float w = on ? fmaf(wj.x, uk.x, fmaf(wj.x, uk.y, wj.y * uk.x)) : 0.f;
      const float mult = axis ? (on ? 1.f : 0.f) : w;  // the weight rides on the x profile
      // Profile of the stamp's own K-pixel window, window pixel m spanning edges m and m+1
      // at offsets (m - H -+ 1/2) - f from the stamp centre: tails E = erfc(|w|) at the edges
      // off the centre pixel, and erf F = erf(|w|) at the four edges around the centre pixel H.
      // Twice the pixel integrals are differences of left tails (m < H-1), of right tails
      // (m > H+1), and sums / differences of erf for the centre pixel and its two neighbours.
      // The tails of the centre pixel's own edges H and H+1 enter only where erf is out of its
      // range (|w| >= kErfMaxArg, a PSF narrower than ~0.85 px), so they are evaluated only
      // when some lane of the warp needs them.  Edges are taken in pairs (packed arithmetic).
      float E[K + 1], F[K + 1], Wd[K + 1];
      constexpr int NT = K - 1;  // edges 0..H-1 and H+2..K
      float fh, fl;
      split_offset(f, fh, fl);
      const float c1 = -fl * gh;
      const float2 c2 = f2(2.f * c1, 2.f * c1);
#pragma unroll
      for (int i = 0; i < NT; i += 2) {
        const int m0 = i < H ? i : i + 2, m1 = i + 1 < H ? i + 1 : i + 3;
        float2 wh, wl2;
        edge_arg2_split(f2((float)(m0 - H) - 0.5f, (float)(m1 - H) - 0.5f), fh, gh, gl2, c1, c2, wh, wl2);
        // edges one or more pixels from the centre (|e - f| >= 1): the cheaper rational when the
        // plan found every such argument within its fit
        float2 t;
        if (FAR)
          t = tail2x2_w2_far(wh, wl2);
        else
          t = tail2x2_w2(wh, wl2);
        E[m0] = t.x;
        E[m1] = t.y;
        Wd[m0] = wh.x;
        Wd[m1] = wh.y;
      }
      {
        float2 wc, wlc2;  // edges H and H+1
        edge_arg2_split(f2(-0.5f, 0.5f), fh, gh, gl2, c1, c2, wc, wlc2);
        Wd[H] = wc.x;
        Wd[H + 1] = wc.y;
        const bool far = fabsf(wc.x) >= kErfMaxArg || fabsf(wc.y) >= kErfMaxArg;
        if (__any_sync(0xffffffffu, far)) {
          const float2 t = tail2x2_w2(wc, wlc2);
          E[H] = t.x;
          E[H + 1] = t.y;
        } else {
          E[H] = E[H + 1] = 0.f;  // not read: every F below comes from the polynomial
        }
      }
      if constexpr (K >= 3) {
        const float2 fa = erf_small2(f2(Wd[H - 1], Wd[H])), fb = erf_small2(f2(Wd[H + 1], Wd[H + 2]));
        F[H - 1] = fabsf(Wd[H - 1]) < kErfMaxArg ? fa.x : 1.f - E[H - 1];
        F[H] = fabsf(Wd[H]) < kErfMaxArg ? fa.y : 1.f - E[H];
        F[H + 1] = fabsf(Wd[H + 1]) < kErfMaxArg ? fb.x : 1.f - E[H + 1];
        F[H + 2] = fabsf(Wd[H + 2]) < kErfMaxArg ? fb.y : 1.f - E[H + 2];
      } else {
        const float2 fa = erf_small2(f2(Wd[0], Wd[1]));
        F[0] = fabsf(Wd[0]) < kErfMaxArg ? fa.x : 1.f - E[0];
        F[1] = fabsf(Wd[1]) < kErfMaxArg ? fa.y : 1.f - E[1];
      }
      float win[K];
#pragma unroll
      for (int m = 0; m < K; ++m) {
        float v;
        if (m < H - 1) v = E[m + 1] - E[m];
        else if (m == H - 1) v = F[m] - F[m + 1];
        else if (m == H) v = F[m] + F[m + 1];
        else if (m == H + 1) v = F[m + 1] - F[m];
        else v = E[m] - E[m + 1];
        win[m] = v;
      }
#pragma unroll
      for (int m = 0; m + 1 < K; m += 2) {
        const float2 p2 = __fmul2_rn(f2(mult, mult), f2(win[m], win[m + 1]));
        win[m] = p2.x;
        win[m + 1] = p2.y;
      }
      win[K - 1] *= mult;
      // exchange: each lane publishes its window at its offset o (0..D) in a zeroed row, then
      // reads the two x profiles whole and its own rows of the two y profiles
      {
        const int oc = min(o, D);
#pragma unroll
        for (int q4 = 0; q4 < RC; ++q4) reinterpret_cast<float4*>(myrow)[q4] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int m = 0; m < K; ++m) myrow[oc + m] = win[m];
      }
      __syncwarp();
      float xa[4 * RXC], xb[4 * RXC], ya[RY4], yb[RY4];
#pragma unroll
      for (int q4 = 0; q4 < RXC; ++q4) {
        const float4 va = reinterpret_cast<const float4*>(qrow)[q4];
        const float4 vb = reinterpret_cast<const float4*>(qrow + 2 * kXchStride)[q4];
        xa[4 * q4] = va.x; xa[4 * q4 + 1] = va.y; xa[4 * q4 + 2] = va.z; xa[4 * q4 + 3] = va.w;
        xb[4 * q4] = vb.x; xb[4 * q4 + 1] = vb.y; xb[4 * q4 + 2] = vb.z; xb[4 * q4 + 3] = vb.w;
      }
      load_rows<RY4>(qrow + kXchStride + qi * RY4, ya);
      load_rows<RY4>(qrow + 3 * kXchStride + qi * RY4, yb);
      __syncwarp();  // the exchange rows are rewritten by the next step
#pragma unroll
      for (int r = 0; r < RY4; ++r) {
        const float2 yya = f2(ya[r], ya[r]), yyb = f2(yb[r], yb[r]);
#pragma unroll
        for (int c = 0; c + 1 < RX; c += 2) {
          float2 v = __ffma2_rn(yya, f2(xa[c], xa[c + 1]), f2(acc[r][c], acc[r][c + 1]));
          v = __ffma2_rn(yyb, f2(xb[c], xb[c + 1]), v);
          acc[r][c] = v.x;
          acc[r][c + 1] = v.y;
        }
        if constexpr (RX % 2 == 1) {
          acc[r][RX - 1] = fmaf(ya[r], xa[RX - 1], acc[r][RX - 1]);
          acc[r][RX - 1] = fmaf(yb[r], xb[RX - 1], acc[r][RX - 1]);
        }
      }
    }
    __syncwarp();  // the staging is reused by the next task
    // flush this lane's rows of the run tile as exact fixed-point increments
    const int nrow = min(RY4, RY - qi * RY4);
    if (xmn != (1 << 30) && nrow > 0) {
      const int gx0 = xmn - H - it.bx0, gy0 = ymn - H - it.by0 + qi * RY4;
      const bool inside = gx0 >= 0 && gx0 + RX <= it.bw && gy0 >= 0 && gy0 + nrow <= it.bh;
#pragma unroll
      for (int r = 0; r < RY4; ++r) {
        const int gy = gy0 + r;
        if constexpr (CHECK) {  // outside the box is legitimate only off the detector
          if (r < nrow && !inside && (gy < 0 || gy >= it.bh)) {
            const int Y = it.by0 + gy;
#pragma unroll
            for (int c = 0; c < RX; ++c) {
              const int X = it.bx0 + gx0 + c;
              if (acc[r][c] != 0.f && X >= 0 && X < S.W && Y >= 0 && Y < S.H) atomicAdd(a.err, 1);
            }
          }
        }
        if (r >= nrow || (!inside && (gy < 0 || gy >= it.bh))) continue;
        int* rowh = boxh + gy * it.bw + gx0;
        unsigned* rowl = boxl + gy * it.bw + gx0;
#pragma unroll
        for (int c = 0; c < RX; c += 2) {
          int2 hw;
          uint2 lw;
          fixed_split2(make_float2(acc[r][c], c + 1 < RX ? acc[r][c + 1] : 0.f), sc, sc_hi, hw, lw);
#pragma unroll
          for (int h = 0; h < 2 && c + h < RX; ++h) {
            const int cc = c + h;
            if constexpr (CHECK) {
              const int X = it.bx0 + gx0 + cc;
              if (!inside && (gx0 + cc < 0 || gx0 + cc >= it.bw) && acc[r][cc] != 0.f && X >= 0 && X < S.W)
                atomicAdd(a.err, 1);
            }
            if (!inside && (gx0 + cc < 0 || gx0 + cc >= it.bw)) continue;
            atomicAdd(rowh + cc, h ? hw.y : hw.x);
            atomicAdd(rowl + cc, h ? lw.y : lw.x);
          }
        }
      }
    }
  }
  __syncthreads();
  // box value = (hi word * 2^22 + lo word) * 2^-P, written as an unevaluated FP32 pair
  float2* out = a.store + it.store_off;
  const float inv = ldexpf(1.f, -Psh);
  for (int p = tid; p < area; p += kThreads) out[p] = fixed_to_pair(boxh[p], boxl[p], inv);
  if (mg.count) fused_merge_epilogue<kThreads>(mg, a.store, it, S.det);
}


template <int K, int DX, int DY, bool CHECK, bool FAR>
static cudaError_t launch_one(const MixedArgs& a, const MergeArgs& mg, int n_items, size_t smem, cudaStream_t st) {
  auto kern = k_render_mixed<K, DX, DY, CHECK, FAR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_items + mg.n_zero, kThreads, smem, st>>>(FusedArgs{a, mg});
  return cudaGetLastError();
}

// Debug-check instantiations (render_mixed_check.cu) and the cheaper-tail ones of windows
// K >= 3 (render_mixed_far.cu: production, render_mixed_check_far.cu: debug checks), each a
// translation unit of its own so that the instantiations compile in parallel.
cudaError_t launch_render_mixed_checked(int K, int DX, int DY, const MixedArgs& a, const MergeArgs& mg, int n_items,
                                        size_t smem, cudaStream_t st);
cudaError_t launch_render_mixed_far(int K, int DX, int DY, bool check, const MixedArgs& a, const MergeArgs& mg,
                                    int n_items, size_t smem, cudaStream_t st);
cudaError_t launch_render_mixed_far_checked(int K, int DX, int DY, const MixedArgs& a, const MergeArgs& mg,
                                            int n_items, size_t smem, cudaStream_t st);

// The tile variants (K, DX, DY) the library instantiates.
#define E2E_MIXED_VARIANTS(V)                                                                           \
  V(1, 0, 0) V(3, 0, 0) V(5, 0, 0) V(7, 0, 0) V(9, 0, 0) V(11, 0, 0) V(13, 0, 0) V(15, 0, 0)            \
  V(1, 1, 1) V(3, 1, 1) V(5, 1, 1) V(7, 1, 1) V(9, 1, 1) V(11, 1, 1) V(13, 1, 1)                        \
  V(1, 1, 2) V(3, 1, 2) V(5, 1, 2) V(7, 1, 2) V(9, 1, 2) V(11, 1, 2) V(13, 1, 2)                        \
  V(1, 1, 3) V(3, 1, 3) V(5, 1, 3) V(7, 1, 3) V(9, 1, 3) V(11, 1, 3)                                    \
  V(1, 2, 2) V(3, 2, 2) V(5, 2, 2) V(7, 2, 2) V(9, 2, 2)

// The variants with tail edges (K >= 3), instantiated a second time with FAR = true.
#define E2E_MIXED_FAR_VARIANTS(V)                                                                       \
  V(3, 0, 0) V(5, 0, 0) V(7, 0, 0) V(9, 0, 0) V(11, 0, 0) V(13, 0, 0) V(15, 0, 0)                       \
  V(3, 1, 1) V(5, 1, 1) V(7, 1, 1) V(9, 1, 1) V(11, 1, 1) V(13, 1, 1)                                   \
  V(3, 1, 2) V(5, 1, 2) V(7, 1, 2) V(9, 1, 2) V(11, 1, 2) V(13, 1, 2)                                   \
  V(3, 1, 3) V(5, 1, 3) V(7, 1, 3) V(9, 1, 3) V(11, 1, 3)                                               \
  V(3, 2, 2) V(5, 2, 2) V(7, 2, 2) V(9, 2, 2)

}  // namespace e2e
