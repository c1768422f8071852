// Elliptical (rotated) Gaussian PSF: the mixed-precision tiled renderer and the plain FP64
// renderer.
//
// The PSF of an order-slice is a bivariate normal with widths sigma_a(lt), sigma_b(lt) along
// axes rotated by theta (the asymmetric Gaussian of Sec. 2.2, with a rotation).  Its pixel
// integral is no product of 1-D integrals.  Write the density as the x-marginal times the
// conditional density of y given x:
//
//   x ~ N(x_c, vx),   y | x ~ N(y_c + beta (x - x_c), s_c^2),   beta = cxy / vx,   s_c^2 = vy - beta cxy.
//
// Over pixel column m, x = x_c + tb + tau with tb = i0 + m - x_c the column centre and
// |tau| <= 1/2, and with eps = beta / s_c,
//
//   I[m, n] = int dtau phi_x(tb + tau) [Phi(V_{n+1} - eps tau) - Phi(V_n - eps tau)],
//   V_n = (r0 + n - 1/2 - y_c - beta tb) / s_c.
//
// Taylor in eps tau about the column centre, Phi(V - eps tau) = sum_k (-eps tau)^k / k! Phi^(k)(V)
// with Phi^(k)(V) = (-1)^(k-1) He_(k-1)(V) phi(V) (probabilists' Hermite polynomials), gives
//
//   I[m, n] = mu0[m] { Phi(V_{n+1}) - Phi(V_n) + phi(V_{n+1}) G_m(V_{n+1}) - phi(V_n) G_m(V_n) },
//   G_m(V)  = sum_{k >= 1} a_k He_(k-1)(V),   a_k = -eps^k mom_k[m] / k!,
//
// where mu0[m] is the column's x-integral and mom_k[m] the k-th moment of tau under phi_x
// restricted to the column, normalised by its mass (Gauss-Legendre on the column).  The same
// holds with the edges V_n taken at any reference abscissa tb' near the column and tau
// replaced by the offset u = tb + tau - tb' from it.  The FP32 kernel takes tb' at the centre of
// a pair of columns (u = tau -+ 1/2, |u| <= 1), so the pair's two columns share their K + 1
// row edges and differ only in their moments; with |eps| <= 0.2 (checked when the model is
// loaded) the series cut after k = 7, with 5-point Gauss-Legendre moments, stays below 2e-8 of
// the pixel value.  The FP64 kernel takes each column's own centre (|u| <= 1/2), k <= 9 and
// 12-point moments.  The Phi differences carry the full accuracy: they are formed exactly like
// the separable PSF's pixel integrals (tails subtracted on one side of the conditional mean,
// erf across it), only with a per-pair (FP32) or per-column (FP64) centre.
#include "e2e_device.cuh"
#include "e2e_kernels.h"
#include "mixed_common.cuh"
#include "phi32.cuh"
#include "quad_coeffs.h"

namespace e2e {

constexpr int kEThreads = 128;
constexpr int kEWarps = kEThreads / 32;
constexpr float kSqrt2Ln2 = 1.17741002f;         // V = w sqrt(2 ln 2) for w in log2 units
constexpr float kTwoOverSqrt2Pi = 0.797884561f;  // 2 phi(V) / exp(-V^2 / 2)

// ------------------------------------------------------------------------------ mixed

// Shared-memory layout of one CTA (bytes), identical on host and device.  Lane groups of
// (K + 1) / 2 lanes (lane j owning window columns 2j and 2j + 1) stage the 16 stamps of a run
// each and keep their sample's series constants: 32 / ((K + 1) / 2) groups per warp.
struct EllipLayout {
  size_t tabP, tabS, tabW, tabU, tabE, stage, cser, boxh, boxl, total;
  __host__ __device__ EllipLayout(int J, int NK, int nd, int area, int K) {
    const int ng = kEWarps * (32 / ((K + 1) / 2));  // lane groups per CTA
    size_t o = 0;
    tabP = o; o += (size_t)J * nd * 16;        // P_b(lt) of x and y per sample, split_xy pairs
    tabS = o; o += (size_t)NK * 8;              // s of each slit point, (hi, lo) floats
    tabW = o; o += (size_t)J * 8;               // flux x bin width / 4 per sample, (hi, lo)
    tabU = o; o += (size_t)NK * 8;              // slit weights, (hi, lo)
    o = (o + 15) & ~(size_t)15;
    tabE = o; o += (size_t)J * 32;              // two float4 of PSF constants per sample
    stage = o; o += (size_t)ng * 16 * 16;       // mapped stamps of the groups' runs
    cser = o; o += (size_t)ng * kGlKmax * 8;    // the groups' series constants c_k (left, right)
    boxh = o; o += (size_t)area * 4;
    boxl = o; o += (size_t)area * 4;
    total = o;
  }
};

// Twice the x-integral of window column m from its edges' tails E and erf values F (left
// edge L, right edge R), by the separable profile's formulas.
template <int H>
__device__ __forceinline__ float column_x(int m, float EL, float FL, float ER, float FR) {
  return m < H - 1 ? ER - EL : (m == H - 1 ? FL - FR : (m == H ? FL + FR : (m == H + 1 ? FR - FL : EL - ER)));
}

// One CTA per work item (<= 32 wavelength samples x <= 16 slit points, at most 512 stamps,
// so no box pixel gets more than 512 fixed-point deposits).  A warp holds 32 / ((K + 1) / 2)
// groups of (K + 1) / 2 lanes; lane j of a group owns the window's column pair (2j, 2j + 1)
// (the last pair of an odd K has no right column).  A group takes one wavelength sample and
// walks the run of its slit points in order: the run's stamps are mapped into the group's
// staging, then for each stamp every lane evaluates its column pair: x-edges 2j and 2j + 1
// (edge 2j + 2 from the next lane by a shuffle), the moments of each column about the pair's
// centre, and the K + 1 row edges of the pair's conditional profile, shared by both columns,
// in packed pairs; each column's series term is a degree-6 polynomial per edge.  The lane adds
// the 2K pixels to its registers; consecutive slit points mostly share their window origin, so
// the lanes deposit their columns into the item's box (exact fixed point, shared-memory
// integer atomics) only when the origin moves and at the end of the run.
//
// Row edges: the pair's conditional centre f = f_y + beta t_p (t_p the pair's centre offset; a
// double-float, |f| can exceed 1/2) is split once into fc, f rounded to 19 fractional bits,
// and the rest ff (|ff| <= 2^-20).  Each edge offset e - fc (e a half-integer) is then exact
// in FP32 for |e - fc| < 32, and the argument w = (e - f) g_c is the exact product
// (e - fc) g_ch with its FMA error, plus (e - fc) g_cl - ff g_ch: six FP32 operations per edge.
template <int K>
__global__ void __launch_bounds__(kEThreads, 5) k_render_ellip(const MixedArgs a) {
  constexpr int H = K / 2;
  constexpr int GL = (K + 1) / 2;  // lanes per group: column pairs of the window
  constexpr int NG = 32 / GL;      // lane groups per warp
  extern __shared__ __align__(16) unsigned char smem[];
  const Item it = a.items[blockIdx.x];
  const DevSlice& S = a.slices[it.slice];
  const int area = it.bw * it.bh;
  const int nd = S.degree + 1;
  const EllipLayout L(32, a.nk_max, a.max_deg + 1, area, K);
  float4* tabP = reinterpret_cast<float4*>(smem + L.tabP);
  float2* tabS = reinterpret_cast<float2*>(smem + L.tabS);
  float2* tabW = reinterpret_cast<float2*>(smem + L.tabW);
  float2* tabU = reinterpret_cast<float2*>(smem + L.tabU);
  float4* tabE = reinterpret_cast<float4*>(smem + L.tabE);
  int4* stage = reinterpret_cast<int4*>(smem + L.stage);
  float2* cser = reinterpret_cast<float2*>(smem + L.cser);
  int* boxh = reinterpret_cast<int*>(smem + L.boxh);
  unsigned* boxl = reinterpret_cast<unsigned*>(smem + L.boxl);
  __shared__ double s_w[kEWarps], s_u[kEWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int p = tid; p < area; p += kEThreads) {
    boxh[p] = 0;
    boxl[p] = 0u;
  }
  const double* flux = a.flux_tab[S.flux_slot];
  const double* u = a.u_all + S.u_off;
  const double inv_ns = 1.0 / (double)S.n_slit;
  double usum = 0.0;
  for (int kk = tid; kk < it.nk; kk += kEThreads) {
    const double uk = u[it.k0 + kk];
    tabS[kk] = split_df(norm_sample_r(it.k0 + kk, S.n_slit, inv_ns));
    tabU[kk] = split_df(uk);
    usum += fabs(uk);
  }
  {  // mapping coefficients and PSF constants of the item's samples (per-model tables)
    const int w = nd + 2;
    const float4* rows = S.samples + (int64_t)it.j0 * w;
    for (int e = tid; e < it.nj * w; e += kEThreads) {
      const int jj = e / w, b = e - jj * w;
      if (b < nd) tabP[jj * nd + b] = rows[e];
      else tabE[2 * jj + (b - nd)] = rows[e];
    }
  }
  double wsum = 0.0;
  for (int jj = tid; jj < it.nj; jj += kEThreads) {
    const double wj = flux[it.j0 + jj] * S.dlam;
    tabW[jj] = split_df(wj * 0.25);  // the column and row integrals below are both doubled
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
  for (int q = 0; q < kEWarps; ++q) {
    wtot += s_w[q];
    utot += s_u[q];
  }
  const double total = wtot * utot;
  int ex = 0;
  frexp(total, &ex);
  const int Psh = total > 0.0 ? max(-100, min(100, 52 - ex)) : 0;
  const float sc = ldexpf(1.f, Psh), sc_hi = ldexpf(1.f, Psh - 22);

  const int g = lane / GL, j = lane - g * GL;  // group and column pair (g == NG: spare lane)
  const bool in_group = g < NG;
  const int m0 = 2 * j;                        // the pair's left column
  const bool has_r = in_group && m0 + 1 < K;   // the pair has a right column
  const int gidx = warp * NG + (in_group ? g : 0);
  int4* gst = stage + gidx * 16;
  float2* gcs = cser + gidx * kGlKmax;
  float2 acc[K];  // window row n of the left (.x) and right (.y) column
  // the groups of a warp take samples kEWarps apart, so their columns rarely share a box pixel
  const int n_rounds = (it.nj + kEWarps * NG - 1) / (kEWarps * NG);
  for (int round = 0; round < n_rounds && total > 0.0; ++round) {
    const int jj = warp + kEWarps * (g + NG * round);
    const bool active = in_group && jj < it.nj;  // uniform over the group
    if (active) {
      // map the run's stamps (double-float, as the planner), lane j taking b = j, j + GL, ...
      for (int b = j; b < it.nk; b += GL) {
        int ci, ri;
        float fx, fy;
        map_stamp_df(tabP + jj * nd, S.degree, tabS[b], ci, fx, ri, fy);
        gst[b] = make_int4(ci, ri, __float_as_int(fx), __float_as_int(fy));
      }
      // the sample's series constants c_k = -(2 / sqrt(2 pi)) eps_c^k / k! of the left
      // (eps_c = -eps, moments mirrored) and right (eps_c = eps) column, k = 1..kGlKmax
      const float eps = tabE[2 * jj + 1].z;
      for (int k = j + 1; k <= kGlKmax; k += GL) {
        float p = kTwoOverSqrt2Pi;
        for (int i = 1; i <= k; ++i) p *= eps / (float)i;
        gcs[k - 1] = f2((k & 1) ? p : -p, -p);
      }
    }
    __syncwarp();
    float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0;
    float2 wj = make_float2(0.f, 0.f);
    if (active) {
      e0 = tabE[2 * jj];
      e1 = tabE[2 * jj + 1];
      wj = tabW[jj];
    }
    int cx = kOffFrame, cy = kOffFrame;  // origin of the stamps held in acc (uniform over the group)
#pragma unroll
    for (int n = 0; n < K; ++n) acc[n] = f2(0.f, 0.f);
    auto flush = [&]() {
      const int bx = cx - H + m0 - it.bx0, by0 = cy - H - it.by0;
      const bool inl = in_group && bx >= 0 && bx < it.bw, inr = has_r && bx + 1 >= 0 && bx + 1 < it.bw;
#pragma unroll
      for (int n = 0; n < K; ++n) {
        const int by = by0 + n;
        const bool rowin = by >= 0 && by < it.bh;
        const int q = by * it.bw + bx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float v = h ? acc[n].y : acc[n].x;
          if ((h ? inr : inl) && rowin) {
            box_deposit(boxh + q + h, boxl + q + h, v, sc, sc_hi);
          } else if (a.err && v != 0.f) {  // outside the box: legitimate only off the detector
            const int X = it.bx0 + bx + h, Y = it.by0 + by;
            if (X >= 0 && X < S.W && Y >= 0 && Y < S.H) atomicAdd(a.err, 1);
          }
        }
        acc[n] = f2(0.f, 0.f);
      }
    };
    for (int b = 0; b < it.nk; ++b) {
      const int4 st = active ? gst[b] : make_int4(kOffFrame, kOffFrame, 0, 0);
      const bool valid = st.x != kOffFrame && st.y != kOffFrame;
      if (valid && (st.x != cx || st.y != cy)) {
        if (cx != kOffFrame) flush();
        cx = st.x;
        cy = st.y;
      }
      const float2 uk = tabU[b];
      const float w = valid && in_group ? fmaf(wj.x, uk.x, fmaf(wj.x, uk.y, wj.y * uk.x)) : 0.f;
      const float fx = __int_as_float(st.z), fy = __int_as_float(st.w);

      // twice the x-integrals of columns 2j and 2j + 1 from x-edges 2j, 2j + 1 (this lane,
      // packed) and 2j + 2 (the next lane), times the stamp's weight
      float2 wq;
      {
        float2 wxh, wxl;
        edge_arg2(f2((float)(m0 - H) - 0.5f, (float)(m0 - H) + 0.5f), fx, e0.x, e0.y, wxh, wxl);
        const float2 EX = tail2x2(wxh, wxl);
        float2 FX = f2(1.f - EX.x, 1.f - EX.y);
        const bool n0 = fabsf(wxh.x) < kErfMaxArg, n1 = fabsf(wxh.y) < kErfMaxArg;
        if (n0 || n1) {
          const float2 fe = erf_small2(wxh);
          FX = f2(n0 ? fe.x : FX.x, n1 ? fe.y : FX.y);
        }
        const float E2 = __shfl_down_sync(0xffffffffu, EX.x, 1), F2 = __shfl_down_sync(0xffffffffu, FX.x, 1);
        wq = f2(w * column_x<H>(m0, EX.x, FX.x, EX.y, FX.y),
                has_r ? w * column_x<H>(m0 + 1, EX.y, FX.y, E2, F2) : 0.f);
      }

      // the pair's centre offset tp = (2j - H + 1/2) - fx as a double-float (Fast2Sum:
      // |2j - H + 1/2| >= 1/2 >= |fx|)
      const float ep = (float)(m0 - H) + 0.5f;
      const float th = ep - fx;
      const float tl = (ep - th) - fx;

      // moments of u = tau -+ 1/2 (the offset from the pair's centre) on the left / right
      // column under phi_x(tc + tau) / phi_x(tc) = 2^(al (tc tau + tau^2 / 2)), tc = tp -+ 1/2
      // the column's centre, 5-point Gauss-Legendre; the left column's odd moments come out
      // mirrored (s_k (-1)^k), which its series constants absorb
      const float al = e1.w, q2 = 0.5f * al;
      const float2 c0 = f2(al * (th - 0.5f), al * (th + 0.5f));
      float2 s[kGlKmax + 1];
#pragma unroll
      for (int k = 0; k <= kGlKmax; ++k) s[k] = f2(kGlC[k], kGlC[k]);
#define E2E_GL_NODE(T, TSQ, A, B)                                                               \
  {                                                                                             \
    const float2 cl = __fmul2_rn(c0, f2(T, T));                                                 \
    const float2 cc = f2(q2 * TSQ, q2 * TSQ);                                                   \
    const float2 xp = __fadd2_rn(cc, cl), xm = __fadd2_rn(cc, neg2(cl));                        \
    const float2 ep2 = f2(ex2_approx(xp.x), ex2_approx(xp.y)), em2 = f2(ex2_approx(xm.x), ex2_approx(xm.y)); \
    const float2 pa = f2(em2.x, ep2.y), pb = f2(ep2.x, em2.y);                                 \
    _Pragma("unroll") for (int k = 0; k <= kGlKmax; ++k) {                                     \
      s[k] = __ffma2_rn(pa, f2(A[k], A[k]), s[k]);                                              \
      s[k] = __ffma2_rn(pb, f2(B[k], B[k]), s[k]);                                              \
    }                                                                                           \
  }
      E2E_GL_NODE(kGlT0, kGlT0Sq, kGlA0, kGlB0)
      E2E_GL_NODE(kGlT1, kGlT1Sq, kGlA1, kGlB1)
#undef E2E_GL_NODE
      // a_k = c_k s_k / s_0, and G(V) = sum_k a_k He_(k-1)(V) as a polynomial in V
      float2 gc0, gc1, gc2, gc3, gc4, gc5, gc6;
      {
        const float2 r = f2(rcp_approx(s[0].x), rcp_approx(s[0].y));
        float2 av[kGlKmax + 1];
#pragma unroll
        for (int k = 1; k <= kGlKmax; ++k) av[k] = __fmul2_rn(__fmul2_rn(s[k], r), gcs[k - 1]);
        const float2 c3 = f2(3.f, 3.f), c6 = f2(-6.f, -6.f), c10 = f2(-10.f, -10.f), c15 = f2(15.f, 15.f);
        const float2 m15 = f2(-15.f, -15.f), c45 = f2(45.f, 45.f);
        gc0 = __ffma2_rn(av[7], m15, __ffma2_rn(av[5], c3, __fadd2_rn(av[1], neg2(av[3]))));
        gc1 = __ffma2_rn(av[6], c15, __ffma2_rn(av[4], f2(-3.f, -3.f), av[2]));
        gc2 = __ffma2_rn(av[7], c45, __ffma2_rn(av[5], c6, av[3]));
        gc3 = __ffma2_rn(av[6], c10, av[4]);
        gc4 = __ffma2_rn(av[7], m15, av[5]);
        gc5 = av[6];
        gc6 = av[7];
      }
      // conditional centre of the pair relative to the window centre: f = fy + beta tp (double-float)
      float fh, fl;
      {
        const float bh = e1.x, bl = e1.y;
        const float ph = bh * th;
        const float pl = fmaf(bh, th, -ph) + fmaf(bh, tl, bl * th);
        float se;
        two_sum(fy, ph, fh, se);
        fl = se + pl;
      }
      const float gch = e0.z, gcl = e0.w;
      // f = fc + ff, fc on a 2^-19 grid (exact split), ff g_ch in FP32
      const float fc = rintf(fh * 524288.f) * (1.f / 524288.f);
      const float ffg = ((fh - fc) + fl) * gch;
      // the K + 1 row edges in pairs (n, n + 1), shared by both columns; pixel n spans edges n and n + 1
      float Ep = 0.f, Fp = 0.f, whp = 0.f;
      float2 hp = f2(0.f, 0.f);
#pragma unroll
      for (int n = 0; n <= K; n += 2) {
        // w = (e - f) g_c for the half-integers e = n - H -+ 1/2: e - fc exact, its product with
        // g_ch exact as a pair, the small terms added to the low part; wn = fl(w)
        const float2 dc = __fadd2_rn(f2((float)(n - H) - 0.5f, (float)(n - H) + 0.5f), f2(-fc, -fc));
        const float2 gg = f2(gch, gch);
        const float2 wh = __fmul2_rn(dc, gg);
        const float2 wl = __fadd2_rn(__ffma2_rn(dc, gg, neg2(wh)), __ffma2_rn(dc, f2(gcl, gcl), f2(-ffg, -ffg)));
        const float2 wn = __fadd2_rn(wh, wl);
        // tails only off the conditional centre (a near edge's tail is never read), erf only near
        // it; each skipped when no lane of the warp needs it
        const bool near0 = fabsf(wn.x) < kErfMaxArg, near1 = fabsf(wn.y) < kErfMaxArg;
        float2 dens, E = f2(0.f, 0.f);
        if (__any_sync(0xffffffffu, !(near0 && near1)))
          E = tail2x2_dens_n(wh, wl, wn, dens);
        else
          dens = dens2x2(wh, wl);
        float2 F = f2(1.f - E.x, 1.f - E.y);
        if (__any_sync(0xffffffffu, near0 || near1)) {
          const float2 fe = erf_small2(wn);
          F = f2(near0 ? fe.x : F.x, near1 ? fe.y : F.y);
        }
        const float2 V = __fmul2_rn(wn, f2(kSqrt2Ln2, kSqrt2Ln2));
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int ne = n + e;
          const float Ee = e ? E.y : E.x, Fe = e ? F.y : F.x, we = e ? wn.y : wn.x;
          const float2 Vb = e ? f2(V.y, V.y) : f2(V.x, V.x);
          float2 G = __ffma2_rn(gc6, Vb, gc5);
          G = __ffma2_rn(G, Vb, gc4);
          G = __ffma2_rn(G, Vb, gc3);
          G = __ffma2_rn(G, Vb, gc2);
          G = __ffma2_rn(G, Vb, gc1);
          G = __ffma2_rn(G, Vb, gc0);
          const float de = e ? dens.y : dens.x;
          const float2 h = __fmul2_rn(f2(de, de), G);
          if (ne > 0 && ne <= K) {
            // tails subtracted on one side of the conditional centre (erf near it), erf summed
            // across it; the pair's two columns share this and differ in the series term
            const bool same = (we < 0.f) == (whp < 0.f);
            const bool small = fminf(fabsf(we), fabsf(whp)) < kErfMaxArg;
            const float pa = same && !small ? Ep : Fp;
            const float pb = same ? (small ? Fe : Ee) : -Fe;
            const float t = fabsf(pa - pb);
            acc[ne - 1] = __ffma2_rn(wq, __fadd2_rn(f2(t, t), __fadd2_rn(h, neg2(hp))), acc[ne - 1]);
          }
          Ep = Ee;
          Fp = Fe;
          hp = h;
          whp = we;
        }
      }
    }
    if (cx != kOffFrame) flush();
    __syncwarp();  // the staging is reused by the next round
  }
  __syncthreads();
  float2* out = a.store + it.store_off;
  const float inv = ldexpf(1.f, -Psh);
  for (int p = tid; p < area; p += kEThreads) out[p] = fixed_to_pair(boxh[p], boxl[p], inv);
}

size_t ellip_smem_bytes(int area, int nk_max, int nd, int k_min) {
  return EllipLayout(32, nk_max, nd, area, k_min).total;
}

template <int K>
static cudaError_t launch_ellip_one(const MixedArgs& a, int n_items, size_t smem, cudaStream_t st) {
  auto kern = k_render_ellip<K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_items, kEThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_render_ellip(int K, const DevSlice* slices, const double* const* flux_tab, const double* u_all,
                                const Item* items, int n_items, float2* store, int nk_max, int max_deg, size_t smem,
                                cudaStream_t st, int* err) {
  if (n_items == 0) return cudaSuccess;
  MixedArgs a{slices, flux_tab, u_all, items, store, 0, 1, nk_max, max_deg, err};
  switch (K) {
#define E2E_CASE(KK) \
  case KK: return launch_ellip_one<KK>(a, n_items, smem, st);
    E2E_CASE(1) E2E_CASE(3) E2E_CASE(5) E2E_CASE(7) E2E_CASE(9) E2E_CASE(11) E2E_CASE(13) E2E_CASE(15)
#undef E2E_CASE
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------------------ FP64

// P(a < Z < b) for a standard normal Z from E = erfc(|t| / sqrt2) at both ends (tails
// subtracted on one side of the mean, 1 minus both tails across it).
__device__ __forceinline__ double interval_e(double ta, double tb, double ea, double eb) {
  if (ta >= 0.0) return 0.5 * (ea - eb);
  if (tb <= 0.0) return 0.5 * (eb - ea);
  return 1.0 - 0.5 * (ea + eb);
}

// One thread per (stamp, window column), all in FP64: mapping, erfc, exp, 12-point
// Gauss-Legendre moments, the series to k = 9, FP64 atomic deposits into the frame.
template <int K>
__global__ void __launch_bounds__(256) k_render_fp64_ellip(const DevSlice* __restrict__ slices,
                                                           const double* const* __restrict__ flux_tab,
                                                           const double* __restrict__ u_all, double* const* acc,
                                                           const int64_t* __restrict__ pitch) {
  constexpr int NT = 10;  // a_1 .. a_9
  const DevSlice& S = slices[blockIdx.y];
  if (S.K != K) return;
  const double* flux = flux_tab[S.flux_slot];
  const double* u = u_all + S.u_off;
  const int64_t n = (int64_t)S.n_lambda * S.n_slit * K;
  double* frame = acc[S.det];
  const int64_t P = pitch[S.det];
  const double r2 = 0.70710678118654752440, rs2pi = 0.39894228040143267794;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t stamp = idx / K;
    const int m = (int)(idx - stamp * K);
    const int j = (int)(stamp / S.n_slit);
    const int k = (int)(stamp - (int64_t)j * S.n_slit);
    const double lt = norm_sample(j, S.n_lambda);
    const double s = norm_sample(k, S.n_slit);
    double x = 0.0, y = 0.0;
    for (int b = S.degree; b >= 0; --b) {
      x = fma(x, s, poly_lt_for_b(S.cx, S.degree, b, lt));
      y = fma(y, s, poly_lt_for_b(S.cy, S.degree, b, lt));
    }
    x = clamp_coord(x);
    y = clamp_coord(y);
    const int i0 = (int)floor(x + 0.5) - K / 2;
    const int r0 = (int)floor(y + 0.5) - K / 2;
    const int i = i0 + m;
    if (i < 0 || i >= S.W || r0 + K <= 0 || r0 >= S.H) continue;
    const EllipParams p = ellip_params(S, lt);
    const double w = flux[j] * S.dlam * u[k];
    const double tb = (double)i - x;
    const double ta = (tb - 0.5) / p.gx, tc = (tb + 0.5) / p.gx;
    const double mu0 = interval_e(ta, tc, erfc(fabs(ta) * r2), erfc(fabs(tc) * r2));
    double mom[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) mom[q] = 0.0;
    for (int q = 0; q < kGl12; ++q) {
      const double t = kGl12T[q];
      const double e = kGl12W[q] * exp(-(tb * t + 0.5 * t * t) / p.vx);
      double tp = e;
#pragma unroll
      for (int kk = 0; kk < NT; ++kk) {
        mom[kk] += tp;
        tp *= t;
      }
    }
    double a[NT];
    {
      double c = 1.0;
      a[0] = 0.0;
#pragma unroll
      for (int kk = 1; kk < NT; ++kk) {
        c *= p.eps / (double)kk;
        a[kk] = -c * mom[kk] / mom[0];
      }
    }
    const double yb = y + p.beta * tb;  // conditional centre of the column
    double Vp = 0.0, Ep = 0.0, hp = 0.0;
    for (int nn = 0; nn <= K; ++nn) {
      const double V = ((double)(r0 + nn) - 0.5 - yb) / p.sc;
      const double E = erfc(fabs(V) * r2);
      // G(V) = sum_k a_k He_(k-1)(V) by the Hermite recurrence
      double h0 = 1.0, h1 = V, G = a[1] + a[2] * V;
#pragma unroll
      for (int kk = 3; kk < NT; ++kk) {
        const double h2 = V * h1 - (double)(kk - 2) * h0;
        G = fma(a[kk], h2, G);
        h0 = h1;
        h1 = h2;
      }
      const double h = rs2pi * exp(-0.5 * V * V) * G;
      if (nn > 0) {
        const int r = r0 + nn - 1;
        if (r >= 0 && r < S.H) atomicAdd(frame + (int64_t)r * P + i, w * mu0 * (interval_e(Vp, V, Ep, E) + h - hp));
      }
      Vp = V;
      Ep = E;
      hp = h;
    }
  }
}

cudaError_t launch_render_fp64_ellip(int K, int n_slices, int64_t max_stamps, const DevSlice* slices,
                                     const double* const* flux_tab, const double* u_all, double* const* acc,
                                     const int64_t* pitch, cudaStream_t st) {
  if (n_slices == 0 || max_stamps == 0) return cudaSuccess;
  int64_t bx = (max_stamps * K + 255) / 256;
  if (bx > 8192) bx = 8192;
  dim3 grid((unsigned)bx, (unsigned)n_slices);
  switch (K) {
#define E2E_CASE(KK) \
  case KK: k_render_fp64_ellip<KK><<<grid, 256, 0, st>>>(slices, flux_tab, u_all, acc, pitch); break;
    E2E_CASE(1) E2E_CASE(3) E2E_CASE(5) E2E_CASE(7) E2E_CASE(9) E2E_CASE(11) E2E_CASE(13) E2E_CASE(15)
#undef E2E_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace e2e
