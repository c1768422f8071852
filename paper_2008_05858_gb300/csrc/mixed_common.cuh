// Device helpers shared by the mixed-precision renderers (separable and elliptical PSF):
// exact-split FP32 pairs, the fixed-point box format and the kernel argument block.
#pragma once
#include "e2e_device.cuh"

namespace e2e {

// Normalised coordinate of bin-centred sample j of n, (2j + 1 - n) / n, as a product with the
// correctly rounded reciprocal (the plan and the render compute it identically).
__device__ __forceinline__ double norm_sample_r(int j, int n, double inv_n) { return (double)(2 * j + 1 - n) * inv_n; }

struct MixedArgs {
  const DevSlice* slices;
  const double* const* flux_tab;
  const double* u_all;
  const Item* items;
  float2* store;
  int B;        // slit points per run
  int JB;       // largest number of 32-sample blocks in an item
  int nk_max;   // largest number of slit points in an item
  int max_deg;  // largest degree among the launched slices
  int* err;     // debug checks: counts deposits the plan did not foresee (nullptr = off)
  int far_tails;  // separable kernel: the cheaper rational on the tail edges (>= 1 px from the centre)
};

// 16-byte asynchronous copy from global to shared memory (cp.async, bypassing L1); both
// addresses 16-byte aligned.  Completed by cp_async_wait_all in the issuing thread.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ float2 split_df(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// a + b as an unevaluated pair (s, e), s = fl(a + b), a + b = s + e exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi * 2^22 + lo) * scale as an FP32 pair (h, l) with h + l exact to ~2^-48: the 54-bit
// integer is cut into four 16-bit pieces (each exact in FP32) and summed with TwoSum.
__device__ __forceinline__ float2 fixed_to_pair(int hi, unsigned lo, float scale) {
  const float t1 = (float)(hi >> 16) * 274877906944.f;  // 2^38
  const float t2 = (float)(hi & 0xFFFF) * 4194304.f;    // 2^22
  const float t3 = (float)(lo >> 16) * 65536.f;         // 2^16
  const float t4 = (float)(lo & 0xFFFFu);
  float s, e, e2;
  two_sum(t1, t2, s, e);
  two_sum(s, t3, s, e2);
  e += e2;
  two_sum(s, t4, s, e2);
  e += e2;
  return make_float2(s * scale, e * scale);
}

// Fixed-point deposit of val into a box pixel: the value scaled by 2^P is cut into a high
// word (multiples of 2^22, signed) and a low word (< 2^22, unsigned), both added with
// integer atomics, so the sums are exact and independent of the order of the deposits.
__device__ __forceinline__ void box_deposit(int* hi, unsigned* lo, float val, float sc, float sc_hi) {
  const float hf = floorf(val * sc_hi);
  const float lf = fmaf(-hf, 4194304.f, val * sc);
  atomicAdd(hi, __float2int_rz(hf));
  atomicAdd(lo, __float2uint_rn(lf));
}

// ---- the stamp mapping of the mixed-precision kernels and their planner, in double-float
// FP32 arithmetic (x and y together, packed FP32x2): FP64 runs at 1/64 of the FP32 rate on
// this part, and a double-float (~48 significant bits) keeps the mapped centre within
// ~1e-10 px at 9216 px.  The planner and every mixed kernel call these same functions, so
// they agree on every window origin.

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// The coefficients P_b(lt) of x and y of one wavelength sample, as (xh, yh, xl, yl).
__device__ __forceinline__ float4 split_xy(double px, double py) {
  const float xh = (float)px, yh = (float)py;
  return make_float4(xh, yh, (float)(px - (double)xh), (float)(py - (double)yh));
}

// v = h + l (|l| <= ulp(h)/2) split into the window-centre pixel c = floor(v + 1/2) and the
// offset f = v - c in [-1/2, 1/2), rounded to FP32; |v| >= 2^15 px or not finite: kOffFrame.
__device__ __forceinline__ void split_coord_df(float h, float l, int& c, float& f) {
  if (!(fabsf(h) < 32768.f)) {
    c = kOffFrame;
    f = 0.f;
    return;
  }
  const int ci = __float2int_rd(h + 0.5f);  // within one of floor(v + 1/2)
  const float f0 = h - (float)ci;            // exact: |h - ci| <= 1
  float fr = f0 + l;
  int cc = ci;
  if (fr < -0.5f) {
    cc = ci - 1;
    fr = (f0 + 1.f) + l;
  } else if (fr >= 0.5f) {
    cc = ci + 1;
    fr = (f0 - 1.f) + l;
  }
  c = cc;
  f = fr;
}

// Horner in s = (sh, sl) over P[b] = split_xy(P_b of x, P_b of y), b = 0..d: the stamp's x and
// y as double-floats, each step a double-float product (FMA error terms) and a TwoSum.
__device__ __forceinline__ void map_xy_df(const float4* P, int d, float2 s, float2& hi, float2& lo) {
  float4 c = P[d];
  float2 qh = make_float2(c.x, c.y), ql = make_float2(c.z, c.w);
  const float2 sh = make_float2(s.x, s.x), sl = make_float2(s.y, s.y);
  for (int b = d - 1; b >= 0; --b) {
    const float2 ph = __fmul2_rn(qh, sh);
    float2 pe = __ffma2_rn(qh, sh, neg2(ph));
    pe = __ffma2_rn(qh, sl, pe);
    pe = __ffma2_rn(ql, sh, pe);
    c = P[b];
    const float2 bh = make_float2(c.x, c.y), bl = make_float2(c.z, c.w);
    const float2 t = __fadd2_rn(ph, bh);
    const float2 bb = __fadd2_rn(t, neg2(ph));
    const float2 e = __fadd2_rn(__fadd2_rn(ph, neg2(__fadd2_rn(t, neg2(bb)))), __fadd2_rn(bh, neg2(bb)));
    const float2 e2 = __fadd2_rn(e, __fadd2_rn(pe, bl));
    qh = __fadd2_rn(t, e2);
    ql = __fadd2_rn(e2, neg2(__fadd2_rn(qh, neg2(t))));
  }
  hi = qh;
  lo = ql;
}

// map_xy_df for coefficients held in registers (P[0..d], d <= 8): the loop unrolled over
// b = 8..0 with every index static, doing exactly map_xy_df's operations.
__device__ __forceinline__ void map_xy_df_regs(const float4 (&P)[9], int d, float2 s, float2& hi, float2& lo) {
  float2 qh = make_float2(0.f, 0.f), ql = qh;
  const float2 sh = make_float2(s.x, s.x), sl = make_float2(s.y, s.y);
#pragma unroll
  for (int b = 8; b >= 0; --b) {
    if (b == d) {
      qh = make_float2(P[b].x, P[b].y);
      ql = make_float2(P[b].z, P[b].w);
    } else if (b < d) {
      const float2 ph = __fmul2_rn(qh, sh);
      float2 pe = __ffma2_rn(qh, sh, neg2(ph));
      pe = __ffma2_rn(qh, sl, pe);
      pe = __ffma2_rn(ql, sh, pe);
      const float2 bh = make_float2(P[b].x, P[b].y), bl = make_float2(P[b].z, P[b].w);
      const float2 t = __fadd2_rn(ph, bh);
      const float2 bb = __fadd2_rn(t, neg2(ph));
      const float2 e = __fadd2_rn(__fadd2_rn(ph, neg2(__fadd2_rn(t, neg2(bb)))), __fadd2_rn(bh, neg2(bb)));
      const float2 e2 = __fadd2_rn(e, __fadd2_rn(pe, bl));
      qh = __fadd2_rn(t, e2);
      ql = __fadd2_rn(e2, neg2(__fadd2_rn(qh, neg2(t))));
    }
  }
  hi = qh;
  lo = ql;
}

// map_xy_df for N slit coordinates at once: one coefficient load per step for all N, the N
// Horner chains interleaved for instruction-level parallelism; per coordinate exactly
// map_xy_df's operations, so the same bits.
template <int N>
__device__ __forceinline__ void map_xy_df_n(const float4* P, int d, const float2 (&s)[N], float2 (&hi)[N],
                                            float2 (&lo)[N]) {
  float4 c = P[d];
  float2 qh[N], ql[N];
#pragma unroll
  for (int n = 0; n < N; ++n) {
    qh[n] = make_float2(c.x, c.y);
    ql[n] = make_float2(c.z, c.w);
  }
  for (int b = d - 1; b >= 0; --b) {
    c = P[b];
    const float2 bh = make_float2(c.x, c.y), bl = make_float2(c.z, c.w);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const float2 sh = make_float2(s[n].x, s[n].x), sl = make_float2(s[n].y, s[n].y);
      const float2 ph = __fmul2_rn(qh[n], sh);
      float2 pe = __ffma2_rn(qh[n], sh, neg2(ph));
      pe = __ffma2_rn(qh[n], sl, pe);
      pe = __ffma2_rn(ql[n], sh, pe);
      const float2 t = __fadd2_rn(ph, bh);
      const float2 bb = __fadd2_rn(t, neg2(ph));
      const float2 e = __fadd2_rn(__fadd2_rn(ph, neg2(__fadd2_rn(t, neg2(bb)))), __fadd2_rn(bh, neg2(bb)));
      const float2 e2 = __fadd2_rn(e, __fadd2_rn(pe, bl));
      qh[n] = __fadd2_rn(t, e2);
      ql[n] = __fadd2_rn(e2, neg2(__fadd2_rn(qh[n], neg2(t))));
    }
  }
#pragma unroll
  for (int n = 0; n < N; ++n) {
    hi[n] = qh[n];
    lo[n] = ql[n];
  }
}

// Window-centre pixels and FP32 offsets of a stamp (map_xy_df, then split_coord_df).
__device__ __forceinline__ void map_stamp_df(const float4* P, int d, float2 s, int& ci, float& fx, int& ri,
                                             float& fy) {
  float2 hi, lo;
  map_xy_df(P, d, s, hi, lo);
  split_coord_df(hi.x, lo.x, ci, fx);
  split_coord_df(hi.y, lo.y, ri, fy);
}

// Covariance of the rotated PSF at lt and the conditional parameters derived from it.
struct EllipParams {
  double vx, gx, beta, sc, eps;
};

__device__ __forceinline__ EllipParams ellip_params(const DevSlice& S, double lt) {
  const double sa = fma(fma(S.sx[2], lt, S.sx[1]), lt, S.sx[0]);
  const double sb = fma(fma(S.sy[2], lt, S.sy[1]), lt, S.sy[0]);
  const double a2 = sa * sa, b2 = sb * sb, c = S.cos_t, s = S.sin_t;
  EllipParams p;
  p.vx = a2 * c * c + b2 * s * s;
  const double vy = a2 * s * s + b2 * c * c;
  const double cxy = (a2 - b2) * s * c;
  p.gx = sqrt(p.vx);
  p.beta = cxy / p.vx;
  p.sc = sqrt(vy - p.beta * cxy);
  p.eps = p.beta / p.sc;
  return p;
}

// Field node pair and weight of normalised wavelength lt (the end node beyond the ends).
__device__ __forceinline__ void field_weight(const double* lt_nodes, int F, double lt, int& f0, int& f1, double& wf) {
  f0 = 0;
  f1 = 0;
  wf = 0.0;
  if (lt <= lt_nodes[0]) return;
  if (lt >= lt_nodes[F - 1]) {
    f0 = f1 = F - 1;
    return;
  }
  while (f0 + 1 < F && lt_nodes[f0 + 1] <= lt) ++f0;
  f1 = f0 + 1;
  wf = (lt - lt_nodes[f0]) / (lt_nodes[f1] - lt_nodes[f0]);
}

// box_deposit's fixed-point words of two values at once: the same operations on each
// component (packed FP32x2 for the multiplies and the FMA), so the same words.
__device__ __forceinline__ void fixed_split2(float2 val, float sc, float sc_hi, int2& hi, uint2& lo) {
  const float2 t = __fmul2_rn(val, make_float2(sc_hi, sc_hi));
  const float2 hf = make_float2(floorf(t.x), floorf(t.y));
  const float2 lf = __ffma2_rn(hf, make_float2(-4194304.f, -4194304.f), __fmul2_rn(val, make_float2(sc, sc)));
  hi = make_int2(__float2int_rz(hf.x), __float2int_rz(hf.y));
  lo = make_uint2(__float2uint_rn(lf.x), __float2uint_rn(lf.y));
}

}  // namespace e2e
