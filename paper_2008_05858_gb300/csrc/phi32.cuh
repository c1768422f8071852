// FP32 Gaussian tail for a double-float argument, in log2 units.
//
// A stamp's pixel integrals are differences of the normal CDF at the pixel edges (the
// pixel-integrated PSF of Sec. 2.2).  In FP32 an edge argument carries a relative error of
// ~1e-7, which the factor exp(-a^2) amplifies by 2a^2 (1e-6 at a = 2), so the kernels keep
// the argument as a double-float and form the exponent exactly.  The argument is scaled by
// sqrt(log2 e): with w = a sqrt(log2 e),
//
//   erfc(a) = 2^(-w^2) * erfcx(w / sqrt(log2 e)),
//   w^2 = p + e exactly to ~2^-48 (FMA error terms), 2^(-p) on the SFU (ex2.approx,
//   2.4 ulp measured), 2^(-e) ~= 1 - e ln2 (|e| < 1e-5),
//   erfcx by the rational P4/Q5 of tail_coeffs.h (fit error 2e-9; rcp.approx on the SFU).
//
// Worst-case relative error is a few FP32 ulp for every a, independent of a (no 2a^2
// amplification); the test-suite checks it against CUDA's FP64 erfc on the GPU.
#pragma once
#include "tail_coeffs.h"

namespace e2e {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// erfc(|w| / sqrt(log2 e)) for w = wh + wl, |wl| <= a few ulp(wh).
__device__ __forceinline__ float tail2(float wh, float wl) {
  const float p = wh * wh;
  float e = fmaf(wh, wh, -p);      // exact error of p
  e = fmaf(wh + wh, wl, e);        // + 2 wh wl  (wl^2 negligible)
  const float ex = ex2_approx(-p) * fmaf(e, -0.693147181f, 1.f);
  const float x = fminf(fabsf(wh), 40.f);
  float P = kTailP4;
  P = fmaf(P, x, kTailP3);
  P = fmaf(P, x, kTailP2);
  P = fmaf(P, x, kTailP1);
  P = fmaf(P, x, kTailP0);
  float Q = kTailQ5;
  Q = fmaf(Q, x, kTailQ4);
  Q = fmaf(Q, x, kTailQ3);
  Q = fmaf(Q, x, kTailQ2);
  Q = fmaf(Q, x, kTailQ1);
  Q = fmaf(Q, x, kTailQ0);
  return (ex * P) * rcp_approx(Q);
}

// tail2 with the cheaper rational PF3/QF4 of tail_coeffs.h, for |w| >= kTailFarMinArg (fit
// error 4.9e-8 there): the tail edges (one or more pixels from a stamp's centre), when the
// model's widest PSF keeps their arguments in that range.
__device__ __forceinline__ float tail2_far(float wh, float wl) {
  const float p = wh * wh;
  float e = fmaf(wh, wh, -p);
  e = fmaf(wh + wh, wl, e);
  const float ex = ex2_approx(-p) * fmaf(e, -0.693147181f, 1.f);
  const float x = fminf(fabsf(wh), 40.f);
  float P = kTailFarP3;
  P = fmaf(P, x, kTailFarP2);
  P = fmaf(P, x, kTailFarP1);
  P = fmaf(P, x, kTailFarP0);
  float Q = kTailFarQ4;
  Q = fmaf(Q, x, kTailFarQ3);
  Q = fmaf(Q, x, kTailFarQ2);
  Q = fmaf(Q, x, kTailFarQ1);
  Q = fmaf(Q, x, kTailFarQ0);
  return (ex * P) * rcp_approx(Q);
}

// As tail2, also returning 2^(-w^2) = exp(-a^2) (the Gaussian density up to a constant).
__device__ __forceinline__ float tail2_dens(float wh, float wl, float& dens) {
  const float p = wh * wh;
  float e = fmaf(wh, wh, -p);
  e = fmaf(wh + wh, wl, e);
  const float ex = ex2_approx(-p) * fmaf(e, -0.693147181f, 1.f);
  dens = ex;
  const float x = fminf(fabsf(wh), 40.f);
  float P = kTailP4;
  P = fmaf(P, x, kTailP3);
  P = fmaf(P, x, kTailP2);
  P = fmaf(P, x, kTailP1);
  P = fmaf(P, x, kTailP0);
  float Q = kTailQ5;
  Q = fmaf(Q, x, kTailQ4);
  Q = fmaf(Q, x, kTailQ3);
  Q = fmaf(Q, x, kTailQ2);
  Q = fmaf(Q, x, kTailQ1);
  Q = fmaf(Q, x, kTailQ0);
  return (ex * P) * rcp_approx(Q);
}

// erf(|w| / sqrt(log2 e)) for |w| <= kErfMaxArg (odd polynomial, fit error 5e-9): near the window
// centre the pixel integrals are sums and differences of erf, which do not cancel there the
// way differences of erfc values close to 1 do.
__device__ __forceinline__ float erf_small(float w) {
  const float a = fabsf(w);
  const float z = a * a;
  float S = kErfS5;
  S = fmaf(S, z, kErfS4);
  S = fmaf(S, z, kErfS3);
  S = fmaf(S, z, kErfS2);
  S = fmaf(S, z, kErfS1);
  S = fmaf(S, z, kErfS0);
  return a * S;
}

// Edge argument as a double-float: w = (e - f) * g with e a half-integer (exact), f the
// FP32 sub-pixel offset, g = gh + gl.  e - f is split exactly (|e| >= 1/2 >= |f|, so
// Fast2Sum applies); the product keeps its FMA error term.
__device__ __forceinline__ void edge_arg(float e, float f, float gh, float gl, float& wh, float& wl) {
  const float dh = e - f;
  const float dl = (e - dh) - f;
  wh = dh * gh;
  wl = fmaf(dh, gh, -wh) + fmaf(dh, gl, dl * gh);
}

// ---- the same functions on two arguments at once (packed FP32x2 arithmetic, sm_100+: one
// issue slot for two lanes' worth of FMAs); per component the arithmetic is the scalar
// functions' own, operation by operation, so the results are the same bits.

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// tail2 of (wh.x, wl.x) and (wh.y, wl.y).
__device__ __forceinline__ float2 tail2x2(float2 wh, float2 wl) {
  const float2 p = __fmul2_rn(wh, wh);
  float2 e = __ffma2_rn(wh, wh, f2(-p.x, -p.y));
  e = __ffma2_rn(__fadd2_rn(wh, wh), wl, e);
  const float2 ex = __fmul2_rn(f2(ex2_approx(-p.x), ex2_approx(-p.y)),
                               __ffma2_rn(e, f2(-0.693147181f, -0.693147181f), f2(1.f, 1.f)));
  const float2 x = f2(fminf(fabsf(wh.x), 40.f), fminf(fabsf(wh.y), 40.f));
  float2 P = f2(kTailP4, kTailP4);
  P = __ffma2_rn(P, x, f2(kTailP3, kTailP3));
  P = __ffma2_rn(P, x, f2(kTailP2, kTailP2));
  P = __ffma2_rn(P, x, f2(kTailP1, kTailP1));
  P = __ffma2_rn(P, x, f2(kTailP0, kTailP0));
  float2 Q = f2(kTailQ5, kTailQ5);
  Q = __ffma2_rn(Q, x, f2(kTailQ4, kTailQ4));
  Q = __ffma2_rn(Q, x, f2(kTailQ3, kTailQ3));
  Q = __ffma2_rn(Q, x, f2(kTailQ2, kTailQ2));
  Q = __ffma2_rn(Q, x, f2(kTailQ1, kTailQ1));
  Q = __ffma2_rn(Q, x, f2(kTailQ0, kTailQ0));
  return __fmul2_rn(__fmul2_rn(ex, P), f2(rcp_approx(Q.x), rcp_approx(Q.y)));
}

// tail2x2 of arguments whose low parts come doubled (wl2 = 2 wl, exactly): the same
// operations with the doubling of wh folded into the argument.
__device__ __forceinline__ float2 tail2x2_w2(float2 wh, float2 wl2) {
  const float2 p = __fmul2_rn(wh, wh);
  float2 e = __ffma2_rn(wh, wh, f2(-p.x, -p.y));
  e = __ffma2_rn(wh, wl2, e);
  const float2 ex = __fmul2_rn(f2(ex2_approx(-p.x), ex2_approx(-p.y)),
                               __ffma2_rn(e, f2(-0.693147181f, -0.693147181f), f2(1.f, 1.f)));
  const float2 x = f2(fminf(fabsf(wh.x), 40.f), fminf(fabsf(wh.y), 40.f));
  float2 P = f2(kTailP4, kTailP4);
  P = __ffma2_rn(P, x, f2(kTailP3, kTailP3));
  P = __ffma2_rn(P, x, f2(kTailP2, kTailP2));
  P = __ffma2_rn(P, x, f2(kTailP1, kTailP1));
  P = __ffma2_rn(P, x, f2(kTailP0, kTailP0));
  float2 Q = f2(kTailQ5, kTailQ5);
  Q = __ffma2_rn(Q, x, f2(kTailQ4, kTailQ4));
  Q = __ffma2_rn(Q, x, f2(kTailQ3, kTailQ3));
  Q = __ffma2_rn(Q, x, f2(kTailQ2, kTailQ2));
  Q = __ffma2_rn(Q, x, f2(kTailQ1, kTailQ1));
  Q = __ffma2_rn(Q, x, f2(kTailQ0, kTailQ0));
  return __fmul2_rn(__fmul2_rn(ex, P), f2(rcp_approx(Q.x), rcp_approx(Q.y)));
}

// tail2x2 that also returns 2^(-w^2) of each argument, for an argument held as a pair
// (wh, wl) whose low part may exceed ulp(wh) (|wl| <= ~1e-6 |wh|, so wl^2 stays negligible):
// the exponent is formed from the pair, the rational from wn = fl(wh + wl).
// 2^(-w^2) of two arguments held as pairs (wh, wl), |wl| <= ~1e-6 |wh|: the exponent's square
// formed exactly from the pair, 2^(-p) on the SFU, 2^(-e) ~= 1 - e ln2.
__device__ __forceinline__ float2 dens2x2(float2 wh, float2 wl) {
  const float2 p = __fmul2_rn(wh, wh);
  float2 e = __ffma2_rn(wh, wh, f2(-p.x, -p.y));
  e = __ffma2_rn(__fadd2_rn(wh, wh), wl, e);
  return __fmul2_rn(f2(ex2_approx(-p.x), ex2_approx(-p.y)),
                    __ffma2_rn(e, f2(-0.693147181f, -0.693147181f), f2(1.f, 1.f)));
}

__device__ __forceinline__ float2 tail2x2_dens_n(float2 wh, float2 wl, float2 wn, float2& dens) {
  const float2 ex = dens2x2(wh, wl);
  dens = ex;
  const float2 x = f2(fminf(fabsf(wn.x), 40.f), fminf(fabsf(wn.y), 40.f));
  float2 P = f2(kTailP4, kTailP4);
  P = __ffma2_rn(P, x, f2(kTailP3, kTailP3));
  P = __ffma2_rn(P, x, f2(kTailP2, kTailP2));
  P = __ffma2_rn(P, x, f2(kTailP1, kTailP1));
  P = __ffma2_rn(P, x, f2(kTailP0, kTailP0));
  float2 Q = f2(kTailQ5, kTailQ5);
  Q = __ffma2_rn(Q, x, f2(kTailQ4, kTailQ4));
  Q = __ffma2_rn(Q, x, f2(kTailQ3, kTailQ3));
  Q = __ffma2_rn(Q, x, f2(kTailQ2, kTailQ2));
  Q = __ffma2_rn(Q, x, f2(kTailQ1, kTailQ1));
  Q = __ffma2_rn(Q, x, f2(kTailQ0, kTailQ0));
  return __fmul2_rn(__fmul2_rn(ex, P), f2(rcp_approx(Q.x), rcp_approx(Q.y)));
}

// tail2x2 that also returns 2^(-w^2) of each argument (tail2_dens on two arguments).
__device__ __forceinline__ float2 tail2x2_dens(float2 wh, float2 wl, float2& dens) {
  return tail2x2_dens_n(wh, wl, wh, dens);
}

// erf_small of w.x and w.y.
__device__ __forceinline__ float2 erf_small2(float2 w) {
  const float2 a = f2(fabsf(w.x), fabsf(w.y));
  const float2 z = __fmul2_rn(a, a);
  float2 S = f2(kErfS5, kErfS5);
  S = __ffma2_rn(S, z, f2(kErfS4, kErfS4));
  S = __ffma2_rn(S, z, f2(kErfS3, kErfS3));
  S = __ffma2_rn(S, z, f2(kErfS2, kErfS2));
  S = __ffma2_rn(S, z, f2(kErfS1, kErfS1));
  S = __ffma2_rn(S, z, f2(kErfS0, kErfS0));
  return __fmul2_rn(a, S);
}

// edge_arg of the half-integers e.x and e.y against the same offset f and factor (gh, gl).
__device__ __forceinline__ void edge_arg2(float2 e, float f, float gh, float gl, float2& wh, float2& wl) {
  const float2 ff = f2(f, f), g = f2(gh, gh);
  const float2 dh = __fadd2_rn(e, f2(-f, -f));
  const float2 dl = __fadd2_rn(__fadd2_rn(e, f2(-dh.x, -dh.y)), f2(-ff.x, -ff.y));
  wh = __fmul2_rn(dh, g);
  wl = __fadd2_rn(__ffma2_rn(dh, g, f2(-wh.x, -wh.y)), __ffma2_rn(dh, f2(gl, gl), __fmul2_rn(dl, g)));
}

// tail2x2_w2 with the cheaper rational (tail2_far on two arguments, per component the same
// operations as tail2_far).
__device__ __forceinline__ float2 tail2x2_w2_far(float2 wh, float2 wl2) {
  const float2 p = __fmul2_rn(wh, wh);
  float2 e = __ffma2_rn(wh, wh, f2(-p.x, -p.y));
  e = __ffma2_rn(wh, wl2, e);
  const float2 ex = __fmul2_rn(f2(ex2_approx(-p.x), ex2_approx(-p.y)),
                               __ffma2_rn(e, f2(-0.693147181f, -0.693147181f), f2(1.f, 1.f)));
  const float2 x = f2(fminf(fabsf(wh.x), 40.f), fminf(fabsf(wh.y), 40.f));
  float2 P = f2(kTailFarP3, kTailFarP3);
  P = __ffma2_rn(P, x, f2(kTailFarP2, kTailFarP2));
  P = __ffma2_rn(P, x, f2(kTailFarP1, kTailFarP1));
  P = __ffma2_rn(P, x, f2(kTailFarP0, kTailFarP0));
  float2 Q = f2(kTailFarQ4, kTailFarQ4);
  Q = __ffma2_rn(Q, x, f2(kTailFarQ3, kTailFarQ3));
  Q = __ffma2_rn(Q, x, f2(kTailFarQ2, kTailFarQ2));
  Q = __ffma2_rn(Q, x, f2(kTailFarQ1, kTailFarQ1));
  Q = __ffma2_rn(Q, x, f2(kTailFarQ0, kTailFarQ0));
  return __fmul2_rn(__fmul2_rn(ex, P), f2(rcp_approx(Q.x), rcp_approx(Q.y)));
}

// Offset split for edge arguments: f = fh + fl with fh on the 2^-20 grid (a magic-number
// rounding: f + 12 lies in [8, 16), where the FP32 spacing is 2^-20), so that e - fh is exact
// for every half-integer |e| <= 15/2 (|e - fh| <= 8 needs at most 23 bits) and fl = f - fh is
// exact too (|fl| <= 2^-21).
__device__ __forceinline__ void split_offset(float f, float& fh, float& fl) {
  fh = __fsub_rn(__fadd_rn(f, 12.f), 12.f);
  fl = __fsub_rn(f, fh);
}

// Edge arguments of the half-integers e.x and e.y, w = (e - f) g as (wh, 2 wl), from the split
// offset: e - f = dh - fl with dh = e - fh exact.  wh = fl(dh gh + c1), c1 = -fl gh per stamp,
// is w rounded once (within ~1.3 ulp, as edge_arg2's); its residual dh gh - wh is of the size
// of c1 plus half an ulp of wh, so the FMA forms it to ~2^-45 g; the low part adds c1 back
// and dh gl (gl2 = 2 gl and c2 = 2 c1 per stamp; fl gl, below 2^-45 g, is dropped).  w to
// ~2^-45 g absolute, in five packed operations instead of edge_arg2's eight.
__device__ __forceinline__ void edge_arg2_split(float2 e, float fh, float gh, float2 gl2, float c1, float2 c2,
                                                float2& wh, float2& wl2) {
  const float2 g = f2(gh, gh);
  const float2 dh = __fadd2_rn(e, f2(-fh, -fh));
  wh = __ffma2_rn(dh, g, f2(c1, c1));
  const float2 err = __ffma2_rn(dh, g, f2(-wh.x, -wh.y));
  wl2 = __ffma2_rn(err, f2(2.f, 2.f), __ffma2_rn(dh, gl2, c2));
}

}  // namespace e2e
