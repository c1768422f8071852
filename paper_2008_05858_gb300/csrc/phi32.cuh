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

// erf(|w| / sqrt(log2 e)) for |w| <= kErfMaxArg (odd polynomial, ~1.7 ulp): near the window
// centre the pixel integrals are sums and differences of erf, which do not cancel there the
// way differences of erfc values close to 1 do.
__device__ __forceinline__ float erf_small(float w) {
  const float a = fabsf(w);
  const float z = a * a;
  float S = kErfS4;
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

}  // namespace e2e
