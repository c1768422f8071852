// FP32 Gaussian tail erfc(|u|) for a double-float argument u = uh + ul.
//
// A stamp's pixel integrals are differences of the normal CDF at the pixel edges (the
// pixel-integrated PSF of Sec. 2.2).  In FP32 the edge argument u = (edge - centre)/(sqrt2
// sigma) carries a relative error of ~1e-7, which the factor exp(-u^2) amplifies by 2u^2
// (1e-6 at u = 2).  So u is kept as a double-float and the exponent is formed exactly:
//
//   erfc(a) = exp(-a^2) * erfcx(a),        a = |u|
//   exp(-a^2) = 2^(zh + zl),  zh + zl = -(a^2) log2(e) to ~2^-48 (FMA error terms),
//   2^zh by the SFU (ex2.approx, 2.4 ulp measured), 2^zl ~= 1 + zl ln2 (|zl| < 1e-5),
//   erfcx(a) by the rational P4/Q5 of tail_coeffs.h (fit error 2e-9; rcp.approx on the SFU).
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

// erfc(|uh + ul|), |ul| <= ulp(uh).
__device__ __forceinline__ float erfc_df(float uh, float ul) {
  const float a = fabsf(uh);
  const float al = uh < 0.f ? -ul : ul;  // a + al = |u|
  const float p = a * a;
  float e = fmaf(a, a, -p);             // exact error of p
  e = fmaf(a + a, al, e);               // + 2 a al  (al^2 negligible)
  const float L = -1.44269502163f;      // -log2(e), FP32 part
  const float Llo = -1.925963e-08f;     // -log2(e) - L
  const float zh = p * L;
  float zl = fmaf(p, L, -zh);
  zl = fmaf(p, Llo, zl);
  zl = fmaf(e, L, zl);
  const float ex = ex2_approx(zh) * fmaf(zl, 0.693147181f, 1.f);
  const float x = fminf(a, 30.f);
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

// Twice the probability that a standard normal lies between two edges, from the edges'
// signed arguments ta <= tb and their tails Ea = erfc(|ta|), Eb = erfc(|tb|): on one side
// of the mean a difference of the (small) tails, across the mean 2 minus both tails.
__device__ __forceinline__ float twice_interval(float ta, float tb, float ea, float eb) {
  return ta >= 0.f ? ea - eb : (tb <= 0.f ? eb - ea : 2.f - ea - eb);
}

// Edge argument as a double-float: u = (e - f) * g with e a half-integer (exact), f the
// FP32 sub-pixel offset, g = gh + gl = 1/(sqrt2 sigma).  e - f is split exactly
// (|e| >= 1/2 >= |f|, so Fast2Sum applies); the product keeps its FMA error term.
__device__ __forceinline__ void edge_arg(float e, float f, float gh, float gl, float& uh, float& ul) {
  const float dh = e - f;
  const float dl = (e - dh) - f;
  uh = dh * gh;
  ul = fmaf(dh, gh, -uh) + fmaf(dh, gl, dl * gh);
}

}  // namespace e2e
