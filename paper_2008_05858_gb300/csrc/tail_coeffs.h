// Generated by gen_tail_coeffs.py -- do not edit.
// erfcx(w / sqrt(log2 e)) ~= P(w)/Q(w) on w in [0, 6.5 sqrt(log2 e)], degrees (4, 5), max relative fit error 2.01e-09
#pragma once
namespace e2e {
constexpr float kTailP0 = 1.000000002e+00f;
constexpr float kTailP1 = 9.964022297e-01f;
constexpr float kTailP2 = 4.774524070e-01f;
constexpr float kTailP3 = 1.206712217e-01f;
constexpr float kTailP4 = 1.377431187e-02f;
constexpr float kTailQ0 = 1.000000000e+00f;
constexpr float kTailQ1 = 1.935839690e+00f;
constexpr float kTailQ2 = 1.602902543e+00f;
constexpr float kTailQ3 = 7.188032186e-01f;
constexpr float kTailQ4 = 1.780958689e-01f;
constexpr float kTailQ5 = 2.032556214e-02f;
constexpr float kTailMaxArg = 7.8073f;  // largest w the fit covers
// tail edges of narrow PSFs: erfcx(w / sqrt(log2 e)) ~= PF(w)/QF(w) on w in [0.40, 6.5 sqrt(log2 e)], degrees (3, 4), max relative fit error 4.91e-08
constexpr float kTailFarP0 = 9.999673184e-01f;
constexpr float kTailFarP1 = 8.650136613e-01f;
constexpr float kTailFarP2 = 3.418012716e-01f;
constexpr float kTailFarP3 = 5.964265918e-02f;
constexpr float kTailFarQ0 = 1.000000000e+00f;
constexpr float kTailFarQ1 = 1.804167850e+00f;
constexpr float kTailFarQ2 = 1.344621157e+00f;
constexpr float kTailFarQ3 = 5.040287026e-01f;
constexpr float kTailFarQ4 = 8.802431055e-02f;
constexpr float kTailFarMinArg = 0.40f;  // smallest w that fit covers
constexpr float kSqrtLog2e = 1.201122409f;
constexpr double kSqrtLog2eD = 1.2011224087864498;
// erf(w / sqrt(log2 e)) ~= w * S(w^2) for |w| <= 1.00, 6 terms, max relative fit error 4.78e-09
constexpr float kErfS0 = 9.394372742e-01f;
constexpr float kErfS1 = -2.170557832e-01f;
constexpr float kErfS2 = 4.513187456e-02f;
constexpr float kErfS3 = -7.433231989e-03f;
constexpr float kErfS4 = 9.731278067e-04f;
constexpr float kErfS5 = -8.515646385e-05f;
constexpr float kErfMaxArg = 1.00f;
}  // namespace e2e
