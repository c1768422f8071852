// Generated by gen_tail_coeffs.py -- do not edit.
// erfcx(a) ~= P(a)/Q(a) on [0, 6.5], degrees (4, 5), max relative fit error 2.01e-09
#pragma once
namespace e2e {
constexpr float kTailP0 = 1.000000002e+00f;
constexpr float kTailP1 = 1.196801051e+00f;
constexpr float kTailP2 = 6.888182247e-01f;
constexpr float kTailP3 = 2.091055320e-01f;
constexpr float kTailP4 = 2.866942590e-02f;
constexpr float kTailQ0 = 1.000000000e+00f;
constexpr float kTailQ1 = 2.325180436e+00f;
constexpr float kTailQ2 = 2.312499560e+00f;
constexpr float kTailQ3 = 1.245580569e+00f;
constexpr float kTailQ4 = 3.706832211e-01f;
constexpr float kTailQ5 = 5.081347772e-02f;
constexpr float kTailMaxArg = 6.5f;
}  // namespace e2e
