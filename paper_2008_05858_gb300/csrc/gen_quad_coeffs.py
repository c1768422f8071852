"""Write ``quad_coeffs.h``: Gauss-Legendre rules on [-1/2, 1/2] for the elliptical PSF.

The kernels integrate the x-marginal density of the rotated Gaussian over one pixel column
(width 1) to get the conditional moments of the in-column offset tau.  Nodes and weights
come from numpy.polynomial.legendre.leggauss (Golub-Welsch), mapped from [-1, 1] to
[-1/2, 1/2] (nodes / 2, weights / 2).

  * 5 points for the FP32 kernel, which takes the moments of u = tau -+ 1/2 (the offset from
    the centre of a pair of columns): the two positive nodes T_i and T_i^2, and the weighted
    node powers W_i (1/2 + T_i)^k, W_i (1/2 - T_i)^k and W_C (1/2)^k, k = 0..8.
  * 12 points for the FP64 kernel, as __constant__ arrays.

Run:  python gen_quad_coeffs.py   (needs numpy; only at build-authoring time).
"""
import os

import numpy as np

KMAX = 7  # highest moment of the FP32 kernel's series


def rule(q):
    x, w = np.polynomial.legendre.leggauss(q)
    return x / 2.0, w / 2.0


def main():
    out = []
    out.append("// Generated by gen_quad_coeffs.py: Gauss-Legendre rules on [-1/2, 1/2]. Do not edit.")
    out.append("#pragma once")
    out.append("")
    out.append("namespace e2e {")
    x5, w5 = rule(5)
    wc = w5[np.argmin(np.abs(x5))]
    pos = sorted((t, wt) for t, wt in zip(x5, w5) if t > 1e-12)
    out.append(f"constexpr int kGlKmax = {KMAX};")
    for i, (t, wt) in enumerate(pos):
        out.append(f"constexpr float kGlT{i} = {t:.9e}f, kGlT{i}Sq = {t * t:.9e}f;")
        out.append(f"__device__ constexpr float kGlA{i}[{KMAX + 1}] = {{" +
                   ", ".join(f"{wt * (0.5 + t) ** k:.9e}f" for k in range(KMAX + 1)) + "};")
        out.append(f"__device__ constexpr float kGlB{i}[{KMAX + 1}] = {{" +
                   ", ".join(f"{wt * (0.5 - t) ** k:.9e}f" for k in range(KMAX + 1)) + "};")
    out.append(f"__device__ constexpr float kGlC[{KMAX + 1}] = {{" +
               ", ".join(f"{wc * 0.5 ** k:.9e}f" for k in range(KMAX + 1)) + "};  // node tau = 0")
    x12, w12 = rule(12)
    out.append("constexpr int kGl12 = 12;")
    out.append("__constant__ double kGl12T[12] = {" + ", ".join(f"{v:.17e}" for v in x12) + "};")
    out.append("__constant__ double kGl12W[12] = {" + ", ".join(f"{v:.17e}" for v in w12) + "};")
    out.append("}  // namespace e2e")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "quad_coeffs.h")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
