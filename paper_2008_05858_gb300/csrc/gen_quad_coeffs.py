"""Write ``quad_coeffs.h``: Gauss-Legendre rules on [-1/2, 1/2] for the elliptical PSF.

The kernels integrate the x-marginal density of the rotated Gaussian over one pixel column
(width 1) to get the conditional moments of the in-column offset tau.  Nodes and weights
come from numpy.polynomial.legendre.leggauss (Golub-Welsch), mapped from [-1, 1] to
[-1/2, 1/2] (nodes / 2, weights / 2).

  * 5 points for the FP32 kernel: the centre weight and the two positive nodes (the rule is
    symmetric), with the nodes' powers tau^k, k = 1..6.
  * 12 points for the FP64 kernel, as __constant__ arrays.

Run:  python gen_quad_coeffs.py   (needs numpy; only at build-authoring time).
"""
import os

import numpy as np


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
    out.append(f"constexpr float kGl5WC = {w5[np.argmin(np.abs(x5))]:.9e}f;  // node tau = 0")
    pos = [(t, wt) for t, wt in zip(x5, w5) if t > 1e-12]
    pos.sort()
    for i, (t, wt) in enumerate(pos):
        out.append(f"constexpr float kGl5W{i} = {wt:.9e}f;")
        for k in range(1, 7):
            out.append(f"constexpr float kGl5T{i}P{k} = {t ** k:.9e}f;")
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
