"""Generate the rational approximation of the scaled complementary error function used by
the FP32 PSF kernels, and write ``tail_coeffs.h``.

    erfcx(a) = exp(a^2) erfc(a)  ~=  P4(a) / Q5(a),   a in [0, 6.5],  Q5(0) = 1

Method: linearised rational least squares (Loeb's method: minimise the weighted residual
P(a) - f(a) Q(a) with weights 1 / (f Q_prev)), iterated with Lawson's reweighting toward
the minimax relative error, on Chebyshev points.  Reference values: scipy.special.erfcx.
Run:  python gen_tail_coeffs.py   (needs numpy and scipy; only at build-authoring time).
"""
import os

import numpy as np
from scipy import special

M, N, A = 4, 5, 6.5


def fit(m=M, n=N, amax=A, iters=120, npts=6000):
    k = np.arange(npts)
    a = 0.5 * amax * (1 - np.cos(np.pi * (k + 0.5) / npts))
    f = special.erfcx(a)
    w = np.ones_like(a)
    q_prev = np.ones_like(a)
    best = None
    for _ in range(iters):
        V = np.concatenate([a[:, None] ** np.arange(m + 1)[None, :],
                            -(f[:, None] * a[:, None] ** np.arange(1, n + 1)[None, :])], axis=1)
        W = w / (f * q_prev)
        sol, *_ = np.linalg.lstsq(V * W[:, None], f * W, rcond=None)
        p = sol[: m + 1]
        q = np.concatenate([[1.0], sol[m + 1:]])
        Q = np.polyval(q[::-1], a)
        err = np.polyval(p[::-1], a) / Q / f - 1
        e = float(np.max(np.abs(err)))
        if best is None or e < best[0]:
            best = (e, p.copy(), q.copy())
        q_prev = Q
        w = w * np.abs(err) ** 0.5 + 1e-30
        w /= w.max()
    return best


def main():
    e, p, q = fit()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_tail_coeffs.py -- do not edit.",
        "// erfcx(a) ~= P(a)/Q(a) on [0, %.1f], degrees (%d, %d), max relative fit error %.2e" % (A, M, N, e),
        "#pragma once",
        "namespace e2e {",
        *["constexpr float kTailP%d = %.9ef;" % (i, c) for i, c in enumerate(p)],
        *["constexpr float kTailQ%d = %.9ef;" % (i, c) for i, c in enumerate(q)],
        "constexpr float kTailMaxArg = %.1ff;" % A,
        "}  // namespace e2e",
        "",
    ]
    with open(os.path.join(here, "tail_coeffs.h"), "w") as fh:
        fh.write("\n".join(lines))
    print("max relative fit error %.3e" % e)


if __name__ == "__main__":
    main()
