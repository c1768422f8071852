"""Generate the rational approximation of the scaled complementary error function used by
the FP32 PSF kernels, and write ``tail_coeffs.h``.

The kernels carry the edge argument in log2 units, w = a * sqrt(log2 e), so that
exp(-a^2) = 2^(-w^2) needs no extra scaling; the rational is fitted in that variable:

    erfcx(w / sqrt(log2 e)) = exp(a^2) erfc(a)  ~=  P4(w) / Q5(w),   w in [0, 6.5 sqrt(log2 e)],  Q5(0) = 1

Method: linearised rational least squares (Loeb's method: minimise the weighted residual
P(a) - f(a) Q(a) with weights 1 / (f Q_prev)), iterated with Lawson's reweighting toward
the minimax relative error, on Chebyshev points.  Reference values: scipy.special.erfcx.
Near the window centre the kernels use erf itself, as an odd polynomial in w fitted the
same way (relative error, Lawson-reweighted least squares on Chebyshev points):

    erf(w / sqrt(log2 e))  ~=  w * S5(w^2),   |w| <= 1.0

Run:  python gen_tail_coeffs.py   (needs numpy and scipy; only at build-authoring time).
"""
import os

import numpy as np
from scipy import special

M, N, A = 4, 5, 6.5
KAPPA = float(np.sqrt(np.log2(np.e)))  # w = a * KAPPA


def fit(m=M, n=N, amax=A * KAPPA, iters=120, npts=6000, amin=0.0):
    k = np.arange(npts)
    a = amin + 0.5 * (amax - amin) * (1 - np.cos(np.pi * (k + 0.5) / npts))  # the fit variable w
    f = special.erfcx(a / KAPPA)
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


ERF_W, ERF_TERMS = 1.0, 6

# Tail edges (one or more pixels from the stamp centre) of a model whose widest PSF keeps their
# arguments at or above FAR_W: a cheaper (3, 4) rational on [FAR_W, 6.5 sqrt(log2 e)].
FAR_M, FAR_N, FAR_W = 3, 4, 0.4


def fit_erf(wmax=ERF_W, nt=ERF_TERMS, iters=80, npts=4000):
    k = np.arange(npts)
    w = 0.5 * wmax * (1 - np.cos(np.pi * (k + 0.5) / npts)) + 1e-6
    target = special.erf(w / KAPPA) / w
    V = (w * w)[:, None] ** np.arange(nt)[None, :]
    wt = np.ones_like(w)
    best = None
    for _ in range(iters):
        sol, *_ = np.linalg.lstsq(V * (wt / target)[:, None], wt, rcond=None)
        err = V @ sol / target - 1
        e = float(np.max(np.abs(err)))
        if best is None or e < best[0]:
            best = (e, sol.copy())
        wt = wt * np.abs(err) ** 0.5 + 1e-30
        wt /= wt.max()
    return best


def main():
    e, p, q = fit()
    ef, pf, qf = fit(m=FAR_M, n=FAR_N, amin=FAR_W)
    ee, sc = fit_erf()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_tail_coeffs.py -- do not edit.",
        "// erfcx(w / sqrt(log2 e)) ~= P(w)/Q(w) on w in [0, %.1f sqrt(log2 e)], degrees (%d, %d),"
        " max relative fit error %.2e" % (A, M, N, e),
        "#pragma once",
        "namespace e2e {",
        *["constexpr float kTailP%d = %.9ef;" % (i, c) for i, c in enumerate(p)],
        *["constexpr float kTailQ%d = %.9ef;" % (i, c) for i, c in enumerate(q)],
        "constexpr float kTailMaxArg = %.4ff;  // largest w the fit covers" % (A * KAPPA),
        "// tail edges of narrow PSFs: erfcx(w / sqrt(log2 e)) ~= PF(w)/QF(w) on w in [%.2f, %.1f sqrt(log2 e)],"
        " degrees (%d, %d),"
        " max relative fit error %.2e" % (FAR_W, A, FAR_M, FAR_N, ef),
        *["constexpr float kTailFarP%d = %.9ef;" % (i, c) for i, c in enumerate(pf)],
        *["constexpr float kTailFarQ%d = %.9ef;" % (i, c) for i, c in enumerate(qf)],
        "constexpr float kTailFarMinArg = %.2ff;  // smallest w that fit covers" % FAR_W,
        "constexpr float kSqrtLog2e = %.9ff;" % KAPPA,
        "constexpr double kSqrtLog2eD = %.17g;" % KAPPA,
        "// erf(w / sqrt(log2 e)) ~= w * S(w^2) for |w| <= %.2f, %d terms, max relative fit error %.2e"
        % (ERF_W, ERF_TERMS, ee),
        *["constexpr float kErfS%d = %.9ef;" % (i, c) for i, c in enumerate(sc)],
        "constexpr float kErfMaxArg = %.2ff;" % ERF_W,
        "}  // namespace e2e",
        "",
    ]
    with open(os.path.join(here, "tail_coeffs.h"), "w") as fh:
        fh.write("\n".join(lines))
    print("erfcx rational: max relative fit error %.3e; tail-edge rational: %.3e; erf polynomial: %.3e"
          % (e, ef, ee))


if __name__ == "__main__":
    main()
