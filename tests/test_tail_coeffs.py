"""The committed FP32 approximation coefficients (csrc/tail_coeffs.h) against scipy, on the
CPU: each approximation, evaluated in FP64 with its coefficients as the kernels hold them
(FP32), stays within its stated range's error; and the generator reproduces the header."""
import os
import re

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2008_05858_gb300", "csrc")


def _consts():
    txt = open(os.path.join(CSRC, "tail_coeffs.h")).read()
    out = {}
    for name, val in re.findall(r"constexpr (?:float|double) (k\w+) = ([-+0-9.eE]+)f?;", txt):
        out[name] = float(val)
    return out


C = _consts()
KAPPA = np.sqrt(np.log2(np.e))  # the kernels' arguments are in log2 units, w = a sqrt(log2 e)


def _poly(prefix, n, x):
    c = [np.float64(np.float32(C[f"{prefix}{i}"])) for i in range(n + 1)]
    return np.polyval(c[::-1], x)


def test_log2e_constant():
    assert abs(C["kSqrtLog2e"] - KAPPA) < 1e-9
    assert abs(C["kSqrtLog2eD"] - KAPPA) < 1e-15


def test_general_erfcx_rational():
    w = np.linspace(0.0, C["kTailMaxArg"], 200001)
    r = _poly("kTailP", 4, w) / _poly("kTailQ", 5, w)
    rel = np.abs(r / special.erfcx(w / KAPPA) - 1).max()
    assert rel < 2e-8, rel  # fit 2.0e-9, plus the FP32 rounding of the coefficients


def test_tail_edge_erfcx_rational():
    w = np.linspace(C["kTailFarMinArg"], C["kTailMaxArg"], 200001)
    r = _poly("kTailFarP", 3, w) / _poly("kTailFarQ", 4, w)
    rel = np.abs(r / special.erfcx(w / KAPPA) - 1).max()
    assert rel < 8e-8, rel  # fit 4.9e-8, plus the FP32 rounding of the coefficients
    # below its range the cheaper rational is not meant to be used: it is visibly worse there
    w0 = np.linspace(0.0, 0.1, 1001)
    r0 = _poly("kTailFarP", 3, w0) / _poly("kTailFarQ", 4, w0)
    assert np.abs(r0 / special.erfcx(w0 / KAPPA) - 1).max() > 10 * rel


def test_erf_polynomial_near_the_centre():
    w = np.linspace(1e-6, C["kErfMaxArg"], 100001)
    s = _poly("kErfS", 5, w * w) * w
    rel = np.abs(s / special.erf(w / KAPPA) - 1).max()
    assert rel < 2e-8, rel  # fit 4.8e-9


def test_generator_reproduces_the_header():
    import sys

    sys.path.insert(0, CSRC)
    try:
        import gen_tail_coeffs as g
    finally:
        sys.path.pop(0)
    _, p, q = g.fit()
    _, pf, qf = g.fit(m=g.FAR_M, n=g.FAR_N, amin=g.FAR_W)
    _, sc = g.fit_erf()
    for pre, vals in (("kTailP", p), ("kTailQ", q), ("kTailFarP", pf), ("kTailFarQ", qf), ("kErfS", sc)):
        for i, v in enumerate(vals):
            assert abs(C[f"{pre}{i}"] - v) <= 1e-9 * max(1.0, abs(v)), (pre, i)
